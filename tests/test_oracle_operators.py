"""Pins of the oracle's Kronecker-sum operators (Section 2, eqs. disk/sphere/ball/cylinder).

* M applied to samples of a smooth function equals the continuous curvilinear
  Laplacian (eqs. lapdisk, lapsphere, lapball, lapcyl) to second order;
* every Kronecker term equals its fibre description (scale factor times the
  1-D matrix along one mode), the form the split step uses;
* the mass weights derived from Proposition 1's Xi annihilate every term
  (left null vectors under Neumann/periodic boundaries).
"""
import numpy as np
import pytest

from oracle.operators import Grid


def _mesh(g):
    pts = [g.points[mu] for mu in range(g.ndim, 0, -1)]       # numpy axis order
    return np.meshgrid(*pts, indexing="ij")


def _g(R):
    # Radial profile with g'(1) = 0, g'''(1) = 0 and g ~ rho^2 at 0.  The
    # Neumann rows (mirrored ghost value) are second-order consistent only when
    # the third derivative vanishes at the wall, as in the 1-D checks.
    return R**2 - 5 / 7 * R**4 + 1 / 7 * R**6


def _smooth_case(kind, g):
    """Smooth f with the Neumann conditions of the grid, and its exact Laplacian."""
    if kind == "disk":
        TH, R = _mesh(g)
        return _g(R) * np.cos(2 * TH), (-60 / 7 * R**2 + 32 / 7 * R**4) * np.cos(2 * TH)
    if kind == "sphere":
        PH, TH = _mesh(g)
        f = np.sin(PH) ** 2 * np.cos(2 * TH) + np.cos(PH)       # Y_2^2 and Y_1^0 parts
        return f, -6 * np.sin(PH) ** 2 * np.cos(2 * TH) - 2 * np.cos(PH)
    if kind == "ball":
        PH, TH, R = _mesh(g)
        Y = np.sin(PH) ** 2 * np.cos(2 * TH)
        # (g'' + 2 g'/rho - 6 g/rho^2) Y
        return _g(R) * Y, (-10 * R**2 + 36 / 7 * R**4) * Y
    if kind == "cylinder":
        Z, TH, R = _mesh(g)
        gR = _g(R)
        f = gR * np.cos(2 * TH) * np.cos(np.pi * Z)
        return f, (-60 / 7 * R**2 + 32 / 7 * R**4 - np.pi**2 * gR) * np.cos(2 * TH) * np.cos(np.pi * Z)
    raise ValueError(kind)


SIZES = {
    "disk": [(12, 24), (24, 48), (48, 96)],
    "sphere": [(24, 12), (48, 24), (96, 48)],
    "ball": [(8, 16, 8), (16, 32, 16), (32, 64, 32)],
    "cylinder": [(8, 16, 8), (16, 32, 16), (32, 64, 32)],
}


@pytest.mark.parametrize("kind", ["disk", "sphere", "ball", "cylinder"])
def test_laplacian_second_order(kind):
    errs = []
    for n in SIZES[kind]:
        g = Grid(kind, n)
        f, lap = _smooth_case(kind, g)
        errs.append(np.max(np.abs(g.apply_M(f) - lap)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates > 1.7), (kind, errs, rates)


@pytest.mark.parametrize("kind,n", [("disk", (5, 7)), ("sphere", (6, 5)), ("ball", (4, 6, 5)),
                                    ("cylinder", (4, 6, 5))])
def test_kronecker_terms_equal_fibre_form(kind, n):
    g = Grid(kind, n)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(g.shape)
    for mu in range(1, g.ndim + 1):
        axis = g.ndim - mu
        fib = np.moveaxis(np.moveaxis(w, axis, -1) @ g.A[mu].T, -1, axis)
        fib = np.broadcast_to(g.scale[mu], w.shape) * fib
        kr = (g.M[mu] @ w.ravel()).reshape(g.shape)
        assert np.allclose(fib, kr, rtol=1e-13, atol=1e-13 * np.abs(kr).max())


def _mass_weights(g):
    """Left null vectors: m_rho2 = (1,3,...,2n-3,n-1), m_rho3 = (1,4,...,(n-1)^2, n(n-1)/2),
    m_theta = 1, m_z (Neumann caps) = (1/2, 1, ..., 1, 1/2), m_phi = Xi^{-2} 1 (numeric)."""
    from oracle import axes as ax
    def m_rho2(n):
        return np.array([2 * i - 1.0 for i in range(1, n)] + [n - 1.0])
    def m_rho3(n):
        return np.array([i * i * 1.0 for i in range(1, n)] + [n * (n - 1) / 2.0])
    def m_phi(A):
        xi = ax.xi_diagonal(A)
        return xi**-2.0
    if g.kind == "disk":
        return np.ones((g.n[1], 1)) * m_rho2(g.n[0])[None, :]
    if g.kind == "sphere":
        return m_phi(g.A[2])[:, None] * np.ones((1, g.n[0]))
    if g.kind == "ball":
        return m_phi(g.A[3])[:, None, None] * np.ones((1, g.n[1], 1)) * m_rho3(g.n[0])[None, None, :]
    if g.kind == "cylinder":
        mz = np.ones(g.n[2])
        mz[0] = mz[-1] = 0.5
        return mz[:, None, None] * np.ones((1, g.n[1], 1)) * m_rho2(g.n[0])[None, None, :]


@pytest.mark.parametrize("kind,n", [("disk", (7, 9)), ("sphere", (8, 7)), ("ball", (5, 6, 7)),
                                    ("cylinder", (5, 6, 7))])
def test_mass_weights_are_left_null_vectors(kind, n):
    g = Grid(kind, n)
    m = _mass_weights(g).ravel()
    for mu in range(1, g.ndim + 1):
        r = g.M[mu].T @ m
        assert np.max(np.abs(r)) < 1e-11 * abs(g.M[mu]).max() * np.max(m)
