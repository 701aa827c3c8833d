"""Pins of the oracle's split exponential Euler step (Section 4 and Section 5.1).

P1  one step equals w + tau phi_1(tau d M_1)...phi_1(tau d M_d) F with every
    factor from dense expm of the assembled Kronecker term (tiny grids);
    reversing the factor order gives a different result (Section 4).
P2  the splitting error ||phi_1(tau M) - prod phi_1(tau M_mu)|| is O(tau^2)
    (eq. splitorder).
P3  exponential Euler is exact for w' = A w + c with constant c: data that
    the other directions annihilate reduces the split scheme to it.
P4  Neumann/periodic boundaries conserve the weighted mass m^T w exactly.
P5  first-order convergence; the printed errors of Fig. 1 (golden file).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import reactions as R
from oracle.operators import Grid
from oracle.stepper import Problem, rhs, run, step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_splitee_errors.txt")
TINY = [("disk", (6, 8)), ("sphere", (6, 5)), ("ball", (4, 6, 5)), ("cylinder", (4, 6, 5))]


def phi1_expm(X):
    n = X.shape[0]
    aug = np.zeros((2 * n, 2 * n))
    aug[:n, :n] = X
    aug[:n, n:] = np.eye(n)
    return sla.expm(aug)[:n, n:]


def _gray_scott(W, t):
    return R.gray_scott(W, 0.04, 0.06)


@pytest.mark.parametrize("kind,n", TINY)
def test_P1_step_equals_dense_product(kind, n):
    g = Grid(kind, n)
    d = [0.7, 0.3]
    tau = 0.01
    rng = np.random.default_rng(1)
    W = 0.5 + 0.1 * rng.standard_normal((2,) + g.shape)
    p = Problem(g, d, _gray_scott, tau)
    got = step(p, W)
    Md = {mu: g.M[mu].toarray() for mu in g.M}
    Mfull = sum(Md.values())
    G = _gray_scott(W, 0.0)
    for s in range(2):
        F = d[s] * Mfull @ W[s].ravel() + G[s].ravel()
        P = np.eye(g.npts)
        for mu in range(1, g.ndim + 1):        # phi_1(tau d M_1) ... phi_1(tau d M_d)
            P = P @ phi1_expm(tau * d[s] * Md[mu])
        ref = W[s].ravel() + tau * P @ F
        assert np.max(np.abs(got[s].ravel() - ref)) < 1e-13 * np.max(np.abs(ref))
        # the reversed order is a different method
        Prev = np.eye(g.npts)
        for mu in range(g.ndim, 0, -1):
            Prev = Prev @ phi1_expm(tau * d[s] * Md[mu])
        rev = W[s].ravel() + tau * Prev @ F
        assert np.max(np.abs(rev - ref)) > 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind,n", TINY)
def test_P2_splitting_error_is_second_order(kind, n):
    g = Grid(kind, n)
    Md = {mu: g.M[mu].toarray() for mu in g.M}
    Mfull = sum(Md.values())
    errs = []
    taus = [4e-5, 2e-5, 1e-5]          # tau ||M|| << 1: asymptotic regime
    for tau in taus:
        P = np.eye(g.npts)
        for mu in range(1, g.ndim + 1):
            P = P @ phi1_expm(tau * Md[mu])
        errs.append(np.linalg.norm(phi1_expm(tau * Mfull) - P, 2))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9) and np.all(rates < 2.1), rates


@pytest.mark.parametrize("kind,n,mu", [("disk", (7, 9), 1), ("sphere", (8, 7), 2), ("ball", (6, 5, 7), 1),
                                       ("cylinder", (6, 5, 7), 3)])
def test_P3_exact_for_linear_constant_forcing(kind, n, mu):
    """Data and forcing varying only along mode mu: every other M_nu annihilates them."""
    g = Grid(kind, n)
    rng = np.random.default_rng(2)
    axis = g.ndim - mu
    prof_w = rng.standard_normal(g.n[mu - 1])
    prof_c = rng.standard_normal(g.n[mu - 1])
    shape1 = [1] * g.ndim
    shape1[axis] = g.n[mu - 1]
    w0 = np.broadcast_to(prof_w.reshape(shape1), g.shape).copy()
    c = np.broadcast_to(prof_c.reshape(shape1), g.shape).copy()
    d, tau, steps = 0.3, 0.02, 7
    p = Problem(g, [d], lambda W, t: [c], tau)
    got = run(p, w0[None], steps)[0]
    T = steps * tau
    A = d * g.A[mu] * g.scale[mu].ravel()[0]     # the direction's own scale is 1 here
    ref_prof = sla.expm(T * A) @ prof_w + T * phi1_expm(T * A) @ prof_c
    ref = np.broadcast_to(ref_prof.reshape(shape1), g.shape)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind,n", [("disk", (7, 9)), ("sphere", (8, 7)), ("ball", (5, 6, 7)),
                                    ("cylinder", (5, 6, 7))])
def test_P4_mass_conservation(kind, n):
    from tests.test_oracle_operators import _mass_weights
    g = Grid(kind, n)
    m = _mass_weights(g)
    rng = np.random.default_rng(3)
    W = rng.random((1,) + g.shape)
    p = Problem(g, [0.8], lambda W, t: [np.zeros_like(W[0])], 0.05)
    m0 = np.sum(m * W[0])
    W = run(p, W, 40)
    assert abs(np.sum(m * W[0]) - m0) < 1e-13 * abs(m0) * 40


def _fig1_error(nr, nt, m):
    g = Grid("disk", (nr, nt))
    rho = g.points[1][None, :]
    th = g.points[2][:, None]

    def reac(W, t):                        # sources evaluated at t_n (explicit)
        b = R.bvam(W)
        s = R.bvam_sources(t, rho, th)
        return [b[0] + s[0], b[1] + s[1]]

    p = Problem(g, [R.BVAM["gamma"], R.BVAM["delta"]], reac, 1.0 / m)
    W = run(p, np.array(R.bvam_exact(0.0, rho, th)), m)
    E = np.array(R.bvam_exact(1.0, rho, th))
    wgt = rho + 0 * th                     # polar area element rho d rho d theta
    e = [np.sqrt(np.sum(wgt * (W[s] - E[s]) ** 2) / np.sum(wgt * E[s] ** 2)) for s in range(2)]
    return float(np.hypot(e[0], e[1]))


def test_P5_fig1_printed_errors():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    got = {}
    for nr, nt, m, err in rows:
        val = _fig1_error(int(nr), int(nt), int(m))
        got[(nr, nt, m)] = val
        assert abs(val / float(err) - 1) < 5e-3, (nr, nt, m, val, err)
    # first order in tau: slope -1 between the extreme step counts
    for nr, nt in [("25", "50"), ("40", "80")]:
        slope = np.log(got[(nr, nt, "3000")] / got[(nr, nt, "200")]) / np.log(3000 / 200)
        assert -1.05 < slope < -0.95


def test_P5_self_convergence_schnakenberg_disk():
    g = Grid("disk", (16, 24))
    rng = np.random.default_rng(4)
    a, b, gamma = 0.1, 0.9, 100.0
    W0 = np.array([np.full(g.shape, a + b), np.full(g.shape, b / (a + b) ** 2)])
    W0 = W0 + rng.uniform(-0.01, 0.01, W0.shape)
    reac = lambda W, t: R.schnakenberg(W, gamma, a, b)
    T = 0.02
    sols = []
    for m in [80, 160, 320, 640]:
        sols.append(run(Problem(g, [1.0, 10.0], reac, T / m), W0, m))
    e = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(3)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(rates - 1) < 0.15), rates


def test_rhs_zero_at_schnakenberg_steady_state():
    g = Grid("disk", (6, 8))
    a, b = 0.1, 0.9
    W = np.array([np.full(g.shape, a + b), np.full(g.shape, b / (a + b) ** 2)])
    p = Problem(g, [1.0, 10.0], lambda W, t: R.schnakenberg(W, 100.0, a, b), 1e-4)
    F = rhs(p, W)
    assert max(np.abs(f).max() for f in F) < 1e-10
