"""Pins of the bulk-surface DIB oracle (Section 5.6).

D1: the bottom-flux term, 2 g / h on the z = 0 plane, makes the discrete cylinder operator exact on
    a quadratic in z with zero top value and normal derivative g at z = 0 (2 at every node);
    without it the bottom row is off by 4c/h.
D2: a discrete divergence theorem for the coupled right-hand side: with the bulk reactions off,
    the trapezoid-in-z, disk-null-vector-in-(rho, theta) sum of F_u equals minus the top outflow
    minus alpha3 times the surface sum of F_r (what the bulk loses through z = 0 the surface gains,
    scaled by alpha3); likewise for v with delta and beta3.  Fixes the sign, the factor 2/h and
    the scaling between the two sides.
D3: zeta1 = 0 reduces the coupled step to the uncoupled cylinder and disk steps.
D4: the homogeneous equilibrium (alpha2, beta2, 0, zeta5), with eta4 from the printed formula, is
    a fixed point; p and q vanish there.
"""
import numpy as np
import pytest

from oracle.coupled_dib import CoupledCylinder
from oracle.stepper import rhs, step


def m_rho2(n):
    """Closed-form left null vector of the disk radial axis, (1, 3, ..., 2n-3, n-1)."""
    return np.array([2 * i - 1.0 for i in range(1, n)] + [n - 1.0])


@pytest.mark.parametrize("n", [(5, 6, 7), (6, 8, 11)])
@pytest.mark.parametrize("c0", [0.3, -1.7])
def test_D1_bottom_flux_exact_on_quadratic(n, c0):
    cc = CoupledCylinder(n, 1e-3, rho_star=2.0, z_star=3.0)
    g = cc.bulk
    z = g.points[3]
    zs = 3.0
    u = np.broadcast_to(((z - zs) * (z + zs - 2 * c0))[:, None, None], g.shape).copy()
    gn = 2.0 * c0                                   # grad u . n = -u'(0)
    lap = g.apply_M(u) + cc.bottom_flux(np.full((n[1], n[0]), gn))
    scale = np.max(np.abs(u)) / cc.h**2
    assert np.max(np.abs(lap - 2.0)) < 1e-11 * scale
    plain = g.apply_M(u)
    assert np.allclose(plain[0] - 2.0, -4.0 * c0 / cc.h)


@pytest.mark.parametrize("delta", [1.0, 3.0])
def test_D2_discrete_divergence_theorem(delta):
    n = (6, 7, 9)
    cc = CoupledCylinder(n, 1e-3, rho_star=2.0, z_star=3.0, alpha1=0.0, beta1=0.0, delta=delta, zeta1=1.3,
                         alpha3=0.4, beta3=0.7)
    rng = np.random.default_rng(11)
    Wb = 0.3 * rng.standard_normal((2,) + cc.bulk.shape)
    Ws = 0.5 + 0.3 * rng.standard_normal((2,) + cc.surface.shape)
    Fb = rhs(cc.pb, Wb)
    Fs = rhs(cc.ps, Ws)
    ab, as_ = cc.coupling(Wb, Ws)
    Fb = [Fb[q] + ab[q] for q in range(2)]
    Fs = [Fs[q] + as_[q] for q in range(2)]
    W2 = np.ones((n[1], 1)) * m_rho2(n[0])[None, :]
    mz = np.ones(n[2])
    mz[0] = 0.5
    h = cc.h
    d = [1.0, delta]
    scal = [cc.c["alpha3"], cc.c["beta3"]]
    for q in range(2):
        bulk = h * np.sum(mz[:, None, None] * W2[None] * Fb[q])
        top = d[q] * np.sum(W2 * Wb[q][-1]) / h
        surf = d[q] * scal[q] * np.sum(W2 * Fs[q])
        ref = max(abs(bulk), abs(top), abs(surf))
        assert abs(bulk + top + surf) < 1e-11 * ref, (q, bulk, top, surf)


def test_D3_no_coupling_is_two_uncoupled_steps():
    cc = CoupledCylinder((5, 6, 7), 1e-2, zeta1=0.0)
    rng = np.random.default_rng(5)
    Wb = 1e-2 * rng.standard_normal((2,) + cc.bulk.shape)
    Ws = np.stack([1e-2 * rng.uniform(0, 1, cc.surface.shape), 0.5 + 1e-2 * rng.uniform(0, 1, cc.surface.shape)])
    b, s = cc.step(Wb, Ws)
    assert np.max(np.abs(b - step(cc.pb, Wb))) <= 1e-15 * np.max(np.abs(b))
    assert np.max(np.abs(s - step(cc.ps, Ws))) <= 1e-15 * np.max(np.abs(s))


def test_D4_equilibrium_is_a_fixed_point():
    cc = CoupledCylinder((6, 8, 5), 0.025)
    ue, ve, re, se = cc.equilibrium()
    assert (ue, ve, re, se) == (1.0, 1.0, 0.0, 0.5)
    assert abs(cc.p(ue, re, se)) == 0.0
    assert abs(cc.q(ve, re, se)) < 1e-15
    Wb = np.zeros((2,) + cc.bulk.shape)             # lifted: w = (u - alpha2, v - beta2)
    Ws = np.stack([np.full(cc.surface.shape, re), np.full(cc.surface.shape, se)])
    b, s = cc.run(Wb, Ws, 5)
    assert np.max(np.abs(b)) < 1e-14 and np.max(np.abs(s - Ws)) < 1e-14


def test_D5_surface_sees_the_bottom_plane_only():
    """The surface kinetics read the bulk at z = 0 (node k = 1 of eq. A_z) and nowhere else, and
    the flux enters only that plane."""
    cc = CoupledCylinder((5, 6, 7), 1e-3)
    rng = np.random.default_rng(9)
    Wb = 0.1 * rng.standard_normal((2,) + cc.bulk.shape)
    Ws = np.stack([0.2 + 0.1 * rng.uniform(0, 1, cc.surface.shape), 0.5 + 0.1 * rng.uniform(0, 1, cc.surface.shape)])
    ab, as_ = cc.coupling(Wb, Ws)
    for q in range(2):
        assert np.all(ab[q][1:] == 0.0)
    W2 = Wb.copy()
    W2[:, 1:] += 0.3                                 # every plane but the bottom one changed
    ab2, as2 = cc.coupling(W2, Ws)
    assert all(np.array_equal(as_[q], as2[q]) and np.array_equal(ab[q], ab2[q]) for q in range(2))
    W3 = Wb.copy()
    W3[:, 0] += 0.3                                  # the bottom plane changed
    ab3, as3 = cc.coupling(W3, Ws)
    assert all(np.max(np.abs(as3[q] - as_[q])) > 1e-3 for q in range(2))
