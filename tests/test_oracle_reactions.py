"""Pins of the oracle's reaction terms: each vanishes at the homogeneous states its model is built
around, found from the model's own equations (not by re-evaluating the code's formula elsewhere).
The manufactured BVAM sources are pinned through the Fig. 1 errors (tests/test_oracle_stepper.py).
"""
import numpy as np
import pytest

from oracle import reactions as R


def point(*values):
    return np.array([[v] for v in values])


@pytest.mark.parametrize("gamma,a,b", [(100.0, 0.1, 0.9), (200.0, 0.12, 0.85), (500.0, 0.14, 1.34)])
def test_schnakenberg_steady_state(gamma, a, b):
    """f = g = 0 at (a + b, b / (a + b)^2): g = 0 gives u^2 v = b, then f = 0 gives u = a + b."""
    f, g = R.schnakenberg(point(a + b, b / (a + b) ** 2), gamma, a, b)
    assert abs(f[0]) < 1e-12 * gamma and abs(g[0]) < 1e-12 * gamma
    f, g = R.schnakenberg(point(a + b + 1e-3, b / (a + b) ** 2), gamma, a, b)
    assert f[0] != 0.0 and g[0] != 0.0


@pytest.mark.parametrize("F,k", [(0.04, 0.06), (0.03, 0.055), (0.025, 0.05)])
def test_gray_scott_equilibria(F, k):
    """The homogeneous states of f = -u v^2 + F(1 - u), g = u v^2 - (F + k) v: the trivial (1, 0),
    and, where F^2 >= 4 F (F + k)^2, the roots of (F + k) v^2 - F v + F (F + k) = 0 with
    u = (F + k) / v (u v = F + k from g = 0 with v != 0, then f = 0); at the benchmark's
    F = 0.04, k = 0.06 the two coincide at (0.5, 0.2)."""
    f, g = R.gray_scott(point(1.0, 0.0), F, k)
    assert f[0] == 0.0 and g[0] == 0.0
    disc = F * F - 4.0 * F * (F + k) ** 2
    if disc >= 0:
        for v in ((F + np.sqrt(disc)) / (2 * (F + k)), (F - np.sqrt(disc)) / (2 * (F + k))):
            f, g = R.gray_scott(point((F + k) / v, v), F, k)
            assert abs(f[0]) < 1e-15 and abs(g[0]) < 1e-15, (v, f, g)
    if (F, k) == (0.04, 0.06):
        f, g = R.gray_scott(point(0.5, 0.2), F, k)
        assert abs(f[0]) < 1e-16 and abs(g[0]) < 1e-16
    f, g = R.gray_scott(point(0.7, 0.1), F, k)          # away from them, the terms differ from 0
    assert f[0] != 0.0 and g[0] != 0.0


def test_linear_cubic_equilibria():
    """f_i = sum_j K_ij u_j - u_i^3 vanishes at 0 and, for a diagonal K = diag(kappa), at
    u_i = +-sqrt(kappa_i) in every combination of signs."""
    kappa = [0.5, 2.0, 1.25]
    K = np.diag(kappa)
    assert all(x[0] == 0.0 for x in R.linear_cubic(point(0.0, 0.0, 0.0), K))
    for signs in ((1, 1, 1), (1, -1, 1), (-1, -1, 1)):
        u = point(*[s * np.sqrt(k) for s, k in zip(signs, kappa)])
        assert all(abs(x[0]) < 1e-15 for x in R.linear_cubic(u, K))
    K2 = K + np.array([[0.0, 0.3, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])   # an off-diagonal coupling shows
    assert abs(R.linear_cubic(u, K2)[0][0] - 0.3 * u[1][0]) < 1e-15


def test_bvam_vanishes_at_the_origin():
    """b(0, 0) = c(0, 0) = 0 (eq. BVAMnl has no constant term), and both are linear to first order."""
    b, c = R.bvam(point(0.0, 0.0))
    assert b[0] == 0.0 and c[0] == 0.0
    p = R.BVAM
    e = 1e-7
    b, c = R.bvam(point(e, 0.0))
    assert abs(b[0] - p["alpha1"] * e) < 1e-20 and abs(c[0] - p["beta2"] * e) < 1e-20
    b, c = R.bvam(point(0.0, e))
    assert abs(b[0] - e) < 1e-20 and abs(c[0] - p["beta1"] * e) < 1e-20
