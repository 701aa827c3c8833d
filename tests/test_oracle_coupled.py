"""Pins of the bulk-surface coupled oracle (Section 5.5).

C1: the boundary-flux term of the bulk operator, (2/h + 2/rho_*) g on the outer shell, makes the
    discrete ball Laplacian exact on u = rho^2 (normal derivative 2 rho_*): 6 at every node.
C2: with zeta1 = 0 the coupled step is the uncoupled ball and sphere split steps.
C3: the homogeneous equilibrium (u_e, v_e, u_e, v_e) is a fixed point of the coupled step.
"""
import numpy as np
import pytest

from oracle.coupled import Coupled
from oracle.stepper import step


@pytest.mark.parametrize("n", [(5, 6, 7), (9, 8, 6)])
@pytest.mark.parametrize("rho_star", [1.0, 0.7])
def test_C1_flux_term_exact_on_rho_squared(n, rho_star):
    c = Coupled(n, 1e-3, rho_star=rho_star)
    g = c.ball
    rho = g.points[1]
    u = np.broadcast_to((rho**2)[None, None, :], g.shape).copy()
    lap = g.apply_M(u) + c.radial_flux(np.full((n[2], n[1]), 2.0 * rho_star))
    assert np.max(np.abs(lap - 6.0)) < 1e-9 * max(1.0, 1.0 / c.h**2)


def test_C2_no_coupling_is_two_uncoupled_steps():
    c = Coupled((5, 6, 7), 1e-3, zeta1=0.0)
    rng = np.random.default_rng(4)
    ue, ve = c.equilibrium()
    Wb = np.stack([ue + 1e-2 * rng.standard_normal(c.ball.shape), ve + 1e-2 * rng.standard_normal(c.ball.shape)])
    Ws = np.stack([ue + 1e-2 * rng.standard_normal(c.sphere.shape), ve + 1e-2 * rng.standard_normal(c.sphere.shape)])
    b, s = c.step(Wb, Ws)
    assert np.max(np.abs(b - step(c.pb, Wb))) < 1e-14 * np.max(np.abs(b))
    assert np.max(np.abs(s - step(c.ps, Ws))) < 1e-14 * np.max(np.abs(s))


def test_C3_equilibrium_is_a_fixed_point():
    c = Coupled((6, 8, 7), 1e-3)
    ue, ve = c.equilibrium()
    Wb = np.stack([np.full(c.ball.shape, ue), np.full(c.ball.shape, ve)])
    Ws = np.stack([np.full(c.sphere.shape, ue), np.full(c.sphere.shape, ve)])
    b, s = c.run(Wb, Ws, 5)
    assert np.max(np.abs(b - Wb)) < 1e-12 and np.max(np.abs(s - Ws)) < 1e-12
