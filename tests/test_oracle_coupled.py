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


@pytest.mark.parametrize("delta", [1.0, 10.0])
def test_C4_discrete_divergence_theorem(delta):
    """With the reactions off, the ball's left null vector m_rho3 = (1, 4, ..., (n-1)^2, n(n-1)/2)
    times the angular weights (Xi^-2 1 of A_phi, the sphere's as well) annihilates the bulk
    Laplacian, so only the flux row survives: m_n (2/h + 2/rho_*) = (n^2 - 1)/h.  Hence
    sum W_b F_u = -(n^2 - 1)/h sum W_ang F_r, and likewise v with s (delta grad v . n is the
    exchanged quantity) — this fixes the flux factor, its sign and the pairing with the surface."""
    from oracle import axes as ax
    n = (6, 8, 7)
    c = Coupled(n, 1e-3, delta=delta, rho_star=0.8)
    zero = lambda W, t: [0.0 * W[0], 0.0 * W[1]]
    c.pb.reaction = zero
    c.ps.reaction = zero
    rng = np.random.default_rng(13)
    Wb = 1.0 + 0.2 * rng.standard_normal((2,) + c.ball.shape)
    Ws = 1.0 + 0.2 * rng.standard_normal((2,) + c.sphere.shape)
    from oracle.stepper import rhs
    Fb, Fs = rhs(c.pb, Wb), rhs(c.ps, Ws)
    ab, as_ = c.coupling(Wb, Ws)
    Fb = [Fb[q] + ab[q] for q in range(2)]
    Fs = [Fs[q] + as_[q] for q in range(2)]
    m_rho3 = np.array([i * i * 1.0 for i in range(1, n[0])] + [n[0] * (n[0] - 1) / 2.0])
    m_phi = ax.xi_diagonal(c.sphere.A[2]) ** -2.0
    W_ang = m_phi[:, None] * np.ones((1, n[1]))                  # sphere layout (phi, theta)
    W_b = W_ang[:, :, None] * m_rho3[None, None, :]               # ball layout (phi, theta, rho)
    for q in range(2):
        bulk = np.sum(W_b * Fb[q])
        surf = -(n[0] ** 2 - 1) / c.h * np.sum(W_ang * Fs[q])
        assert abs(bulk - surf) < 1e-10 * max(abs(bulk), abs(surf)), (q, bulk, surf)


def test_C5_coupling_reads_and_writes_the_outer_shell_only():
    c = Coupled((6, 8, 7), 1e-3)
    rng = np.random.default_rng(21)
    Wb = 1.0 + 0.1 * rng.standard_normal((2,) + c.ball.shape)
    Ws = 1.0 + 0.1 * rng.standard_normal((2,) + c.sphere.shape)
    ab, as_ = c.coupling(Wb, Ws)
    for q in range(2):
        assert np.all(ab[q][:, :, :-1] == 0.0)
    W2 = Wb.copy()
    W2[:, :, :, :-1] += 0.3                          # every shell but the outer one changed
    ab2, as2 = c.coupling(W2, Ws)
    assert all(np.array_equal(as_[q], as2[q]) and np.array_equal(ab[q], ab2[q]) for q in range(2))
    W3 = Wb.copy()
    W3[:, :, :, -1] += 0.3                           # the outer shell changed
    ab3, as3 = c.coupling(W3, Ws)
    assert all(np.max(np.abs(as3[q] - as_[q])) > 1e-3 for q in range(2))
