"""Bulk-surface Schnakenberg system on the ball and its boundary sphere (paper Section 5.5,
eqs. bulkball, bulkballsys, bulkballnl).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Bulk species u, v on the ball (Laplacian, eq. ball; diffusion 1 and delta; reactions alpha1 b,
alpha1 c), surface species r, s on the sphere rho = rho_* (Laplace-Beltrami / rho_*^2, eq.
sphere; diffusion 1/rho_*^2 and eps/rho_*^2), coupled by the boundary conditions
grad u . n = zeta1 (zeta2 r - zeta3 u), delta grad v . n = zeta1 (eta1 s - eta2 v) and by the
surface reactions p = b(r, s) - (zeta2 r - zeta3 u), q = c(r, s) - (eta1 s - eta2 v), with
b(x, y) = alpha2 - x + x^2 y, c(x, y) = beta1 - x^2 y.

The paper leaves the coupled discretisation out ("We omit the details").  Reading used:
* the bulk radial axis keeps eq. ball_discr, whose last row is the homogeneous Neumann row
  obtained from a virtual point rho_{n+1}; a normal derivative g enters that row through the
  same virtual point, u_{n+1} = u_{n-1} + 2 h g, which adds b_n 2 h g = (2/h + 2/rho_*) g to
  (A_rho3 u)_n (b_n the printed super-diagonal coefficient (n+1)/(n h^2), rho_* = n h);
* the surface grid is the ball's outermost shell: theta and phi as the ball's, so u at
  (rho_*, theta_j, phi_k) is the bulk node (n_rho, j, k);
* every coupling term is evaluated explicitly at t_n with the reactions, and each component is
  advanced by its own geometry's split step (eqs. ee_ball, ee_sphere): the linear operators act
  on each component separately, as the paper remarks.

Pins (tests/test_oracle_coupled.py): the flux term makes the discrete bulk operator exact on
u = rho^2 with its normal derivative (Laplacian 6 at every node); zeta1 = 0 reduces the step to
the two uncoupled split steps; the homogeneous equilibrium is a fixed point; a discrete divergence
theorem ties the bulk's gain through the outer row, (n^2 - 1)/h times the exchanged flux, to the
surface's loss (flux factor, sign, pairing); the coupling reads and writes the outer shell only.
"""
import numpy as np

from . import reactions as R
from .operators import Grid
from .stepper import Problem, advance, rhs


class Coupled:
    """The two grids, their problems and the coupling constants."""

    def __init__(self, n, tau, alpha1=55.0, alpha2=0.1, beta1=0.9, delta=10.0, eps=10.0, zeta1=55.0,
                 zeta2=5.0 / 12.0, zeta3=5.0 / 12.0, eta1=5.0, eta2=5.0, rho_star=1.0):
        n_rho, n_theta, n_phi = n
        self.ball = Grid("ball", (n_rho, n_theta, n_phi), rho_star=rho_star)
        self.sphere = Grid("sphere", (n_theta, n_phi))
        self.rho_star = rho_star
        self.h = rho_star / n_rho
        self.c = dict(alpha1=alpha1, alpha2=alpha2, beta1=beta1, delta=delta, eps=eps, zeta1=zeta1,
                      zeta2=zeta2, zeta3=zeta3, eta1=eta1, eta2=eta2)
        self.pb = Problem(self.ball, [1.0, delta], lambda W, t: R.schnakenberg(W, alpha1, alpha2, beta1), tau)
        self.ps = Problem(self.sphere, [1.0 / rho_star**2, eps / rho_star**2],
                          lambda W, t: R.schnakenberg(W, zeta1, alpha2, beta1), tau)
        self.tau = tau

    def radial_flux(self, g):
        """The bulk operator's extra term for a normal derivative g (shape (n_phi, n_theta)) on rho_*."""
        out = np.zeros(self.ball.shape)
        out[:, :, -1] = (2.0 / self.h + 2.0 / self.rho_star) * g
        return out

    def coupling(self, Wb, Ws):
        """Terms added to F of u, v (bulk, boundary nodes) and of r, s (surface)."""
        c = self.c
        ub, vb = Wb[0][:, :, -1], Wb[1][:, :, -1]
        r, s = Ws[0], Ws[1]
        ju = c["zeta1"] * (c["zeta2"] * r - c["zeta3"] * ub)           # grad u . n
        jv = c["zeta1"] * (c["eta1"] * s - c["eta2"] * vb)             # delta grad v . n
        # F_u = 1 * (M u + flux(ju)); F_v = delta * (M v + flux(jv / delta)) = delta M v + flux(jv)
        return [self.radial_flux(ju), self.radial_flux(jv)], [-ju, -jv]

    def step(self, Wb, Ws, t=0.0):
        Fb = rhs(self.pb, Wb, t)
        Fs = rhs(self.ps, Ws, t)
        ab, as_ = self.coupling(Wb, Ws)
        Fb = [Fb[q] + ab[q] for q in range(2)]
        Fs = [Fs[q] + as_[q] for q in range(2)]
        return advance(self.pb, Wb, Fb), advance(self.ps, Ws, Fs)

    def run(self, Wb, Ws, n_steps):
        for _ in range(n_steps):
            Wb, Ws = self.step(Wb, Ws)
        return Wb, Ws

    def equilibrium(self):
        a2, b1 = self.c["alpha2"], self.c["beta1"]
        return a2 + b1, b1 / (a2 + b1) ** 2
