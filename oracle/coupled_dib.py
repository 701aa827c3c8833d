"""Bulk-surface DIB model on the cylinder and its bottom disk (paper Section 5.6, eqs. bulkcyl,
bulkcylsys, bulkcylnl).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Bulk species u, v on the cylinder of radius rho_* and height z_* (Laplacian eq. lapcyl, diffusion
1 and delta, reactions b(u) = -alpha1 (u - alpha2), c(v) = -beta1 (v - beta2)); Dirichlet values
u = alpha2, v = beta2 on the top disk z = z_*; homogeneous Neumann on the lateral surface; on the
bottom disk z = 0 the flux conditions grad u . n = -zeta1 alpha3 p(u, r, s) and
grad v . n = -zeta1 beta3 q(v, r, s).  Surface species r, s on the bottom disk (Laplacian eq.
disk, diffusion 1 and eps, homogeneous Neumann on its rim) with reactions zeta1 p, zeta1 q:

    p(u, r, s) = zeta2 u (1 - s) r - zeta3 r^3 - zeta4 (s - zeta5)
    q(v, r, s) = eta1 v (1 + eta2 r) (1 - s) (1 - eta3 (1 - s)) - eta4 (1 + eta5 r) s (1 + eta3 s)

The paper leaves the coupled discretisation out.  Reading used:
* the z axis is eq. A_z (z_k = (k - 1) h, h = z_*/n, Neumann row at z = 0, Dirichlet value at
  z_* = n h); the bulk state is lifted, w = (u - alpha2, v - beta2), so the top value is the
  homogeneous Dirichlet end of A_z and the bulk reactions become -alpha1 w_u, -beta1 w_v;
* the surface grid is the cylinder's rho x theta grid at z = 0, so u on the bottom disk at
  (rho_i, theta_j) is the bulk node (i, j, 1);
* the flux enters the Neumann row k = 1 through the virtual value at z_0 = -h that gives its
  b_1 = 2/h^2: with g = grad u . n = -du/dz at z = 0, u_0 = u_2 + 2 h g, which adds 2 g / h to
  (A_z u)_1; a species of diffusion d gains d * 2 g / h in F;
* every coupling term is explicit at t_n with the reactions, and each component takes its own
  geometry's split step (eqs. ee_cylinder, ee_disk).

Pins (tests/test_oracle_coupled_dib.py): the flux term makes the discrete z operator exact (2 at
every node) on a quadratic with zero top value and a given normal derivative at z = 0; a discrete
divergence theorem ties the bulk's loss through z = 0 to the surface's gain (sign, 2/h, alpha3,
beta3, delta); zeta1 = 0 reduces the step to the uncoupled cylinder and disk steps; the
homogeneous equilibrium (alpha2, beta2, 0, zeta5), with eta4 from the printed formula, is a fixed
point; the coupling reads and writes the bottom plane only.
"""
import numpy as np

from .operators import Grid
from .stepper import Problem, advance, rhs

# Section 5.6 parameters as printed; eta4 follows from the others.
DIB = dict(alpha1=1.0, alpha2=1.0, alpha3=0.1, beta1=1.0, beta2=1.0, beta3=0.1, delta=1.0, eps=20.0,
           zeta1=1.0, zeta2=10.0, zeta3=1.0, zeta4=30.0, zeta5=0.5,
           eta1=3.0, eta2=2.5, eta3=0.2, eta5=1.5)


def eta4_for_equilibrium(c):
    """eta4 = beta2 eta1 (1 - zeta5) (1 - eta3 + eta3 zeta5) / (zeta5 (1 + eta3 zeta5)), as printed."""
    return (c["beta2"] * c["eta1"] * (1.0 - c["zeta5"]) * (1.0 - c["eta3"] + c["eta3"] * c["zeta5"])
            / (c["zeta5"] * (1.0 + c["eta3"] * c["zeta5"])))


class CoupledCylinder:
    """The cylinder (n_rho, n_theta, n_z), its bottom disk (n_rho, n_theta) and the constants."""

    def __init__(self, n, tau, rho_star=15.0, z_star=25.0, **params):
        c = dict(DIB)
        c.update(params)
        if "eta4" not in c:
            c["eta4"] = eta4_for_equilibrium(c)
        self.c = c
        n_rho, n_theta, n_z = n
        self.bulk = Grid("cylinder", (n_rho, n_theta, n_z), rho_star=rho_star, z_star=z_star, z_bc="paper")
        self.surface = Grid("disk", (n_rho, n_theta), rho_star=rho_star)
        self.h = z_star / n_z
        self.pb = Problem(self.bulk, [1.0, c["delta"]],
                          lambda W, t: [-c["alpha1"] * W[0], -c["beta1"] * W[1]], tau)
        self.ps = Problem(self.surface, [1.0, c["eps"]], lambda W, t: [0.0 * W[0], 0.0 * W[1]], tau)
        self.tau = tau

    def p(self, u, r, s):
        c = self.c
        return c["zeta2"] * u * (1.0 - s) * r - c["zeta3"] * r ** 3 - c["zeta4"] * (s - c["zeta5"])

    def q(self, v, r, s):
        c = self.c
        return (c["eta1"] * v * (1.0 + c["eta2"] * r) * (1.0 - s) * (1.0 - c["eta3"] * (1.0 - s))
                - c["eta4"] * (1.0 + c["eta5"] * r) * s * (1.0 + c["eta3"] * s))

    def bottom_flux(self, g):
        """The bulk z operator's extra term for a normal derivative g (shape (n_theta, n_rho)) on z = 0."""
        out = np.zeros(self.bulk.shape)
        out[0] = 2.0 * g / self.h
        return out

    def coupling(self, Wb, Ws):
        """Terms added to F of w_u, w_v (bulk, bottom plane) and of r, s (surface)."""
        c = self.c
        u = Wb[0][0] + c["alpha2"]                  # bulk values on the bottom disk (lifting undone)
        v = Wb[1][0] + c["beta2"]
        r, s = Ws[0], Ws[1]
        P, Q = self.p(u, r, s), self.q(v, r, s)
        gu = -c["zeta1"] * c["alpha3"] * P           # grad u . n on z = 0
        gv = -c["zeta1"] * c["beta3"] * Q
        bulk = [1.0 * self.bottom_flux(gu), c["delta"] * self.bottom_flux(gv)]
        return bulk, [c["zeta1"] * P, c["zeta1"] * Q]

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
        """(u_e, v_e, r_e, s_e) = (alpha2, beta2, 0, zeta5)."""
        c = self.c
        return c["alpha2"], c["beta2"], 0.0, c["zeta5"]
