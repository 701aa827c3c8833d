"""Split exponential Euler step (paper Section 4, eqs. ee, splitorder and ee_disk/ee_sphere/ee_ball/ee_cylinder).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For species s with diffusion d_s the semidiscrete system is
w_s' = d_s M w_s + g_s(w), M = M_1 + ... + M_d.  One step is

    F_s = d_s M w_s + g_s(w_n)                                   (eq. ee)
    w_s <- w_s + tau phi_1(tau d_s M_1) ... phi_1(tau d_s M_d) F_s  (eq. splitorder)

so phi_1(tau d_s M_d) acts first.  Each factor acts fibre by fibre: along
mode mu every fibre is multiplied by phi_1(tau d_s s A_mu), s being the
fibre's diagonal factor (rho_i^-2, sin^-2 phi_k or their product), which
equals phi_1 of the Kronecker term (mixed-product property, Section 4).
phi_1(t s A_mu) is applied through A_mu = V diag(lam) V^{-1}
(``oracle.phi.eigen``): y = V diag(phi_1(t s lam)) V^{-1} x.

Pins (tests/test_oracle_stepper.py): one step equals w + tau prod phi_1 F
with each phi_1 of the assembled Kronecker term taken from dense expm on
tiny grids; the splitting error is O(tau^2); exactness for linear problems
with constant forcing on data that the other directions annihilate; mass
conservation under Neumann boundaries; first-order convergence and the
printed errors of the manufactured-solution experiment (Fig. 1).
"""
import numpy as np

from .phi import eigen, phi1


class Problem:
    """Grid + per-species diffusion + reaction callback + step size.

    ``reaction(W, t)`` returns a list of per-species arrays; ``d`` is a
    sequence of diffusion coefficients (may be complex for complex-step).
    """

    def __init__(self, grid, d, reaction, tau):
        self.grid = grid
        self.d = list(d)
        self.reaction = reaction
        self.tau = tau
        self._eig = {mu: eigen(grid.A[mu]) for mu in grid.A}

    @property
    def S(self):
        return len(self.d)


def apply_phi1_mode(X, grid, eig, mu, t):
    """phi_1(t M_mu) X, fibre by fibre along mode mu (numpy axis ndim - mu)."""
    lam, V, Vinv = eig
    axis = X.ndim - mu
    s = np.broadcast_to(grid.scale[mu], X.shape)
    Xm = np.moveaxis(X, axis, -1)
    sm = np.moveaxis(s, axis, -1)
    assert np.all(sm == sm[..., :1]), "scale factor must be constant along the fibre"
    Z = Xm @ Vinv.T                                 # to the eigenbasis of A_mu
    Z = Z * phi1(t * sm[..., :1] * lam)             # diag(phi_1(t s lam)) per fibre
    Y = Z @ V.T                                     # back
    return np.moveaxis(Y, -1, axis)


def rhs(problem, W, t=0.0):
    """F_s = d_s M w_s + g_s(W) for every species (first line of eqs. ee_*)."""
    G = problem.reaction(W, t)
    return [problem.d[s] * problem.grid.apply_M(W[s]) + G[s] for s in range(problem.S)]


def _to_fp32(x):
    return x.astype(np.float32).astype(np.float64)


def step(problem, W, t=0.0, fp32_storage=False):
    """One split exponential Euler step; W has shape (S, *grid.shape). Returns a new array.

    fp32_storage=True is a precision-emulation switch for error modelling
    only: F, the result of every direction and the increment are rounded to
    FP32 (the state stays FP64), i.e. the storage precision of a mixed
    FP32/FP64 implementation, with the arithmetic itself still exact.
    """
    grid = problem.grid
    F = rhs(problem, W, t)
    out = np.array(W, copy=True)
    for s in range(problem.S):
        X = _to_fp32(F[s]) if fp32_storage else F[s]
        for mu in range(grid.ndim, 0, -1):          # phi_1(tau d M_d) first, phi_1(tau d M_1) last
            X = apply_phi1_mode(X, grid, problem._eig[mu], mu, problem.tau * problem.d[s])
            if fp32_storage:
                X = _to_fp32(X)
        out[s] = W[s] + (_to_fp32(problem.tau * X) if fp32_storage else problem.tau * X)
    return out


def run(problem, W0, n_steps, t0=0.0, fp32_storage=False):
    """n_steps split exponential Euler steps from W0 (time-dependent reactions see t_n)."""
    W = np.array(W0, copy=True)
    for n in range(n_steps):
        W = step(problem, W, t0 + n * problem.tau, fp32_storage)
    return W


def advance(problem, W, F):
    """w_s + tau phi_1(tau d_s M_1) ... phi_1(tau d_s M_d) F_s for every species, for a given F
    (the split update of eq. splitorder; used where F carries terms from outside the grid, as in
    the bulk-surface coupling of Section 5.5)."""
    grid = problem.grid
    out = np.array(W, copy=True)
    for s in range(problem.S):
        X = F[s]
        for mu in range(grid.ndim, 0, -1):
            X = apply_phi1_mode(X, grid, problem._eig[mu], mu, problem.tau * problem.d[s])
        out[s] = W[s] + problem.tau * X
    return out
