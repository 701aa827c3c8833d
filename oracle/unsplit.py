"""Unsplit exponential Euler (paper Section 4, eq. ee with phi_1 of the whole operator).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The accuracy baseline that the splitting of eq. splitorder approximates: for
species s with diffusion d_s, one step is

    F_s = d_s M w_s + g_s(w_n),     w_s <- w_s + tau phi_1(tau d_s M) F_s,

with M = M_1 + ... + M_d the assembled Kronecker sum of the geometry
(``Grid.M_total``).  phi_1(X) is the upper-right block of
expm([[X, I], [0, 0]]) (scipy's expm is the library primitive of this step).
Dense, hence tiny and medium grids only.

Pins (tests/test_oracle_unsplit.py): exact for the linear problem with
constant forcing on any data (closed form e^{T A} w_0 + T phi_1(T A) c); equal
to the split step on data that only M_1 acts on; the split stepper converges
to it at second order in tau (phi_1 of a sum and the product of the phi_1
differ at O(tau^2)).
"""
import numpy as np
import scipy.linalg as sla

from .stepper import rhs


def phi1_dense(X):
    """phi_1(X) of a dense matrix: upper-right block of expm([[X, I], [0, 0]])."""
    n = X.shape[0]
    aug = np.zeros((2 * n, 2 * n))
    aug[:n, :n] = X
    aug[:n, n:] = np.eye(n)
    return sla.expm(aug)[:n, n:]


def phi1_operators(problem):
    """phi_1(tau d_s M) for every species (dense N x N)."""
    M = problem.grid.M_total.toarray()
    return [phi1_dense(problem.tau * problem.d[s] * M) for s in range(problem.S)]


def run_unsplit(problem, W0, n_steps, t0=0.0, P=None):
    """n_steps unsplit exponential Euler steps from W0 (time-dependent reactions see t_n)."""
    if P is None:
        P = phi1_operators(problem)
    W = np.array(W0, copy=True)
    for n in range(n_steps):
        F = rhs(problem, W, t0 + n * problem.tau)
        W = np.stack([W[s] + problem.tau * (P[s] @ F[s].ravel()).reshape(W[s].shape) for s in range(problem.S)])
    return W
