"""Pins of the unsplit exponential Euler oracle (the splitting's accuracy baseline).

U1: exact for w' = A w + c on arbitrary data: n steps of size tau equal the closed form
    e^{T A} w_0 + T phi_1(T A) c, with A = d M assembled from the Kronecker terms and e^{T A}
    taken separately from expm (exponential Euler is exact for linear constant forcing).
U2: on data varying along rho only (annihilated by every other Kronecker term), the split step and
    the unsplit step agree to rounding: the splitting has nothing to split there.
U3: the split stepper converges to the unsplit one at second order in tau (fixed final time): both
    are first-order methods, but phi_1(tau (A + B)) - phi_1(tau A) phi_1(tau B) = O(tau^2) (their
    Taylor series agree through tau (A + B)/2), so the per-step difference is O(tau^3).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import reactions as R
from oracle.operators import Grid
from oracle.stepper import Problem, run
from oracle.unsplit import run_unsplit


@pytest.mark.parametrize("kind,n", [("disk", (6, 8)), ("sphere", (7, 6)), ("ball", (4, 5, 6)), ("cylinder", (4, 6, 5))])
def test_U1_exact_for_linear_constant_forcing(kind, n):
    g = Grid(kind, n)
    rng = np.random.default_rng(5)
    w0 = rng.standard_normal(g.shape)
    c = rng.standard_normal(g.shape)
    d, tau, steps = 0.05, 0.01, 6
    p = Problem(g, [d], lambda W, t: [c], tau)
    got = run_unsplit(p, w0[None], steps)[0]
    T = steps * tau
    A = d * g.M_total.toarray()
    Ta = T * A
    # phi_1(T A) = (T A)^-1 (e^{T A} - I) is singular here (M has a null space), so its action
    # on c comes from the block exponential of [[T A, T c], [0, 0]] (last column, top rows)
    aug = np.zeros((g.npts + 1, g.npts + 1))
    aug[:-1, :-1] = Ta
    aug[:-1, -1] = T * c.ravel()
    ref = sla.expm(Ta) @ w0.ravel() + sla.expm(aug)[:-1, -1]
    assert np.max(np.abs(got.ravel() - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind,n", [("disk", (6, 8)), ("ball", (4, 5, 6)), ("cylinder", (4, 6, 5))])
def test_U2_split_equals_unsplit_on_radial_data(kind, n):
    g = Grid(kind, n)
    rng = np.random.default_rng(6)
    # a profile along rho only (mode 1): every other Kronecker term annihilates it (the theta, phi
    # and Neumann z matrices have zero row sums), so only M_1 acts and nothing is split
    shape1 = [1] * g.ndim
    shape1[g.ndim - 1] = g.n[0]
    W0 = np.stack([np.broadcast_to(1.0 + 0.1 * rng.standard_normal(shape1), g.shape) for _ in range(2)])
    p = Problem(g, [1e-2, 3e-2], lambda W, t: R.gray_scott(W, 0.04, 0.06), 0.05)
    a = run(p, W0, 4)
    b = run_unsplit(p, W0, 4)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(a - W0)) > 1e-4        # the data did evolve


def test_U3_split_converges_to_unsplit_second_order():
    g = Grid("disk", (8, 12))
    rng = np.random.default_rng(7)
    a_, b_ = 0.1, 0.9
    W0 = np.stack([(a_ + b_) + 0.01 * rng.uniform(-1, 1, g.shape), b_ / (a_ + b_) ** 2 + 0.01 * rng.uniform(-1, 1, g.shape)])
    T = 0.02
    errs = []
    for steps in (20, 40, 80):
        p = Problem(g, [1.0, 10.0], lambda W, t: R.schnakenberg(W, 100.0, a_, b_), T / steps)
        errs.append(np.linalg.norm(run(p, W0, steps) - run_unsplit(p, W0, steps)) / np.linalg.norm(W0))
    rates = [np.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert errs[0] > 1e-8                      # a splitting error is there to measure
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)
