"""Pins of the oracle's complex-step gradients (the reference for the library's adjoint).

* against central finite differences of the real oracle (h ~ 1e-6 relative,
  O(h^2) truncation);
* for a linear problem (no reaction) against the closed form: the step map is
  W -> (I + tau P d M) W per species, so d<c, W_N>/dW_0 = ((I + tau P d M)^T)^N c,
  with P and M assembled dense (phi_1 factors from expm of the Kronecker terms).
"""
import numpy as np
import scipy.linalg as sla

from oracle import adjoint as A
from oracle.operators import Grid
from oracle.stepper import run


def _loss(c):
    return lambda W: np.sum(c * W)


def test_complex_step_matches_central_differences():
    g = Grid("disk", (6, 8))
    rng = np.random.default_rng(0)
    a, b = 0.1, 0.9
    W0 = np.array([np.full(g.shape, a + b), np.full(g.shape, b / (a + b) ** 2)]) + rng.uniform(-0.01, 0.01, (2,) + g.shape)
    c = rng.standard_normal(W0.shape)
    params = [100.0, a, b, 1.0, 10.0]
    build = A.problem_builder(g, "schnakenberg", 1e-4, 3)
    L = _loss(c)
    for q in range(len(params)):
        cs = A.complex_step_param(build, params, q, W0, 5, L)
        h = 1e-6 * abs(params[q])
        pp, pm = list(params), list(params)
        pp[q] += h
        pm[q] -= h
        fd = (L(run(build(np.array(pp)), W0, 5)) - L(run(build(np.array(pm)), W0, 5))) / (2 * h)
        assert abs(cs - fd) <= 1e-6 * max(abs(fd), 1e-12), (q, cs, fd)
    delta = rng.standard_normal(W0.shape)
    cs = A.complex_step_state(build, params, W0, delta, 5, L)
    h = 1e-6
    fd = (L(run(build(np.array(params)), W0 + h * delta, 5)) - L(run(build(np.array(params)), W0 - h * delta, 5))) / (2 * h)
    assert abs(cs - fd) <= 1e-6 * abs(fd)


def test_linear_problem_closed_form_gradient():
    g = Grid("ball", (4, 5, 3))
    rng = np.random.default_rng(1)
    d, tau, N = 0.7, 0.01, 4
    W0 = rng.standard_normal((1,) + g.shape)
    c = rng.standard_normal(W0.shape)
    build = A.problem_builder(g, "none", tau, 0)
    Md = {mu: g.M[mu].toarray() for mu in g.M}
    Mfull = sum(Md.values())
    n = g.npts
    P = np.eye(n)
    for mu in range(1, g.ndim + 1):
        aug = np.zeros((2 * n, 2 * n))
        aug[:n, :n] = tau * d * Md[mu]
        aug[:n, n:] = np.eye(n)
        P = P @ sla.expm(aug)[:n, n:]
    Sm = np.eye(n) + tau * P @ (d * Mfull)
    grad = c[0].ravel()
    for _ in range(N):
        grad = Sm.T @ grad
    delta = rng.standard_normal(W0.shape)
    cs = A.complex_step_state(build, [d], W0, delta, N, _loss(c))
    assert abs(cs - grad @ delta[0].ravel()) <= 1e-12 * abs(cs)
