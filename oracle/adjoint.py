"""Gradients of a scalar loss of the final state by complex-step differentiation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The oracle's stepper is dtype-generic, so running it with a parameter (or the
initial state) perturbed by i*h, h tiny, gives
    d L / d p = Im(L(p + i h)) / h
to rounding accuracy, with no transposed code path of its own: this is the
reference for the library's discrete adjoint.  Pins (tests/test_oracle_adjoint.py):
agreement with central finite differences of the real oracle, and the closed
form of the gradient for a linear problem (no reaction), where the step map is
W -> (I + tau P d M) W and d L/d W_0 = (I + tau P d M)^T ... c.
"""
import numpy as np

from .stepper import Problem, run

H = 1e-30


def complex_step_param(build, params, q, W0, steps, loss, h=H):
    """d loss(W_N) / d params[q]; build(params) -> Problem (params may be complex)."""
    p = np.array(params, dtype=complex)
    p[q] += 1j * h
    WN = run(build(p), np.asarray(W0, dtype=complex), steps)
    return float(np.imag(loss(WN)) / h)


def complex_step_state(build, params, W0, delta, steps, loss, h=H):
    """Directional derivative <d loss / d W_0, delta>."""
    WN = run(build(np.asarray(params, dtype=complex)), np.asarray(W0, dtype=complex) + 1j * h * delta, steps)
    return float(np.imag(loss(WN)) / h)


def problem_builder(grid, reaction, tau, n_reaction_params):
    """build(params) for a parameter vector (reaction parameters..., d_1, ..., d_S)."""
    from . import reactions as R

    def build(params):
        rp = params[:n_reaction_params]
        d = list(params[n_reaction_params:])
        if reaction == "schnakenberg":
            reac = lambda W, t: R.schnakenberg(W, rp[0], rp[1], rp[2])
        elif reaction == "gray_scott":
            reac = lambda W, t: R.gray_scott(W, rp[0], rp[1])
        elif reaction == "linear_cubic":
            S = len(d)
            K = np.asarray(rp).reshape(S, S)
            reac = lambda W, t: R.linear_cubic(W, K)
        else:
            reac = lambda W, t: [np.zeros_like(W[0]) for _ in range(len(d))]
        return Problem(grid, d, reac, tau)

    return build
