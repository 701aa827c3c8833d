"""The split precision is chosen by measured error (error model of the product arithmetic, against
the exact oracle): two BF16 pieces with three products miss the 1e-6 target on a Gray-Scott ball,
three TF32-split products meet it, three BF16 pieces with six products meet it too (and are not
built for cost reasons: twice the MMA issues from producer-bound kernels)."""
import numpy as np
import pytest

from oracle.operators import Grid
from oracle.stepper import Problem, run as oracle_run
from paper_2604_11558_gb300 import workloads as wl
from tests.gpu_helpers import oracle_reaction
from tests.precision_emulation import run as emulated_run


def rel(W, ref):
    return max(np.linalg.norm(W[s] - ref[s]) / np.linalg.norm(ref[s]) for s in range(ref.shape[0]))


@pytest.fixture(scope="module")
def ball():
    w = wl.gray_scott_ball(n=(40, 40, 40), steps=20)
    g = Grid(w["geometry"], w["n"])
    p = Problem(g, w["d"], oracle_reaction(w, g), w["tau"])
    return p, w, oracle_run(p, w["W0"], w["steps"])


def test_tf32x3_meets_the_target(ball):
    p, w, ref = ball
    assert rel(emulated_run(p, w["W0"], w["steps"], "tf32x3"), ref) < 1e-6


def test_bf16_two_pieces_miss_the_target(ball):
    p, w, ref = ball
    assert rel(emulated_run(p, w["W0"], w["steps"], "bf16x3"), ref) > 1e-6


def test_bf16_three_pieces_meet_it(ball):
    p, w, ref = ball
    e6 = rel(emulated_run(p, w["W0"], w["steps"], "bf16x6"), ref)
    e3 = rel(emulated_run(p, w["W0"], w["steps"], "tf32x3"), ref)
    assert e6 < 1e-6 and e6 < 2 * e3
