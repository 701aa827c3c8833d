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


def test_truncating_accumulation_model():
    """The 'rz8' accumulation model: with inputs whose pieces and partial sums are exact in FP32 it
    equals the exact product; with positive operands it never exceeds the exact product (rounding
    toward zero) and stays within one FP32 ulp of it per accumulation step."""
    import numpy as np
    from tests.precision_emulation import matmul
    rng = np.random.default_rng(3)
    A = rng.integers(-64, 64, (5, 24)).astype(np.float64)
    B = rng.integers(-64, 64, (24, 7)).astype(np.float64)
    assert np.array_equal(matmul(A, B, accumulate="rz8"), A @ B)
    A = rng.uniform(0.5, 1.0, (6, 40))
    B = rng.uniform(0.5, 1.0, (40, 9))
    exact = A.astype(np.float32).astype(np.float64) @ B.astype(np.float32).astype(np.float64)
    got = matmul(A, B, accumulate="rz8")
    assert np.all(got <= exact * (1 + 1e-7))
    steps = 3 * (40 // 8)
    assert np.all(exact - got <= steps * np.spacing(exact.astype(np.float32)).astype(np.float64) + 1e-6 * exact)
