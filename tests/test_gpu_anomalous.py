"""Anomalous diffusion on the disk (Section 5.3, the second extension): Delta_lambda with
homogeneous Dirichlet at rho_* (eq. A_lambda), D_rho = rho^(-2-lambda), and the lifted
Schnakenberg system of eq. (schnak) (state w = u - (u_e, v_e)); both GPU paths against the
oracle.  The split path evaluates the lifted reaction in its exact expansion about (u_e, v_e),
so the 1e-5 perturbations keep FP32 relative accuracy."""
import numpy as np
import pytest

from paper_2604_11558_gb300 import workloads as wl
from tests.gpu_helpers import assert_parity, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split_tf32", 1e-6)])
def test_anomalous_schnakenberg_matches_oracle(precision, tol):
    w = wl.anomalous_disk(n=(40, 36), steps=23, seed=41)
    assert_parity(gpu_run(w, precision), oracle_run(w), w["W0"], tol)


def test_anomalous_paper_size_a_few_steps():
    """The paper's 160 x 160 grid on the FP64 path; the split path takes n_rho <= 128 (one
    tensor-memory accumulator set per slab), checked at 128 x 160."""
    w = wl.anomalous_disk(steps=4, seed=42)
    assert_parity(gpu_run(w, "fp64"), oracle_run(w), w["W0"], 1e-12)
    # split path on this random field (rough data): the relative 2-norm error within 1e-6.  Elementwise,
    # every step's increment is about the size of the state (the strongly damped rough modes), and
    # each split-TF32 product carries up to ~2^-21 relative error (hi + lo keep 22 bits, lo*lo is
    # dropped): the bound is 8 x 2^-21 x (max increment / max state) per step, over the steps.
    from tests.gpu_helpers import rel_errors
    w = wl.anomalous_disk(n=(128, 160), steps=4, seed=42)
    ref = oracle_run(w)
    got = gpu_run(w, "split_tf32")
    assert max(rel_errors(got, ref)) <= 1e-6, rel_errors(got, ref)
    ref1 = oracle_run(w, steps=1)
    for s in range(2):
        m = np.max(np.abs(ref[s]))
        inc = np.max(np.abs(ref1[s] - w["W0"][s])) / np.max(np.abs(ref1[s]))
        em = np.max(np.abs(got[s] - ref[s])) / m
        bound = max(1e-6, 8 * 2.0 ** -21 * inc * w["steps"])
        print("anomalous 128x160 species", s, "max-abs", em, "per-step increment / state", inc, "bound", bound)
        assert em <= bound, (s, em, bound)


@pytest.mark.parametrize("lam", [0.0, 0.5, -1.0])
def test_other_exponents_and_generic_offsets(lam):
    """Subdiffusion, the Dirichlet Laplacian (lambda = 0) and a Gray-Scott reaction with generic
    lifting offsets (FP64 path)."""
    w = wl.anomalous_disk(n=(23, 31), steps=9, seed=43, lam=lam, tau=1e-4)
    w = dict(w, reaction="gray_scott", params=[0.04, 0.06], d=[2e-3, 1e-3], offsets=[0.3, 0.2],
             W0=0.1 * np.abs(np.random.default_rng(3).standard_normal(w["W0"].shape)))
    assert_parity(gpu_run(w, "fp64"), oracle_run(w), w["W0"], 1e-12)


def test_invalid_anomalous_setups():
    from paper_2604_11558_gb300 import binding
    assert binding.setup_status("ball", (8, 8, 8), [1.0, 2.0], "gray_scott", [0.04, 0.06], 1e-3, "fp64",
                                lam=-1.0) == 1
    assert binding.setup_status("disk", (8, 8), [1.0, 2.0], "gray_scott", [0.04, 0.06], 1e-3, "fp64",
                                lam=1.0) == 1
