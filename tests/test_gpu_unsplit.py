"""GPU parity of the unsplit exponential Euler baseline (precision SEXPE_UNSPLIT_FP64) against the
oracle's unsplit stepper, and the splitting error it measures on the paper's disk workload.

The unsplit step is eq. ee with phi_1 of the whole operator: w_s += tau phi_1(tau d_s M) F_s, the
phi_1 formed densely at setup.  FP64 on both sides: 1e-12 relative.
"""
import numpy as np
import pytest

from oracle.operators import Grid
from oracle.stepper import Problem
from oracle.unsplit import run_unsplit
from paper_2604_11558_gb300 import workloads as wl
from tests.gpu_helpers import gpu_run, oracle_reaction, rel_errors
from tests.test_gpu_bvam import bvam_case

pytestmark = pytest.mark.gpu


def oracle_unsplit(w, steps=None):
    g = Grid(w["geometry"], w["n"], z_bc=w.get("z_bc", "neumann"), lam=w.get("lam"))
    p = Problem(g, w["d"], oracle_reaction(w, g), w["tau"])
    return run_unsplit(p, w["W0"], w["steps"] if steps is None else steps)


CASES = [
    ("disk", wl.schnakenberg_disk(n=(8, 12), steps=10, seed=51)),
    ("sphere", wl.schnakenberg_sphere(n=(8, 10), steps=10, seed=52)),
    ("ball", wl.gray_scott_ball(n=(5, 6, 7), steps=6, seed=53)),
    ("cylinder", wl.linear_cubic_cylinder(n=(5, 6, 6), steps=6, seed=54)),
    ("anomalous_disk", wl.anomalous_disk(n=(9, 10), steps=8, seed=55, tau=1e-4)),
    ("bvam_manufactured", bvam_case(9, 12, 8, steps=6)[0]),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_unsplit_matches_oracle(name, w):
    got = gpu_run(w, "unsplit_fp64")
    ref = oracle_unsplit(w)
    assert np.all(np.isfinite(got))
    e = rel_errors(got, ref)
    assert max(e) <= 1e-12, e
    for s in range(ref.shape[0]):
        assert np.max(np.abs(got[s] - ref[s])) <= 1e-12 * np.max(np.abs(ref[s])), (s, e)


def test_unsplit_limits():
    from paper_2604_11558_gb300 import binding
    assert binding.setup_status("disk", (48, 48), [1.0, 10.0], "schnakenberg", [100.0, 0.1, 0.9], 1e-4,
                                "unsplit_fp64") == 5      # SEXPE_EUNSUPPORTED: more than 2048 points
    w = wl.schnakenberg_disk(n=(8, 12), steps=2, seed=51)
    plan = binding.Plan.from_workload(w, precision="unsplit_fp64")
    with pytest.raises(RuntimeError):
        plan.set_stencil(4, 0)
    plan.close()


def test_splitting_error_on_the_paper_disk():
    """Disk 32 x 64, Schnakenberg (gamma 100, a 0.1, b 0.9, d = (1, 10)), tau = 1e-4, 200 steps: the
    split FP64 GPU path against the unsplit GPU baseline, and again at tau / 2 (400 steps): the
    splitting error (difference of two first-order methods) falls at second order."""
    errs = []
    for tau, steps in ((1e-4, 200), (5e-5, 400)):
        w = wl.schnakenberg_disk(steps=steps, tau=tau)
        split = gpu_run(w, "fp64")
        unsplit = gpu_run(w, "unsplit_fp64")
        errs.append(max(rel_errors(split, unsplit)))
    ratio = errs[0] / errs[1]
    print("disk 32x64 splitting error (relative, max over species): tau 1e-4:", errs[0], "tau 5e-5:", errs[1],
          "ratio", ratio)
    assert errs[0] > 1e-10
    assert 3.0 < ratio < 5.0, (errs, ratio)
