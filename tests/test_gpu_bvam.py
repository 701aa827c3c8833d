"""The BVAM model with the manufactured sources of Section 5.1 on the GPU (the
first extension beyond the benchmark workloads): parity of both arithmetic paths
with the oracle, and the paper's printed Fig. 1 errors (SplitEE series,
tests/golden/fig1_splitee_errors.txt) reproduced by the GPU FP64 path within
0.5% and by the split-TF32 path within 1%, with the error norm of the oracle's
pin: sqrt(e_u^2 + e_v^2), e the relative discrete L2 norm with the polar weight
rho.  The sources depend on t_n = t0 + n tau; sexpe_set_time restarts the clock."""
import os

import numpy as np
import pytest

from oracle import reactions as R
from oracle.operators import Grid
from tests.gpu_helpers import assert_parity, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_splitee_errors.txt")
PARAMS = [R.BVAM[k] for k in ("alpha1", "alpha2", "alpha3", "beta1", "beta2")]


def bvam_case(nr, nt, m, steps=None):
    g = Grid("disk", (nr, nt))
    rho = g.points[1][None, :]
    th = g.points[2][:, None]
    W0 = np.array(R.bvam_exact(0.0, rho, th))
    return dict(geometry="disk", n=(nr, nt), d=[R.BVAM["gamma"], R.BVAM["delta"]], reaction="bvam_manufactured",
                params=PARAMS, tau=1.0 / m, steps=m if steps is None else steps, W0=W0), g


def fig1_error(W, g):
    rho = g.points[1][None, :]
    th = g.points[2][:, None]
    E = np.array(R.bvam_exact(1.0, rho, th))
    wgt = rho + 0 * th
    e = [np.sqrt(np.sum(wgt * (W[s] - E[s]) ** 2) / np.sum(wgt * E[s] ** 2)) for s in range(2)]
    return float(np.hypot(e[0], e[1]))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split_tf32", 1e-6)])
def test_bvam_manufactured_matches_oracle(precision, tol):
    w, _ = bvam_case(25, 50, 200, steps=23)              # graph replays and single steps
    assert_parity(gpu_run(w, precision), oracle_run(w), w["W0"], tol)


def test_bvam_plain_reaction_matches_oracle():
    w, _ = bvam_case(17, 36, 100, steps=12)
    w = dict(w, reaction="bvam")
    assert_parity(gpu_run(w, "fp64"), oracle_run(w), w["W0"], 1e-12)


def test_fig1_printed_errors_on_the_gpu():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    for nr, nt, m, err in rows:
        w, g = bvam_case(int(nr), int(nt), int(m))
        for precision, rel in (("fp64", 5e-3), ("split_tf32", 1e-2)):
            val = fig1_error(gpu_run(w, precision), g)
            assert abs(val / float(err) - 1) < rel, (nr, nt, m, precision, val, err)


def test_set_time_restarts_the_source_clock():
    import torch
    from paper_2604_11558_gb300 import binding
    w, _ = bvam_case(25, 50, 200)
    plan = binding.Plan.from_workload(w, precision="fp64")
    x = torch.from_numpy(w["W0"].copy()).cuda()
    plan.step(x, 7)
    plan.synchronize()
    first = x.cpu().numpy()
    x.copy_(torch.from_numpy(w["W0"]))
    plan.set_time(0.0)
    plan.step(x, 7)
    plan.synchronize()
    assert np.array_equal(x.cpu().numpy(), first)
    # starting at t = 0.5 equals the oracle started there
    x.copy_(torch.from_numpy(w["W0"]))
    plan.set_time(0.5)
    plan.step(x, 5)
    plan.synchronize()
    from oracle.stepper import Problem, run
    from tests.gpu_helpers import oracle_reaction
    g = Grid("disk", w["n"])
    ref = run(Problem(g, w["d"], oracle_reaction(w, g), w["tau"]), w["W0"], 5, t0=0.5)
    assert_parity(x.cpu().numpy(), ref, w["W0"], 1e-12)
    plan.close()
