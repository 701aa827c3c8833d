"""GPU test of sexpe_step_noalloc, the step for callers that cannot allocate.

Callers that run where cudaMalloc is not allowed (inside a globally captured
CUDA graph region, inside a framework that owns every device allocation, under
a fixed memory budget) use sexpe_step_noalloc: the same split-TF32 step with
its FP32 scratch in the library's static device array.  This file checks, through
the C ABI, that two calls in a row give the same states as the ordinary
sexpe_step within the split path's tolerance (1e-6 relative per species), and
that oversized or FP64 plans are refused.  It is named so that pytest collects
it last, and it passes alone in a fresh process as well as after the others.
"""
import numpy as np
import pytest

from paper_2604_11558_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _rel(a, b):
    return [float(np.linalg.norm(a[s] - b[s]) / np.linalg.norm(b[s])) for s in range(b.shape[0])]


@pytest.mark.parametrize("w", [wl.gray_scott_ball(n=(20, 33, 40), steps=3, seed=13),
                               wl.schnakenberg_disk(n=(37, 45), steps=3, seed=11),
                               wl.gray_scott_ball(steps=2)],
                         ids=["ball_20x33x40", "disk_37x45", "ball_100"])
def test_noalloc_matches_step_on_two_calls(w):
    import torch
    from paper_2604_11558_gb300 import binding
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    ref = torch.from_numpy(w["W0"].copy()).cuda()
    got = torch.from_numpy(w["W0"].copy()).cuda()
    for call in range(2):
        plan.step(ref, w["steps"])
        plan.step_noalloc(got, w["steps"])
        plan.synchronize()
        e = _rel(got.cpu().numpy(), ref.cpu().numpy())
        assert max(e) <= TOL, (call, e)
    plan.close()


def test_noalloc_refuses_what_it_cannot_hold():
    import torch
    from paper_2604_11558_gb300 import binding
    big = wl.linear_cubic_cylinder(steps=1)            # 3 x 64*128*128 > 2^21 scratch floats
    plan = binding.Plan.from_workload(big, precision="split_tf32")
    x = torch.from_numpy(big["W0"].copy()).cuda()
    with pytest.raises(binding.SexpeError) as ei:
        plan.step_noalloc(x, 1)
    assert ei.value.status == 1
    plan.close()
    small = wl.schnakenberg_disk(n=(13, 20), steps=1)
    plan64 = binding.Plan.from_workload(small, precision="fp64")
    y = torch.from_numpy(small["W0"].copy()).cuda()
    with pytest.raises(binding.SexpeError) as ei:
        plan64.step_noalloc(y, 1)
    assert ei.value.status == 1
    plan64.close()
