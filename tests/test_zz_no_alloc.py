"""GPU test of sexpe_step_noalloc, the step for callers that cannot allocate.

Callers that run where cudaMalloc is not allowed (inside a globally captured
CUDA graph region, inside a framework that owns every device allocation, under
a fixed memory budget) use sexpe_step_noalloc: the same split-TF32 kernels as
sexpe_step with the FP32 scratch in the library's static device array.  This
file checks, through the C ABI, that two calls in a row give exactly the states
of the ordinary sexpe_step on every geometry (and with time-dependent sources),
also after an earlier call left non-finite values in the shared array, and that
oversized, FP64 and misaligned requests are refused before anything runs.  It
is named so that pytest collects it last, and it passes alone in a fresh
process as well as after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_2604_11558_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _bvam_disk(nr=25, nt=50, steps=4):
    from oracle import reactions as R
    from oracle.operators import Grid
    g = Grid("disk", (nr, nt))
    W0 = np.array(R.bvam_exact(0.0, g.points[1][None, :], g.points[2][:, None]))
    params = [R.BVAM[k] for k in ("alpha1", "alpha2", "alpha3", "beta1", "beta2")]
    return dict(geometry="disk", n=(nr, nt), d=[R.BVAM["gamma"], R.BVAM["delta"]], reaction="bvam_manufactured",
                params=params, tau=1.0 / 200, steps=steps, W0=W0)


CASES = [
    ("ball_20x33x40", wl.gray_scott_ball(n=(20, 33, 40), steps=3, seed=13)),
    ("disk_37x45_padded", wl.schnakenberg_disk(n=(37, 45), steps=3, seed=11)),
    ("ball_100", wl.gray_scott_ball(steps=2)),
    ("sphere_24x13", wl.schnakenberg_sphere(n=(24, 13), steps=3, seed=12)),
    ("sphere_30x17_padded", wl.schnakenberg_sphere(n=(30, 17), steps=3, seed=12)),
    ("cylinder_9x14x11_padded", wl.linear_cubic_cylinder(n=(9, 14, 11), steps=3, seed=14)),
    ("bvam_manufactured_disk", _bvam_disk()),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_noalloc_equals_step_on_two_calls(name, w):
    """Two plans from the same workload (their step clocks both start at 0), one stepped by
    sexpe_step and one by sexpe_step_noalloc: bit-identical states after each of two calls."""
    import torch
    from paper_2604_11558_gb300 import binding
    pa = binding.Plan.from_workload(w, precision="split_tf32")
    pb = binding.Plan.from_workload(w, precision="split_tf32")
    ref = torch.from_numpy(w["W0"].copy()).cuda()
    got = torch.from_numpy(w["W0"].copy()).cuda()
    for call in range(2):
        pa.step(ref, w["steps"])
        pb.step_noalloc(got, w["steps"])
        pa.synchronize()
        pb.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), (name, call)
        assert np.array_equal(a, b), (name, call, float(np.max(np.abs(a - b))))
    pa.close()
    pb.close()


def test_noalloc_after_a_call_that_left_nan_in_the_array():
    """A call on a NaN state fills the shared array with NaN; a following call on a plan whose rho
    lines are padded (n_rho = 37, padded to 40) must still equal sexpe_step exactly."""
    import torch
    from paper_2604_11558_gb300 import binding
    big = wl.gray_scott_ball(n=(20, 33, 40), steps=1, seed=13)
    pbig = binding.Plan.from_workload(big, precision="split_tf32")
    bad = torch.full(big["W0"].shape, float("nan"), dtype=torch.float64, device="cuda")
    pbig.step_noalloc(bad, 2)
    pbig.synchronize()
    assert torch.isnan(bad).all()
    pbig.close()
    w = wl.schnakenberg_disk(n=(37, 45), steps=3, seed=11)
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    ref = torch.from_numpy(w["W0"].copy()).cuda()
    got = torch.from_numpy(w["W0"].copy()).cuda()
    plan.step(ref, w["steps"])
    plan.step_noalloc(got, w["steps"])
    plan.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())
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


def test_misaligned_state_is_refused_before_any_launch():
    """A state pointer that is not 8-byte aligned gives SEXPE_EINVAL from both step entry points,
    and the buffer it points into is left untouched."""
    import torch
    from paper_2604_11558_gb300 import binding
    w = wl.schnakenberg_disk(n=(13, 20), steps=1)
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    raw = torch.zeros(w["W0"].size + 1, dtype=torch.float64, device="cuda")
    raw[:-1] = torch.from_numpy(w["W0"].ravel())
    before = raw.clone()
    L = binding.lib()
    st = torch.cuda.current_stream().cuda_stream
    odd = ctypes.c_void_p(raw.data_ptr() + 4)
    assert L.sexpe_step_noalloc(plan.handle, odd, 1, st) == 1
    assert L.sexpe_step(plan.handle, odd, 1, st) == 1
    torch.cuda.synchronize()
    assert torch.equal(raw, before)
    plan.close()
