"""GPU parity of the batched disk stepper (sexpe_batch_setup + one persistent launch per step).

Every instance is compared with the oracle stepping it alone, 1e-6 relative per
species (the split path's target); odd and even step counts exercise the
ping-pong of the two state buffers, n_theta > 128 the two-tile theta products,
and 12 steps the captured-graph replay (bit-identical to single steps).
"""
import numpy as np
import pytest

from paper_2604_11558_gb300 import workloads as wl
from tests.gpu_helpers import oracle_run, rel_errors

pytestmark = pytest.mark.gpu


def _instances(sizes, steps, seed=31):
    rng = np.random.default_rng(seed)
    out = []
    for q, (nr, nt) in enumerate(sizes):
        w = wl.schnakenberg_disk(n=(nr, nt), steps=steps, seed=seed + q,
                                 a=float(rng.uniform(0.05, 0.2)), b=float(rng.uniform(0.7, 1.0)),
                                 d=(1.0, float(rng.uniform(8, 20))))
        out.append(w)
    return out


def _run_batch(ws, steps, single=False):
    import torch
    from paper_2604_11558_gb300 import binding
    plan = binding.BatchPlan(ws)
    off = plan.offsets()
    x = torch.from_numpy(np.concatenate([w["W0"].ravel() for w in ws])).cuda()
    if single:
        for _ in range(steps):
            plan.step(x, 1)
    else:
        plan.step(x, steps)
    plan.synchronize()
    flat = x.cpu().numpy()
    plan.close()
    return [flat[off[q]:off[q + 1]].reshape(w["W0"].shape) for q, w in enumerate(ws)]


SIZES = [(5, 8), (17, 33), (40, 140), (96, 256), (23, 64), (64, 97), (90, 140), (128, 136)]


@pytest.mark.parametrize("steps", [4, 5])
def test_batch_matches_oracle(steps):
    ws = _instances(SIZES, steps)
    got = _run_batch(ws, steps)
    for q, w in enumerate(ws):
        e = rel_errors(got[q], oracle_run(w))
        assert max(e) <= 1e-6, (q, w["n"], e)


def test_batch_graph_replay_equals_single_steps():
    ws = _instances(SIZES[:4], 12)
    a = _run_batch(ws, 12)
    b = _run_batch(ws, 12, single=True)
    for q in range(len(ws)):
        assert np.array_equal(a[q], b[q])


def test_batch_full_workload_sampled():
    ws = wl.batched_disks(steps=10)
    got = _run_batch(ws, 10)
    for q in [0, 17, 100, 255]:
        e = rel_errors(got[q], oracle_run(ws[q]))
        assert max(e) <= 1e-6, (q, ws[q]["n"], e)


def test_batch_plan_reports_tuned_configuration():
    """sexpe_batch_setup times every feasible (ring depths, stencil tile height, work-list order)
    and keeps the fastest; sexpe_plan_info reports the kept choice and its measured step time."""
    from paper_2604_11558_gb300 import binding
    plan = binding.BatchPlan(wl.batched_disks(steps=1))
    info = plan.info()
    plan.close()
    print("batch tuner choice", info["stencil_tile_j"], info["ring_slots"], info["batch_order"],
          info["batch_step_us"])
    assert info["stencil_tile_j"] in (8, 16, 32)
    assert info["batch_order"] in (0, 1)
    nm, nd = info["ring_slots"]
    assert 2 <= nm <= nd <= 4
    assert 0.0 < info["batch_step_us"] < 5000.0
