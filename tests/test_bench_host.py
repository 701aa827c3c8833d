"""Host logic of bench.py on CPU: the max-over-ranks reduction used for the
timed region, with two gloo ranks (replicas only: no collective on the data
path), the algorithmic-work table used for the roofline, and the JSON line of the
reference arm (the oracle on the host cores)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank, world)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.5


def test_kernel_work_table():
    import bench
    wk = bench.kernel_work((100, 100, 100), 2)
    dof = 2 * 10**6
    # algorithmic bytes: the state read by the stencil, read and written by the slab's update
    assert wk["stencil"]["bytes"] == 8 * dof and wk["k_tc_mode3"]["bytes"] == 0
    assert wk["k_tc_slab"]["bytes"] == 16 * dof
    assert wk["k_tc_slab"]["bytes_with_intermediates"] == 20 * dof
    assert wk["k_tc_mode3"]["flops"] == 3 * 2 * 2 * 100 * dof
    # split-TF32 flops per DOF of the whole chain: 3 passes x 2 x (2 n_phi + 2 n_theta + n_rho)
    total = sum(v["flops"] for v in wk.values()) / dof
    assert total == 3 * 2 * (2 * 100 + 2 * 100 + 100)


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores, one timed step) prints one JSON
    line with the contract's keys, the workload of our own arm and a reference-arm e2e entry."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    import bench
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
