"""Write the oracle's final-time references of the benchmark workloads (tests/golden/final_time_*.npz).

Runs ONLY the FP64 CPU oracle (``oracle/``) on the seeded workloads of
``paper_2604_11558_gb300.workloads`` to their final times and stores, per workload,
the exact per-species 2-norms of the final state, its values at a seeded sample
of grid points (the full states are 2-25 MB each; the sample lets the GPU tests and
the benchmark state the error of a full-size run at the final time without running
the oracle for minutes) and the storage floor of an FP32-intermediate chain: the
per-species relative 2-norm error, over the whole final state, of the oracle run with
F, every direction's result and the increment rounded to FP32 (its precision-emulation
switch), which is what any implementation that keeps those intermediates in FP32 cannot
be expected to beat; for the ball also an FP64 evaluation-order floor (rowsum_exact_floor):

* ball 100^3 Gray-Scott, 500 steps (tau 0.5, t_* = 250);
* cylinder 64 x 128 x 128, 3 species, 1000 steps (tau 0.05, t_* = 50);
* sphere 256 x 512 Schnakenberg (gamma 200), 1000 steps (tau 1e-4, t_* = 0.1);
* 16 of the 256 batched disks (a seeded choice), 500 steps each (tau 1e-4).

Usage: python tests/golden/make_final_time_refs.py [ball|cylinder|sphere|batch ...]
(about 5-20 minutes per workload on 8 cores)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2604_11558_gb300 import workloads as wl  # noqa: E402
from tests.gpu_helpers import oracle_run  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLES = 2048          # sampled points per species of a single-grid workload
BATCH_PICK = 16         # batched disks checked
BATCH_SAMPLES = 256     # sampled points per species of each checked disk
SAMPLE_SEED = 2604


def sample_indices(npts, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(npts, size=min(k, npts), replace=False))


def storage_floor(w, ref):
    """Per-species relative 2-norm error of the oracle run with FP32 storage of every intermediate."""
    emu = oracle_run(w, fp32_storage=True)
    return np.array([np.linalg.norm(emu[s] - ref[s]) / np.linalg.norm(ref[s]) for s in range(ref.shape[0])])


def rowsum_exact_floor(w, ref):
    """Per-species relative 2-norm difference, at the final time, between the oracle and the same
    oracle with d M w evaluated per direction with every row of each Kronecker term summing to exactly
    0 (the two are equal in exact arithmetic; every row of the benchmark grids is a Neumann or
    periodic row): how far two FP64 evaluations of the same operator drift apart over the run."""
    import scipy.sparse as sp
    from oracle.operators import Grid
    from oracle.stepper import Problem, run
    from tests.gpu_helpers import oracle_reaction
    g = Grid(w["geometry"], w["n"], z_bc=w.get("z_bc", "neumann"), lam=w.get("lam"))
    Ms = {}
    for mu, M in g.M.items():
        M = sp.csr_matrix(M)
        Ms[mu] = M - sp.diags(np.asarray(M.sum(axis=1)).ravel())
    g.apply_M = lambda x: sum((Ms[mu] @ x.ravel()).reshape(x.shape) for mu in sorted(Ms))
    alt = run(Problem(g, w["d"], oracle_reaction(w, g), w["tau"]), w["W0"], w["steps"])
    return np.array([np.linalg.norm(alt[s] - ref[s]) / np.linalg.norm(ref[s]) for s in range(ref.shape[0])])


def single(name, w, fp64_floor=False):
    t0 = time.time()
    ref = oracle_run(w)
    S = ref.shape[0]
    flat = ref.reshape(S, -1)
    idx = sample_indices(flat.shape[1], SAMPLES, SAMPLE_SEED)
    floor = storage_floor(w, ref)
    extra = {}
    if fp64_floor:
        extra["floor64"] = rowsum_exact_floor(w, ref)
        print(name, "FP64 evaluation-order floor per species", extra["floor64"], flush=True)
    np.savez_compressed(os.path.join(HERE, f"final_time_{name}.npz"), idx=idx, values=flat[:, idx],
                        norms=np.linalg.norm(flat, axis=1), maxabs=np.max(np.abs(flat), axis=1),
                        floor=floor, steps=w["steps"], n=np.array(w["n"]), seed=w["seed"], **extra)
    print(name, "FP32-storage floor per species", floor, flush=True)
    print(name, "done in", round(time.time() - t0), "s", flush=True)


def batch():
    t0 = time.time()
    ws = wl.batched_disks()
    pick = np.sort(np.random.Generator(np.random.PCG64(SAMPLE_SEED)).choice(len(ws), BATCH_PICK, replace=False))
    out = dict(pick=pick, steps=ws[0]["steps"])
    for q in pick:
        ref = oracle_run(ws[q])
        flat = ref.reshape(ref.shape[0], -1)
        idx = sample_indices(flat.shape[1], BATCH_SAMPLES, SAMPLE_SEED + int(q))
        out[f"idx_{q}"] = idx
        out[f"values_{q}"] = flat[:, idx]
        out[f"norms_{q}"] = np.linalg.norm(flat, axis=1)
        out[f"maxabs_{q}"] = np.max(np.abs(flat), axis=1)
        out[f"floor_{q}"] = storage_floor(ws[q], ref)
    np.savez_compressed(os.path.join(HERE, "final_time_batch.npz"), **out)
    print("batch done in", round(time.time() - t0), "s", flush=True)


def main(which):
    for name in which:
        if name == "ball":
            single("ball", wl.gray_scott_ball(), fp64_floor=True)
        elif name == "cylinder":
            single("cylinder", wl.linear_cubic_cylinder())
        elif name == "sphere":
            single("sphere", wl.schnakenberg_sphere())
        elif name == "batch":
            batch()
        else:
            raise SystemExit(f"unknown workload {name}")


if __name__ == "__main__":
    main(sys.argv[1:] or ["ball", "cylinder", "sphere", "batch"])
