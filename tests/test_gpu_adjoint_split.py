"""GPU tests of the split-TF32 discrete adjoint of the sphere step (the differentiation workload).

The split adjoint differentiates the split-TF32 forward: its transposed chain runs on the
tensor-core kernels in split TF32 with FP32 accumulation (lambda and the parameter sums FP64).
Reference gradients: the oracle's complex-step derivatives (FP64, exact to rounding) on small
grids, and at the full 256 x 512, 1000-step size the FP64 GPU adjoint (itself checked against
the oracle's complex step and against central differences in tests/test_gpu_adjoint.py) and
central differences of the FP64 GPU forward (h = 1e-4).  Tolerance: 1e-4 relative (the
FP32 arithmetic of the transposed chain and of the split forward's trajectory).
"""
import time

import numpy as np
import pytest

from oracle import adjoint as OA
from oracle.operators import Grid
from paper_2604_11558_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _adjoint(w, precision, gT, every, params=None, d=None):
    import torch
    from paper_2604_11558_gb300 import binding
    prm = w["params"] if params is None else params
    plan = binding.Plan(w["geometry"], w["n"], w["d"] if d is None else d, w["reaction"], prm, w["tau"], precision)
    x = torch.from_numpy(w["W0"].copy()).cuda()
    n_ckpt = w["steps"] // every
    ckpt = torch.empty((n_ckpt,) + tuple(x.shape), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.step_checkpointed(x, w["steps"], every, ckpt)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    WT = x.cpu().numpy()
    g = torch.from_numpy(gT(WT)).cuda()
    g0 = torch.empty_like(g)
    gp = plan.adjoint(ckpt, n_ckpt, every, g, g0)          # first call builds the adjoint tables
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gp2 = plan.adjoint(ckpt, n_ckpt, every, g, torch.empty_like(g))
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    plan.synchronize()
    out = dict(g0=g0.cpu().numpy(), gp=np.array(gp), gp2=np.array(gp2), WT=WT, t_fwd=t_fwd, t_adj=t_adj)
    plan.close()
    return out


@pytest.mark.parametrize("n,steps,every", [((24, 13), 10, 5), ((40, 33), 8, 4)])
def test_split_sphere_adjoint_matches_complex_step(n, steps, every):
    w = wl.schnakenberg_sphere(n=n, steps=steps, seed=22)
    c = np.random.default_rng(5).standard_normal(w["W0"].shape)
    r = _adjoint(w, "split_tf32", lambda WT: c, every)
    # a second call repeats the first (up to the order of the FP64 atomic reductions)
    assert np.allclose(r["gp"], r["gp2"], rtol=1e-12, atol=0)
    g = Grid("sphere", n)
    params = list(w["params"]) + list(w["d"])
    build = OA.problem_builder(g, w["reaction"], w["tau"], len(w["params"]))
    loss = lambda W: np.sum(c * W)
    ref = np.array([OA.complex_step_param(build, params, q, w["W0"], steps, loss) for q in range(len(params))])
    err = np.abs(r["gp"] - ref) / np.abs(ref)
    print("split sphere", n, "parameter gradient rel. errors", err)
    assert np.all(err <= TOL), (r["gp"], ref)
    rng = np.random.default_rng(7)
    for t in range(3):
        delta = rng.standard_normal(w["W0"].shape)
        cs = OA.complex_step_state(build, params, w["W0"], delta, steps, loss)
        e = abs(np.sum(r["g0"] * delta) - cs) / abs(cs)
        print("  directional derivative", t, "rel. error", e)
        assert e <= TOL


def test_split_sphere_adjoint_full_size():
    """Sphere 256 x 512, Schnakenberg (gamma 200), 1000 steps, checkpoints every 50; loss
    ||u(T) - u_target||^2 with u_target from a run at a = 0.12, b = 0.85 (split forward).  The
    split adjoint's gradient with respect to (a, b, d_v) and W_0 against the FP64 GPU adjoint of
    the same loss and against central differences of the FP64 GPU forward; its cost against the
    split forward is printed (the benchmark reports it)."""
    import torch
    from paper_2604_11558_gb300 import binding
    w = wl.schnakenberg_sphere()
    steps, every = w["steps"], 50
    gamma, a, b = w["params"]
    d = list(w["d"])

    def forward(prm, W0, precision):
        plan = binding.Plan("sphere", w["n"], prm[3:], "schnakenberg", prm[:3], w["tau"], precision)
        x = torch.from_numpy(W0.copy()).cuda()
        plan.step(x, steps)
        plan.synchronize()
        out = x.cpu().numpy()
        plan.close()
        return out

    target = forward([gamma, 0.12, 0.85] + d, w["W0"], "split_tf32")[0]

    def gT(WT):
        g = np.zeros_like(WT)
        g[0] = 2.0 * (WT[0] - target)
        return g

    rs = _adjoint(w, "split_tf32", gT, every)
    r64 = _adjoint(w, "fp64", gT, every)
    print(f"split forward {rs['t_fwd']:.4f} s, split adjoint {rs['t_adj']:.4f} s, ratio {rs['t_adj'] / rs['t_fwd']:.2f}; "
          f"FP64 adjoint {r64['t_adj']:.3f} s")
    for q in (1, 2, 4):                                  # a, b, d_v
        e = abs(rs["gp"][q] - r64["gp"][q]) / abs(r64["gp"][q])
        print("param", q, "split", rs["gp"][q], "fp64", r64["gp"][q], "rel", e)
        assert e <= TOL
    e0 = np.linalg.norm(rs["g0"] - r64["g0"]) / np.linalg.norm(r64["g0"])
    print("dL/dW0 rel. 2-norm error vs FP64 adjoint", e0)
    assert e0 <= TOL
    params = [gamma, a, b] + d

    def loss(prm):
        return float(np.sum((forward(prm, w["W0"], "fp64")[0] - target) ** 2))

    for q in (1, 2, 4):
        h = 1e-4 * abs(params[q])
        pp, pm = list(params), list(params)
        pp[q] += h
        pm[q] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        e = abs(rs["gp"][q] - fd) / abs(fd)
        print("param", q, "central difference", fd, "rel", e)
        assert e <= TOL
