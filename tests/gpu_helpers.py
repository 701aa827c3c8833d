"""Shared helpers of the GPU parity tests: run one workload on the CUDA path
(through the C-ABI binding) and on the CPU oracle, and compare."""
import numpy as np

from oracle import reactions as R
from oracle.operators import Grid
from oracle.stepper import Problem, run


def oracle_reaction(w, g=None):
    """The workload's reaction for the oracle; with lifting offsets c_s it sees W_s + c_s.  That
    evaluation runs in extended precision (numpy longdouble) and is rounded once: for W small
    against c the FP64 formula would cancel to ~eps |c| / |W| relative accuracy."""
    base = _oracle_reaction(w, g)
    off = w.get("offsets")
    if off is None:
        return base

    def lifted(W, t):
        ext = [np.asarray(W[s], dtype=np.longdouble) + np.longdouble(off[s]) for s in range(len(W))]
        return [np.asarray(r, dtype=np.float64) for r in base(ext, t)]
    return lifted


def _oracle_reaction(w, g=None):
    p = w["params"]
    if w["reaction"] in ("bvam", "bvam_manufactured"):
        prm = dict(R.BVAM, alpha1=p[0], alpha2=p[1], alpha3=p[2], beta1=p[3], beta2=p[4],
                   gamma=w["d"][0], delta=w["d"][1])
        if w["reaction"] == "bvam":
            return lambda W, t: R.bvam(W, prm)
        rho = g.points[1][None, :]
        th = g.points[2][:, None]

        def mms(W, t):                      # sources evaluated at t_n (explicit)
            b = R.bvam(W, prm)
            src = R.bvam_sources(t, rho, th, prm)
            return [b[0] + src[0], b[1] + src[1]]
        return mms
    if w["reaction"] == "schnakenberg":
        return lambda W, t: R.schnakenberg(W, p[0], p[1], p[2])
    if w["reaction"] == "gray_scott":
        return lambda W, t: R.gray_scott(W, p[0], p[1])
    if w["reaction"] == "linear_cubic":
        S = len(w["d"])
        K = np.array(p).reshape(S, S)
        return lambda W, t: R.linear_cubic(W, K)
    return lambda W, t: [np.zeros_like(W[0]) for _ in range(len(w["d"]))]


def oracle_run(w, steps=None, fp32_storage=False):
    g = Grid(w["geometry"], w["n"], z_bc=w.get("z_bc", "neumann"), lam=w.get("lam"))
    p = Problem(g, w["d"], oracle_reaction(w, g), w["tau"])
    return run(p, w["W0"], w["steps"] if steps is None else steps, fp32_storage=fp32_storage)


def emulated_fp32_errors(w, ref, increments=False):
    """Per-species relative error of the oracle run with FP32 storage of F, of every
    direction's result and of the increment (the storage floor of an FP32 chain); with
    `increments`, also the relative error of W_n - W_0."""
    g = Grid(w["geometry"], w["n"], z_bc=w.get("z_bc", "neumann"), lam=w.get("lam"))
    p = Problem(g, w["d"], oracle_reaction(w, g), w["tau"])
    emu = run(p, w["W0"], w["steps"], fp32_storage=True)
    if not increments:
        return rel_errors(emu, ref)
    return rel_errors(emu, ref), increment_errors(emu, ref, w["W0"])


def increment_errors(got, ref, W0):
    return [float(np.linalg.norm((got[s] - W0[s]) - (ref[s] - W0[s])) / max(np.linalg.norm(ref[s] - W0[s]), 1e-300))
            for s in range(ref.shape[0])]


def gpu_run(w, precision, steps=None, single_calls=False, stencil=None, theta_split=None):
    """stencil: optional (tile_j, planes) forced through sexpe_set_stencil; theta_split: optional
    sphere theta-kernel split forced through sexpe_set_theta_split."""
    import torch
    from paper_2604_11558_gb300 import binding
    plan = binding.Plan(w["geometry"], w["n"], w["d"], w["reaction"], w["params"], w["tau"], precision,
                        z_bc=w.get("z_bc", "neumann"), lam=w.get("lam"), offsets=w.get("offsets"))
    if stencil is not None:
        plan.set_stencil(*stencil)
    if theta_split is not None:
        plan.set_theta_split(theta_split)
        assert plan.info()["theta_split"] == theta_split
    x = torch.from_numpy(np.ascontiguousarray(w["W0"])).cuda()
    n = w["steps"] if steps is None else steps
    if single_calls:
        for _ in range(n):
            plan.step(x, 1)
    else:
        plan.step(x, n)
    plan.synchronize()
    out = x.cpu().numpy()
    plan.close()
    return out


def rel_errors(got, ref):
    return [float(np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s])) for s in range(ref.shape[0])]


def assert_parity(got, ref, W0, tol_state, tol_incr=None):
    """State: per-species relative 2-norm error <= tol_state and elementwise
    |got - ref| <= tol_state * max|ref|.  Increment W_n - W_0 likewise with tol_incr."""
    assert np.all(np.isfinite(got))
    e = rel_errors(got, ref)
    assert max(e) <= tol_state, ("state", e)
    for s in range(ref.shape[0]):
        assert np.max(np.abs(got[s] - ref[s])) <= tol_state * np.max(np.abs(ref[s])), ("max-abs", s)
    if tol_incr is not None:
        di = [float(np.linalg.norm((got[s] - W0[s]) - (ref[s] - W0[s])) / max(np.linalg.norm(ref[s] - W0[s]), 1e-300))
              for s in range(ref.shape[0])]
        assert max(di) <= tol_incr, ("increment", di)
    return e
