"""GPU tests of the discrete adjoint (sexpe_step_checkpointed + sexpe_adjoint).

The loss is L = <c, W_N> for a seeded c (so dL/dW_N = c).  Every parameter
gradient (reaction parameters and diffusion coefficients) and the gradient with
respect to W_0 along seeded directions are compared with the oracle's
complex-step derivatives (exact to rounding), relative tolerance 1e-8 -- the
FP64 adjoint accumulates rounding over O(steps x products) operations.  The
sphere workload at its full size (256 x 512, 1000 steps, checkpoints every 50)
is checked against central finite differences of the GPU FP64 forward.
"""
import numpy as np
import pytest

from oracle import adjoint as OA
from oracle.operators import Grid
from paper_2604_11558_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [
    ("disk", wl.schnakenberg_disk(n=(9, 12), steps=6, seed=21)),
    ("sphere", wl.schnakenberg_sphere(n=(12, 9), steps=6, seed=22)),
    ("ball", wl.gray_scott_ball(n=(7, 8, 9), steps=6, seed=23, tau=0.5)),
    ("cylinder", wl.linear_cubic_cylinder(n=(7, 8, 9), steps=6, seed=24)),
]


def _gpu_adjoint(w, c, every):
    import torch
    from paper_2604_11558_gb300 import binding
    plan = binding.Plan.from_workload(w, precision="fp64")
    x = torch.from_numpy(w["W0"].copy()).cuda()
    n_ckpt = w["steps"] // every
    ckpt = torch.empty((n_ckpt,) + tuple(x.shape), dtype=torch.float64, device="cuda")
    plan.step_checkpointed(x, w["steps"], every, ckpt)
    g = torch.from_numpy(c.copy()).cuda()
    g0 = torch.empty_like(g)
    gp = plan.adjoint(ckpt, n_ckpt, every, g, g0)
    plan.synchronize()
    out = g0.cpu().numpy(), gp, x.cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_complex_step(name, w):
    rng = np.random.default_rng(5)
    c = rng.standard_normal(w["W0"].shape)
    g0, gp, _ = _gpu_adjoint(w, c, every=2)
    g = Grid(w["geometry"], w["n"])
    params = list(w["params"]) + list(w["d"])
    build = OA.problem_builder(g, w["reaction"], w["tau"], len(w["params"]))
    loss = lambda W: np.sum(c * W)
    ref = np.array([OA.complex_step_param(build, params, q, w["W0"], w["steps"], loss) for q in range(len(params))])
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(gp - ref)) <= 1e-8 * scale, (name, gp, ref)
    for t in range(3):
        delta = rng.standard_normal(w["W0"].shape)
        cs = OA.complex_step_state(build, params, w["W0"], delta, w["steps"], loss)
        assert abs(np.sum(g0 * delta) - cs) <= 1e-8 * abs(cs), (name, t)


def test_autograd_function_matches_adjoint():
    import torch
    from paper_2604_11558_gb300 import binding
    w = wl.schnakenberg_disk(n=(9, 12), steps=6, seed=21)
    plan = binding.Plan.from_workload(w, precision="fp64")
    W0 = torch.from_numpy(w["W0"].copy()).cuda().requires_grad_(True)
    params = torch.tensor(list(w["params"]) + list(w["d"]), dtype=torch.float64, requires_grad=True)
    c = torch.from_numpy(np.random.default_rng(5).standard_normal(w["W0"].shape)).cuda()
    WN = binding.evolve(plan, W0, params, 6, 3)
    loss = (c * WN).sum()
    loss.backward()
    g0, gp, _ = _gpu_adjoint(w, c.cpu().numpy(), every=3)
    assert np.allclose(W0.grad.cpu().numpy(), g0, rtol=0, atol=1e-12 * np.abs(g0).max())
    assert np.allclose(params.grad.numpy(), gp, rtol=1e-12)
    plan.close()


def test_sphere_full_size_adjoint_against_finite_differences():
    """Sphere 256 x 512, Schnakenberg (gamma 200), 1000 steps, checkpoints every 50;
    loss ||u(T) - u_target||^2 with u_target from a run at a = 0.12, b = 0.85."""
    import time
    import torch
    from paper_2604_11558_gb300 import binding
    w = wl.schnakenberg_sphere()
    steps, every = w["steps"], 50
    gamma, a, b = w["params"]
    d = w["d"]

    def forward(prm, W0):
        plan = binding.Plan("sphere", w["n"], prm[3:], "schnakenberg", prm[:3], w["tau"], "fp64")
        x = torch.from_numpy(W0.copy()).cuda()
        plan.step(x, steps)
        plan.synchronize()
        out = x.cpu().numpy()
        plan.close()
        return out

    target = forward([gamma, 0.12, 0.85, d[0], d[1]], w["W0"])[0]
    params = [gamma, a, b, d[0], d[1]]
    plan = binding.Plan("sphere", w["n"], d, "schnakenberg", [gamma, a, b], w["tau"], "fp64")
    x = torch.from_numpy(w["W0"].copy()).cuda()
    ckpt = torch.empty((steps // every,) + tuple(x.shape), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.step_checkpointed(x, steps, every, ckpt)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    WT = x.cpu().numpy()
    gT = np.zeros_like(WT)
    gT[0] = 2.0 * (WT[0] - target)
    g = torch.from_numpy(gT).cuda()
    g0 = torch.empty_like(g)
    t0 = time.perf_counter()
    gp = plan.adjoint(ckpt, steps // every, every, g, g0)    # first call also builds the adjoint tables
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    gp2 = plan.adjoint(ckpt, steps // every, every, g, torch.empty_like(g))
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    assert np.allclose(gp, gp2, rtol=1e-12)
    print(f"sphere 256x512, 1000 steps: forward {t_fwd:.3f} s, adjoint {t_adj:.3f} s (first call with setup "
          f"{t_first:.3f} s), adjoint / forward {t_adj / t_fwd:.2f}")
    plan.close()

    def loss(prm, W0):
        return float(np.sum((forward(prm, W0)[0] - target) ** 2))

    for q in [1, 2, 4]:                                  # a, b, d_v
        h = 1e-4 * abs(params[q])
        pp, pm = list(params), list(params)
        pp[q] += h
        pm[q] -= h
        fd = (loss(pp, w["W0"]) - loss(pm, w["W0"])) / (2 * h)
        assert abs(gp[q] - fd) <= 1e-5 * abs(fd) + 1e-12, (q, gp[q], fd)
    delta = np.random.default_rng(9).standard_normal(w["W0"].shape)
    h = 1e-4
    fd = (loss(params, w["W0"] + h * delta) - loss(params, w["W0"] - h * delta)) / (2 * h)
    assert abs(np.sum(g0.cpu().numpy() * delta) - fd) <= 1e-5 * abs(fd)
