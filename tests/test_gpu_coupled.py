"""GPU parity of the bulk-surface coupled step (Section 5.5, eqs. bulkball) against the oracle's
``Coupled`` stepper.

Species u, v on the ball and r, s on its boundary sphere, coupled through the flux boundary
conditions (entering the ball's outer radial row through the virtual point of eq. ball_discr) and
the surface reactions, explicit at t_n; each component then takes its own split step (eqs. ee_ball,
ee_sphere).  FP64 on both sides: the state within 1e-12 relative, and the increment W_n - W_0
(of size ~tau |F|, far below the state near the equilibrium) within 1e-9 relative.  Split-TF32
chains (FP32 F, TF32 hi/lo products): the state within 1e-6 relative; the increment within 1e-5
over a few steps and 1e-4 over 200, on data 5e-2 away from the equilibrium (nearer to it the FP32
reaction, alpha1 b(u, v) with |b| ~ 1e-3 formed from O(1) terms, loses digits to cancellation).
"""
import numpy as np
import pytest

from oracle.coupled import Coupled
from paper_2604_11558_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def plan_for(w, precision="fp64"):
    from paper_2604_11558_gb300 import binding
    rs = w["rho_star"]
    return binding.CoupledPlan(w["n"], w["d_bulk"], w["bulk_params"], [d / rs**2 for d in w["d_surface"]],
                               w["surface_params"], w["coupling"], w["tau"], rho_star=rs, precision=precision)


def flat(Wb, Ws):
    return np.concatenate([np.ascontiguousarray(Wb).ravel(), np.ascontiguousarray(Ws).ravel()])


def split_state(x, n):
    nb = int(np.prod(n))
    ns = n[1] * n[2]
    return x[:2 * nb].reshape((2,) + tuple(reversed(n))), x[2 * nb:2 * nb + 2 * ns].reshape((2, n[2], n[1]))


def gpu_coupled(w, steps, single_calls=False, precision="fp64"):
    import torch
    plan = plan_for(w, precision)
    x = torch.from_numpy(flat(w["Wb"], w["Ws"])).cuda()
    info = plan.info()
    assert info["state_elems"] == x.numel()
    if single_calls:
        for _ in range(steps):
            plan.step(x, 1)
    else:
        plan.step(x, steps)
    plan.synchronize()
    out = x.cpu().numpy()
    plan.close()
    return split_state(out, w["n"])


def oracle_coupled(w, steps):
    c = w["coupling"]
    a1, a2, b1 = w["bulk_params"]
    o = Coupled(w["n"], w["tau"], alpha1=a1, alpha2=a2, beta1=b1, delta=w["d_bulk"][1], eps=w["d_surface"][1],
                zeta1=c["zeta1"], zeta2=c["zeta2"], zeta3=c["zeta3"], eta1=c["eta1"], eta2=c["eta2"],
                rho_star=w["rho_star"])
    assert w["surface_params"][0] == c["zeta1"]
    return o.run(w["Wb"].copy(), w["Ws"].copy(), steps)


def check(got, ref, W0, tol_state=1e-12, tol_incr=1e-9):
    errs = []
    for g, r, w0 in zip(got, ref, W0):
        assert np.all(np.isfinite(g))
        for s in range(2):
            err = np.max(np.abs(g[s] - r[s])) / np.max(np.abs(r[s]))
            inc = np.linalg.norm((g[s] - w0[s]) - (r[s] - w0[s])) / max(np.linalg.norm(r[s] - w0[s]), 1e-300)
            errs.append((float(err), float(inc)))
    print("state / increment errors (u, v, r, s):", errs)
    for err, inc in errs:
        assert err <= tol_state, errs
        assert inc <= tol_incr, errs


def case(n, steps, tau, seed, rho_star=1.0, noise=1e-3):
    w = wl.bulk_surface_ball(n=n, steps=steps, seed=seed, tau=tau)
    if noise != 1e-3:                      # larger perturbations: the coupling terms well above rounding
        w["Wb"] = w["Wb"] + (noise / 1e-3 - 1.0) * (w["Wb"] - w["Wb"].mean(axis=(1, 2, 3), keepdims=True))
        w["Ws"] = w["Ws"] + (noise / 1e-3 - 1.0) * (w["Ws"] - w["Ws"].mean(axis=(1, 2), keepdims=True))
    w["rho_star"] = rho_star
    return w


CASES = [
    ("small", case((5, 6, 7), 4, 1e-3, 61)),
    ("rho_star_0p7", case((9, 8, 6), 5, 1e-3, 62, rho_star=0.7, noise=5e-2)),
    ("ragged_tiles", case((33, 40, 37), 3, 2e-4, 63, noise=5e-2)),
    ("paper_30x50x30", case((30, 50, 30), 200, 1e-4, 8)),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_coupled_matches_oracle(name, w):
    got = gpu_coupled(w, w["steps"])
    ref = oracle_coupled(w, w["steps"])
    check(got, ref, (w["Wb"], w["Ws"]))


SPLIT_CASES = [
    ("small", case((5, 6, 7), 4, 1e-3, 71, noise=5e-2), 1e-5),
    ("rho_star_0p7", case((9, 8, 6), 5, 1e-3, 72, rho_star=0.7, noise=1e-2), 1e-5),
    ("ragged_tiles", case((33, 40, 37), 3, 2e-4, 73, noise=5e-2), 1e-5),
    ("paper_30x50x30", case((30, 50, 30), 200, 1e-4, 74, noise=5e-2), 1e-4),
]


@pytest.mark.parametrize("name,w,tol_incr", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_coupled_split_tf32_matches_oracle(name, w, tol_incr):
    got = gpu_coupled(w, w["steps"], precision="split_tf32")
    ref = oracle_coupled(w, w["steps"])
    check(got, ref, (w["Wb"], w["Ws"]), tol_state=1e-6, tol_incr=tol_incr)


def test_coupled_split_tf32_rough_coarse_grid():
    """White noise of 5e-2 on the coarse 9 x 8 x 6 ball with rho_* = 0.7: the Laplacian terms of such
    a field reach ~1e4 near the axis and the poles, so the FP32 evaluation of F leaves ~1e-6 at those
    few points.  As for the other noisy split-TF32 fields, the state is held to 1e-6 in the relative
    2-norm per species (the stated target) and the increment to 1e-5; pointwise to 1e-5 of max|W|."""
    w = case((9, 8, 6), 5, 1e-3, 72, rho_star=0.7, noise=5e-2)
    got = gpu_coupled(w, w["steps"], precision="split_tf32")
    ref = oracle_coupled(w, w["steps"])
    out = []
    for g, r, w0 in zip(got, ref, (w["Wb"], w["Ws"])):
        for s in range(2):
            e2 = np.linalg.norm(g[s] - r[s]) / np.linalg.norm(r[s])
            inc = np.linalg.norm((g[s] - w0[s]) - (r[s] - w0[s])) / np.linalg.norm(r[s] - w0[s])
            em = np.max(np.abs(g[s] - r[s])) / np.max(np.abs(r[s]))
            out.append((float(e2), float(inc), float(em)))
    print("2-norm state / increment / max-abs errors (u, v, r, s):", out)
    for e2, inc, em in out:
        assert e2 <= 1e-6 and inc <= 1e-5 and em <= 1e-5, out


@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_coupled_single_calls_equal_one_call(precision):
    w = case((7, 10, 9), 12, 1e-3, 64, noise=2e-2)       # one call: a 10-step graph, then 2 steps
    a = gpu_coupled(w, 12, precision=precision)
    b = gpu_coupled(w, 12, single_calls=True, precision=precision)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_coupled_split_two_streams_equal_one_stream():
    """Split coupled steps run the surface component on a second stream beside the bulk's; profiled
    steps keep one stream.  Both orders give the same state bit for bit (the kernels and their
    inputs are the same; only their overlap differs)."""
    import torch
    w = case((7, 10, 9), 6, 1e-3, 66, noise=2e-2)
    out = []
    for profiled in (False, True):
        plan = plan_for(w, precision="split_tf32")
        x = torch.from_numpy(flat(w["Wb"], w["Ws"])).cuda()
        if profiled:
            plan.profile_begin(6)
        for _ in range(6):
            plan.step(x, 1)
        if profiled:
            plan.profile_end()
        plan.synchronize()
        out.append(x.cpu().numpy())
        plan.close()
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1])


def test_coupled_step_host_equals_device():
    w = case((6, 9, 8), 3, 1e-3, 65, noise=2e-2)
    dev = gpu_coupled(w, 3)
    plan = plan_for(w)
    x = flat(w["Wb"], w["Ws"])
    plan.step_host(x, 3)
    plan.close()
    host = split_state(x, w["n"])
    for a, b in zip(dev, host):
        assert np.array_equal(a, b)


def test_coupled_equilibrium_stays_fixed():
    """The homogeneous equilibrium is a fixed point of the coupled step up to rounding.  With
    zeta2 = zeta3 and eta1 = eta2 the coupling terms vanish exactly there; what remains is the FP64
    rounding of the operators' row sums (ball entries up to ~1e4 near the axis on this grid, times
    tau, over 10 steps), of order 1e-12."""
    w = case((8, 10, 12), 10, 1e-3, 66)
    ue, ve = 0.1 + 0.9, 0.9 / (0.1 + 0.9) ** 2
    w["Wb"] = np.stack([np.full_like(w["Wb"][0], ue), np.full_like(w["Wb"][1], ve)])
    w["Ws"] = np.stack([np.full_like(w["Ws"][0], ue), np.full_like(w["Ws"][1], ve)])
    got = gpu_coupled(w, 10)
    assert np.max(np.abs(got[0] - w["Wb"])) < 1e-10
    assert np.max(np.abs(got[1] - w["Ws"])) < 1e-10


def test_coupled_setup_errors():
    from paper_2604_11558_gb300 import binding
    w = case((5, 6, 7), 1, 1e-3, 67)
    base = dict(n=w["n"], d_bulk=w["d_bulk"], bulk_params=w["bulk_params"], d_surface=w["d_surface"],
                surface_params=w["surface_params"], coupling=w["coupling"], tau=w["tau"])
    st = binding.coupled_setup_status
    assert st(**base) == 0
    assert st(**dict(base, precision="split_tf32")) == 0
    assert st(**dict(base, precision="unsplit_fp64")) == 5       # SEXPE_EUNSUPPORTED
    assert st(**dict(base, d_bulk=[1.0, 10.0, 3.0])) == 1        # SEXPE_EINVAL: three bulk species
    assert st(**dict(base, coupling=dict(w["coupling"], zeta2=float("nan")))) == 1
    assert st(**dict(base, tau=-1.0)) == 1
    assert st(**dict(base, n=(2, 6, 7))) == 1
    plan = plan_for(w, "split_tf32")
    with pytest.raises(RuntimeError):                            # the stencil belongs to the sub-grids
        plan.set_stencil(4, 0)
    import torch
    with pytest.raises(RuntimeError):                            # no static-scratch variant
        plan.step_noalloc(torch.zeros(plan.info()["state_elems"], dtype=torch.float64, device="cuda"), 1)
    plan.close()
    plan = plan_for(w)
    with pytest.raises(RuntimeError):                            # no adjoint for the coupled system
        import torch
        x = torch.zeros(plan.info()["state_elems"], dtype=torch.float64, device="cuda")
        g = torch.zeros_like(x)
        plan.adjoint(x, 1, 1, g, torch.zeros_like(x))
    plan.close()
