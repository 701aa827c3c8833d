"""GPU parity of the bulk-surface DIB step on the cylinder and its bottom disk (Section 5.6, eqs.
bulkcyl) against the oracle's ``CoupledCylinder``.

Bulk w = (u - alpha2, v - beta2) on the cylinder with the Dirichlet top of eq. A_z (LINEAR reaction
K = diag(-alpha1, -beta1)), surface r, s on the bottom disk; the DIB kinetics p, q and the bottom
fluxes -zeta1 alpha3 p, -zeta1 beta3 q are formed by the coupling kernel, explicit at t_n; each
component then takes its own split step (eqs. ee_cylinder, ee_disk).

FP64: state within max(1e-12, 4 x floor) of its largest value, increment W_n - W_0 within
max(1e-9, 4 x floor), the floor being the oracle's own rounding: the difference between two
evaluations of d M w that are equal in exact arithmetic, the oracle's assembled sparse Kronecker sum
and the per-direction product with every Neumann/periodic row summing to exactly 0 (the library's
difference form).  The DIB kinetics amplify it: r and w are driven by zeta4 (s - zeta5) with
s ~ zeta5, so the assembled operator's rounded row sums acting on s ~ 0.5 (a smooth per-ring
source, ~1e-13 absolute) reappear in r and w at ~1e-11 of their (small) size on the paper's grid.
Split-TF32 (n_rho <= 128): state within max(1e-6, 8 x floor), increment within max(1e-5, 8 x
floor), the floor being the oracle run with the split chain's arithmetic emulated (F rounded to
FP32; every product as three TF32 products hi hi + hi lo + lo hi accumulated in FP32; each
direction's result and the increment rounded to FP32).  On the 120 x 140 x 25 grid the chain's
error is characterised instead (see that test).
"""
import numpy as np
import pytest

from oracle.coupled_dib import CoupledCylinder
from paper_2604_11558_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def plan_for(w, precision="fp64"):
    from paper_2604_11558_gb300 import binding
    return binding.CoupledPlan(w["n"], w["d_bulk"], w["bulk_params"], w["d_surface"], w["surface_params"],
                               w["coupling"], w["tau"], rho_star=w["rho_star"], precision=precision,
                               reaction=w["bulk_reaction"], surface_reaction=w["surface_reaction"],
                               geometry="cylinder", z_star=w["z_star"])


def split_state(x, n):
    nb = int(np.prod(n))
    ns = n[0] * n[1]
    return x[:2 * nb].reshape((2,) + tuple(reversed(n))), x[2 * nb:2 * nb + 2 * ns].reshape((2, n[1], n[0]))


def gpu_dib(w, steps, precision="fp64", single_calls=False):
    import torch
    plan = plan_for(w, precision)
    x = torch.from_numpy(np.concatenate([w["Wb"].ravel(), w["Ws"].ravel()])).cuda()
    assert plan.info()["state_elems"] == x.numel()
    if single_calls:
        for _ in range(steps):
            plan.step(x, 1)
    else:
        plan.step(x, steps)
    plan.synchronize()
    out = x.cpu().numpy()
    plan.close()
    return split_state(out, w["n"])


def oracle_dib(w, steps):
    o = CoupledCylinder(w["n"], w["tau"], rho_star=w["rho_star"], z_star=w["z_star"], **w["oracle_params"])
    return o.run(w["Wb"].copy(), w["Ws"].copy(), steps)


def oracle_dib_rowsum_exact(w, steps):
    """The oracle with d M w evaluated per direction, each direction's rows summing to exactly 0
    except the Dirichlet top rows of eq. A_z (equal to the oracle's result in exact arithmetic)."""
    import scipy.sparse as sp
    o = CoupledCylinder(w["n"], w["tau"], rho_star=w["rho_star"], z_star=w["z_star"], **w["oracle_params"])
    for g in (o.bulk, o.surface):
        Ms = {}
        for mu, M in g.M.items():
            M = sp.csr_matrix(M)
            rs = np.asarray(M.sum(axis=1)).ravel()
            if g.kind == "cylinder" and mu == 3:
                rs[(g.n[2] - 1) * g.n[0] * g.n[1]:] = 0.0
            Ms[mu] = M - sp.diags(rs)
        g.apply_M = lambda x, Ms=Ms: sum((Ms[mu] @ x.ravel()).reshape(x.shape) for mu in sorted(Ms))
    return o.run(w["Wb"].copy(), w["Ws"].copy(), steps)


def oracle_dib_split_emulated(w, steps):
    """The oracle step with the split chain's arithmetic emulated (an error model, not a reference)."""
    from oracle.stepper import rhs
    from tests.precision_emulation import advance

    o = CoupledCylinder(w["n"], w["tau"], rho_star=w["rho_star"], z_star=w["z_star"], **w["oracle_params"])
    Wb, Ws = w["Wb"].copy(), w["Ws"].copy()
    for _ in range(steps):
        Fb, Fs = rhs(o.pb, Wb), rhs(o.ps, Ws)
        ab, as_ = o.coupling(Wb, Ws)
        Wb, Ws = (advance(o.pb, Wb, [Fb[q] + ab[q] for q in range(2)]),
                  advance(o.ps, Ws, [Fs[q] + as_[q] for q in range(2)]))
    return Wb, Ws


def errors(got, ref, W0):
    out = []
    for g, r, w0 in zip(got, ref, W0):
        for s in range(2):
            err = np.max(np.abs(g[s] - r[s])) / np.max(np.abs(r[s]))
            inc = np.linalg.norm((g[s] - w0[s]) - (r[s] - w0[s])) / max(np.linalg.norm(r[s] - w0[s]), 1e-300)
            out.append((float(err), float(inc)))
    return out


FP64_CASES = [
    ("small", wl.dib_cylinder(n=(5, 6, 7), steps=4, seed=81, bulk_noise=1e-2)),
    ("ragged_tiles", wl.dib_cylinder(n=(33, 40, 19), steps=3, seed=82, bulk_noise=1e-2)),
    ("paper_140x140x25", wl.dib_cylinder(steps=20, seed=9)),
]


@pytest.mark.parametrize("name,w", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_dib_fp64_matches_oracle(name, w):
    got = gpu_dib(w, w["steps"])
    ref = oracle_dib(w, w["steps"])
    W0 = (w["Wb"], w["Ws"])
    floor = errors(oracle_dib_rowsum_exact(w, w["steps"]), ref, W0)
    e = errors(got, ref, W0)
    print("state / increment errors (w_u, w_v, r, s):", e, "oracle floor:", floor)
    for (err, inc), (fe, fi) in zip(e, floor):
        assert err <= max(1e-12, 4 * fe) and inc <= max(1e-9, 4 * fi), (e, floor)


SPLIT_CASES = [
    ("small", wl.dib_cylinder(n=(5, 6, 7), steps=4, seed=83, bulk_noise=1e-2)),
    ("ragged_tiles", wl.dib_cylinder(n=(33, 40, 19), steps=3, seed=84, bulk_noise=1e-2)),
]


@pytest.mark.parametrize("name,w", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_dib_split_tf32_matches_oracle(name, w):
    got = gpu_dib(w, w["steps"], precision="split_tf32")
    ref = oracle_dib(w, w["steps"])
    W0 = (w["Wb"], w["Ws"])
    floor = errors(oracle_dib_split_emulated(w, w["steps"]), ref, W0)
    e = errors(got, ref, W0)
    print("state / increment errors (w_u, w_v, r, s):", e, "emulated floor:", floor)
    for (err, inc), (fe, fi) in zip(e, floor):
        assert err <= max(1e-6, 8 * fe) and inc <= max(1e-5, 8 * fi), (e, floor)


def _dib_120x140x25():
    w = wl.dib_cylinder(n=(120, 140, 25), steps=20, seed=85)
    got = gpu_dib(w, w["steps"], precision="split_tf32")
    ref = oracle_dib(w, w["steps"])
    e = errors(got, ref, (w["Wb"], w["Ws"]))
    print("state / increment errors (w_u, w_v, r, s):", e)
    return e


@pytest.mark.xfail(strict=True, reason="known accuracy defect of the split DIB chain near the axis: r, w_u, w_v "
                   "reach ~1e-5 on 120 x 140 x 25 (mechanism in the characterisation test below)")
def test_dib_split_tf32_meets_target_on_120x140x25():
    """The 1e-6 target on the 120 x 140 x 25 grid: not met by this build (strict expected failure, so
    that a fix shows as an unexpected pass)."""
    (wu, wui), (wv, wvi), (r, ri), (s, si) = _dib_120x140x25()
    assert max(wu, wv, r, s) <= 1e-6


def test_dib_split_tf32_characterised_on_120x140x25():
    """Characterisation of the defect, not the 1e-6 target: on the 120 x 140 x 25 grid (rho_* = 15,
    tau = 0.025, 20 steps) the surface species s, which the chain computes directly, stays within
    1e-6 (measured 8.8e-8), but r, w_u, w_v reach ~1e-5 of their own size (measured 0.90-0.99e-5).
    Mechanism: near the axis the F of rough surface data is dominated by the theta-Laplacian (~1e4,
    zero theta-mean); r and w are driven by zeta4 (s - zeta5) with s ~ zeta5 and are ~1e-2 of s, so a
    coherent error in the undamped theta-mean of s reappears ~100x larger in them.  The tensor cores'
    truncating FP32 accumulation biases that cancelling sum; the slab pass of these plans forms the
    theta-mean coefficient by compensated summation on the producers instead (this took the errors
    from 0.8-1.0e-4 to ~1e-5); the rest is attributed to the same truncation in the later products
    (an emulation with the accumulator rounded toward zero per 8-wide K step grows with the steps as
    the GPU error does; with round-to-nearest it decays).  These bounds hold the measured values with
    a margin of ~3 so that a regression shows; the FP64 path is the one to use for this model."""
    (wu, wui), (wv, wvi), (r, ri), (s, si) = _dib_120x140x25()
    assert s <= 1e-6 and si <= 5e-6
    assert max(wu, wv, r) <= 3e-5 and max(wui, wvi, ri) <= 1.2e-5


@pytest.mark.parametrize("precision", ["fp64", "split_tf32"])
def test_dib_single_calls_equal_one_call(precision):
    w = wl.dib_cylinder(n=(9, 12, 8), steps=12, seed=86, bulk_noise=1e-2)
    a = gpu_dib(w, 12, precision)
    b = gpu_dib(w, 12, precision, single_calls=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_dib_equilibrium_stays_fixed():
    """(alpha2, beta2, 0, zeta5) is a fixed point: p vanishes there exactly, q up to the rounding of
    eta4, and the lifted bulk stays 0."""
    w = wl.dib_cylinder(n=(10, 12, 9), steps=10, seed=87)
    w["Ws"] = np.stack([np.zeros_like(w["Ws"][0]), np.full_like(w["Ws"][1], 0.5)])
    got = gpu_dib(w, 10)
    assert np.max(np.abs(got[0])) < 1e-12
    assert np.max(np.abs(got[1] - w["Ws"])) < 1e-12


def test_dib_setup_errors():
    from paper_2604_11558_gb300 import binding
    w = wl.dib_cylinder(n=(5, 6, 7), steps=1, seed=88)
    args = (w["n"], w["d_bulk"], w["bulk_params"], w["d_surface"], w["surface_params"], w["coupling"], w["tau"])
    kw = dict(rho_star=w["rho_star"], reaction="linear", surface_reaction="none", z_star=w["z_star"])
    st = binding.coupled_setup_status
    assert st(*args, geometry="cylinder", **kw) == 0
    assert st(*args, geometry="ball", **kw) == 1                              # the DIB coupling needs a cylinder
    assert st(*args, geometry="cylinder", precision="split_tf32", **kw) == 0
    big = (140, 140, 25)
    assert st(big, *args[1:], geometry="cylinder", precision="split_tf32", **kw) == 5   # n_rho > 128
    assert st(big, *args[1:], geometry="cylinder", **kw) == 0                 # FP64 takes the paper's grid
    assert st(*args[:2], [-1.0, 0.0, 0.0], *args[3:], geometry="cylinder", **kw) == 1   # LINEAR needs S^2 params
