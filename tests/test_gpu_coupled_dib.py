"""GPU parity of the bulk-surface DIB step on the cylinder and its bottom disk (Section 5.6, eqs.
bulkcyl) against the oracle's ``CoupledCylinder``.

Bulk w = (u - alpha2, v - beta2) on the cylinder with the Dirichlet top of eq. A_z (LINEAR reaction
K = diag(-alpha1, -beta1)), surface r, s on the bottom disk; the DIB kinetics p, q and the bottom
fluxes -zeta1 alpha3 p, -zeta1 beta3 q are formed by the coupling kernel, explicit at t_n; each
component then takes its own split step (eqs. ee_cylinder, ee_disk).  FP64: state within 1e-12 of
its largest value, increment W_n - W_0 within 1e-9 relative.  Split-TF32 (n_rho <= 128): state
within 1e-6, increment within 1e-5.
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


def check(got, ref, W0, tol_state, tol_incr):
    errs = []
    for g, r, w0 in zip(got, ref, W0):
        assert np.all(np.isfinite(g))
        for s in range(2):
            err = np.max(np.abs(g[s] - r[s])) / np.max(np.abs(r[s]))
            inc = np.linalg.norm((g[s] - w0[s]) - (r[s] - w0[s])) / max(np.linalg.norm(r[s] - w0[s]), 1e-300)
            errs.append((float(err), float(inc)))
    print("state / increment errors (w_u, w_v, r, s):", errs)
    for err, inc in errs:
        assert err <= tol_state, errs
        assert inc <= tol_incr, errs


FP64_CASES = [
    ("small", wl.dib_cylinder(n=(5, 6, 7), steps=4, seed=81, bulk_noise=1e-2)),
    ("ragged_tiles", wl.dib_cylinder(n=(33, 40, 19), steps=3, seed=82, bulk_noise=1e-2)),
    ("paper_140x140x25", wl.dib_cylinder(steps=20, seed=9)),
]


@pytest.mark.parametrize("name,w", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_dib_fp64_matches_oracle(name, w):
    got = gpu_dib(w, w["steps"])
    ref = oracle_dib(w, w["steps"])
    check(got, ref, (w["Wb"], w["Ws"]), 1e-12, 1e-9)


SPLIT_CASES = [
    ("small", wl.dib_cylinder(n=(5, 6, 7), steps=4, seed=83, bulk_noise=1e-2)),
    ("ragged_tiles", wl.dib_cylinder(n=(33, 40, 19), steps=3, seed=84, bulk_noise=1e-2)),
    ("120x140x25", wl.dib_cylinder(n=(120, 140, 25), steps=20, seed=85)),
]


@pytest.mark.parametrize("name,w", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_dib_split_tf32_matches_oracle(name, w):
    got = gpu_dib(w, w["steps"], precision="split_tf32")
    ref = oracle_dib(w, w["steps"])
    check(got, ref, (w["Wb"], w["Ws"]), 1e-6, 1e-5)


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
