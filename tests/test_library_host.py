"""CPU tests of the C-ABI library: it loads, exports every symbol the header
declares, validates arguments without touching a GPU, and its FP64 setup
stage (axes, phi_1 by Pade, eigenbases) matches the oracle's independent
route (Proposition 1 symmetrisation + numpy eigh) -- row A0 of the hot path.
"""
import os

import numpy as np
import pytest

from oracle import axes as oax
from oracle.phi import phi1_matrix

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    from paper_2604_11558_gb300 import binding as b
    if not os.path.exists(b.LIB_PATH):
        from paper_2604_11558_gb300 import build_lib
        build_lib.build()
    b.lib()
    return b


def test_exports_every_declared_symbol(binding):
    names = binding.header_functions()
    assert len(names) >= 12
    L = binding.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(binding):
    L = binding.lib()
    for code in range(7):
        assert len(L.sexpe_status_string(code)) > 0
    assert L.sexpe_status_string(99) == b"unknown status"


@pytest.mark.parametrize("kw,code", [
    (dict(geometry="disk", n=(10, 12), d=[1.0, 2.0], reaction="schnakenberg", params=[1, 2, 3], tau=-1.0), 1),
    (dict(geometry="disk", n=(10, 12), d=[1.0, 2.0], reaction="schnakenberg", params=[1, 2, 3], tau=float("nan")), 1),
    (dict(geometry="disk", n=(2, 12), d=[1.0, 2.0], reaction="schnakenberg", params=[1, 2, 3], tau=1e-3), 1),
    (dict(geometry="ball", n=(10, 12, 600), d=[1.0, 2.0], reaction="gray_scott", params=[0.04, 0.06], tau=1e-3), 1),
    (dict(geometry="disk", n=(10, 12), d=[1.0, -2.0], reaction="schnakenberg", params=[1, 2, 3], tau=1e-3), 1),
    (dict(geometry="disk", n=(10, 12), d=[1.0], reaction="schnakenberg", params=[1, 2, 3], tau=1e-3), 1),
    (dict(geometry="disk", n=(10, 12), d=[1.0, 2.0], reaction="gray_scott", params=[1, 2, 3], tau=1e-3), 1),
    (dict(geometry="cylinder", n=(8, 8, 8), d=[1.0] * 3, reaction="linear_cubic", params=[0.0] * 4, tau=1e-3), 1),
    (dict(geometry="disk", n=(10, 12), d=[1.0] * 5, reaction="none", params=[], tau=1e-3), 1),
    (dict(geometry="disk", n=(10, 12), d=[1.0, 1.0], reaction="none", params=[], tau=1e-3, rho_star=0.0), 1),
])
def test_setup_rejects_invalid_arguments(binding, kw, code):
    assert binding.setup_status(**kw) == code


def test_null_pointers_rejected(binding):
    L = binding.lib()
    assert L.sexpe_step(None, None, 1, None) == 1
    assert L.sexpe_destroy(None) == 1
    assert L.sexpe_synchronize(None, None) == 1
    assert L.sexpe_axis_matrix(9, 5, 1.0, None) == 1


AXES = {"theta": lambda n: oax.theta_axis(n)[1], "rho2": lambda n: oax.rho2_axis(n)[1],
        "rho3": lambda n: oax.rho3_axis(n)[1], "phi": lambda n: oax.phi_axis(n)[1],
        "z_neumann": lambda n: oax.z_axis_neumann(n)[1], "z_paper": lambda n: oax.z_axis_paper(n)[1]}


@pytest.mark.parametrize("axis", list(AXES))
def test_axis_matrices_match_oracle(binding, axis):
    for n in [3, 7, 32, 100]:
        A = binding.axis_matrix(axis, n)
        R = AXES[axis](n)
        assert np.max(np.abs(A - R)) <= 1e-13 * np.max(np.abs(R))


@pytest.mark.parametrize("axis", list(AXES))
@pytest.mark.parametrize("t", [1e-5, 1e-3, 0.05, 2.0])
def test_pade_phi1_matches_oracle_eigen_route(binding, axis, t):
    """Two independent phi_1 routes: Pade [13/13] on [[tA, I], [0, 0]] (library) and
    V diag(phi_1(t lam)) V^{-1} through Proposition 1 (oracle)."""
    # ||t A|| reaches ~1e5 at t = 2, n = 100: 14 squarings; both routes then agree to a few 1e-12
    tol = 1e-12 if t <= 0.05 else 5e-12
    for n in [5, 33, 100]:
        P = binding.axis_phi1(axis, n, t)
        R = phi1_matrix(AXES[axis](n), t)
        assert np.max(np.abs(P - R)) <= tol * np.max(np.abs(R)), (axis, n, t)


@pytest.mark.parametrize("axis", list(AXES))
def test_library_eigenbasis(binding, axis):
    for n in [4, 9, 64, 100]:
        lam, V, Vinv = binding.axis_eigen(axis, n)
        A = AXES[axis](n)
        scale = np.max(np.abs(A))
        assert np.max(np.abs(V @ Vinv - np.eye(n))) < 1e-11
        assert np.max(np.abs((V * lam) @ Vinv - A)) < 1e-11 * scale
        ref = np.sort(np.linalg.eigvals(A).real)
        assert np.max(np.abs(np.sort(lam) - ref)) < 1e-10 * scale
    if axis == "theta":      # orthogonal real Fourier basis: V^{-1} = V^T
        assert np.allclose(Vinv, V.T, atol=1e-14)


def test_batch_setup_rejects_invalid(binding):
    from paper_2604_11558_gb300 import workloads as wl
    good = wl.schnakenberg_disk(n=(10, 12), steps=1)
    ball = wl.gray_scott_ball(n=(5, 6, 7), steps=1)
    assert binding.batch_setup_status([good, ball]) == 1                  # not a disk
    bad = dict(good, d=[1.0, -1.0])
    assert binding.batch_setup_status([good, bad]) == 1                   # negative diffusion
    big = wl.schnakenberg_disk(n=(10, 300), steps=1)
    assert binding.batch_setup_status([big]) == 5                         # theta > 256 unsupported
    assert binding.batch_setup_status([good], precision="fp64") == 5      # batched FP64 not built


def test_coupled_setup_rejects_invalid(binding):
    """sexpe_coupled_setup validates everything on the host before it touches a GPU."""
    from paper_2604_11558_gb300 import workloads as wl
    b = wl.bulk_surface_ball(n=(5, 6, 7), steps=1)
    ball = dict(n=b["n"], d_bulk=b["d_bulk"], bulk_params=b["bulk_params"], d_surface=b["d_surface"],
                surface_params=b["surface_params"], coupling=b["coupling"], tau=b["tau"])
    st = binding.coupled_setup_status
    assert st(**dict(ball, precision="unsplit_fp64")) == 5
    assert st(**dict(ball, d_bulk=[1.0, 10.0, 3.0])) == 1                         # three bulk species
    assert st(**dict(ball, d_surface=[1.0])) == 1                                 # one surface species
    assert st(**dict(ball, coupling=dict(b["coupling"], zeta2=float("nan")))) == 1
    assert st(**dict(ball, coupling=dict(b["coupling"], eta2=float("inf")))) == 1
    assert st(**dict(ball, tau=0.0)) == 1
    assert st(**dict(ball, n=(5, 2, 7))) == 1                                     # theta < 3
    assert st(**dict(ball, geometry="cylinder")) == 1                             # the ball kind needs a ball
    assert st(**dict(ball, reaction="bvam_manufactured", bulk_params=[1.0, 0.2, 0.2, 1.0, 1.0])) == 1
    d = wl.dib_cylinder(n=(5, 6, 7), steps=1)
    dib = dict(n=d["n"], d_bulk=d["d_bulk"], bulk_params=d["bulk_params"], d_surface=d["d_surface"],
               surface_params=d["surface_params"], coupling=d["coupling"], tau=d["tau"], rho_star=d["rho_star"],
               reaction=d["bulk_reaction"], surface_reaction=d["surface_reaction"], geometry="cylinder",
               z_star=d["z_star"])
    assert st(**dict(dib, geometry="ball")) == 1                                  # the DIB kind needs a cylinder
    assert st(**dict(dib, z_bc="neumann")) == 1                                   # and the Dirichlet top of A_z
    assert st(**dict(dib, z_star=-1.0)) == 1
    assert st(**dict(dib, bulk_params=[-1.0, 0.0, 0.0])) == 1                     # LINEAR takes S^2 params
    assert st(**dict(dib, coupling=dict(d["coupling"], alpha3=float("nan")))) == 1
    assert st(**dict(dib, coupling=dict(d["coupling"], u_top=float("inf")))) == 1
    assert st(**dict(dib, precision="unsplit_fp64")) == 5
    L = binding.lib()
    assert L.sexpe_coupled_setup(None, None, None, None, 1e-3, 0, None, None) == 1


def test_coupling_terms_match_the_oracles(binding):
    """The coupling arithmetic the kernels run (shared with sexpe_coupling_terms, host evaluation)
    against the two coupled oracles, point by point: Section 5.5 (ball + sphere, rho_* = 0.8) and
    Section 5.6 (cylinder + bottom disk, lifted bulk)."""
    from oracle.coupled import Coupled
    from oracle.coupled_dib import CoupledCylinder
    from paper_2604_11558_gb300 import workloads as wl
    rng = np.random.default_rng(31)
    # Section 5.5
    n = (6, 8, 7)
    c = Coupled(n, 1e-3, delta=10.0, rho_star=0.8)
    Wb = 1.0 + 0.3 * rng.standard_normal((2,) + c.ball.shape)
    Ws = 1.0 + 0.3 * rng.standard_normal((2,) + c.sphere.shape)
    ab, as_ = c.coupling(Wb, Ws)
    b = wl.bulk_surface_ball(n=n, steps=1)
    got = binding.coupling_terms("ball", n, [1.0, 10.0], b["coupling"], Wb[0][:, :, -1], Wb[1][:, :, -1],
                                 Ws[0], Ws[1], rho_star=0.8)
    ref = [ab[0][:, :, -1], ab[1][:, :, -1], as_[0], as_[1]]
    for g, r in zip(got, ref):
        assert np.allclose(g, r.ravel(), rtol=1e-14, atol=1e-14 * np.abs(r).max())
    # Section 5.6
    d = wl.dib_cylinder(n=(6, 8, 7), steps=1)
    cc = CoupledCylinder(d["n"], d["tau"], rho_star=d["rho_star"], z_star=d["z_star"], **d["oracle_params"])
    Wb = 0.05 * rng.standard_normal((2,) + cc.bulk.shape)
    Ws = np.stack([0.1 * rng.uniform(0, 1, cc.surface.shape), 0.5 + 0.1 * rng.uniform(0, 1, cc.surface.shape)])
    ab, as_ = cc.coupling(Wb, Ws)
    got = binding.coupling_terms("cylinder", d["n"], d["d_bulk"], d["coupling"], Wb[0][0], Wb[1][0], Ws[0], Ws[1],
                                 rho_star=d["rho_star"], z_star=d["z_star"])
    ref = [ab[0][0], ab[1][0], as_[0], as_[1]]
    for g, r in zip(got, ref):
        assert np.allclose(g, r.ravel(), rtol=1e-13, atol=1e-13 * np.abs(r).max())
    # arguments are checked on the host
    with pytest.raises(RuntimeError):
        binding.coupling_terms("ball", d["n"], d["d_bulk"], d["coupling"], Wb[0][0], Wb[1][0], Ws[0], Ws[1])
    L = binding.lib()
    assert L.sexpe_coupling_terms(None, None, None, 0, *([None] * 8)) == 1
