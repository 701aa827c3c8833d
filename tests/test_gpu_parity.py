"""GPU parity of the split exponential Euler step against the FP64 oracle.

Every case runs the CUDA path through the C-ABI binding and the oracle on the
same seeded inputs and compares element by element.  Tolerances:
* FP64 path: 1e-12 relative per species (the stated target).
* split-TF32 path, smooth or patch data: 1e-6 relative per species (the
  stated target); the increment W_n - W_0 within 1e-5 relative (three TF32
  products per mu-mode product carry ~2^-21 relative error each, times the
  3-5 products of the chain and the FP32 rounding of F).
* split-TF32 path on rough random data, where the strongly damped phi_1
  factors amplify the relative error of every FP32 intermediate: per species
  within max(1e-6, 8 x the error of the oracle run with F, every direction's
  result and the increment rounded to FP32) -- the storage-precision floor
  of any FP32-intermediate chain, times the 3xTF32 product factor.
* split-TF32 over hundreds of steps: whole-state relative error within 1e-6;
  a species that decays towards zero (here to ~1e-12) accumulates the bias of
  the tensor cores' truncating FP32 accumulation, so it is held to 4x an
  emulation of that arithmetic.
Sizes span several 128-row tiles and 16-wide K-chunks with ragged tails, the
two-tile theta case (n_theta > 128), the largest supported sizes and n = 3.
"""
import numpy as np
import pytest

from paper_2604_11558_gb300 import workloads as wl
from tests.gpu_helpers import (assert_parity, emulated_fp32_errors, gpu_run, increment_errors, oracle_run,
                               rel_errors)

pytestmark = pytest.mark.gpu


def disk(n, steps=5, seed=11):
    return wl.schnakenberg_disk(n=n, steps=steps, seed=seed)


def sphere(n, steps=5, seed=12):
    return wl.schnakenberg_sphere(n=n, steps=steps, seed=seed)


def ball(n, steps=5, seed=13, tau=0.5):
    return wl.gray_scott_ball(n=n, steps=steps, seed=seed, tau=tau)


def cyl(n, steps=5, seed=14):
    return wl.linear_cubic_cylinder(n=n, steps=steps, seed=seed)


FP64_CASES = [
    ("disk", disk((13, 20))),
    ("disk_cfg0_full", disk((32, 64), steps=200, seed=2)),
    ("sphere", sphere((24, 13))),
    ("sphere_min", sphere((3, 3))),
    ("ball", ball((11, 13, 10))),
    ("ball_min", ball((3, 3, 3))),
    ("cylinder", cyl((9, 14, 11))),
    ("cylinder_dirichlet_cap", dict(cyl((9, 14, 11)), z_bc="paper")),
]


@pytest.mark.parametrize("name,w", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_matches_oracle(name, w):
    got = gpu_run(w, "fp64")
    ref = oracle_run(w)
    assert_parity(got, ref, w["W0"], 1e-12, 1e-10)


SPLIT_CASES = [
    ("disk", disk((37, 45))),
    ("disk_two_theta_tiles", disk((40, 200))),
    ("disk_min", disk((3, 3))),
    ("disk_rho128_theta136", disk((128, 136))),
    ("ball", ball((20, 33, 40))),
    ("ball_rho128", ball((128, 16, 16), steps=3)),
    ("ball_phi256", ball((8, 12, 256), steps=3)),
    ("ball_min", ball((3, 3, 3))),
    ("sphere", sphere((24, 13))),
    ("sphere_min", sphere((3, 3))),
    ("sphere_two_theta_tiles", sphere((130, 70))),
]


@pytest.mark.parametrize("name,w", SPLIT_CASES, ids=[c[0] for c in SPLIT_CASES])
def test_split_tf32_matches_oracle(name, w):
    got = gpu_run(w, "split_tf32")
    ref = oracle_run(w)
    assert_parity(got, ref, w["W0"], 1e-6, 1e-5)


ROUGH_CASES = [
    ("cylinder", cyl((24, 40, 37))),
    ("cylinder_theta256", cyl((16, 256, 18), steps=3)),
    ("sphere_theta256_phi300", sphere((256, 300), steps=3)),
]


@pytest.mark.parametrize("name,w", ROUGH_CASES, ids=[c[0] for c in ROUGH_CASES])
def test_split_tf32_rough_data_within_fp32_floor(name, w):
    """State within max(1e-6, 8 x floor) and increment W_n - W_0 within max(1e-5, 8 x its floor),
    the floors being the oracle's own errors with FP32 storage of every intermediate."""
    got = gpu_run(w, "split_tf32")
    ref = oracle_run(w)
    floor, ifloor = emulated_fp32_errors(w, ref, increments=True)
    e, ie = rel_errors(got, ref), increment_errors(got, ref, w["W0"])
    print(name, "split errors", e, ie, "fp32-storage floors", floor, ifloor)
    for s in range(len(e)):
        assert e[s] <= max(1e-6, 8 * floor[s]), (s, e, floor)
        assert ie[s] <= max(1e-5, 8 * ifloor[s]), (s, ie, ifloor)


def test_sphere_full_size_split():
    """The 256 x 512 sphere of the differentiation workload on the split path, a few steps.  The
    relative 2-norm error of the state is held to 1e-6.  This field is noisy and the theta terms
    next to the poles carry sin^-2 phi factors of ~10^4, so elementwise and increment errors are
    held to 8 x the oracle's own errors with FP32 storage of every intermediate (the worst points
    of both sit on the first and last phi rows)."""
    from oracle.stepper import Problem, run
    from oracle.operators import Grid
    from tests.gpu_helpers import oracle_reaction
    w = wl.schnakenberg_sphere(steps=3)
    ref = oracle_run(w)
    got = gpu_run(w, "split_tf32")
    assert np.all(np.isfinite(got))
    e = rel_errors(got, ref)
    assert max(e) <= 1e-6, e
    p = Problem(Grid(w["geometry"], w["n"]), w["d"], oracle_reaction(w), w["tau"])
    emu = run(p, w["W0"], w["steps"], fp32_storage=True)
    for s in range(2):
        m = np.max(np.abs(ref[s]))
        em, fm = np.max(np.abs(got[s] - ref[s])) / m, np.max(np.abs(emu[s] - ref[s])) / m
        ie, fi = increment_errors(got, ref, w["W0"])[s], increment_errors(emu, ref, w["W0"])[s]
        print("sphere 256x512 species", s, "max-abs", em, "floor", fm, "increment", ie, "floor", fi)
        assert em <= max(1e-6, 8 * fm), (s, em, fm)
        assert ie <= max(1e-5, 8 * fi), (s, ie, fi)


def test_ball_full_size_split_and_fp64():
    """The 100^3 ball workload in the launch configuration the benchmark times, a few steps."""
    w = wl.gray_scott_ball(steps=3)
    ref = oracle_run(w)
    assert_parity(gpu_run(w, "split_tf32"), ref, w["W0"], 1e-6, 1e-5)
    assert_parity(gpu_run(w, "fp64", steps=3), ref, w["W0"], 1e-12, 1e-10)


def test_cylinder_full_size_split():
    w = wl.linear_cubic_cylinder(steps=2)
    ref = oracle_run(w)
    got = gpu_run(w, "split_tf32")
    floor = emulated_fp32_errors(w, ref)
    e = rel_errors(got, ref)
    print("cylinder 64x128x128 split errors", e, "fp32-storage floor", floor)
    for s in range(len(e)):
        assert e[s] <= max(1e-6, 8 * floor[s]), (s, e, floor)


def test_ball_500_steps_split_vs_oracle_reduced_grid():
    """Final-time parity over the full step count on a reduced ball (oracle in seconds).  The whole
    state and u are held to the 1e-6 target.  The decaying species v (to ~1e-12 at t_* = 250) is held
    to 4x an emulation of the chain's arithmetic (tests/precision_emulation.py: F and intermediates
    FP32, three TF32 products per product, the accumulator rounded toward zero after every 8-wide
    K step as in the tensor cores; the rho direction as one plain phi_1 product as on the GPU):
    truncation biases every product's magnitude low, and v's relative error accumulates that bias
    over the steps (the full-size ball at t_* is tested in tests/test_gpu_final_time.py)."""
    from oracle.operators import Grid
    from oracle.stepper import Problem
    from tests.gpu_helpers import oracle_reaction
    from tests.precision_emulation import run as emulate
    w = wl.gray_scott_ball(n=(24, 20, 16), steps=500)
    ref = oracle_run(w)
    got = gpu_run(w, "split_tf32")
    whole = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    e = rel_errors(got, ref)
    g = Grid(w["geometry"], w["n"])
    emu = emulate(Problem(g, w["d"], oracle_reaction(w, g), w["tau"]), w["W0"], w["steps"], accumulate="rz8",
                  plain=(1,))
    fe = rel_errors(emu, ref)
    print("split vs oracle, ball 24x20x16, 500 steps: whole", whole, "per species", e, "emulated", fe)
    assert whole <= 1e-6
    assert e[0] <= 1e-6
    assert e[1] <= max(1e-6, 4 * fe[1])


def test_graph_replay_equals_single_steps():
    w = ball((20, 33, 40), steps=25)
    a = gpu_run(w, "split_tf32")
    b = gpu_run(w, "split_tf32", single_calls=True)
    assert np.array_equal(a, b)
    w = disk((13, 20), steps=23)
    assert np.array_equal(gpu_run(w, "fp64"), gpu_run(w, "fp64", single_calls=True))


def test_step_host_equals_step():
    import torch
    from paper_2604_11558_gb300 import binding
    w = ball((20, 33, 40), steps=4)
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    host = torch.from_numpy(w["W0"].copy()).pin_memory()
    plan.step_host(host, 4)
    dev = gpu_run(w, "split_tf32")
    assert np.array_equal(host.numpy(), dev)
    plan.close()


def test_unsupported_and_invalid_on_gpu():
    from paper_2604_11558_gb300 import binding
    assert binding.setup_status("sphere", (300, 16), [1.0, 2.0], "schnakenberg", [1, 2, 3], 1e-3,
                                "split_tf32") == 5
    assert binding.setup_status("ball", (130, 16, 16), [1.0, 2.0], "gray_scott", [0.04, 0.06], 1e-3,
                                "split_tf32") == 5
    assert binding.setup_status("disk", (16, 300), [1.0, 2.0], "schnakenberg", [1, 2, 3], 1e-3,
                                "split_tf32") == 5


def test_plan_info_reports_measured_tile_choices():
    """The split plan times every feasible stencil tile height at setup and keeps the fastest."""
    from paper_2604_11558_gb300 import binding
    for w in (ball((20, 24, 18)), disk((30, 40))):
        plan = binding.Plan.from_workload(w, precision="split_tf32")
        inf = plan.info()
        plan.close()
        assert 1 <= inf["stencil_tile_j"] <= min(32, w["n"][1])
        assert inf["stencil_tile_us"] > 0
        assert inf["ring_slots"][0] >= 2 and inf["ring_slots"][1] >= 2


STENCIL_CASES = [
    ("ball", ball((37, 29, 23)), [(1, 0), (7, 0), (2, 2), (4, 4), (10, 8, 2), (16, 16), (24, 2, 2),
                                  (1, 2, 0), (5, 3, 0), (24, 16, 0)]),
    ("cylinder", cyl((24, 40, 37), steps=3), [(3, 0), (2, 16, 2), (8, 4), (24, 8, 2), (3, 4, 0), (20, 12, 0)]),
    ("ball_even_rho", ball((36, 29, 23)), [(7, 0), (4, 4), (10, 8, 2), (1, 2, 0), (5, 3, 0), (24, 16, 0)]),
]


@pytest.mark.parametrize("name,w,configs", STENCIL_CASES, ids=[c[0] for c in STENCIL_CASES])
def test_every_stencil_configuration_matches_oracle(name, w, configs):
    """The stencil kernels (tiled: planes = 0; rolling window: planes > 0, registers capped for one
    or two CTAs per SM; k-marching: planes > 0, ctas_per_sm = 0, with one column per thread for odd
    n_rho and two for even n_rho), forced through sexpe_set_stencil at several tile shapes with ragged last
    tiles, give the oracle's result; the
    F they write is the same whatever the shape (the rest of the step is identical)."""
    ref = oracle_run(w)
    outs = []
    for cfg in configs:
        got = gpu_run(w, "split_tf32", stencil=cfg)
        if name.startswith("ball"):
            assert_parity(got, ref, w["W0"], 1e-6, 1e-5)
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_march_stencil_state_alignment():
    """A state that is 8- but not 16-byte aligned takes the one-column marching kernel (the
    two-column kernel's 16-byte copies need 16-byte alignment): same result bit for bit."""
    import torch
    from paper_2604_11558_gb300 import binding
    w = ball((36, 29, 23), steps=4)
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    plan.set_stencil(5, 3, 0)
    x = torch.from_numpy(np.ascontiguousarray(w["W0"])).cuda()
    buf = torch.zeros(x.numel() + 1, dtype=torch.float64, device="cuda")
    y = buf[1:].view(x.shape)
    y.copy_(x)
    assert x.data_ptr() % 16 == 0 and y.data_ptr() % 16 == 8
    plan.step(x, w["steps"])
    plan.step(y, w["steps"])
    plan.synchronize()
    assert torch.equal(x, y)
    plan.close()


SPECIES_CASES = [
    ("cylinder_1species", wl.linear_cubic_cylinder(n=(20, 24, 18), steps=3, seed=21, d=(2e-3,)),
     [(3, 0), (2, 4, 2), (4, 3, 0), (16, 8, 0)]),
    ("cylinder_4species", wl.linear_cubic_cylinder(n=(20, 24, 18), steps=3, seed=22, d=(1e-3, 3e-3, 5e-3, 2e-2)),
     [(3, 0), (2, 4, 1), (5, 3, 0), (16, 6, 0)]),
]


@pytest.mark.parametrize("name,w,configs", SPECIES_CASES, ids=[c[0] for c in SPECIES_CASES])
def test_species_counts_every_stencil_kernel(name, w, configs):
    """One and four species (the marching stencil is instantiated per species count): every stencil
    kernel gives the same F, and the step stays within 8x the FP32-storage floor of the oracle
    (rough N(0, 0.01^2) data, as for the 3-species cylinder)."""
    ref = oracle_run(w)
    floor = emulated_fp32_errors(w, ref)
    outs = [gpu_run(w, "split_tf32", stencil=cfg) for cfg in configs]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    e = rel_errors(outs[0], ref)
    for s in range(len(e)):
        assert e[s] <= max(1e-6, 8 * floor[s]), (s, e, floor)


def test_every_theta_split_matches_oracle():
    """The sphere's theta kernel with its output columns split over 1, 2, 4 and 8 CTAs (120 theta
    points padded to 128: 128, 64, 32 and 16 columns per CTA, the last group ragged; 150 phi rows,
    two row tiles) gives the oracle's result, and the same result at every split (each column's
    products see the same operands in the same order)."""
    w = sphere((120, 150), steps=4)
    ref = oracle_run(w)
    outs = []
    for split in (1, 2, 4, 8):
        got = gpu_run(w, "split_tf32", theta_split=split)
        assert_parity(got, ref, w["W0"], 1e-6, 1e-5)
        outs.append(got)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_set_theta_split_rejects_unbuilt_splits():
    from paper_2604_11558_gb300 import binding
    w = sphere((130, 70))
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    assert plan.info()["theta_split"] == 1     # 144 padded columns: only the unsplit kernel
    for bad in (0, 2, 3, 16):
        with pytest.raises(RuntimeError):
            plan.set_theta_split(bad)
    plan.set_theta_split(1)
    plan.close()
    for other, prec in ((sphere((24, 13)), "fp64"), (ball((20, 24, 18)), "split_tf32")):
        p = binding.Plan.from_workload(other, precision=prec)
        assert p.info()["theta_split"] == 0
        with pytest.raises(RuntimeError):
            p.set_theta_split(1)
        p.close()


def test_set_stencil_rejects_untimed_configurations():
    from paper_2604_11558_gb300 import binding
    w = ball((20, 24, 18))
    plan = binding.Plan.from_workload(w, precision="split_tf32")
    for bad in [(0, 0), (17, 0), (3, 2), (4, 3), (4, 32), (40, 2), (4, 4, 3), (4, 0, 2), (4, 5, 0), (30, 2, 0),
                (4, 0, 0)]:
        with pytest.raises(RuntimeError):
            plan.set_stencil(*bad)
    plan.set_stencil(4, 4)
    assert plan.info()["stencil_planes"] == 4 and plan.info()["stencil_tile_j"] == 4
    plan.set_stencil(6, 3, 0)
    inf = plan.info()
    assert (inf["stencil_tile_j"], inf["stencil_planes"], inf["stencil_ctas_per_sm"]) == (6, 3, 0)
    plan.close()
    p64 = binding.Plan.from_workload(w, precision="fp64")
    with pytest.raises(RuntimeError):
        p64.set_stencil(4, 0)
    p64.close()
