"""Seeded synthetic inputs for the benchmark and parity workloads.

This module holds random draws and constants only: none of the method's
arithmetic (no grids, matrices, phi_1 or reaction evaluation).  Both the
CUDA path's tests/bench and the CPU oracle's tests take their inputs from
here, so the two sides see bit-identical initial data.

Every workload is a plain dict:

    geometry   'disk' | 'sphere' | 'ball' | 'cylinder'
    n          points per mode, mode 1 first (disk: (n_rho, n_theta),
               sphere: (n_theta, n_phi), ball: (n_rho, n_theta, n_phi),
               cylinder: (n_rho, n_theta, n_z))
    d          diffusion coefficient per species
    reaction   'schnakenberg' | 'gray_scott' | 'linear_cubic' | 'none'
    params     reaction parameters (see below)
    tau, steps time step and number of steps
    W0         float64 array (S, *reversed(n)): mode 1 is the last axis
    seed       numpy PCG64 seed

Reaction parameters: schnakenberg (gamma, a, b); gray_scott (F, k);
linear_cubic (K as a row-major S x S list).
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _shape(n):
    return tuple(reversed(tuple(n)))


def schnakenberg_disk(n=(32, 64), steps=200, seed=2, gamma=100.0, a=0.1, b=0.9, d=(1.0, 10.0), tau=1e-4):
    """Polar disk, Schnakenberg, steady state (a+b, b/(a+b)^2) plus U(-0.01, 0.01) noise per point."""
    rng = _rng(seed)
    shp = _shape(n)
    u = (a + b) + rng.uniform(-0.01, 0.01, shp)
    v = b / (a + b) ** 2 + rng.uniform(-0.01, 0.01, shp)
    return dict(geometry="disk", n=tuple(n), d=list(d), reaction="schnakenberg", params=[gamma, a, b],
                tau=tau, steps=steps, W0=np.stack([u, v]), seed=seed, name="disk_schnakenberg")


def gray_scott_ball(n=(100, 100, 100), steps=500, seed=3, F=0.04, k=0.06, d=(2e-3, 1e-3), tau=0.5):
    """Ball, Gray-Scott: u = 1, v = 0 except a seeded patch where v = 0.25 + U(-0.01, 0.01).

    The patch is a box in index space: each side about a fifth of the points
    of its mode, at a uniformly drawn corner (periodic wrap along theta,
    clipped along rho and phi).
    """
    rng = _rng(seed)
    shp = _shape(n)
    u = np.ones(shp)
    v = np.zeros(shp)
    n1, n2, n3 = n
    w1, w2, w3 = max(1, n1 // 5), max(1, n2 // 5), max(1, n3 // 5)
    i0 = int(rng.integers(0, n1 - w1 + 1))
    j0 = int(rng.integers(0, n2))
    k0 = int(rng.integers(0, n3 - w3 + 1))
    noise = rng.uniform(-0.01, 0.01, (w3, w2, w1))
    for jl in range(w2):
        v[k0:k0 + w3, (j0 + jl) % n2, i0:i0 + w1] = 0.25 + noise[:, jl, :]
    return dict(geometry="ball", n=tuple(n), d=list(d), reaction="gray_scott", params=[F, k],
                tau=tau, steps=steps, W0=np.stack([u, v]), seed=seed, name="ball_gray_scott")


def linear_cubic_cylinder(n=(64, 128, 128), steps=1000, seed=4, d=(1e-3, 5e-3, 20e-3), tau=0.05):
    """Cylinder, 3 species, f_i = sum_j K_ij u_j - u_i^3 with K = N(0, 0.5^2) + 0.5 I; u_i ~ N(0, 0.01^2)."""
    rng = _rng(seed)
    S = len(d)
    K = rng.normal(0.0, 0.5, (S, S)) + 0.5 * np.eye(S)
    W0 = rng.normal(0.0, 0.01, (S,) + _shape(n))
    return dict(geometry="cylinder", n=tuple(n), d=list(d), reaction="linear_cubic",
                params=[float(x) for x in K.ravel()], tau=tau, steps=steps, W0=W0, seed=seed,
                name="cylinder_linear_cubic")


def batched_disks(count=256, steps=500, seed=5, n_rho=(16, 96), n_theta=(32, 256), gamma=100.0, tau=1e-4):
    """Independent Schnakenberg disks of uneven sizes.

    Per instance: n_rho ~ U{16..96}, n_theta ~ U{32..256}, a ~ U(0.05, 0.2),
    b ~ U(0.7, 1.0), d_v ~ U(8, 20), d_u = 1, gamma = 100; steady state plus
    U(-0.01, 0.01) noise.  Returns a list of workload dicts.
    """
    rng = _rng(seed)
    out = []
    for _ in range(count):
        nr = int(rng.integers(n_rho[0], n_rho[1] + 1))
        nt = int(rng.integers(n_theta[0], n_theta[1] + 1))
        a = float(rng.uniform(0.05, 0.2))
        b = float(rng.uniform(0.7, 1.0))
        dv = float(rng.uniform(8.0, 20.0))
        shp = (nt, nr)
        u = (a + b) + rng.uniform(-0.01, 0.01, shp)
        v = b / (a + b) ** 2 + rng.uniform(-0.01, 0.01, shp)
        out.append(dict(geometry="disk", n=(nr, nt), d=[1.0, dv], reaction="schnakenberg",
                        params=[gamma, a, b], tau=tau, steps=steps, W0=np.stack([u, v]), seed=seed,
                        name="batched_disks"))
    return out


def schnakenberg_sphere(n=(256, 512), steps=1000, seed=6, gamma=200.0, a=0.1, b=0.9, d=(1.0, 10.0), tau=1e-4):
    """Unit sphere (Laplace-Beltrami), Schnakenberg, steady state plus U(-0.01, 0.01) noise."""
    rng = _rng(seed)
    shp = _shape(n)
    noise = rng.uniform(-0.01, 0.01, (2,) + shp)
    u = (a + b) + noise[0]
    v = b / (a + b) ** 2 + noise[1]
    return dict(geometry="sphere", n=tuple(n), d=list(d), reaction="schnakenberg", params=[gamma, a, b],
                tau=tau, steps=steps, W0=np.stack([u, v]), seed=seed, name="sphere_schnakenberg",
                noise=noise)


def anomalous_disk(n=(160, 160), steps=25000, seed=7, lam=-1.95, tau=1e-5):
    """Schnakenberg with anomalous diffusion on the unit disk (Section 5.3, eq. schnak):
    u_t = Delta_lambda u + alpha1 b(u, v), v_t = delta Delta_lambda v + alpha1 c(u, v),
    b = alpha2 - u + u^2 v, c = beta1 - u^2 v, alpha1 = 500, alpha2 = 0.14, beta1 = 1.34,
    delta = 50, lambda = -1.95; boundary values (u_e, v_e) = (alpha2 + beta1, beta1/(alpha2 + beta1)^2),
    the uniform steady state.  The state is lifted, w = (u - u_e, v - v_e), with homogeneous
    Dirichlet boundary values; the reaction sees w + (u_e, v_e).  Initial data: 1e-5 U(0, 1) per
    point and species.  (The paper does not state tau; 25000 steps are its step count.)"""
    rng = _rng(seed)
    a1, a2, b1, delta = 500.0, 0.14, 1.34, 50.0
    ue, ve = a2 + b1, b1 / (a2 + b1) ** 2
    shp = _shape(n)
    W0 = np.stack([1e-5 * rng.uniform(0.0, 1.0, shp), 1e-5 * rng.uniform(0.0, 1.0, shp)])
    return dict(geometry="disk", n=tuple(n), d=[1.0, delta], reaction="schnakenberg", params=[a1, a2, b1],
                tau=tau, steps=steps, W0=W0, seed=seed, lam=lam, offsets=[ue, ve], name="anomalous_disk")


def random_state(geometry, n, S=2, seed=7, scale=0.1, offset=0.5):
    """Generic seeded field for parity tests: offset + scale * N(0, 1) per point and species."""
    rng = _rng(seed)
    return offset + scale * rng.standard_normal((S,) + _shape(n))


def bulk_surface_ball(n=(30, 50, 30), steps=150000, seed=8, tau=1e-4):
    """Bulk-surface Schnakenberg on the unit ball and its boundary sphere (Section 5.5, eqs. bulkball):
    bulk u, v on the ball n = (n_rho, n_theta, n_phi) with diffusion (1, delta) and reaction
    alpha1 (b, c); surface r, s on the ball's theta x phi grid with diffusion (1, eps) / rho_*^2 and
    reaction zeta1 (b, c); alpha1 = zeta1 = 55, alpha2 = 0.1, beta1 = 0.9, zeta2 = zeta3 = 5/12,
    eta1 = eta2 = 5, delta = eps = 10, rho_* = 1.  Initial data: the homogeneous equilibrium
    (alpha2 + beta1, beta1 / (alpha2 + beta1)^2) for both pairs plus 1e-3 N(0, 1) per point and
    species.  t_* = 15 in 150000 steps (tau = 1e-4).  Wb: (2, n_phi, n_theta, n_rho), Ws: (2, n_phi,
    n_theta); the flat state is Wb then Ws."""
    rng = _rng(seed)
    a1, a2, b1, delta, eps = 55.0, 0.1, 0.9, 10.0, 10.0
    z1, z2, z3, e1, e2 = 55.0, 5.0 / 12.0, 5.0 / 12.0, 5.0, 5.0
    ue, ve = a2 + b1, b1 / (a2 + b1) ** 2
    shb, shs = _shape(n), _shape(n[1:])
    eq = np.array([ue, ve])[:, None, None, None]
    Wb = eq + 1e-3 * rng.standard_normal((2,) + shb)
    Ws = eq[:, :, :, 0] + 1e-3 * rng.standard_normal((2,) + shs)
    return dict(geometry="ball+sphere", n=tuple(n), rho_star=1.0, tau=tau, steps=steps, seed=seed,
                d_bulk=[1.0, delta], bulk_params=[a1, a2, b1], d_surface=[1.0, eps], surface_params=[z1, a2, b1],
                coupling=dict(zeta1=z1, zeta2=z2, zeta3=z3, eta1=e1, eta2=e2), Wb=Wb, Ws=Ws,
                name="bulk_surface_ball")


def dib_cylinder(n=(140, 140, 25), steps=10000, seed=9, tau=0.025, bulk_noise=0.0):
    """Bulk-surface DIB model on the cylinder rho_* = 15, z_* = 25 and its bottom disk (Section 5.6,
    eqs. bulkcyl): bulk u, v (diffusion 1, delta = 1; b = -alpha1 (u - alpha2), c = -beta1 (v - beta2);
    u = alpha2, v = beta2 on the top) held lifted, w = (u - alpha2, v - beta2), so the bulk reaction
    is LINEAR with K = diag(-alpha1, -beta1); surface r, s (diffusion 1, eps = 20, no reaction of
    their own: the DIB kinetics zeta1 p, zeta1 q come through the coupling).  Parameters as printed:
    alpha1 = alpha2 = delta = beta1 = beta2 = zeta1 = zeta3 = 1, alpha3 = beta3 = 0.1, eps = 20,
    zeta2 = 10, zeta4 = 30, zeta5 = 0.5, eta1 = 3, eta2 = 2.5, eta3 = 0.2, eta5 = 1.5 and eta4 from
    the equilibrium condition.  Initial data: u = alpha2, v = beta2 (w = 0; optionally plus
    bulk_noise N(0, 1)), r = 1e-2 U(0, 1), s = zeta5 + 1e-2 U(0, 1).  t_* = 250 in 10000 steps.
    Wb: (2, n_z, n_theta, n_rho), Ws: (2, n_theta, n_rho); the flat state is Wb then Ws."""
    rng = _rng(seed)
    a1, a2, a3, b1, b2, b3, delta, eps = 1.0, 1.0, 0.1, 1.0, 1.0, 0.1, 1.0, 20.0
    z = [1.0, 10.0, 1.0, 30.0, 0.5]
    e1, e2, e3, e5 = 3.0, 2.5, 0.2, 1.5
    e4 = b2 * e1 * (1.0 - z[4]) * (1.0 - e3 + e3 * z[4]) / (z[4] * (1.0 + e3 * z[4]))
    shb, shs = _shape(n), _shape(n[:2])
    Ws = np.stack([1e-2 * rng.uniform(0.0, 1.0, shs), z[4] + 1e-2 * rng.uniform(0.0, 1.0, shs)])
    Wb = np.zeros((2,) + shb)
    if bulk_noise:
        Wb = Wb + bulk_noise * rng.standard_normal((2,) + shb)
    coupling = dict(kind="dib_cylinder", alpha3=a3, beta3=b3, u_top=a2, v_top=b2, eta4=e4,
                    **{f"zeta{q + 1}": z[q] for q in range(5)}, eta1=e1, eta2=e2, eta3=e3, eta5=e5)
    return dict(geometry="cylinder+disk", n=tuple(n), rho_star=15.0, z_star=25.0, tau=tau, steps=steps, seed=seed,
                d_bulk=[1.0, delta], bulk_reaction="linear", bulk_params=[-a1, 0.0, 0.0, -b1],
                d_surface=[1.0, eps], surface_reaction="none", surface_params=[], coupling=coupling,
                oracle_params=dict(alpha1=a1, alpha2=a2, alpha3=a3, beta1=b1, beta2=b2, beta3=b3, delta=delta,
                                   eps=eps, zeta1=z[0], zeta2=z[1], zeta3=z[2], zeta4=z[3], zeta5=z[4],
                                   eta1=e1, eta2=e2, eta3=e3, eta5=e5),
                Wb=Wb, Ws=Ws, name="dib_cylinder")


def bvam_disk(n=(40, 80), steps=5000, seed=10, tau=0.16):
    """BVAM model on the unit disk without sources (Section 5.2, eq. BVAM): diffusion (gamma, delta)
    and the reaction of eq. BVAMnl with the parameters printed in Section 5.1 (gamma 3.87e-3, delta
    7.5e-3, alpha1 0.899, alpha2 0.2, alpha3 0.2, beta1 -0.91, beta2 -0.899); initial data
    1e-2 N(0, 1) per point and species about the equilibrium (0, 0); t_* = 800 in 5000 steps."""
    rng = _rng(seed)
    W0 = 1e-2 * rng.standard_normal((2,) + _shape(n))
    return dict(geometry="disk", n=tuple(n), d=[3.87e-3, 7.5e-3], reaction="bvam",
                params=[0.899, 0.2, 0.2, -0.91, -0.899], tau=tau, steps=steps, W0=W0, seed=seed, name="bvam_disk")
