"""Reaction terms g(w) of the coupled systems (paper Section 5 and the benchmark workloads).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Each returns a list of arrays, one per species, evaluated pointwise.  They are
dtype-generic so that the complex-step gradients in ``adjoint`` go through
them unchanged.  Pins: tests/test_oracle_reactions.py checks the steady
states each model is built around and, for the manufactured BVAM sources,
that the exact solution satisfies the source-augmented PDE.
"""
import numpy as np


def schnakenberg(W, gamma, a, b):
    """f = gamma (a - u + u^2 v), g = gamma (b - u^2 v)."""
    u, v = W[0], W[1]
    u2v = u * u * v
    return [gamma * (a - u + u2v), gamma * (b - u2v)]


def gray_scott(W, F, k):
    """f = -u v^2 + F (1 - u), g = u v^2 - (F + k) v."""
    u, v = W[0], W[1]
    uv2 = u * v * v
    return [-uv2 + F * (1.0 - u), uv2 - (F + k) * v]


def linear_cubic(W, K):
    """f_i = sum_j K_ij u_j - u_i^3 for an S x S matrix K."""
    S = len(W)
    return [sum(K[i][j] * W[j] for j in range(S)) - W[i] ** 3 for i in range(S)]


# BVAM model of Section 5.1, eq. (BVAMnl), parameters as printed there.
BVAM = dict(gamma=3.87e-3, delta=7.5e-3, alpha1=8.99e-1, alpha2=2e-1, alpha3=2e-1,
            beta1=-9.1e-1, beta2=-8.99e-1)


def bvam(W, p=BVAM):
    """b(u,v) = a1 u (1 - a2 v^2) + v (1 - a3 u); c(u,v) = b1 v (1 + a1 a2/b1 u v) + u (b2 + a3 v)."""
    u, v = W[0], W[1]
    a1, a2, a3, b1, b2 = p["alpha1"], p["alpha2"], p["alpha3"], p["beta1"], p["beta2"]
    bb = a1 * u * (1.0 - a2 * v * v) + v * (1.0 - a3 * u)
    cc = b1 * v * (1.0 + a1 * a2 / b1 * u * v) + u * (b2 + a3 * v)
    return [bb, cc]


def bvam_exact(t, rho, theta):
    """Manufactured solution of Section 5.1: u = e^-t (1-rho)^2 e^{cos(theta)/10}, v likewise with sin."""
    R = (1.0 - rho) ** 2
    return [np.exp(-t) * R * np.exp(np.cos(theta) / 10.0), np.exp(-t) * R * np.exp(np.sin(theta) / 10.0)]


def bvam_sources(t, rho, theta, p=BVAM):
    """b_s, c_s such that the manufactured solution solves eq. (BVAMsys).

    b_s = du/dt - gamma Lap_D u - b(u, v) with the polar Laplacian of
    eq. (lapdisk) applied analytically to u = e^-t R(rho) T(theta):
    Lap_D u = e^-t [(R'' + R'/rho) T + R T''/rho^2]; likewise for v.
    """
    R = (1.0 - rho) ** 2
    dR = -2.0 * (1.0 - rho)
    d2R = 2.0 * np.ones_like(rho)
    T = np.exp(np.cos(theta) / 10.0)
    d2T = T * (np.sin(theta) ** 2 / 100.0 - np.cos(theta) / 10.0)
    Sv = np.exp(np.sin(theta) / 10.0)
    d2S = Sv * (np.cos(theta) ** 2 / 100.0 - np.sin(theta) / 10.0)
    e = np.exp(-t)
    u = e * R * T
    v = e * R * Sv
    lap_u = e * ((d2R + dR / rho) * T + R * d2T / rho**2)
    lap_v = e * ((d2R + dR / rho) * Sv + R * d2S / rho**2)
    bb, cc = bvam([u, v], p)
    return [-u - p["gamma"] * lap_u - bb, -v - p["delta"] * lap_v - cc]
