"""Pins of the oracle's phi_1 (Section 4).

* scalar: phi_1(0) = 1, phi_1(1) = e - 1, the series 1 + x/2 + x^2/6 near 0;
* phi_1 of every axis matrix (route: Proposition 1 symmetrisation + eigh)
  against the upper-right block of expm([[X, I], [0, 0]]), a textbook
  identity that shares nothing with the eigen route.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import axes as ax
from oracle.phi import eigen, phi1, phi1_matrix


def phi1_expm(X):
    n = X.shape[0]
    aug = np.zeros((2 * n, 2 * n), dtype=X.dtype)
    aug[:n, :n] = X
    aug[:n, n:] = np.eye(n)
    return sla.expm(aug)[:n, n:]


def test_phi1_scalar():
    assert phi1(np.array([0.0]))[0] == 1.0
    assert np.isclose(phi1(np.array([1.0]))[0], np.e - 1, rtol=1e-15)
    x = np.array([1e-3, -1e-5, 1e-9])
    assert np.allclose(phi1(x), 1 + x / 2 + x**2 / 6, rtol=1e-14)
    big = np.array([-1e8])
    assert np.isclose(phi1(big)[0], 1e-8, rtol=1e-12)


@pytest.mark.parametrize("name", ["theta", "rho2", "rho3", "phi", "z_neumann", "z_paper"])
@pytest.mark.parametrize("t", [1e-5, 1e-3, 0.05])
def test_phi1_matrix_vs_augmented_expm(name, t):
    n = 17
    A = {"theta": ax.theta_axis(n)[1], "rho2": ax.rho2_axis(n)[1], "rho3": ax.rho3_axis(n)[1],
         "phi": ax.phi_axis(n)[1], "z_neumann": ax.z_axis_neumann(n)[1], "z_paper": ax.z_axis_paper(n)[1]}[name]
    P = phi1_matrix(A, t)
    R = phi1_expm(t * A)
    assert np.max(np.abs(P - R)) < 1e-12 * np.max(np.abs(R))


def test_eigen_reconstructs():
    for A in [ax.rho3_axis(30)[1], ax.phi_axis(30)[1], ax.rho2_axis(9)[1]]:
        lam, V, Vinv = eigen(A)
        assert np.allclose(V @ Vinv, np.eye(A.shape[0]), atol=1e-12)
        assert np.allclose((V * lam) @ Vinv, A, atol=1e-10 * np.abs(A).max())
