"""The phi_1 function: scalar form and phi_1 of a 1-D matrix (paper Section 4, Proposition 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Pins (tests/test_oracle_phi.py): the scalar limit and series; phi_1 of every
axis matrix against the upper-right block of ``scipy.linalg.expm`` of the
augmented matrix [[X, I], [0, 0]] (a textbook identity independent of the
eigen route used here); the eigen decomposition reproduces A.
"""
import numpy as np

from .axes import xi_diagonal


def phi1(x):
    """Scalar phi_1(x) = (e^x - 1)/x, with phi_1(0) = 1 (Section 4).

    Works elementwise on real or complex arrays; uses the library expm1.
    """
    x = np.asarray(x)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = np.expm1(x[nz]) / x[nz]
    return out


def eigen(A):
    """A = V diag(lam) V^{-1} through the symmetrisation of Proposition 1.

    S = Xi^{-1} A Xi is symmetric; its orthogonal eigenvectors Q give
    V = Xi Q and V^{-1} = Q^T Xi^{-1} (the relation quoted after eq. ee_ball).
    Returns (lam, V, Vinv), eigenvalues ascending.
    """
    xi = xi_diagonal(A)
    S = (A * xi[None, :]) / xi[:, None]
    S = 0.5 * (S + S.T)                      # remove rounding asymmetry only
    lam, Q = np.linalg.eigh(S)
    V = xi[:, None] * Q
    Vinv = Q.T / xi[None, :]
    return lam, V, Vinv


def phi1_matrix(A, t):
    """phi_1(t A) = V diag(phi_1(t lam)) V^{-1} for a 1-D axis matrix A and scalar t (may be complex)."""
    lam, V, Vinv = eigen(A)
    return (V * phi1(t * lam)[None, :]) @ Vinv
