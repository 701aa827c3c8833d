"""Kronecker-sum semidiscretisations per geometry (paper Section 2, eqs. disk/sphere/ball/cylinder).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Tensor convention: the state of one species is a numpy array whose *last*
axis is mode 1, so that ``W.ravel()`` is the paper's vector ordering
w_{i + (j-1) n1 + (k-1) n1 n2} (first coordinate fastest).  Mode mu lives on
numpy axis ``ndim - mu``.

``Grid.M[mu]`` is the sparse Kronecker term M_mu exactly as printed
(e.g. ball: M_2 = D_phi (x) A_theta (x) D_rho).  ``Grid.A[mu]`` and
``Grid.scale[mu]`` describe the same term fibre by fibre: along mode mu every
fibre is multiplied by s * A_mu, with s the broadcastable array of diagonal
factors contributed by the other modes.  Tests check that both descriptions
agree (tests/test_oracle_operators.py) and that M approximates the continuous
Laplacians of eqs. lapdisk/lapsphere/lapball/lapcyl to second order.
"""
import numpy as np
import scipy.sparse as sp

from . import axes as ax


def _kron(*mats):
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


class Grid:
    """Grids, 1-D matrices and Kronecker terms of one geometry.

    kind: 'disk' (rho, theta), 'sphere' (theta, phi), 'ball' (rho, theta, phi),
    'cylinder' (rho, theta, z); ``n`` lists the points per mode, mode 1 first.
    ``z_bc`` selects the height axis: 'neumann' (both caps) or 'paper'
    (Neumann at 0, Dirichlet at z_*, eq. A_z).  ``lam`` (disk only) selects the
    anomalous operator Delta_lambda of Section 5.3 (eq. anomalous) with
    homogeneous Dirichlet at rho_*: A_rho from eq. (A_lambda), D_rho = rho^(-2-lam).
    """

    def __init__(self, kind, n, rho_star=1.0, z_star=1.0, z_bc="neumann", lam=None):
        self.kind = kind
        self.n = tuple(int(v) for v in n)
        self.ndim = len(self.n)
        self.shape = tuple(reversed(self.n))          # numpy shape, mode 1 last
        self.A = {}
        self.scale = {}
        self.points = {}
        self.M = {}
        if kind == "disk":
            n1, n2 = self.n
            if lam is None:
                rho, A_rho = ax.rho2_axis(n1, rho_star)
                p = -2.0
            else:
                rho, A_rho = ax.rho_lambda_axis(n1, lam, rho_star)
                p = -2.0 - lam
            theta, A_theta = ax.theta_axis(n2)
            D_rho = np.diag(rho**p)
            I1, I2 = np.eye(n1), np.eye(n2)
            self.points = {1: rho, 2: theta}
            self.A = {1: A_rho, 2: A_theta}
            self.scale = {1: np.ones((1, 1)), 2: (rho**p)[None, :]}
            self.M = {1: _kron(I2, A_rho), 2: _kron(A_theta, D_rho)}        # eq. (disk)
        elif kind == "sphere":
            n1, n2 = self.n
            theta, A_theta = ax.theta_axis(n1)
            phi, A_phi, self.sigma = ax.phi_axis(n2)
            D_phi = np.diag(np.sin(phi) ** -2.0)
            I1 = np.eye(n1)
            self.points = {1: theta, 2: phi}
            self.A = {1: A_theta, 2: A_phi}
            self.scale = {1: (np.sin(phi) ** -2.0)[:, None], 2: np.ones((1, 1))}
            self.M = {1: _kron(D_phi, A_theta), 2: _kron(A_phi, I1)}        # eq. (sphere)
        elif kind == "ball":
            n1, n2, n3 = self.n
            rho, A_rho = ax.rho3_axis(n1, rho_star)
            theta, A_theta = ax.theta_axis(n2)
            phi, A_phi, self.sigma = ax.phi_axis(n3)
            D_rho = np.diag(rho**-2.0)
            D_phi = np.diag(np.sin(phi) ** -2.0)
            I1, I2, I3 = np.eye(n1), np.eye(n2), np.eye(n3)
            self.points = {1: rho, 2: theta, 3: phi}
            self.A = {1: A_rho, 2: A_theta, 3: A_phi}
            self.scale = {
                1: np.ones((1, 1, 1)),
                2: (np.sin(phi) ** -2.0)[:, None, None] * (rho**-2.0)[None, None, :],
                3: (rho**-2.0)[None, None, :],
            }
            self.M = {                                                        # eq. (ball)
                1: _kron(I3, I2, A_rho),
                2: _kron(D_phi, A_theta, D_rho),
                3: _kron(A_phi, I2, D_rho),
            }
        elif kind == "cylinder":
            n1, n2, n3 = self.n
            rho, A_rho = ax.rho2_axis(n1, rho_star)
            theta, A_theta = ax.theta_axis(n2)
            if z_bc == "neumann":
                z, A_z = ax.z_axis_neumann(n3, z_star)
            elif z_bc == "paper":
                z, A_z = ax.z_axis_paper(n3, z_star)
            else:
                raise ValueError(z_bc)
            D_rho = np.diag(rho**-2.0)
            I1, I2, I3 = np.eye(n1), np.eye(n2), np.eye(n3)
            self.points = {1: rho, 2: theta, 3: z}
            self.A = {1: A_rho, 2: A_theta, 3: A_z}
            self.scale = {1: np.ones((1, 1, 1)), 2: (rho**-2.0)[None, None, :], 3: np.ones((1, 1, 1))}
            self.M = {                                                        # eq. (cylinder)
                1: _kron(I3, I2, A_rho),
                2: _kron(I3, A_theta, D_rho),
                3: _kron(A_z, I2, I1),
            }
        else:
            raise ValueError(kind)
        self.M_total = sum(self.M[mu] for mu in range(1, self.ndim + 1))

    @property
    def npts(self):
        return int(np.prod(self.n))

    def apply_M(self, w):
        """M w for one species tensor (Kronecker-sum action)."""
        return (self.M_total @ w.ravel()).reshape(w.shape)
