"""One-dimensional grids and finite-difference matrices (paper Section 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Each builder returns ``(points, A)`` with ``A`` a dense ``n x n`` float64
matrix written entry by entry from the paper's formulas.  Tridiagonal
matrices use the paper's 1-based naming of eq. (tridiag): ``a_l`` on the
diagonal, ``b_l`` at (l, l+1), ``c_l`` at (l+1, l).

Pins (tests/test_oracle_axes.py): second-order consistency of every axis with
the continuous 1-D operator on smooth functions; the closed-form spectra of
A_theta and A_z; the Proposition 1 numbers (positive off-diagonals,
nonpositive real spectrum, nonnegative exponential, ||Xi^{-1}||_2); the
appendix bounds on sigma.
"""
import numpy as np


def tridiag(a, b, c):
    """Dense matrix of eq. (tridiag) from 1-based lists a (n), b (n-1), c (n-1)."""
    n = len(a)
    A = np.zeros((n, n))
    for l in range(1, n + 1):
        A[l - 1, l - 1] = a[l - 1]
        if l <= n - 1:
            A[l - 1, l] = b[l - 1]     # b_l at row l, column l+1
            A[l, l - 1] = c[l - 1]     # c_l at row l+1, column l
    return A


def theta_axis(n):
    """Periodic theta, eq. (A_theta): theta_j = j h, h = 2 pi / n, circulant (-2, 1, 1)/h^2."""
    h = 2.0 * np.pi / n
    theta = np.array([j * h for j in range(1, n + 1)])
    A = np.zeros((n, n))
    for r in range(n):
        A[r, r] += -2.0 / h**2
        A[r, (r + 1) % n] += 1.0 / h**2
        A[r, (r - 1) % n] += 1.0 / h**2
    return theta, A


def rho2_axis(n, rho_star=1.0):
    """Radial axis of the disk/cylinder, eq. (disk_discr): half-point grid, Neumann at rho_*."""
    h = rho_star / (n - 0.5)
    rho = np.array([h / 2.0 + (i - 1) * h for i in range(1, n + 1)])
    a = [-2.0 / h**2] * n
    b = [2.0 * l / ((2.0 * l - 1.0) * h**2) for l in range(1, n)]
    c = [2.0 * l / ((2.0 * l + 1.0) * h**2) for l in range(1, n)]
    c[n - 2] = 2.0 / h**2          # c_{n-1}
    return rho, tridiag(a, b, c)


def rho3_axis(n, rho_star=1.0):
    """Radial axis of the ball, eq. (ball_discr): rho_i = i h, h = rho_*/n, Neumann at rho_*."""
    h = rho_star / n
    rho = np.array([h + (i - 1) * h for i in range(1, n + 1)])
    a = [-2.0 / h**2] * n
    b = [(l + 1.0) / (l * h**2) for l in range(1, n)]
    c = [l / ((l + 1.0) * h**2) for l in range(1, n)]
    c[n - 2] = 2.0 / h**2          # c_{n-1}
    return rho, tridiag(a, b, c)


def rho_lambda_axis(n, lam, rho_star=1.0):
    """Radial axis of the anomalous operator Delta_lambda on the disk, eq. (A_lambda) of
    Section 5.3, with homogeneous Dirichlet at rho_* (after lifting the boundary values):
    rho_i = (1 - lam) h/2 + (i - 1) h, h = rho_*/(n + (1 - lam)/2), so rho_{n+1} = rho_*;
    with x_l = (1 - lam)/2 + l - 1:
    a_l = -2/(x_l^lam h^(2+lam)), b_l = (1 - lam + l - 1)/(x_l^(1+lam) h^(2+lam)),
    c_l = l/(x_{l+1}^(1+lam) h^(2+lam))."""
    h = rho_star / (n + (1.0 - lam) / 2.0)
    rho = np.array([(1.0 - lam) * h / 2.0 + (i - 1) * h for i in range(1, n + 1)])
    x = lambda l: (1.0 - lam) / 2.0 + l - 1.0
    s = h ** (2.0 + lam)
    a = [-2.0 / (x(l) ** lam * s) for l in range(1, n + 1)]
    b = [(1.0 - lam + l - 1.0) / (x(l) ** (1.0 + lam) * s) for l in range(1, n)]
    c = [l / (x(l + 1) ** (1.0 + lam) * s) for l in range(1, n)]
    return rho, tridiag(a, b, c)


def phi_sigma(n):
    """Root sigma in (0, 1/2) of the appendix's f(x) = cot(x pi/(n-1+2x)) - 2(n-1+2x)/pi.

    f decreases strictly on (0, 1/2), tends to +inf at 0 and is negative at
    1/2 (Appendix A), so plain bisection brackets the unique root; it runs
    until the bracket stops shrinking in floating point.
    """
    def f(x):
        return 1.0 / np.tan(x * np.pi / (n - 1 + 2 * x)) - 2.0 * (n - 1 + 2 * x) / np.pi

    lo, hi = 0.0, 0.5
    assert f(hi) < 0.0
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            return mid
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid


def phi_axis(n):
    """Polar-angle axis, eqs. (syscn) and (A_phi): grid avoiding phi = 0, pi."""
    sigma = phi_sigma(n)
    h = np.pi / (n - 1 + 2 * sigma)
    phi = np.array([sigma * h + (k - 1) * h for k in range(1, n + 1)])
    a = [-2.0 / h**2] * n
    b = [1.0 / h**2 + (1.0 / np.tan((sigma + l - 1) * h)) / (2.0 * h) for l in range(1, n)]
    c = [b[(n - l) - 1] for l in range(1, n)]     # c_l = b_{n-l}
    return phi, tridiag(a, b, c), sigma


def z_axis_paper(n, z_star=1.0):
    """Height axis as printed, eq. (A_z): Neumann at 0, Dirichlet at z_*, h = z_*/n."""
    h = z_star / n
    z = np.array([(k - 1) * h for k in range(1, n + 1)])
    a = [-2.0 / h**2] * n
    b = [1.0 / h**2] * (n - 1)
    b[0] = 2.0 / h**2
    c = [1.0 / h**2] * (n - 1)
    return z, tridiag(a, b, c)


def z_axis_neumann(n, z_star=1.0):
    """Height axis with homogeneous Neumann at both caps (the reading used for walls+caps).

    The paper's Neumann end at z = 0 (b_1 = 2/h^2, from the mirrored ghost
    value) is applied at z = z_* as well: node-centred grid z_k = (k-1) h with
    h = z_*/(n-1), c_{n-1} = 2/h^2, every other off-diagonal 1/h^2.
    """
    h = z_star / (n - 1)
    z = np.array([(k - 1) * h for k in range(1, n + 1)])
    a = [-2.0 / h**2] * n
    b = [1.0 / h**2] * (n - 1)
    b[0] = 2.0 / h**2
    c = [1.0 / h**2] * (n - 1)
    c[n - 2] = 2.0 / h**2
    return z, tridiag(a, b, c)


def xi_diagonal(A):
    """Diagonal of Xi from the proof of Proposition 1: xi_1 = 1, xi_{l+1} = sqrt(c_1..c_l / (b_1..b_l)).

    For a symmetric matrix (A_theta, whose corner entries make it
    non-tridiagonal) Xi is the identity.
    """
    n = A.shape[0]
    if np.array_equal(A, A.T):
        return np.ones(n)
    xi = np.ones(n)
    for l in range(1, n):
        b_l = A[l - 1, l]
        c_l = A[l, l - 1]
        xi[l] = xi[l - 1] * np.sqrt(c_l / b_l)
    return xi
