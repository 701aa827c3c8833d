"""Pins of the oracle's 1-D grids and matrices against what the paper and mathematics fix.

* second-order consistency of each axis with its continuous operator
  (Table 1 operators, Section 3);
* closed-form spectra: circulant A_theta (eq. A_theta), A_z as printed
  (eigenpairs stated after eq. A_z), A_z with Neumann caps;
* Proposition 1: positive off-diagonals, e^{tA} >= 0, real nonpositive
  spectrum, ||Xi||_2 = 1 and ||Xi^{-1}||_2 = sqrt(2n-3) (d=2), n-1 (d=3);
* Appendix A: sigma in ((-(n-1)+sqrt(n^2-1))/2, 1/2) and f(sigma) = 0;
* Delta_lambda (Section 5.3): the printed eq. (A_lambda) equals central differences of eq.
  (anomalous) built independently, consistency order, Appendix B's closed-form Xi and bound.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import axes as ax
from oracle.phi import eigen


def _max_err(build, f, Lf, ns):
    errs = []
    for n in ns:
        out = build(n)
        x, A = out[0], out[1]
        errs.append(np.max(np.abs(A @ f(x) - Lf(x))))
    return np.array(errs)


@pytest.mark.parametrize("name", ["theta", "rho2", "rho3", "phi", "z_neumann", "z_paper"])
def test_second_order_consistency(name):
    # smooth test functions obeying each axis's boundary conditions
    if name == "theta":
        build = ax.theta_axis
        f = lambda x: np.exp(np.sin(x))
        Lf = lambda x: np.exp(np.sin(x)) * (np.cos(x) ** 2 - np.sin(x))
    elif name == "rho2":
        build = ax.rho2_axis
        f = lambda r: np.cos(np.pi * r)                       # f'(1) = 0
        Lf = lambda r: -np.pi * np.sin(np.pi * r) / r - np.pi**2 * np.cos(np.pi * r)
    elif name == "rho3":
        build = ax.rho3_axis
        f = lambda r: np.cos(np.pi * r)
        Lf = lambda r: -2 * np.pi * np.sin(np.pi * r) / r - np.pi**2 * np.cos(np.pi * r)
    elif name == "phi":
        build = ax.phi_axis
        f = lambda p: np.cos(p) + np.cos(p) ** 2              # l = 1 and l = 2 zonal parts
        # cot(p) f' + f'' for f = cos p + cos^2 p
        Lf = lambda p: -2 * np.cos(p) + (2 - 6 * np.cos(p) ** 2)
    elif name == "z_neumann":
        build = ax.z_axis_neumann
        f = lambda z: np.cos(np.pi * z)
        Lf = lambda z: -np.pi**2 * np.cos(np.pi * z)
    else:
        build = ax.z_axis_paper
        f = lambda z: np.cos(np.pi * z / 2)                   # f'(0) = 0, f(1) = 0
        Lf = lambda z: -(np.pi**2 / 4) * np.cos(np.pi * z / 2)
    e = _max_err(build, f, Lf, [20, 40, 80, 160])
    rates = np.log2(e[:-1] / e[1:])
    assert np.all(rates > 1.8), (name, e, rates)


def test_theta_closed_form_spectrum():
    for n in [5, 8, 13, 64]:
        _, A = ax.theta_axis(n)
        h = 2 * np.pi / n
        exact = np.sort(-(4 / h**2) * np.sin(np.pi * np.arange(n) / n) ** 2)
        lam, V, Vinv = eigen(A)
        assert np.allclose(np.sort(lam), exact, rtol=0, atol=1e-10 / h**2)
        assert np.allclose(V @ np.diag(lam) @ Vinv, A, atol=1e-9 / h**2)


def test_z_paper_closed_form_eigenpairs():
    for n in [4, 7, 32]:
        _, A = ax.z_axis_paper(n, 1.0)
        h = 1.0 / n
        for k in range(1, n + 1):
            lam = -2 / h**2 + (2 / h**2) * np.cos(np.pi * (k - 0.5) / n)
            v = np.array([np.sin((n - i + 1) * np.pi * (k - 0.5) / n) / np.sin(np.pi * (k - 0.5) / n)
                          for i in range(1, n)] + [1.0])
            assert np.allclose(A @ v, lam * v, rtol=0, atol=1e-9 / h**2 * np.max(np.abs(v)))


def test_z_neumann_closed_form_spectrum():
    for n in [4, 9, 33]:
        _, A = ax.z_axis_neumann(n, 1.0)
        h = 1.0 / (n - 1)
        exact = -(4 / h**2) * np.sin(np.pi * np.arange(n) / (2 * (n - 1))) ** 2
        lam, _, _ = eigen(A)
        assert np.allclose(np.sort(lam), np.sort(exact), rtol=0, atol=1e-10 / h**2)


@pytest.mark.parametrize("name", ["rho2", "rho3", "phi", "z_neumann", "z_paper", "theta"])
def test_proposition_1(name):
    n = 23
    A = {"rho2": lambda: ax.rho2_axis(n)[1], "rho3": lambda: ax.rho3_axis(n)[1],
         "phi": lambda: ax.phi_axis(n)[1], "z_neumann": lambda: ax.z_axis_neumann(n)[1],
         "z_paper": lambda: ax.z_axis_paper(n)[1], "theta": lambda: ax.theta_axis(n)[1]}[name]()
    off = A - np.diag(np.diag(A))
    assert np.all(off[off != 0] > 0)                                   # item 1
    for t in [1e-4, 1e-2, 1.0]:
        assert np.min(sla.expm(t * A)) > -1e-12                        # item 2
    ev = np.linalg.eigvals(A)
    assert np.max(np.abs(ev.imag)) < 1e-8 * np.max(np.abs(ev))         # items 3-4: real spectrum
    assert np.max(ev.real) < 1e-8 * np.max(np.abs(ev))                 # item 5
    xi = ax.xi_diagonal(A)
    S = (A * xi[None, :]) / xi[:, None]
    assert np.allclose(S, S.T, rtol=1e-12, atol=1e-12 * np.max(np.abs(A)))


def test_xi_norms_radial():
    for n in [5, 10, 50, 100]:
        xi2 = ax.xi_diagonal(ax.rho2_axis(n)[1])
        xi3 = ax.xi_diagonal(ax.rho3_axis(n)[1])
        assert np.isclose(np.max(xi2), 1.0) and np.isclose(np.max(xi3), 1.0)
        assert np.isclose(np.max(1 / xi2), np.sqrt(2 * n - 3), rtol=1e-12)
        assert np.isclose(np.max(1 / xi3), n - 1, rtol=1e-12)


def test_sigma_appendix_bounds():
    for n in [3, 5, 10, 50, 100, 512]:
        s = ax.phi_sigma(n)
        lower = (-(n - 1) + np.sqrt(n * n - 1.0)) / 2
        assert lower < s < 0.5
        h = np.pi / (n - 1 + 2 * s)
        # second equation of eq. (syscn): -cot(sigma h)/(2h) + 1/h^2 = 0
        assert abs(-1 / np.tan(s * h) / (2 * h) + 1 / h**2) < 1e-9 / h**2
    # the first equation of (syscn) holds by construction of h
    n = 17
    s = ax.phi_sigma(n)
    h = np.pi / (n - 1 + 2 * s)
    assert np.isclose(h, (np.pi - 2 * s * h) / (n - 1))


# ---- anomalous diffusion Delta_lambda on the disk (Section 5.3, Appendix B) ----
LAMBDAS = [-1.95, -1.0, 0.0, 0.5]


def _central_difference_lambda(n, lam, rho_star=1.0):
    """Delta_lambda's radial part (eq. anomalous), (1-lam)/rho^(1+lam) f' + f''/rho^lam, by
    central differences at the grid points of eq. (A_lambda), u = 0 at rho_{n+1} = rho_*:
    built from the definition, independently of the printed a_l, b_l, c_l."""
    h = rho_star / (n + (1.0 - lam) / 2.0)
    rho = (1.0 - lam) * h / 2.0 + h * np.arange(n)
    A = np.zeros((n, n))
    for i in range(n):
        d2 = 1.0 / (rho[i] ** lam * h * h)
        d1 = (1.0 - lam) / (rho[i] ** (1.0 + lam) * 2.0 * h)
        A[i, i] = -2.0 * d2
        if i > 0:
            A[i, i - 1] = d2 - d1
        if i < n - 1:
            A[i, i + 1] = d2 + d1
    return rho, A


@pytest.mark.parametrize("lam", LAMBDAS)
def test_lambda_axis_equals_its_definition(lam):
    """The printed a_l, b_l, c_l of eq. (A_lambda) are the central differences of eq. (anomalous);
    the coefficient of u_0 vanishes (x_1 - (1-lam)/2 = 0), so no condition at rho = 0 is needed."""
    for n in [4, 17, 60]:
        rho, A = ax.rho_lambda_axis(n, lam)
        rho_d, A_d = _central_difference_lambda(n, lam)
        assert np.allclose(rho, rho_d, rtol=0, atol=1e-15)
        assert np.max(np.abs(A - A_d)) <= 1e-12 * np.max(np.abs(A))
        h = 1.0 / (n + (1.0 - lam) / 2.0)
        assert np.isclose(rho[-1] + h, 1.0)                   # Dirichlet point rho_{n+1} = rho_*


@pytest.mark.parametrize("lam", [-1.95, 0.0, 0.5])
def test_lambda_axis_consistency_order(lam):
    """Consistency with the continuous operator on f = cos(pi rho / 2) (f(rho_*) = 0, even at 0):
    second order for lam <= 0; for lam > 0 the coefficient 1/rho^(1+lam) is singular at the
    origin and the first points' error decays like h^(2-lam)."""
    f = lambda r: np.cos(np.pi * r / 2)
    Lf = lambda r: ((1 - lam) / r ** (1 + lam) * (-np.pi / 2 * np.sin(np.pi * r / 2))
                    - (np.pi / 2) ** 2 * np.cos(np.pi * r / 2) / r ** lam)
    errs = _max_err(lambda n: ax.rho_lambda_axis(n, lam), f, Lf, [40, 80, 160])
    ratio = 0.9 * 2.0 ** min(2.0, 2.0 - lam)
    assert errs[0] / errs[1] > ratio and errs[1] / errs[2] > ratio, errs


def test_lambda_axis_appendix_b():
    """Appendix B: xi_l^2 = ((1-lam)/((2l-1)-lam))^(1+lam) (l-1)!/prod_{i<l}(i-lam); the largest entry
    of Xi^{-1} is 1/xi_n for lam < 0, below sqrt(((2n-1-lam)/(1-lam))^(1+lam) e^{-lam(ln(n-1)+1)});
    an essentially nonnegative matrix with negative eigenvalues."""
    from math import lgamma
    for lam in [-1.95, -1.0, -0.3]:
        for n in [5, 40, 160]:
            _, A = ax.rho_lambda_axis(n, lam)
            xi = ax.xi_diagonal(A)
            for l in range(2, n + 1):
                log_p = sum(np.log(i - lam) for i in range(1, l)) - lgamma(l)
                ref = np.sqrt(((1 - lam) / ((2 * l - 1) - lam)) ** (1 + lam) * np.exp(-log_p))
                assert np.isclose(xi[l - 1], ref, rtol=1e-10), (lam, n, l)
            assert np.isclose(np.max(1 / xi), 1 / xi[-1])
            bound = np.sqrt(((2 * n - 1 - lam) / (1 - lam)) ** (1 + lam) * np.exp(-lam * (np.log(n - 1) + 1)))
            assert 1 / xi[-1] < bound
            off = A - np.diag(np.diag(A))
            assert np.all(off >= 0)
            assert np.max(np.linalg.eigvals(A).real) < 0
