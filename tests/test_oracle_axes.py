"""Pins of the oracle's 1-D grids and matrices against what the paper and mathematics fix.

* second-order consistency of each axis with its continuous operator
  (Table 1 operators, Section 3);
* closed-form spectra: circulant A_theta (eq. A_theta), A_z as printed
  (eigenpairs stated after eq. A_z), A_z with Neumann caps;
* Proposition 1: positive off-diagonals, e^{tA} >= 0, real nonpositive
  spectrum, ||Xi||_2 = 1 and ||Xi^{-1}||_2 = sqrt(2n-3) (d=2), n-1 (d=3);
* Appendix A: sigma in ((-(n-1)+sqrt(n^2-1))/2, 1/2) and f(sigma) = 0.
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
