// FP64 host setup: axes (Section 3), eigenbases (Proposition 1) and phi_1
// matrices (Section 4) for the split exponential Euler plan.
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <stdexcept>
#include <thread>

namespace sexpe {

static const double kPi = 3.14159265358979323846;

Mat Axis::dense() const {
    Mat A(n);
    for (int r = 0; r < n; ++r) {
        A(r, r) += diag[r];
        if (r > 0) A(r, r - 1) += lower[r];
        else if (periodic) A(r, n - 1) += lower[r];
        if (r < n - 1) A(r, r + 1) += upper[r];
        else if (periodic) A(r, 0) += upper[r];
    }
    return A;
}

double phi_sigma(int n) {
    // f(x) = cot(x pi/(n-1+2x)) - 2(n-1+2x)/pi decreases on (0, 1/2), f(0+) = +inf,
    // f(1/2) < 0 (Appendix A): bisect until the bracket stops shrinking.
    auto f = [n](double x) {
        return 1.0 / std::tan(x * kPi / (n - 1 + 2 * x)) - 2.0 * (n - 1 + 2 * x) / kPi;
    };
    double lo = 0.0, hi = 0.5;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (f(mid) > 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

Axis build_axis(AxisKind kind, int n, double extent, double lambda) {
    Axis ax;
    ax.n = n;
    ax.pts.assign(n, 0.0);
    ax.lower.assign(n, 0.0);
    ax.diag.assign(n, 0.0);
    ax.upper.assign(n, 0.0);
    double h = 0.0;
    if (kind == AX_RHO_LAMBDA) {
        // eq. (A_lambda): rho_i = (1 - lambda) h/2 + (i - 1) h, h = rho_*/(n + (1 - lambda)/2);
        // x_l = (1 - lambda)/2 + l - 1; a_l = -2/(x_l^lambda h^(2+lambda)),
        // b_l = (1 - lambda + l - 1)/(x_l^(1+lambda) h^(2+lambda)), c_l = l/(x_{l+1}^(1+lambda) h^(2+lambda))
        h = extent / (n + 0.5 * (1.0 - lambda));
        const double s = std::pow(h, 2.0 + lambda);
        auto x = [&](int l) { return 0.5 * (1.0 - lambda) + l - 1.0; };
        for (int i = 0; i < n; ++i) ax.pts[i] = 0.5 * (1.0 - lambda) * h + i * h;
        for (int l = 1; l <= n; ++l) ax.diag[l - 1] = -2.0 / (std::pow(x(l), lambda) * s);
        for (int l = 1; l <= n - 1; ++l) {
            ax.upper[l - 1] = (1.0 - lambda + l - 1.0) / (std::pow(x(l), 1.0 + lambda) * s);   // b_l
            ax.lower[l] = l / (std::pow(x(l + 1), 1.0 + lambda) * s);                       // c_l
        }
        return ax;
    }
    switch (kind) {
    case AX_THETA:  // eq. (A_theta): theta_j = j h, h = 2 pi/n, periodic
        h = 2.0 * kPi / n;
        ax.periodic = true;
        for (int j = 0; j < n; ++j) {
            ax.pts[j] = (j + 1) * h;
            ax.lower[j] = ax.upper[j] = 1.0 / (h * h);
        }
        break;
    case AX_RHO2:   // eq. (disk_discr): rho_i = h/2 + (i-1) h, h = rho_*/(n - 1/2)
        h = extent / (n - 0.5);
        for (int i = 0; i < n; ++i) ax.pts[i] = 0.5 * h + i * h;
        for (int l = 1; l <= n - 1; ++l) {
            ax.upper[l - 1] = 2.0 * l / ((2.0 * l - 1.0) * h * h);   // b_l
            ax.lower[l] = 2.0 * l / ((2.0 * l + 1.0) * h * h);       // c_l
        }
        ax.lower[n - 1] = 2.0 / (h * h);                             // c_{n-1}
        break;
    case AX_RHO3:   // eq. (ball_discr): rho_i = i h, h = rho_*/n
        h = extent / n;
        for (int i = 0; i < n; ++i) ax.pts[i] = (i + 1) * h;
        for (int l = 1; l <= n - 1; ++l) {
            ax.upper[l - 1] = (l + 1.0) / (l * h * h);               // b_l
            ax.lower[l] = l / ((l + 1.0) * h * h);                   // c_l
        }
        ax.lower[n - 1] = 2.0 / (h * h);                             // c_{n-1}
        break;
    case AX_PHI: {  // eqs. (syscn), (A_phi)
        double s = phi_sigma(n);
        ax.sigma = s;
        h = kPi / (n - 1 + 2 * s);
        for (int k = 0; k < n; ++k) ax.pts[k] = s * h + k * h;
        for (int l = 1; l <= n - 1; ++l)                             // b_l
            ax.upper[l - 1] = 1.0 / (h * h) + (1.0 / std::tan((s + l - 1) * h)) / (2.0 * h);
        for (int l = 1; l <= n - 1; ++l) ax.lower[l] = ax.upper[n - l - 1];   // c_l = b_{n-l}
        break;
    }
    case AX_Z_NEUMANN:  // Neumann at both caps: h = z_*/(n-1), mirrored ghost at each end
        h = extent / (n - 1);
        for (int k = 0; k < n; ++k) {
            ax.pts[k] = k * h;
            if (k < n - 1) ax.upper[k] = 1.0 / (h * h);
            if (k > 0) ax.lower[k] = 1.0 / (h * h);
        }
        ax.upper[0] = 2.0 / (h * h);
        ax.lower[n - 1] = 2.0 / (h * h);
        break;
    case AX_RHO_LAMBDA:
        break;                                                       // built above
    case AX_Z_PAPER:    // eq. (A_z): Neumann at 0, Dirichlet at z_*, h = z_*/n
        h = extent / n;
        for (int k = 0; k < n; ++k) {
            ax.pts[k] = k * h;
            if (k < n - 1) ax.upper[k] = 1.0 / (h * h);
            if (k > 0) ax.lower[k] = 1.0 / (h * h);
        }
        ax.upper[0] = 2.0 / (h * h);
        break;
    }
    for (int r = 0; r < n; ++r) ax.diag[r] = -2.0 / (h * h);
    return ax;
}

Eigen theta_eigen(const Axis& ax) {
    // A_theta is circulant: real Fourier vectors cos(2 pi m j/n), sin(2 pi m j/n)
    // with eigenvalue -(4/h^2) sin^2(pi m/n); m = 0 (and m = n/2 for even n) single.
    const int n = ax.n;
    const double h = 2.0 * kPi / n;
    Eigen e;
    e.lam.assign(n, 0.0);
    e.V = Mat(n);
    int col = 0;
    auto lam_of = [&](int m) { double s = std::sin(kPi * m / n); return -(4.0 / (h * h)) * s * s; };
    for (int j = 0; j < n; ++j) e.V(j, col) = 1.0 / std::sqrt((double)n);
    e.lam[col++] = 0.0;
    for (int m = 1; 2 * m < n; ++m) {
        for (int j = 0; j < n; ++j) {
            double a = 2.0 * kPi * (double)((long long)m * j % n) / n;
            e.V(j, col) = std::sqrt(2.0 / n) * std::cos(a);
            e.V(j, col + 1) = std::sqrt(2.0 / n) * std::sin(a);
        }
        e.lam[col] = e.lam[col + 1] = lam_of(m);
        col += 2;
    }
    if (n % 2 == 0) {
        for (int j = 0; j < n; ++j) e.V(j, col) = ((j % 2) ? -1.0 : 1.0) / std::sqrt((double)n);
        e.lam[col++] = lam_of(n / 2);
    }
    e.Vinv = Mat(n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) e.Vinv(r, c) = e.V(c, r);
    return e;
}

// Eigen-decomposition of a symmetric tridiagonal matrix (diagonal d, off-diagonal
// e[i] coupling i and i + 1) by the implicit QL method with Wilkinson-type shifts
// (Bowdler, Martin, Reinsch & Wilkinson, Numer. Math. 11, 1968): each sweep
// chases a plane rotation from the bottom of the unreduced block up to row l.
// On return d holds the eigenvalues and row k of Zt the unit eigenvector of
// d[k] (rows, so every rotation updates two contiguous rows).  False if an
// eigenvalue needs more than 60 sweeps.
static bool tridiag_ql(std::vector<double>& d, std::vector<double> e, Mat& Zt) {
    const int n = (int)d.size();
    e.resize(n, 0.0);
    Zt = Mat(n);
    for (int i = 0; i < n; ++i) Zt(i, i) = 1.0;
    const double eps = std::numeric_limits<double>::epsilon();
    for (int l = 0; l < n; ++l) {
        for (int sweep = 0;; ++sweep) {
            int m = l;
            while (m < n - 1 && std::fabs(e[m]) > eps * (std::fabs(d[m]) + std::fabs(d[m + 1]))) ++m;
            if (m == l) break;
            if (sweep == 60) return false;
            // shift: the eigenvalue of the leading 2 x 2 block nearer to d[l]
            const double theta = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double g = d[m] - d[l] + e[l] / (theta + std::copysign(std::hypot(theta, 1.0), theta));
            double s = 1.0, c = 1.0, p = 0.0;
            bool deflated = false;
            for (int i = m - 1; i >= l; --i) {
                const double f = s * e[i], b = c * e[i];
                const double r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {                  // the bulge vanished: split the block here
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                const double h = d[i + 1] - p;
                const double t = (d[i] - h) * s + 2.0 * c * b;
                p = s * t;
                d[i + 1] = h + p;
                g = c * t - b;
                double* zi = &Zt.a[(size_t)i * n];
                double* zj = zi + n;
                for (int k = 0; k < n; ++k) {
                    const double zk = zj[k];
                    zj[k] = s * zi[k] + c * zk;
                    zi[k] = c * zi[k] - s * zk;
                }
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return true;
}

Eigen tridiag_eigen(const Axis& ax) {
    // Proposition 1: xi_1 = 1, xi_{l+1} = sqrt(c_1..c_l/(b_1..b_l)); S = Xi^{-1} A Xi symmetric.
    const int n = ax.n;
    std::vector<double> xi(n, 1.0);
    for (int l = 1; l < n; ++l) xi[l] = xi[l - 1] * std::sqrt(ax.lower[l] / ax.upper[l - 1]);
    std::vector<double> dg(ax.diag.begin(), ax.diag.end()), off(n > 1 ? n - 1 : 0);
    for (int r = 0; r + 1 < n; ++r) off[r] = std::sqrt(ax.upper[r] * ax.lower[r + 1]);
    Mat Zt;
    if (!tridiag_ql(dg, off, Zt)) {       // no convergence: NaN tables, reported as SEXPE_ENUMERIC
        Eigen bad;
        bad.lam.assign(n, std::nan(""));
        bad.V = Mat(n);
        bad.Vinv = Mat(n);
        for (double& v : bad.V.a) v = std::nan("");
        for (double& v : bad.Vinv.a) v = std::nan("");
        return bad;
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return dg[a] < dg[b]; });
    Eigen e;
    e.lam.resize(n);
    e.V = Mat(n);
    e.Vinv = Mat(n);
    for (int c = 0; c < n; ++c) {
        const int src = order[c];
        e.lam[c] = dg[src];
        const double* q = &Zt.a[(size_t)src * n];
        for (int r = 0; r < n; ++r) {
            e.V(r, c) = xi[r] * q[r];
            e.Vinv(c, r) = q[r] / xi[r];
        }
    }
    return e;
}

// ---- phi_1 by Pade scaling and squaring on the augmented matrix ----------
// Elements of the algebra {[[T, B], [0, c I]]} closed under +, * and inversion
// of the (V - U) factor; expm([[X, I], [0, 0]]) = [[e^X, phi_1(X)], [0, I]].

// Rows are split over host threads for large n (the dense phi_1 of an assembled
// operator); every row is computed in the same order whatever the split.
static Mat matmul(const Mat& A, const Mat& B) {
    const int n = A.n;
    Mat C(n);
    auto rows = [&](int r0, int r1) {
        for (int i = r0; i < r1; ++i) {
            double* ci = &C.a[(size_t)i * n];
            for (int k = 0; k < n; ++k) {
                double aik = A(i, k);
                if (aik == 0.0) continue;
                const double* bk = &B.a[(size_t)k * n];
                for (int j = 0; j < n; ++j) ci[j] += aik * bk[j];
            }
        }
    };
    const int hw = (int)std::thread::hardware_concurrency();
    const int nt = n >= 256 ? std::max(1, std::min(hw, 32)) : 1;
    if (nt == 1) {
        rows(0, n);
        return C;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(rows, (int)((long long)n * t / nt), (int)((long long)n * (t + 1) / nt));
    for (std::thread& th : pool) th.join();
    return C;
}

static Mat axpby(double a, const Mat& X, double b, const Mat& Y) {
    Mat Z(X.n);
    for (size_t i = 0; i < Z.a.size(); ++i) Z.a[i] = a * X.a[i] + b * Y.a[i];
    return Z;
}

struct Aug {
    Mat T, B;
    double c = 0.0;
};

static Aug aug_mul(const Aug& x, const Aug& y) {
    Aug z;
    z.T = matmul(x.T, y.T);
    z.B = axpby(1.0, matmul(x.T, y.B), y.c, x.B);
    z.c = x.c * y.c;
    return z;
}

static Aug aug_lin(double a, const Aug& x, double b, const Aug& y) {
    Aug z;
    z.T = axpby(a, x.T, b, y.T);
    z.B = axpby(a, x.B, b, y.B);
    z.c = a * x.c + b * y.c;
    return z;
}

static Aug aug_identity(int n) {
    Aug z;
    z.T = Mat(n);
    z.B = Mat(n);
    for (int i = 0; i < n; ++i) z.T(i, i) = 1.0;
    z.c = 1.0;
    return z;
}

// Solve P X = R for X (n x n right-hand sides) by LU with partial pivoting: P is
// factored first (multipliers kept below the diagonal, pivots recorded), then
// the right-hand-side columns are eliminated and back-substituted in blocks on
// host threads, every column with the same operations in the same order.
static Mat lu_solve(Mat P, Mat R) {
    const int n = P.n;
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int pk = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(P(i, k)) > std::fabs(P(pk, k))) pk = i;
        if (P(pk, k) == 0.0) throw std::runtime_error("singular Pade denominator");
        piv[k] = pk;
        if (pk != k)
            for (int j = 0; j < n; ++j) std::swap(P(k, j), P(pk, j));
        for (int i = k + 1; i < n; ++i) {
            const double f = P(i, k) / P(k, k);
            P(i, k) = f;
            if (f == 0.0) continue;
            for (int j = k + 1; j < n; ++j) P(i, j) -= f * P(k, j);
        }
    }
    auto cols = [&](int c0, int c1) {
        for (int k = 0; k < n; ++k) {
            if (piv[k] != k)
                for (int j = c0; j < c1; ++j) std::swap(R(k, j), R(piv[k], j));
            for (int i = k + 1; i < n; ++i) {
                const double f = P(i, k);
                if (f == 0.0) continue;
                for (int j = c0; j < c1; ++j) R(i, j) -= f * R(k, j);
            }
        }
        for (int k = n - 1; k >= 0; --k)
            for (int j = c0; j < c1; ++j) {
                double s = R(k, j);
                for (int i = k + 1; i < n; ++i) s -= P(k, i) * R(i, j);
                R(k, j) = s / P(k, k);
            }
    };
    const int hw = (int)std::thread::hardware_concurrency();
    const int nt = n >= 256 ? std::max(1, std::min(hw, 32)) : 1;
    if (nt == 1) {
        cols(0, n);
        return R;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(cols, (int)((long long)n * t / nt), (int)((long long)n * (t + 1) / nt));
    for (std::thread& th : pool) th.join();
    return R;
}

Mat phi1_pade(const Mat& X) {
    const int n = X.n;
    // [13/13] diagonal Pade coefficients b_j = (2m-j)! m! / ((2m)! j! (m-j)!), m = 13,
    // generated by their ratio b_j / b_{j-1} = (m-j+1) / (j (2m-j+1)).
    const int m = 13;
    double b[m + 1];
    b[0] = 1.0;
    for (int j = 1; j <= m; ++j) b[j] = b[j - 1] * (m - j + 1) / (j * (2.0 * m - j + 1));
    // theta_13 of Higham (2005), Table 2.3: backward error below 2^-53 for ||A||_1 <= theta_13.
    const double theta13 = 5.371920351148152;
    double norm1 = 1.0;   // the identity block contributes column sums of 1
    for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += std::fabs(X(r, c));
        norm1 = std::max(norm1, s);
    }
    int sq = 0;
    if (norm1 > theta13) sq = (int)std::ceil(std::log2(norm1 / theta13));
    const double scale = std::ldexp(1.0, -sq);
    Aug A;
    A.T = axpby(scale, X, 0.0, X);
    A.B = Mat(n);
    for (int i = 0; i < n; ++i) A.B(i, i) = scale;
    A.c = 0.0;
    Aug I = aug_identity(n);
    Aug A2 = aug_mul(A, A), A4 = aug_mul(A2, A2), A6 = aug_mul(A4, A2);
    // U = A [A6 (b13 A6 + b11 A4 + b9 A2) + b7 A6 + b5 A4 + b3 A2 + b1 I]
    Aug t1 = aug_lin(b[13], A6, b[11], A4);
    t1 = aug_lin(1.0, t1, b[9], A2);
    Aug t2 = aug_mul(A6, t1);
    t2 = aug_lin(1.0, t2, b[7], A6);
    t2 = aug_lin(1.0, t2, b[5], A4);
    t2 = aug_lin(1.0, t2, b[3], A2);
    t2 = aug_lin(1.0, t2, b[1], I);
    Aug U = aug_mul(A, t2);
    // V = A6 (b12 A6 + b10 A4 + b8 A2) + b6 A6 + b4 A4 + b2 A2 + b0 I
    Aug v1 = aug_lin(b[12], A6, b[10], A4);
    v1 = aug_lin(1.0, v1, b[8], A2);
    Aug V = aug_mul(A6, v1);
    V = aug_lin(1.0, V, b[6], A6);
    V = aug_lin(1.0, V, b[4], A4);
    V = aug_lin(1.0, V, b[2], A2);
    V = aug_lin(1.0, V, b[0], I);
    Aug P = aug_lin(1.0, V, -1.0, U), Qn = aug_lin(1.0, V, 1.0, U);
    // R = P^{-1} Qn in the block algebra: R.c = Qn.c/P.c, R.T = P.T^{-1} Qn.T,
    // R.B = P.T^{-1} (Qn.B - P.B R.c).
    Aug R;
    R.c = Qn.c / P.c;
    R.T = lu_solve(P.T, Qn.T);
    R.B = lu_solve(P.T, axpby(1.0, Qn.B, -R.c, P.B));
    for (int s = 0; s < sq; ++s) R = aug_mul(R, R);
    return R.B;
}

double phi1_scalar(double x) { return x == 0.0 ? 1.0 : std::expm1(x) / x; }

double dphi1_scalar(double x) {
    if (std::fabs(x) < 0.1) {
        double term = 0.5, sum = 0.5;          // k = 0: 1/2!
        for (int k = 1; k <= 12; ++k) {
            term *= x / (k + 2);               // x^k / (k+2)!  (times (k+1), applied below)
            sum += (k + 1) * term;
        }
        return sum;
    }
    return (x + std::expm1(x) * (x - 1.0)) / (x * x);
}

}  // namespace sexpe
