// FP64 host-side setup of the split exponential Euler plan: 1-D axes,
// eigenbases and phi_1 matrices.  Runs once per plan (the paper's
// "once and for all" initialisation, Section 4), never inside a step.
#pragma once
#include <vector>

namespace sexpe {

// Dense row-major n x n matrix.
struct Mat {
    int n = 0;
    std::vector<double> a;
    Mat() = default;
    explicit Mat(int n_) : n(n_), a((size_t)n_ * n_, 0.0) {}
    double& operator()(int r, int c) { return a[(size_t)r * n + c]; }
    double operator()(int r, int c) const { return a[(size_t)r * n + c]; }
};

// One axis: grid points and the tridiagonal (or periodic tridiagonal) matrix
// as lower[r] = A[r][r-1], diag[r] = A[r][r], upper[r] = A[r][r+1];
// periodic axes wrap lower[0] to column n-1 and upper[n-1] to column 0.
struct Axis {
    int n = 0;
    bool periodic = false;
    std::vector<double> pts, lower, diag, upper;
    double sigma = 0.0;   // phi axis only
    Mat dense() const;
};

enum AxisKind { AX_THETA, AX_RHO2, AX_RHO3, AX_PHI, AX_Z_NEUMANN, AX_Z_PAPER, AX_RHO_LAMBDA };

// Section 3: eq. (A_theta), (disk_discr), (ball_discr), (syscn)/(A_phi), (A_z);
// Section 5.3: eq. (A_lambda), Delta_lambda's radial part with Dirichlet at rho_*
// (lambda < 1; the diagonal varies by row).
Axis build_axis(AxisKind kind, int n, double extent, double lambda = 0.0);

// Root of cot(x pi/(n-1+2x)) - 2(n-1+2x)/pi on (0, 1/2) (Appendix A).
double phi_sigma(int n);

// Eigen decomposition A = V diag(lam) Vinv.
struct Eigen {
    std::vector<double> lam;
    Mat V, Vinv;
};
// Closed-form real Fourier eigenbasis of the circulant A_theta (orthogonal, Vinv = V^T).
Eigen theta_eigen(const Axis& ax);
// Proposition 1: S = Xi^{-1} A Xi symmetric tridiagonal, implicit QL on S, V = Xi Q, Vinv = Q^T Xi^{-1}.
Eigen tridiag_eigen(const Axis& ax);

// phi_1(X) by [13/13] Pade scaling and squaring of expm([[X, I], [0, 0]])
// (Higham 2005), exploiting the block structure of the augmented matrix.
Mat phi1_pade(const Mat& X);

// Scalar phi_1(x) = expm1(x)/x, 1 at 0.
double phi1_scalar(double x);

// Derivative phi_1'(x) = phi_1(x) - phi_2(x) = (x + expm1(x)(x - 1))/x^2, 1/2 at 0
// (Taylor series sum_k (k+1) x^k/(k+2)! for |x| < 0.1).
double dphi1_scalar(double x);

}  // namespace sexpe
