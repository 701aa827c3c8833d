// Host-side launch entry points of the kernels (internal to libsexpe).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace sexpe {

// FP64 SIMT path.
cudaError_t launch_rhs64(int geometry, const RhsTables<double>& tb, const double* W, double* F, cudaStream_t st);
cudaError_t launch_gemm64(const Gemm64& g, int n_species, cudaStream_t st);
// Bulk-surface coupling terms added to the bulk and surface F (FP64 chains), or to
// the FP32 F of the split chains (Yb, Ys: layouts [s][k][j][n1q], ys floats per species).
cudaError_t launch_couple64(const CoupleArgs& a, const double* Wb, const double* Ws, double* Fb, double* Fs,
                            cudaStream_t st);
cudaError_t launch_couple_split(const CoupleArgs& a, const double* Wb, const double* Ws, float* Yb, float* Ys,
                                int n1q_b, long long ys_b, int n1q_s, long long ys_s, cudaStream_t st);
// Unsplit baseline: W_s += tau P_s F_s, P_s dense N x N row-major.
cudaError_t launch_matvec64(const double* P, const double* F, double* W, int N, int S, double tau, cudaStream_t st);
// Discrete adjoint (FP64).
cudaError_t launch_adj_lambda(int geometry, const RhsTables<double>& tb, const double* W, const double* mu,
                              double* lam, cudaStream_t st);
cudaError_t launch_adj_params(int geometry, const RhsTables<double>& tb, const double* W, const double* mu,
                              double* acc, cudaStream_t st);
// lambda += d M^T mu + J^T mu and the parameter sums in one pass (np reaction parameters + S <= 8).
cudaError_t launch_adj_fused(int geometry, const RhsTables<double>& tb, const RhsTables<double>& tbT, const double* W,
                             const double* mu, double* lam, double* acc, int np, cudaStream_t st);
// The same for the split-TF32 adjoint in FP32 arithmetic: mu (FP32, chain layout [s][rows][n1q]) with
// M^T in difference form (tbT), M w from split pairs of the state (tbF), lambda and the sums FP64.
cudaError_t launch_adj_fused_split(int geometry, const RhsTables<float>& tbF, const RhsTables<float>& tbT,
                                   const double* W, const float* mu, int n1q, long long ys, double* lam, double* acc,
                                   int np, cudaStream_t st);
cudaError_t launch_wdot(const double* a, const double* b, const double* wt, long long npts, int S, double scale,
                        double* acc, cudaStream_t st);
cudaError_t launch_scale(double* x, double a, long long n, cudaStream_t st);
// Split-TF32 adjoint: the adjoint variable between the FP64 state layout [s][r][n1] and the FP32
// chain layout [s][r][n1q] (ys floats per species), and acc[s] += <a_s, b_s> across the two layouts.
cudaError_t launch_to_chain_f32(const double* src, float* dst, int n1, int n1q, long long ys, long long npts, int S,
                                cudaStream_t st);
cudaError_t launch_from_chain_f32(const float* src, double* dst, int n1, int n1q, long long ys, long long npts, int S,
                                  cudaStream_t st);
cudaError_t launch_dot_state_chain(const double* a, const float* b, int n1, int n1q, long long ys, long long npts,
                                   int S, double* acc, cudaStream_t st);
cudaError_t launch_tick(long long* step, cudaStream_t st);

// Split-TF32 tensor-core path.
// Shared-memory rings and tensor-memory columns of a tensor-core kernel.
struct TcShape {
    uint32_t mat_bytes;    // bytes per matrix slot (hi + lo tiles of the widest product)
    uint32_t data_bytes;   // bytes per data slot
    uint32_t nm, nd;       // slots in the matrix and data rings
    uint32_t tmem_cols;
    uint32_t smem_bytes;
};
TcShape tc_mode3_shape(int geometry, int n1, int n2, int n3);
TcShape tc_slab_shape(int n1, int n2);
uint32_t slab_tmem_cols(int n1, int n2);
// Raise the kernels' dynamic shared-memory limit (once, outside stream capture).
cudaError_t tc_prepare(uint32_t smem_mode3, uint32_t smem_slab);
cudaError_t launch_tc_mode3(const SplitTables& T, const TcShape& sh, cudaStream_t st);
cudaError_t launch_tc_slab(const SplitTables& T, const TcShape& sh, cudaStream_t st);
cudaError_t launch_rhs_split(const SplitTables& T, cudaStream_t st);
cudaError_t launch_wait_selftest(int* err, long long limit_cycles, cudaStream_t st);
// Sphere: phi product (plain), then theta pair (scaled) + update.
TcShape tc_sphere_phi_shape(int nt);
TcShape tc_sphere_theta_shape(int n1, int nt);
cudaError_t tc_prepare_sphere(uint32_t smem_phi, uint32_t smem_theta);
cudaError_t launch_tc_sphere_phi(const SplitTables& T, const TcShape& sh, cudaStream_t st);
cudaError_t launch_tc_sphere_theta(const SplitTables& T, const TcShape& sh, cudaStream_t st);
// Split sphere adjoint: G1 = lambda x_1 Q^T, the Phi and dPhi/dd products x_1 Q, tau P_theta lambda out,
// the two d-derivative dots accumulated (see k_tc_sphere_theta_adj).
TcShape tc_sphere_theta_adj_shape(int n1, int nt);
cudaError_t launch_tc_sphere_theta_adj(const SplitTables& T, const TcShape& sh, const SphereAdjArgs& A,
                                       cudaStream_t st);
int rhs_candidates(const SplitTables& T, int3* out, int max_out);
// Batched disks: one persistent launch per step.
TcShape tc_batch_shape(int max_n1, int max_n2, uint32_t tmem_cols);
int tc_batch_shapes(int max_n1, int max_n2, uint32_t tmem_cols, int max_tj, TcShape* out, int cap);
cudaError_t tc_prepare_batch(uint32_t smem);
cudaError_t launch_tc_batch(const BatchTables& B, const TcShape& sh, int grid, cudaStream_t st);
int batch_grid(const TcShape& sh);

}  // namespace sexpe
