// FP64 SIMT kernels of the split exponential Euler step: stencil + reaction,
// and mu-mode products (tensor x small dense matrix) with optional Hadamard
// factor and fused update.  The comparison leg of the split-TF32 path.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"
#include "couple_terms.cuh"
#include "launch.h"

namespace sexpe {

template <int GEO>
__global__ void __launch_bounds__(256) k_rhs64(RhsTables<double> tb, const double* __restrict__ W,
                                               double* __restrict__ F) {
    const long long npts = tb.npts;
    const long long total = npts * tb.S;
    const double et = GEO == GEO_DISK ? mms_time_factor(tb) : 1.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / npts);
        const long long idx = t - (long long)s * npts;
        const int i = (int)(idx % tb.n1);
        const long long rest = idx / tb.n1;
        const int j = (int)(rest % tb.n2);
        const int k = (int)(rest / tb.n2);
        double f = rhs_point<F64Acc, GEO>(tb, W, s, idx, i, j, k);
        if (GEO == GEO_DISK && tb.reac.kind == R_BVAM_MMS) f += mms_source<double>(tb, i, j, et, s);
        F[t] = f;
    }
}

// Advance the step counter of a plan with time-dependent sources (one thread).
__global__ void k_tick(long long* step) { *step += 1; }

cudaError_t launch_tick(long long* step, cudaStream_t st) {
    k_tick<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}

// C(b, r, c) = sum_k A(b, r, k) B(b, k, c), tiles of 64 x 64, K-chunks of 16,
// 256 threads with 4 x 4 outputs each.  blockIdx.z = species * batch + b.
constexpr int G64_BM = 64, G64_BN = 64, G64_BK = 16;

__global__ void __launch_bounds__(256) k_gemm64(Gemm64 g) {
    __shared__ double As[G64_BK][G64_BM + 1];
    __shared__ double Bs[G64_BK][G64_BN + 1];
    const int s = blockIdx.z / g.batch;
    const int b = blockIdx.z % g.batch;
    const int r0 = blockIdx.y * G64_BM, c0 = blockIdx.x * G64_BN;
    const double* A = g.A + s * g.A_sp + b * g.a_b;
    const double* B = g.B + s * g.B_sp + b * g.b_b;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < g.K; k0 += G64_BK) {
        for (int e = threadIdx.x; e < G64_BM * G64_BK; e += 256) {
            const int rr = e / G64_BK, kk = e % G64_BK;
            const int r = r0 + rr, k = k0 + kk;
            As[kk][rr] = (r < g.R && k < g.K) ? A[r * g.a_r + k * g.a_k] : 0.0;
        }
        for (int e = threadIdx.x; e < G64_BN * G64_BK; e += 256) {
            const int kk = e / G64_BN, cc = e % G64_BN;
            const int c = c0 + cc, k = k0 + kk;
            Bs[kk][cc] = (c < g.C && k < g.K) ? B[k * g.b_k + c * g.b_c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < G64_BK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = As[kk][ty * 4 + q];
#pragma unroll
            for (int q = 0; q < 4; ++q) bb[q] = Bs[kk][tx * 4 + q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], bb[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int r = r0 + ty * 4 + p;
        if (r >= g.R) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + tx * 4 + q;
            if (c >= g.C) continue;
            const long long o = b * g.o_b + r * g.o_r + c * g.o_c;
            double v = acc[p][q];
            if (g.had) v *= g.had[s * g.had_sp + o];
            if (g.upd) g.upd[s * g.upd_sp + o] += g.tau * v;
            else g.out[s * g.out_sp + o] = v;
        }
    }
}

__device__ __forceinline__ long long couple_bulk_node(const CoupleArgs& a, long long q) {
    return a.kind == 0 ? (a.bn1 - 1) + (long long)a.bn1 * q : q;
}

// Bulk-surface coupling for the FP64 chains: one thread per surface point adds the
// terms to the bulk F (buffer of the bulk sub-plan, species stride nb) and the
// surface F (species stride ns), both computed from the state at t_n.
__global__ void k_couple64(CoupleArgs a, const double* __restrict__ Wb, const double* __restrict__ Ws,
                           double* __restrict__ Fb, double* __restrict__ Fs) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.ns) return;
    const long long b = couple_bulk_node(a, q);
    double add[4];
    couple_terms(a, Wb[b], Wb[a.nb + b], Ws[q], Ws[a.ns + q], add);
    Fb[b] += add[0];
    Fb[a.nb + b] += add[1];
    Fs[q] += add[2];
    Fs[a.ns + q] += add[3];
}

cudaError_t launch_couple64(const CoupleArgs& a, const double* Wb, const double* Ws, double* Fb, double* Fs,
                            cudaStream_t st) {
    k_couple64<<<(unsigned)((a.ns + 255) / 256), 256, 0, st>>>(a, Wb, Ws, Fb, Fs);
    return cudaGetLastError();
}

// The same terms for the split-TF32 chains, whose F is FP32 in the padded layout
// [s][k][j][n1q] of each grid: the ball's boundary node (n_rho - 1, j, k) and the
// cylinder's (i, j, 0); the surface point (a, c) = (q mod sn1, q / sn1) at
// c n1q + a.  The terms are added to F in FP64 before rounding to FP32.
__global__ void k_couple_split(CoupleArgs a, const double* __restrict__ Wb, const double* __restrict__ Ws,
                               float* __restrict__ Yb, float* __restrict__ Ys, int n1q_b, long long ys_b, int n1q_s,
                               long long ys_s) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.ns) return;
    const long long b = couple_bulk_node(a, q);
    double add[4];
    couple_terms(a, Wb[b], Wb[a.nb + b], Ws[q], Ws[a.ns + q], add);
    const long long ca = q % a.sn1, cc = q / a.sn1;
    const long long yb = a.kind == 0 ? (cc * a.bn2 + ca) * n1q_b + (a.bn1 - 1) : cc * n1q_b + ca;
    const long long ysq = cc * n1q_s + ca;
    Yb[yb] = (float)((double)Yb[yb] + add[0]);
    Yb[ys_b + yb] = (float)((double)Yb[ys_b + yb] + add[1]);
    Ys[ysq] = (float)((double)Ys[ysq] + add[2]);
    Ys[ys_s + ysq] = (float)((double)Ys[ys_s + ysq] + add[3]);
}

cudaError_t launch_couple_split(const CoupleArgs& a, const double* Wb, const double* Ws, float* Yb, float* Ys,
                                int n1q_b, long long ys_b, int n1q_s, long long ys_s, cudaStream_t st) {
    k_couple_split<<<(unsigned)((a.ns + 255) / 256), 256, 0, st>>>(a, Wb, Ws, Yb, Ys, n1q_b, ys_b, n1q_s, ys_s);
    return cudaGetLastError();
}

// Unsplit baseline: W_s[r] += tau sum_k P_s[r][k] F_s[k] (row-major N x N per
// species), one warp per row, lanes striding the row (coalesced), a warp-shuffle
// reduction, then the update by lane 0.  grid (ceil(N / 8), S), 256 threads.
__global__ void __launch_bounds__(256) k_matvec64(const double* __restrict__ P, const double* __restrict__ F,
                                                  double* __restrict__ W, int N, double tau) {
    const int s = blockIdx.y;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= N) return;
    const double* pr = P + ((long long)s * N + row) * N;
    const double* f = F + (long long)s * N;
    double acc = 0.0;
    for (int k = lane; k < N; k += 32) acc = fma(__ldg(pr + k), __ldg(f + k), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) W[(long long)s * N + row] += tau * acc;
}

cudaError_t launch_matvec64(const double* P, const double* F, double* W, int N, int S, double tau, cudaStream_t st) {
    k_matvec64<<<dim3((N + 7) / 8, S), 256, 0, st>>>(P, F, W, N, tau);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the step (derived from eqs. ee and splitorder; the paper
// has no adjoint).  With mu_s = tau P_s^T lambda_s:
//   lambda_r += d_r (M^T mu_r) + sum_s (dG_s/dW_r) mu_s.
// M^T keeps the Kronecker structure: along mode m, (A^T x)_r = a_r x_r
// + c-entry of row r+1 times x_{r+1} + b-entry of row r-1 times x_{r-1},
// scaled by the point's own diagonal factors of the other modes.

__device__ __forceinline__ double axisT(const StencilAxis<double>& ax, const double* x, long long idx, int r,
                                        long long st) {
    // ax.rs carries the full diagonal a_r here
    double acc = ax.rs[r] * x[idx];
    if (r < ax.n - 1) acc += ax.lower[r + 1] * x[idx + st];
    else if (ax.periodic) acc += ax.lower[0] * x[idx - (long long)(ax.n - 1) * st];
    if (r > 0) acc += ax.upper[r - 1] * x[idx - st];
    else if (ax.periodic) acc += ax.upper[ax.n - 1] * x[idx + (long long)(ax.n - 1) * st];
    return acc;
}

template <int GEO>
__device__ __forceinline__ double laplacianT(const RhsTables<double>& tb, const double* x, long long idx, int i, int j,
                                             int k) {
    const double t0 = axisT(tb.ax[0], x, idx, i, 1);
    const double t1 = axisT(tb.ax[1], x, idx, j, tb.n1);
    if constexpr (GEO == GEO_DISK) return t0 + tb.Dr[i] * t1;
    if constexpr (GEO == GEO_SPHERE) return tb.Dp[j] * t0 + t1;
    const double t2 = axisT(tb.ax[2], x, idx, k, (long long)tb.n1 * tb.n2);
    if constexpr (GEO == GEO_BALL) return t0 + tb.Dr[i] * (tb.Dp[k] * t1 + t2);
    return t0 + tb.Dr[i] * t1 + t2;
}

// sum_s (dG_s/dW_r) mu_s at one point, for species r.
__device__ __forceinline__ double reaction_jt(const ReactionParams<double>& rp, const double* w, const double* mu,
                                              int r) {
    switch (rp.kind) {
    case R_SCHNAKENBERG: {
        const double g = rp.p[0], u = w[0], v = w[1];
        // f = g(a - u + u^2 v), h = g(b - u^2 v)
        return r == 0 ? mu[0] * g * (-1.0 + 2.0 * u * v) - mu[1] * 2.0 * g * u * v
                      : mu[0] * g * u * u - mu[1] * g * u * u;
    }
    case R_GRAY_SCOTT: {
        const double F = rp.p[0], kk = rp.p[1], u = w[0], v = w[1];
        // f = -u v^2 + F(1-u), h = u v^2 - (F+k) v
        return r == 0 ? mu[0] * (-v * v - F) + mu[1] * v * v
                      : mu[0] * (-2.0 * u * v) + mu[1] * (2.0 * u * v - (F + kk));
    }
    case R_LINEAR_CUBIC: {
        double acc = -3.0 * w[r] * w[r] * mu[r];
        for (int i = 0; i < rp.S; ++i) acc += mu[i] * rp.p[i * rp.S + r];
        return acc;
    }
    default:
        return 0.0;
    }
}

template <int GEO>
__global__ void __launch_bounds__(256) k_adj_lambda(RhsTables<double> tb, const double* __restrict__ W,
                                                    const double* __restrict__ mu, double* __restrict__ lam) {
    const long long npts = tb.npts;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < npts;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % tb.n1);
        const long long rest = idx / tb.n1;
        const int j = (int)(rest % tb.n2);
        const int k = (int)(rest / tb.n2);
        double w[kMaxSpecies], m[kMaxSpecies];
        for (int r = 0; r < kMaxSpecies; ++r) {
            w[r] = r < tb.S ? W[r * npts + idx] : 0.0;
            m[r] = r < tb.S ? mu[r * npts + idx] : 0.0;
        }
        for (int r = 0; r < tb.S; ++r)
            lam[r * npts + idx] += tb.d[r] * laplacianT<GEO>(tb, mu + r * npts, idx, i, j, k) +
                                   reaction_jt(tb.reac, w, m, r);
    }
}

// Per-point contributions to the parameter gradient: reaction parameters
// sum_s mu_s dG_s/dp, then <mu_s, (M W_s)> for the diffusion of each species.
template <int GEO>
__global__ void __launch_bounds__(256) k_adj_params(RhsTables<double> tb, const double* __restrict__ W,
                                                    const double* __restrict__ mu, double* __restrict__ acc) {
    constexpr int kSlots = 16 + kMaxSpecies;
    __shared__ double red[kSlots][8];
    double part[kSlots];
    for (int q = 0; q < kSlots; ++q) part[q] = 0.0;
    const long long npts = tb.npts;
    const int np = tb.reac.kind == R_SCHNAKENBERG ? 3 : (tb.reac.kind == R_GRAY_SCOTT ? 2 :
                   (tb.reac.kind == R_LINEAR_CUBIC ? tb.S * tb.S : 0));
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < npts;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % tb.n1);
        const long long rest = idx / tb.n1;
        const int j = (int)(rest % tb.n2);
        const int k = (int)(rest / tb.n2);
        double w[kMaxSpecies], m[kMaxSpecies];
        for (int r = 0; r < kMaxSpecies; ++r) {
            w[r] = r < tb.S ? W[r * npts + idx] : 0.0;
            m[r] = r < tb.S ? mu[r * npts + idx] : 0.0;
        }
        switch (tb.reac.kind) {
        case R_SCHNAKENBERG: {   // params (gamma, a, b)
            const double u2v = w[0] * w[0] * w[1];
            part[0] += m[0] * (tb.reac.p[1] - w[0] + u2v) + m[1] * (tb.reac.p[2] - u2v);
            part[1] += m[0] * tb.reac.p[0];
            part[2] += m[1] * tb.reac.p[0];
            break;
        }
        case R_GRAY_SCOTT:       // params (F, k)
            part[0] += m[0] * (1.0 - w[0]) - m[1] * w[1];
            part[1] += -m[1] * w[1];
            break;
        case R_LINEAR_CUBIC:     // params K (row-major): d f_a / d K_ab = u_b
            for (int a = 0; a < tb.S; ++a)
                for (int b = 0; b < tb.S; ++b) part[a * tb.S + b] += m[a] * w[b];
            break;
        default:
            break;
        }
        for (int r = 0; r < tb.S; ++r)
            part[16 + r] += m[r] * laplacian<F64Acc, GEO>(tb, W + r * npts, idx, i, j, k, W[r * npts + idx]);
    }
    // block reduction (warp shuffles, then across the 8 warps)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kSlots; ++q) {
        double v = part[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSlots) {
        const int q = threadIdx.x;
        if (q < np || (q >= 16 && q < 16 + tb.S)) {
            double v = 0.0;
            for (int w8 = 0; w8 < 8; ++w8) v += red[q][w8];
            atomicAdd(&acc[q], v);
        }
    }
}

// Per-point reaction-parameter derivatives sum_s mu_s dG_s/dp into part[0 .. np).
__device__ __forceinline__ void reaction_param_parts(const ReactionParams<double>& rp, const double* w, const double* m,
                                                     double* part) {
    switch (rp.kind) {
    case R_SCHNAKENBERG: {   // params (gamma, a, b)
        const double u2v = w[0] * w[0] * w[1];
        part[0] += m[0] * (rp.p[1] - w[0] + u2v) + m[1] * (rp.p[2] - u2v);
        part[1] += m[0] * rp.p[0];
        part[2] += m[1] * rp.p[0];
        break;
    }
    case R_GRAY_SCOTT:       // params (F, k)
        part[0] += m[0] * (1.0 - w[0]) - m[1] * w[1];
        part[1] += -m[1] * w[1];
        break;
    case R_LINEAR_CUBIC:     // params K (row-major): d f_a / d K_ab = u_b
        for (int a = 0; a < rp.S; ++a)
            for (int b = 0; b < rp.S; ++b) part[a * rp.S + b] += m[a] * w[b];
        break;
    default:
        break;
    }
}

// One pass of an adjoint step after mu is formed: lambda_r += d_r M^T mu_r + sum_s (dG_s/dW_r) mu_s
// and the parameter sums (reaction parameters, then <mu_s, M W_s> per species) of k_adj_lambda and
// k_adj_params in one read of W and mu, with kFusedSlots partial sums per thread.  tbT carries M^T
// (the full diagonal in rs), tb the difference-form M.  Needs np + S <= kFusedSlots.
constexpr int kFusedSlots = 8;
template <int GEO>
__global__ void __launch_bounds__(256) k_adj_fused(RhsTables<double> tb, RhsTables<double> tbT,
                                                   const double* __restrict__ W, const double* __restrict__ mu,
                                                   double* __restrict__ lam, double* __restrict__ acc, int np) {
    __shared__ double red[kFusedSlots][8];
    double part[kFusedSlots];
#pragma unroll
    for (int q = 0; q < kFusedSlots; ++q) part[q] = 0.0;
    const long long npts = tb.npts;                 // < 2^31 (at most 512^3 points): 32-bit index arithmetic
    const int n1 = tb.n1, n2 = tb.n2, np32 = (int)npts;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < np32; idx += gridDim.x * blockDim.x) {
        const int rest = idx / n1;
        const int i = idx - rest * n1;
        const int k = rest / n2;
        const int j = rest - k * n2;
        double w[kMaxSpecies], m[kMaxSpecies];
        for (int r = 0; r < kMaxSpecies; ++r) {
            w[r] = r < tb.S ? W[r * npts + idx] : 0.0;
            m[r] = r < tb.S ? mu[r * npts + idx] : 0.0;
        }
        reaction_param_parts(tb.reac, w, m, part);
        for (int r = 0; r < tb.S; ++r) {
            part[np + r] += m[r] * laplacian<F64Acc, GEO>(tb, W + r * npts, idx, i, j, k, W[r * npts + idx]);
            lam[r * npts + idx] += tb.d[r] * laplacianT<GEO>(tbT, mu + r * npts, idx, i, j, k) +
                                   reaction_jt(tb.reac, w, m, r);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kFusedSlots; ++q) {
        double v = part[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < np + tb.S) {
        const int q = threadIdx.x;
        double v = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) v += red[q][w8];
        atomicAdd(&acc[q < np ? q : 16 + (q - np)], v);
    }
}

// sum_s (dG_s/dW_r) mu_s at one point, for species r, in the arithmetic type T.
template <class T>
__device__ __forceinline__ T reaction_jt_t(const ReactionParams<T>& rp, const T* w, const T* mu, int r) {
    switch (rp.kind) {
    case R_SCHNAKENBERG: {
        const T g = rp.p[0], u = w[0], v = w[1];
        return r == 0 ? mu[0] * g * ((T)-1 + (T)2 * u * v) - mu[1] * (T)2 * g * u * v
                      : mu[0] * g * u * u - mu[1] * g * u * u;
    }
    case R_GRAY_SCOTT: {
        const T F = rp.p[0], kk = rp.p[1], u = w[0], v = w[1];
        return r == 0 ? mu[0] * (-v * v - F) + mu[1] * v * v
                      : mu[0] * ((T)-2 * u * v) + mu[1] * ((T)2 * u * v - (F + kk));
    }
    case R_LINEAR_CUBIC: {
        T acc = (T)-3 * w[r] * w[r] * mu[r];
        for (int i = 0; i < rp.S; ++i) acc += mu[i] * rp.p[i * rp.S + r];
        return acc;
    }
    default:
        return (T)0;
    }
}

// Per-point reaction-parameter derivatives in FP32, summed into FP64 partials.
__device__ __forceinline__ void reaction_param_parts_f32(const ReactionParams<float>& rp, const float* w,
                                                         const float* m, double* part) {
    switch (rp.kind) {
    case R_SCHNAKENBERG: {
        const float u2v = w[0] * w[0] * w[1];
        part[0] += (double)(m[0] * (rp.p[1] - w[0] + u2v) + m[1] * (rp.p[2] - u2v));
        part[1] += (double)(m[0] * rp.p[0]);
        part[2] += (double)(m[1] * rp.p[0]);
        break;
    }
    case R_GRAY_SCOTT:
        part[0] += (double)(m[0] * (1.f - w[0]) - m[1] * w[1]);
        part[1] += (double)(-m[1] * w[1]);
        break;
    case R_LINEAR_CUBIC:
        for (int a = 0; a < rp.S; ++a)
            for (int b = 0; b < rp.S; ++b) part[a * rp.S + b] += (double)(m[a] * w[b]);
        break;
    default:
        break;
    }
}

// (A^T x)_r of one axis in difference form on FP32 values x (stride st in elements):
// tbT holds the transpose's off-diagonals and its column sums in rs.
__device__ __forceinline__ float axis_term_t32(const StencilAxis<float>& ax, const float* x, int r, long long st) {
    const float c = x[0];
    float acc = ax.rs[r] * c;
    if (r > 0) acc += ax.lower[r] * (x[-st] - c);
    else if (ax.periodic) acc += ax.lower[r] * (x[(long long)(ax.n - 1) * st] - c);
    if (r < ax.n - 1) acc += ax.upper[r] * (x[st] - c);
    else if (ax.periodic) acc += ax.upper[r] * (x[-(long long)(ax.n - 1) * st] - c);
    return acc;
}

// Split-TF32 adjoint, after mu is formed by the tensor-core chain: in one pass per point,
// lambda_r += d_r (M^T mu_r) + sum_s (dG_s/dW_r) mu_s and the parameter sums (reaction parameters,
// then <mu_s, M w_s>), with FP32 arithmetic -- M^T mu in difference form on the FP32 mu of the
// chain layout (tbT), M w from FP64-accurate split pairs of the state (tbF, the forward tables) --
// and FP64 for lambda and the sums.  mu: chain layout [s][rows][n1q], ys floats per species.
template <int GEO>
__global__ void __launch_bounds__(256) k_adj_fused_split(RhsTables<float> tbF, RhsTables<float> tbT,
                                                         const double* __restrict__ W, const float* __restrict__ mu,
                                                         int n1q, long long ys, double* __restrict__ lam,
                                                         double* __restrict__ acc, int np) {
    __shared__ double red[kFusedSlots][8];
    double part[kFusedSlots];
#pragma unroll
    for (int q = 0; q < kFusedSlots; ++q) part[q] = 0.0;
    const long long npts = tbF.npts;
    const int n1 = tbF.n1, n2 = tbF.n2, np32 = (int)npts;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < np32; idx += gridDim.x * blockDim.x) {
        const int rest = idx / n1;
        const int i = idx - rest * n1;
        const int k = rest / n2;
        const int j = rest - k * n2;
        const long long cidx = (long long)rest * n1q + i;
        float w[kMaxSpecies], m[kMaxSpecies];
        float2 wc[kMaxSpecies];
        for (int r = 0; r < kMaxSpecies; ++r) {
            wc[r] = r < tbF.S ? split_f64(__ldg(W + r * npts + idx)) : make_float2(0.f, 0.f);
            w[r] = wc[r].x + wc[r].y;
            m[r] = r < tbF.S ? __ldg(mu + r * ys + cidx) : 0.f;
        }
        reaction_param_parts_f32(tbF.reac, w, m, part);
        for (int r = 0; r < tbF.S; ++r) {
            part[np + r] += (double)m[r] * (double)laplacian<SplitAcc, GEO>(tbF, W + r * npts, idx, i, j, k, wc[r]);
            const float* x = mu + r * ys + cidx;
            const float t0 = axis_term_t32(tbT.ax[0], x, i, 1);
            const float t1 = axis_term_t32(tbT.ax[1], x, j, n1q);
            float mt;
            if constexpr (GEO == GEO_DISK) mt = t0 + tbT.Dr[i] * t1;
            else if constexpr (GEO == GEO_SPHERE) mt = tbT.Dp[j] * t0 + t1;
            else {
                const float t2 = axis_term_t32(tbT.ax[2], x, k, (long long)n1q * n2);
                if constexpr (GEO == GEO_BALL) mt = t0 + tbT.Dr[i] * (tbT.Dp[k] * t1 + t2);
                else mt = t0 + tbT.Dr[i] * t1 + t2;
            }
            lam[r * npts + idx] += (double)(tbF.d[r] * mt + reaction_jt_t<float>(tbF.reac, w, m, r));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kFusedSlots; ++q) {
        double v = part[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < np + tbF.S) {
        const int q = threadIdx.x;
        double v = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) v += red[q][w8];
        atomicAdd(&acc[q < np ? q : 16 + (q - np)], v);
    }
}

// acc[slot + s] += sum_p a[s][p] b[s][p] (wt ? wt[s][p] : 1) * scale for every species s.
__global__ void __launch_bounds__(256) k_wdot(const double* __restrict__ a, const double* __restrict__ b,
                                              const double* __restrict__ wt, long long npts, double scale,
                                              double* __restrict__ acc) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    double v = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
        const long long q = s * npts + p;
        v += a[q] * b[q] * (wt ? wt[q] : 1.0);
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) t += red[w8];
        atomicAdd(&acc[s], t * scale);
    }
}

__global__ void k_scale(double* __restrict__ x, double a, long long n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        x[p] *= a;
}

cudaError_t launch_adj_lambda(int geometry, const RhsTables<double>& tb, const double* W, const double* mu,
                              double* lam, cudaStream_t st) {
    long long blocks = (tb.npts + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    switch (geometry) {
    case GEO_DISK: k_adj_lambda<GEO_DISK><<<(int)blocks, 256, 0, st>>>(tb, W, mu, lam); break;
    case GEO_SPHERE: k_adj_lambda<GEO_SPHERE><<<(int)blocks, 256, 0, st>>>(tb, W, mu, lam); break;
    case GEO_BALL: k_adj_lambda<GEO_BALL><<<(int)blocks, 256, 0, st>>>(tb, W, mu, lam); break;
    default: k_adj_lambda<GEO_CYLINDER><<<(int)blocks, 256, 0, st>>>(tb, W, mu, lam); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_params(int geometry, const RhsTables<double>& tb, const double* W, const double* mu,
                              double* acc, cudaStream_t st) {
    long long blocks = (tb.npts + 255) / 256;
    if (blocks > 152LL * 4) blocks = 152LL * 4;
    switch (geometry) {
    case GEO_DISK: k_adj_params<GEO_DISK><<<(int)blocks, 256, 0, st>>>(tb, W, mu, acc); break;
    case GEO_SPHERE: k_adj_params<GEO_SPHERE><<<(int)blocks, 256, 0, st>>>(tb, W, mu, acc); break;
    case GEO_BALL: k_adj_params<GEO_BALL><<<(int)blocks, 256, 0, st>>>(tb, W, mu, acc); break;
    default: k_adj_params<GEO_CYLINDER><<<(int)blocks, 256, 0, st>>>(tb, W, mu, acc); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_wdot(const double* a, const double* b, const double* wt, long long npts, int S, double scale,
                        double* acc, cudaStream_t st) {
    long long blocks = (npts + 255) / 256;
    if (blocks > 152LL * 2) blocks = 152LL * 2;
    k_wdot<<<dim3((unsigned)blocks, S), 256, 0, st>>>(a, b, wt, npts, scale, acc);
    return cudaGetLastError();
}

cudaError_t launch_scale(double* x, double a, long long n, cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    k_scale<<<(int)blocks, 256, 0, st>>>(x, a, n);
    return cudaGetLastError();
}

cudaError_t launch_rhs64(int geometry, const RhsTables<double>& tb, const double* W, double* F,
                         cudaStream_t st) {
    const long long total = tb.npts * tb.S;
    const int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    switch (geometry) {
    case GEO_DISK: k_rhs64<GEO_DISK><<<(int)blocks, threads, 0, st>>>(tb, W, F); break;
    case GEO_SPHERE: k_rhs64<GEO_SPHERE><<<(int)blocks, threads, 0, st>>>(tb, W, F); break;
    case GEO_BALL: k_rhs64<GEO_BALL><<<(int)blocks, threads, 0, st>>>(tb, W, F); break;
    default: k_rhs64<GEO_CYLINDER><<<(int)blocks, threads, 0, st>>>(tb, W, F); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_gemm64(const Gemm64& g, int n_species, cudaStream_t st) {
    dim3 grid((g.C + G64_BN - 1) / G64_BN, (g.R + G64_BM - 1) / G64_BM, g.batch * n_species);
    k_gemm64<<<grid, 256, 0, st>>>(g);
    return cudaGetLastError();
}

// ---- split-TF32 adjoint helpers: the adjoint variable moves between the FP64 state layout
// [s][j][n1] (rows of n1 values, rows = npts / n1 per species) and the FP32 chain layout
// [s][j][n1q] of the tensor-core kernels (rows padded to n1q; the padding is never written).

// dst[s][r][i] = (float) src[s][r][i] for i < n1.
__global__ void __launch_bounds__(256) k_to_chain_f32(const double* __restrict__ src, float* __restrict__ dst, int n1,
                                                      int n1q, long long rows, long long ys, long long npts, int S) {
    const long long total = (long long)S * npts;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long s = q / npts, rest = q - s * npts;
        const long long r = rest / n1, i = rest - r * n1;
        dst[s * ys + r * n1q + i] = (float)src[q];
    }
    (void)rows;
}

// dst[s][r][i] = src[s][r][i] (FP32 chain layout to the FP64 state layout, exact).
__global__ void __launch_bounds__(256) k_from_chain_f32(const float* __restrict__ src, double* __restrict__ dst, int n1,
                                                        int n1q, long long ys, long long npts, int S) {
    const long long total = (long long)S * npts;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long s = q / npts, rest = q - s * npts;
        const long long r = rest / n1, i = rest - r * n1;
        dst[q] = (double)src[s * ys + r * n1q + i];
    }
}

// acc[s] += sum over the points of a[s][r][i] (FP64 state layout) * b[s][r][i] (FP32 chain layout).
__global__ void __launch_bounds__(256) k_dot_state_chain(const double* __restrict__ a, const float* __restrict__ b,
                                                         int n1, int n1q, long long ys, long long npts,
                                                         double* __restrict__ acc) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    double v = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
        const long long r = p / n1, i = p - r * n1;
        v += a[s * npts + p] * (double)b[s * ys + r * n1q + i];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) t += red[w8];
        atomicAdd(&acc[s], t);
    }
}

static int helper_blocks(long long n, long long cap) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_to_chain_f32(const double* src, float* dst, int n1, int n1q, long long ys, long long npts, int S,
                                cudaStream_t st) {
    k_to_chain_f32<<<helper_blocks((long long)S * npts, 152LL * 8), 256, 0, st>>>(src, dst, n1, n1q, npts / n1, ys,
                                                                                  npts, S);
    return cudaGetLastError();
}

cudaError_t launch_from_chain_f32(const float* src, double* dst, int n1, int n1q, long long ys, long long npts, int S,
                                  cudaStream_t st) {
    k_from_chain_f32<<<helper_blocks((long long)S * npts, 152LL * 8), 256, 0, st>>>(src, dst, n1, n1q, ys, npts, S);
    return cudaGetLastError();
}

cudaError_t launch_dot_state_chain(const double* a, const float* b, int n1, int n1q, long long ys, long long npts,
                                   int S, double* acc, cudaStream_t st) {
    k_dot_state_chain<<<dim3((unsigned)helper_blocks(npts, 152LL * 2), S), 256, 0, st>>>(a, b, n1, n1q, ys, npts, acc);
    return cudaGetLastError();
}

cudaError_t launch_adj_fused(int geometry, const RhsTables<double>& tb, const RhsTables<double>& tbT, const double* W,
                             const double* mu, double* lam, double* acc, int np, cudaStream_t st) {
    if (np + tb.S > kFusedSlots) return cudaErrorInvalidValue;
    long long blocks = (tb.npts + 255) / 256;
    if (blocks > 152LL * 4) blocks = 152LL * 4;
    switch (geometry) {
    case GEO_DISK: k_adj_fused<GEO_DISK><<<(int)blocks, 256, 0, st>>>(tb, tbT, W, mu, lam, acc, np); break;
    case GEO_SPHERE: k_adj_fused<GEO_SPHERE><<<(int)blocks, 256, 0, st>>>(tb, tbT, W, mu, lam, acc, np); break;
    case GEO_BALL: k_adj_fused<GEO_BALL><<<(int)blocks, 256, 0, st>>>(tb, tbT, W, mu, lam, acc, np); break;
    default: k_adj_fused<GEO_CYLINDER><<<(int)blocks, 256, 0, st>>>(tb, tbT, W, mu, lam, acc, np); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_fused_split(int geometry, const RhsTables<float>& tbF, const RhsTables<float>& tbT,
                                   const double* W, const float* mu, int n1q, long long ys, double* lam, double* acc,
                                   int np, cudaStream_t st) {
    if (np + tbF.S > kFusedSlots) return cudaErrorInvalidValue;
    long long blocks = (tbF.npts + 255) / 256;
    if (blocks > 152LL * 4) blocks = 152LL * 4;
    switch (geometry) {
    case GEO_DISK: k_adj_fused_split<GEO_DISK><<<(int)blocks, 256, 0, st>>>(tbF, tbT, W, mu, n1q, ys, lam, acc, np); break;
    case GEO_SPHERE: k_adj_fused_split<GEO_SPHERE><<<(int)blocks, 256, 0, st>>>(tbF, tbT, W, mu, n1q, ys, lam, acc, np); break;
    case GEO_BALL: k_adj_fused_split<GEO_BALL><<<(int)blocks, 256, 0, st>>>(tbF, tbT, W, mu, n1q, ys, lam, acc, np); break;
    default: k_adj_fused_split<GEO_CYLINDER><<<(int)blocks, 256, 0, st>>>(tbF, tbT, W, mu, n1q, ys, lam, acc, np); break;
    }
    return cudaGetLastError();
}

}  // namespace sexpe
