// FP64 SIMT kernels of the split exponential Euler step: stencil + reaction,
// and mu-mode products (tensor x small dense matrix) with optional Hadamard
// factor and fused update.  The comparison leg of the split-TF32 path.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"
#include "launch.h"

namespace sexpe {

template <int GEO>
__global__ void __launch_bounds__(256) k_rhs64(RhsTables<double> tb, const double* __restrict__ W,
                                               double* __restrict__ F) {
    const long long npts = tb.npts;
    const long long total = npts * tb.S;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / npts);
        const long long idx = t - (long long)s * npts;
        const int i = (int)(idx % tb.n1);
        const long long rest = idx / tb.n1;
        const int j = (int)(rest % tb.n2);
        const int k = (int)(rest / tb.n2);
        F[t] = rhs_point<F64Acc, GEO>(tb, W, s, idx, i, j, k);
    }
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

}  // namespace sexpe
