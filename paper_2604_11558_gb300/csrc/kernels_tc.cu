// Split-TF32 tensor-core kernels (tcgen05 + TMEM + TMA bulk copies, sm_103a)
// for the per-step chain of the split exponential Euler method:
//
//   mode-3 pass (ball, cylinder): F = d M w + g(w) at FP64-accurate differences,
//       then F x_3 V_phi^{-1}, Hadamard phi_1(tau d rho_i^-2 lambda_phi), x_3 V_phi
//       (ball, eq. ee_ball) or F x_3 phi_1(tau d A_z) (cylinder, eq. ee_cylinder) -> Y.
//   slab pass (disk, ball, cylinder), one k-slab per CTA:
//       Y x_2 Q_theta^T, Hadamard Phi (theta factor), x_2 Q_theta, x_1 phi_1(tau d A_rho),
//       w += tau * result (eqs. ee_disk, ee_ball, ee_cylinder).
//
// Every mu-mode product is D = A B^T with FP32 accumulation in tensor memory
// and three TF32 MMAs per K-step (lo*hi, hi*lo, hi*hi).  The constant matrix of
// a product arrives by one TMA bulk copy per K-chunk from an image pre-laid in
// the canonical K-major no-swizzle layout; the data operand is written by the
// 128 threads (one row each), split into TF32 hi/lo on the way.  Intermediates
// stay in tensor memory: a row (lane) of one product becomes the row of the
// next operand, so the chain swaps the row mode once (theta -> rho) by putting
// the data in the B operand of the middle product.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"
#include "launch.h"
#include "tc_ptx.cuh"

namespace sexpe {

constexpr int kThreads = 128;
constexpr int kStages = 3;
constexpr uint32_t kHeaderBytes = 1024;   // barriers + tensor-memory slot

struct Pipe {
    uint64_t* tma_bar;
    uint64_t* mma_bar;
    char* stages;
    uint32_t stage_bytes;
    uint32_t g;        // K-chunks issued so far in this CTA (uniform)
    int* err;
    volatile int* aborted;
};

__device__ __forceinline__ void pipe_wait(Pipe& P, uint64_t* bar, uint32_t parity, int code) {
    const long long lim = *P.aborted ? 2000000LL : 4000000000LL;
    if (!mbar_wait_bounded(bar, parity, P.err, code, lim)) *P.aborted = 1;
}

// Row r of a tile pair (hi, lo), 16 K-values starting at the chunk's first column.
__device__ __forceinline__ void store_row16(char* hi, char* lo, int r, const float* v) {
    const uint32_t off = (uint32_t)(r >> 3) * kSBO + (uint32_t)(r & 7) * 16u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_tf32(v[4 * q + e], h[e], l[e]);
        *reinterpret_cast<uint4*>(hi + off + q * kLBO) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + off + q * kLBO) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

struct GemmSpec {
    Image mat;
    int mat_is_A;     // constant matrix is the A operand (data is B) or the B operand
    int data_rows;    // rows of the data tile
    int m_tiles;      // 128-row tiles of A
    int n_pad;        // N of the product (rows of B), multiple of 16
    int k_chunks;
    uint32_t tmem_d;  // tensor-memory address of the accumulator (tile mt at + mt * n_pad)
};

template <class Producer>
__device__ __forceinline__ void run_gemm(Pipe& P, const GemmSpec& G, Producer&& produce) {
    const int tid = threadIdx.x;
    const uint32_t data_bytes = (uint32_t)G.data_rows * kTileRowBytes;
    const uint32_t mat_bytes = (uint32_t)G.mat.rows_pad * kTileRowBytes;
    const int nsub = G.n_pad < 256 ? G.n_pad : 256;
    const int n_halves = G.n_pad / nsub;
    const uint32_t idesc = idesc_tf32(128, nsub);
    for (int c = 0; c < G.k_chunks; ++c) {
        const uint32_t g = P.g;
        const int s = (int)(g % kStages);
        const uint32_t use = g / kStages;
        if (g >= (uint32_t)kStages) pipe_wait(P, &P.mma_bar[s], (use - 1) & 1u, DERR_TIMEOUT_MMA);
        char* st = P.stages + (size_t)s * P.stage_bytes;
        char* dhi = st;
        char* dlo = st + data_bytes;
        char* mhi = st + 2 * data_bytes;
        char* mlo = mhi + mat_bytes;
        if (tid == 0) {
            mbar_arrive_expect_tx(&P.tma_bar[s], 2 * mat_bytes);
            tma_bulk_g2s(mhi, G.mat.ptr + (long long)c * G.mat.chunk_floats, 2 * mat_bytes, &P.tma_bar[s]);
        }
        produce(c, dhi, dlo);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            pipe_wait(P, &P.tma_bar[s], use & 1u, DERR_TIMEOUT_TMA);
            tc_fence_after();
            const uint32_t a_hi = smem_u32(G.mat_is_A ? mhi : dhi), a_lo = smem_u32(G.mat_is_A ? mlo : dlo);
            const uint32_t b_hi = smem_u32(G.mat_is_A ? dhi : mhi), b_lo = smem_u32(G.mat_is_A ? dlo : mlo);
#pragma unroll
            for (int ks = 0; ks < kKC / 8; ++ks) {
#pragma unroll
                for (int pass = 0; pass < 3; ++pass) {      // lo*hi, hi*lo, hi*hi
                    const uint32_t a = (pass == 0) ? a_lo : a_hi;
                    const uint32_t b = (pass == 1) ? b_lo : b_hi;
                    const uint32_t acc = (c | ks | pass) != 0;
                    for (int mt = 0; mt < G.m_tiles; ++mt) {
                        for (int nh = 0; nh < n_halves; ++nh) {
                            const uint64_t ad = smem_desc(a + mt * 16 * kSBO + ks * 2 * kLBO, kLBO, kSBO);
                            const uint64_t bd = smem_desc(b + nh * (nsub / 8) * kSBO + ks * 2 * kLBO, kLBO, kSBO);
                            mma_tf32(G.tmem_d + (uint32_t)(mt * G.n_pad + nh * nsub), ad, bd, idesc, acc);
                        }
                    }
                }
            }
            mma_commit(&P.mma_bar[s]);
        }
        P.g = g + 1;
    }
    const uint32_t gl = P.g - 1;
    pipe_wait(P, &P.mma_bar[gl % kStages], (gl / kStages) & 1u, DERR_TIMEOUT_MMA);
    tc_fence_after();
}

// Kernel prologue/epilogue: carve shared memory, init barriers, allocate TMEM.
struct CtaRes {
    Pipe P;
    uint32_t tmem;
};

__device__ __forceinline__ CtaRes cta_begin(char* smem_raw, uint32_t stage_bytes, uint32_t tmem_cols, int* err) {
    const uint32_t base = smem_u32(smem_raw);
    char* smem = smem_raw + (((base + 1023u) & ~1023u) - base);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kStages * sizeof(uint64_t));
    int* aborted = reinterpret_cast<int*>(smem + 2 * kStages * sizeof(uint64_t) + 16);
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * kStages; ++s) mbar_init(&bars[s], 1);
        *aborted = 0;
        fence_mbar_init();
    }
    if (threadIdx.x / 32 == 0) {
        tmem_alloc(tslot, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    CtaRes r;
    r.P.tma_bar = bars;
    r.P.mma_bar = bars + kStages;
    r.P.stages = smem + kHeaderBytes;
    r.P.stage_bytes = stage_bytes;
    r.P.g = 0;
    r.P.err = err;
    r.P.aborted = aborted;
    r.tmem = *tslot;
    return r;
}

__device__ __forceinline__ void cta_end(const CtaRes& r, uint32_t tmem_cols) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x / 32 == 0) tmem_dealloc(r.tmem, tmem_cols);
}

// ------------------------------------------------------------------------------
// mode-3 pass: rows = 128 consecutive (i, j) points, columns = the k fibre.
template <int GEO>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_mode3(SplitTables T, uint32_t stage_bytes, uint32_t tmem_cols) {
    extern __shared__ char smem_raw[];
    CtaRes R = cta_begin(smem_raw, stage_bytes, tmem_cols, T.err);
    const int tid = threadIdx.x;
    const uint32_t lane_base = (uint32_t)((tid >> 5) * 32) << 16;
    const int s = blockIdx.y;
    const int n1 = T.n1, n3 = T.n3;
    const long long n12 = (long long)T.n1 * T.n2;
    const int n3p = (n3 + 15) & ~15;
    const long long ij = (long long)blockIdx.x * kThreads + tid;
    const bool valid = ij < n12;
    const int i = valid ? (int)(ij % n1) : 0;
    const int j = valid ? (int)(ij / n1) : 0;

    GemmSpec g1{GEO == GEO_BALL ? T.M3a : T.M3b[s], 0, kThreads, 1, n3p, n3p / kKC, R.tmem};
    run_gemm(R.P, g1, [&](int c, char* hi, char* lo) {
        float v[16];
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            const int k = c * 16 + kk;
            v[kk] = (valid && k < n3) ? rhs_point<SplitAcc, GEO>(T.rhs, T.state, s, k * n12 + ij, i, j, k) : 0.f;
        }
        store_row16(hi, lo, tid, v);
    });
    uint32_t last = 0;
    if constexpr (GEO == GEO_BALL) {
        GemmSpec g2{T.M3b[0], 0, kThreads, 1, n3p, n3p / kKC, R.tmem + (uint32_t)n3p};
        const float ci = valid ? T.had_phi[s * n1 + i] : 0.f;
        run_gemm(R.P, g2, [&](int c, char* hi, char* lo) {
            float v[16];
            tmem_ld16(R.tmem + lane_base + (uint32_t)(c * 16), v);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int kp = c * 16 + kk;
                v[kk] = (valid && kp < n3) ? v[kk] * phi1f(ci * T.lam_phi[kp]) : 0.f;
            }
            store_row16(hi, lo, tid, v);
        });
        last = (uint32_t)n3p;
    }
    float* Ys = T.Y + (long long)s * T.npts;
    for (int c = 0; c < n3p / 16; ++c) {
        float v[16];
        tmem_ld16(R.tmem + lane_base + last + (uint32_t)(c * 16), v);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int k = c * 16 + kk;
            if (valid && k < n3) Ys[k * n12 + ij] = v[kk];
        }
    }
    cta_end(R, tmem_cols);
}

// ------------------------------------------------------------------------------
// slab pass: one k-slab (n2 x n1 matrix, rho contiguous) of one species.
struct SlabJob {
    int n1, n2;
    const float* Y;       // F after the earlier directions, slab base
    double* W;            // state slab base (updated)
    Image QT, Q, P;
    const float* had_c;   // per rho-row coefficient c_i: Phi = phi_1(c_i lambda_theta_j)
    const float* lam;     // eigenvalues of A_theta in the column order of Q
    double tau;
};

__device__ __forceinline__ void slab_body(const SlabJob& J, Pipe& P, uint32_t tmem, char* epi) {
    const int tid = threadIdx.x;
    const uint32_t lane_base = (uint32_t)((tid >> 5) * 32) << 16;
    const int n1 = J.n1, n2 = J.n2;
    const int n1p = (n1 + 15) & ~15, n2p = (n2 + 15) & ~15, m2 = (n2 + 127) / 128;
    const uint32_t c1 = 0, c2 = (uint32_t)n2p;
    const uint32_t c3 = (m2 * n1p <= n2p) ? 0u : (uint32_t)(n2p + m2 * n1p);

    // G1: X[i][j'] = sum_j Y[i][j] Q[j][j']          (Y x_2 Q_theta^T), rows i
    GemmSpec g1{J.QT, 0, kThreads, 1, n2p, n2p / kKC, tmem + c1};
    run_gemm(P, g1, [&](int c, char* hi, char* lo) {
        float v[16];
        const int i = tid;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int j = c * 16 + kk;
            v[kk] = (i < n1 && j < n2) ? J.Y[j * n1 + i] : 0.f;
        }
        store_row16(hi, lo, tid, v);
    });
    // G2: Z^T[j][i] = sum_j' Q[j][j'] (Phi o X)[i][j']   (x_2 Q_theta), data in B, rows j
    GemmSpec g2{J.Q, 1, n1p, m2, n1p, n2p / kKC, tmem + c2};
    const float ci = (tid < n1) ? J.had_c[tid] : 0.f;
    run_gemm(P, g2, [&](int c, char* hi, char* lo) {
        float v[16];
        tmem_ld16(tmem + lane_base + c1 + (uint32_t)(c * 16), v);
        const int i = tid;
        if (i < n1p) {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int jp = c * 16 + kk;
                v[kk] = (i < n1 && jp < n2) ? v[kk] * phi1f(ci * J.lam[jp]) : 0.f;
            }
            store_row16(hi, lo, i, v);
        }
    });
    // G3: R^T[j][i'] = sum_i Z^T[j][i] P[i'][i]      (x_1 phi_1(tau d A_rho)), rows j
    GemmSpec g3{J.P, 0, kThreads * m2, m2, n1p, n1p / kKC, tmem + c3};
    run_gemm(P, g3, [&](int c, char* hi, char* lo) {
        for (int mt = 0; mt < m2; ++mt) {
            float v[16];
            tmem_ld16(tmem + lane_base + c2 + (uint32_t)(mt * n1p + c * 16), v);
            const int j = mt * kThreads + tid;
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const int i = c * 16 + kk;
                if (!(j < n2 && i < n1)) v[kk] = 0.f;
            }
            store_row16(hi, lo, mt * kThreads + tid, v);
        }
    });
    // w[k][j][i'] += tau R^T[j][i'], staged through shared memory for coalesced FP64 RMW.
    float* E = reinterpret_cast<float*>(epi);
    const int pitch = n1p + 1;
    for (int mt = 0; mt < m2; ++mt) {
        for (int c = 0; c < n1p / 16; ++c) {
            float v[16];
            tmem_ld16(tmem + lane_base + c3 + (uint32_t)(mt * n1p + c * 16), v);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) E[tid * pitch + c * 16 + kk] = v[kk];
        }
        __syncthreads();
        const int rows = min(kThreads, n2 - mt * kThreads);
        double* Wt = J.W + (long long)mt * kThreads * n1;
        for (int f = tid; f < rows * n1; f += kThreads) {
            const int jl = f / n1, i = f - jl * n1;
            Wt[f] += J.tau * (double)E[jl * pitch + i];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_slab(SplitTables T, uint32_t stage_bytes, uint32_t tmem_cols) {
    extern __shared__ char smem_raw[];
    CtaRes R = cta_begin(smem_raw, stage_bytes, tmem_cols, T.err);
    const int k = blockIdx.x, s = blockIdx.y;
    const long long n12 = (long long)T.n1 * T.n2;
    SlabJob J;
    J.n1 = T.n1;
    J.n2 = T.n2;
    J.Y = T.Y + (long long)s * T.npts + k * n12;
    J.W = T.state_upd + (long long)s * T.npts + k * n12;
    J.QT = T.QT;
    J.Q = T.Q;
    J.P = T.P[s];
    J.had_c = T.had_theta + (long long)s * T.had_theta_sp + (T.geometry == GEO_BALL ? (long long)k * T.n1 : 0);
    J.lam = T.lam_theta;
    J.tau = T.tau_d;
    slab_body(J, R.P, R.tmem, R.P.stages);
    cta_end(R, tmem_cols);
}

// F in FP32 at FP64-accurate differences (disk: the only direction before the slab pass).
template <int GEO>
__global__ void __launch_bounds__(256) k_rhs_split(RhsTables<float> tb, const double* __restrict__ W,
                                                   float* __restrict__ Y) {
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
        Y[t] = rhs_point<SplitAcc, GEO>(tb, W, s, idx, i, j, k);
    }
}

// ------------------------------------------------------------------------------
// Host-side shape logic.

static uint32_t round_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

static uint32_t pow2_cols(uint32_t c) {
    uint32_t p = 32;
    while (p < c) p <<= 1;
    return p;
}

TcShape tc_mode3_shape(int geometry, int n1, int n2, int n3) {
    (void)n1;
    (void)n2;
    TcShape sh{};
    const uint32_t n3p = round_up(n3, 16);
    sh.stage_bytes = round_up(2u * kThreads * kTileRowBytes + 2u * n3p * kTileRowBytes, 1024);
    sh.tmem_cols = pow2_cols(geometry == GEO_BALL ? 2 * n3p : n3p);
    sh.smem_bytes = 1024 + kHeaderBytes + kStages * sh.stage_bytes;
    return sh;
}

TcShape tc_slab_shape(int n1, int n2) {
    TcShape sh{};
    const uint32_t n1p = round_up(n1, 16), n2p = round_up(n2, 16), m2 = (n2 + 127) / 128;
    const uint32_t rows1 = kThreads + n2p;              // G1: data 128 rows, matrix n2p rows
    const uint32_t rows2 = n1p + kThreads * m2;         // G2: data n1p rows, matrix 128 m2 rows
    const uint32_t rows3 = kThreads * m2 + n1p;         // G3
    uint32_t rows = rows1 > rows2 ? rows1 : rows2;
    rows = rows > rows3 ? rows : rows3;
    sh.stage_bytes = round_up(2u * rows * kTileRowBytes, 1024);
    const uint32_t epi = kThreads * (n1p + 1) * 4u;
    uint32_t body = kStages * sh.stage_bytes;
    if (body < epi) {
        sh.stage_bytes = round_up((epi + kStages - 1) / kStages, 1024);
        body = kStages * sh.stage_bytes;
    }
    const uint32_t c3 = (m2 * n1p <= n2p) ? 0 : n2p + m2 * n1p;
    uint32_t cols = n2p + m2 * n1p;
    if (c3 + m2 * n1p > cols) cols = c3 + m2 * n1p;
    sh.tmem_cols = pow2_cols(cols);
    sh.smem_bytes = 1024 + kHeaderBytes + body;
    return sh;
}

cudaError_t tc_prepare(uint32_t smem_mode3, uint32_t smem_slab) {
    cudaError_t e = cudaSuccess;
    if (smem_mode3) {
        e = cudaFuncSetAttribute(k_tc_mode3<GEO_BALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_mode3);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_tc_mode3<GEO_CYLINDER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_mode3);
        if (e != cudaSuccess) return e;
    }
    if (smem_slab) e = cudaFuncSetAttribute(k_tc_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_slab);
    return e;
}

cudaError_t launch_tc_mode3(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    dim3 grid((unsigned)((T.n1 * (long long)T.n2 + kThreads - 1) / kThreads), T.S);
    if (T.geometry == GEO_BALL)
        k_tc_mode3<GEO_BALL><<<grid, kThreads, sh.smem_bytes, st>>>(T, sh.stage_bytes, sh.tmem_cols);
    else
        k_tc_mode3<GEO_CYLINDER><<<grid, kThreads, sh.smem_bytes, st>>>(T, sh.stage_bytes, sh.tmem_cols);
    return cudaGetLastError();
}

cudaError_t launch_tc_slab(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    dim3 grid(T.geometry == GEO_DISK ? 1 : T.n3, T.S);
    k_tc_slab<<<grid, kThreads, sh.smem_bytes, st>>>(T, sh.stage_bytes, sh.tmem_cols);
    return cudaGetLastError();
}

cudaError_t launch_rhs_split(const SplitTables& T, cudaStream_t st) {
    const long long total = T.npts * T.S;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    switch (T.geometry) {
    case GEO_DISK: k_rhs_split<GEO_DISK><<<(int)blocks, 256, 0, st>>>(T.rhs, T.state, T.Y); break;
    case GEO_SPHERE: k_rhs_split<GEO_SPHERE><<<(int)blocks, 256, 0, st>>>(T.rhs, T.state, T.Y); break;
    case GEO_BALL: k_rhs_split<GEO_BALL><<<(int)blocks, 256, 0, st>>>(T.rhs, T.state, T.Y); break;
    default: k_rhs_split<GEO_CYLINDER><<<(int)blocks, 256, 0, st>>>(T.rhs, T.state, T.Y); break;
    }
    return cudaGetLastError();
}

}  // namespace sexpe
