// Split-TF32 tensor-core kernels (tcgen05 + TMEM + TMA bulk copies, sm_103a)
// for the per-step chain of the split exponential Euler method:
//
//   stencil pass (all geometries, SIMT): F = d M w + g(w) in FP32 from FP64-
//       accurate differences, one shared-memory tile per CTA -> Y.
//   mode-3 pass (ball, cylinder), in place on Y: F x_3 V_phi^{-1}, Hadamard
//       Phi_{rho,.,phi}, x_3 V_phi (ball, eq. ee_ball) or F x_3 phi_1(tau d A_z)
//       (cylinder, eq. ee_cylinder).
//   slab pass (disk, ball, cylinder), one k-slab per CTA: Y x_2 Q_theta^T,
//       Hadamard Phi (theta factor), x_2 Q_theta, x_1 phi_1(tau d A_rho),
//       w += tau * result (eqs. ee_disk, ee_ball, ee_cylinder).
//
// Every mu-mode product is D = A B^T with FP32 accumulation in tensor memory
// and three TF32 MMAs per K-step (lo*hi, hi*lo, hi*hi).  The constant matrix of
// a product arrives by one TMA bulk copy per K-chunk from an image pre-laid in
// the canonical K-major no-swizzle layout; the data operand is written by the
// 256 threads (two per row, eight K-columns each), split into TF32 hi/lo on the
// way.  Intermediates stay in tensor memory: a row (lane) of one product
// becomes the row of the next operand, so the chain swaps the row mode once
// (theta -> rho) by putting the data in the B operand of the middle product.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"
#include "launch.h"
#include "tc_ptx.cuh"

namespace sexpe {

constexpr int kRows = 128;                 // MMA M and tensor-memory lanes
constexpr int kThreads = 256;              // producer threads: two per row, columns 0-7 / 8-15 of a chunk
constexpr int kBlock = kThreads + 64;      // + one warp issuing TMA copies ahead, one issuing the MMAs
constexpr int kMaxStages = 3;   // stage ring depth: 3, or 2 when 3 would keep two CTAs off one SM
constexpr uint32_t kHeaderBytes = 128;    // barriers + tensor-memory slot

struct Pipe {
    uint64_t* tma_bar;     // matrix chunk landed (TMA transaction count)
    uint64_t* mma_bar;     // MMAs reading the stage completed (tcgen05.commit)
    uint64_t* data_bar;    // data operand of the stage written (one arrive per producer warp)
    char* stages;
    uint32_t stage_bytes;
    uint32_t nst;      // stages in the ring
    uint32_t raw_bytes;   // raw region at the end of every stage
    uint32_t g;        // K-chunks issued so far in this CTA (uniform)
    int* err;
    volatile int* aborted;
};

__device__ __forceinline__ void pipe_wait(Pipe& P, uint64_t* bar, uint32_t parity, int code) {
    const long long lim = *P.aborted ? 2000000LL : 4000000000LL;
    if (!mbar_wait_bounded(bar, parity, P.err, code, lim)) *P.aborted = 1;
}

// Barrier of the 256 compute threads only (the TMA warp runs on its own).
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Row r, columns 8h..8h+7 of a chunk, of a tile pair (hi, lo).
__device__ __forceinline__ void store_row8(char* hi, char* lo, int r, int h, const float* v) {
    const uint32_t off = (uint32_t)(r >> 3) * kSBO + (uint32_t)(r & 7) * 16u + (uint32_t)(2 * h) * kLBO;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint32_t hb[4], lb[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_tf32(v[4 * q + e], hb[e], lb[e]);
        *reinterpret_cast<uint4*>(hi + off + q * kLBO) = make_uint4(hb[0], hb[1], hb[2], hb[3]);
        *reinterpret_cast<uint4*>(lo + off + q * kLBO) = make_uint4(lb[0], lb[1], lb[2], lb[3]);
    }
}

// Global FP32 rows copied into a stage's raw region next to each K-chunk's
// matrix copy (the producers then read shared memory only): chunk c copies rows
// [16c, min(16c + 16, rows_total)), each `row_floats` floats (a multiple of 4),
// row r of the chunk landing at raw + r * row_floats.
struct AuxCopy {
    const float* src;       // row 0; null = no copy
    long long row_stride;   // floats between consecutive rows in global memory
    int row_floats;
    int rows_total;
};

struct GemmSpec {
    Image mat;
    int mat_is_A;     // constant matrix is the A operand (data is B) or the B operand
    int data_rows;    // rows of the data tile
    int m_tiles;      // 128-row tiles of A
    int n_pad;        // N of the product (rows of B), multiple of 16
    int k_chunks;
    uint32_t tmem_d;  // tensor-memory address of the accumulator (tile mt at + mt * n_pad)
    AuxCopy aux;
};

// Raw region of a stage: 16 rows of the widest staged row (<= 128 floats).
__host__ __device__ constexpr uint32_t raw_bytes_for(int row_floats) { return (uint32_t)kKC * row_floats * 4u; }

// Byte offset of the constant-matrix tiles inside a stage: after the data hi/lo tiles.
__device__ __forceinline__ uint32_t mat_offset(const GemmSpec& G) { return 2u * G.data_rows * kTileRowBytes; }

// Producer side of one product: the 256 producer threads write the data operand
// of each K-chunk into its stage and signal the MMA warp through the stage's
// data barrier; a stage is rewritten only after the MMAs that read it completed.
template <class Producer>
__device__ __forceinline__ void run_gemm(Pipe& P, const GemmSpec& G, Producer&& produce) {
    const uint32_t data_bytes = (uint32_t)G.data_rows * kTileRowBytes;
    for (int c = 0; c < G.k_chunks; ++c) {
        const uint32_t g = P.g;
        const int s = (int)(g % P.nst);
        const uint32_t use = g / P.nst;
        if (g >= P.nst) pipe_wait(P, &P.mma_bar[s], (use - 1) & 1u, DERR_TIMEOUT_MMA);
        char* st = P.stages + (size_t)s * P.stage_bytes;
        if (G.aux.src) pipe_wait(P, &P.tma_bar[s], use & 1u, DERR_TIMEOUT_TMA);
        produce(c, st, st + data_bytes, reinterpret_cast<const float*>(st + P.stage_bytes - P.raw_bytes));
        fence_async_smem();
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&P.data_bar[s]);
        P.g = g + 1;
    }
    const uint32_t gl = P.g - 1;
    pipe_wait(P, &P.mma_bar[gl % P.nst], (gl / P.nst) & 1u, DERR_TIMEOUT_MMA);
    tc_fence_after();
}

// MMA side: one lane of the MMA warp walks the K-chunks of every product in
// order; when a chunk's data operand and matrix copy are both in its stage it
// issues the three TF32 MMAs per K-step and commits them to the stage barrier.
__device__ __forceinline__ void mma_issuer(Pipe& P, const GemmSpec* gs, int n_gemms) {
    if ((threadIdx.x & 31) != 0) return;
    uint32_t g = P.g;
    for (int q = 0; q < n_gemms; ++q) {
        const GemmSpec& G = gs[q];
        const uint32_t data_bytes = (uint32_t)G.data_rows * kTileRowBytes;
        const uint32_t mat_bytes = (uint32_t)G.mat.rows_pad * kTileRowBytes;
        const int nsub = G.n_pad < 256 ? G.n_pad : 256;
        const int n_halves = G.n_pad / nsub;
        const uint32_t idesc = idesc_tf32(128, nsub);
        for (int c = 0; c < G.k_chunks; ++c, ++g) {
            const int s = (int)(g % P.nst);
            const uint32_t use = g / P.nst;
            pipe_wait(P, &P.data_bar[s], use & 1u, DERR_TIMEOUT_MMA);
            pipe_wait(P, &P.tma_bar[s], use & 1u, DERR_TIMEOUT_TMA);
            tc_fence_after();
            char* st = P.stages + (size_t)s * P.stage_bytes;
            char* dhi = st;
            char* dlo = st + data_bytes;
            char* mhi = st + mat_offset(G);
            char* mlo = mhi + mat_bytes;
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
    }
    P.g = g;
}

// TMA side: one lane of the extra warp walks the K-chunks of every product of
// the CTA in order and copies each chunk's matrix image into its stage as soon
// as the stage is free, up to one ring of stages ahead of the MMAs.
__device__ __forceinline__ void tma_issuer(Pipe& P, const GemmSpec* gs, int n_gemms) {
    if ((threadIdx.x & 31) != 0) return;
    uint32_t g = P.g;
    for (int q = 0; q < n_gemms; ++q) {
        const GemmSpec& G = gs[q];
        const uint32_t mat_bytes = (uint32_t)G.mat.rows_pad * kTileRowBytes;
        for (int c = 0; c < G.k_chunks; ++c, ++g) {
            const int s = (int)(g % P.nst);
            const uint32_t use = g / P.nst;
            if (g >= P.nst) pipe_wait(P, &P.mma_bar[s], (use - 1) & 1u, DERR_TIMEOUT_MMA);
            char* st = P.stages + (size_t)s * P.stage_bytes;
            char* mhi = st + mat_offset(G);
            uint32_t tx = 2 * mat_bytes;
            int rows = 0;
            if (G.aux.src) {
                rows = min(kKC, G.aux.rows_total - c * kKC);
                rows = rows > 0 ? rows : 0;
                tx += (uint32_t)rows * G.aux.row_floats * 4u;
            }
            mbar_arrive_expect_tx(&P.tma_bar[s], tx);
            tma_bulk_g2s(mhi, G.mat.ptr + (long long)c * G.mat.chunk_floats, 2 * mat_bytes, &P.tma_bar[s]);
            if (rows > 0) {
                char* raw = st + P.stage_bytes - P.raw_bytes;
                const float* src = G.aux.src + (long long)c * kKC * G.aux.row_stride;
                if (G.aux.row_stride == G.aux.row_floats) {          // contiguous rows: one copy
                    tma_bulk_g2s(raw, src, (uint32_t)rows * G.aux.row_floats * 4u, &P.tma_bar[s]);
                } else {
                    for (int r = 0; r < rows; ++r)
                        tma_bulk_g2s(raw + (size_t)r * G.aux.row_floats * 4, src + r * G.aux.row_stride,
                                     (uint32_t)G.aux.row_floats * 4u, &P.tma_bar[s]);
                }
            }
        }
    }
    P.g = g;
}

// Kernel prologue/epilogue: carve shared memory, init barriers, allocate TMEM.
struct CtaRes {
    Pipe P;
    uint32_t tmem;
};

__device__ __forceinline__ CtaRes cta_begin(char* smem_raw, uint32_t stage_bytes, uint32_t nst, uint32_t raw_bytes,
                                            uint32_t tmem_cols, int* err) {
    const uint32_t base = smem_u32(smem_raw);
    char* smem = smem_raw + (((base + 127u) & ~127u) - base);   // 128-byte aligned ring
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 3 * kMaxStages * sizeof(uint64_t));
    int* aborted = reinterpret_cast<int*>(smem + 3 * kMaxStages * sizeof(uint64_t) + 16);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(&bars[s], 1);                          // tma_bar
            mbar_init(&bars[kMaxStages + s], 1);             // mma_bar
            mbar_init(&bars[2 * kMaxStages + s], kThreads / 32);   // data_bar
        }
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
    r.P.mma_bar = bars + kMaxStages;
    r.P.data_bar = bars + 2 * kMaxStages;
    r.P.nst = nst;
    r.P.raw_bytes = raw_bytes;
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
// stencil pass: F = d_s M w_s + g_s(w) in FP32 for every species of one
// (all i) x TJ x TK tile.  The tile of every species, with a one-point halo in
// j and k, is loaded with many loads in flight per thread and each FP64 value
// is split once into FP32 hi + lo in shared memory; every stencil difference
// is then formed from split pairs at FP32 relative accuracy of the difference.
template <int GEO>
struct TileShape {
    static constexpr bool k3 = (GEO == GEO_BALL || GEO == GEO_CYLINDER);
    static constexpr int TK = k3 ? 8 : 1;
    static constexpr int KH = k3 ? 1 : 0;
    static constexpr bool periodic1 = (GEO == GEO_SPHERE);   // mode 1 is theta on the sphere
    static constexpr bool periodic2 = (GEO != GEO_SPHERE);   // mode 2 is theta elsewhere
};

__device__ __forceinline__ float sdiff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

constexpr int kTileBatch = 8;   // global loads in flight per thread while filling the tile

constexpr int kRhsThreads = 512;   // 128 lanes along rho x 4 line parities

template <int GEO>
__global__ void __launch_bounds__(kRhsThreads) k_rhs_tile(RhsTables<float> tb, const double* __restrict__ Wall,
                                                          float* __restrict__ F, int TJ, int n1q, long long ys) {
    using TS = TileShape<GEO>;
    extern __shared__ float2 tile[];                 // [S][nK][nJ][n1]
    __shared__ float cj[3][32], ck[4][8];            // j- and k-dependent coefficients of the tile
    __shared__ long long row_off[kMaxSpecies * 10 * 34];   // global offset of each tile row, -1 outside
    const int n1 = tb.n1, n2 = tb.n2, n3 = tb.n3, S = tb.S;
    const int j0 = blockIdx.x * TJ, k0 = blockIdx.y * TS::TK;
    const int nJ = TJ + 2, nK = TS::TK + 2 * TS::KH;
    const int rows = S * nK * nJ;
    const long long npts = tb.npts;
    const long long n12 = (long long)n1 * n2;
    constexpr int NP = kRhsThreads / 128;            // line parities
    const int lane = threadIdx.x & 127, rpar = threadIdx.x >> 7;
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const int jj = row % nJ, kk = (row / nJ) % nK, sp = row / (nJ * nK);
        int j = j0 - 1 + jj;
        const int k = k0 - TS::KH + kk;
        if (TS::periodic2) j = j < 0 ? j + n2 : (j >= n2 ? j - n2 : j);
        const bool ok = j >= 0 && j < n2 && k >= 0 && k < n3;
        row_off[row] = ok ? sp * npts + (long long)k * n12 + (long long)j * n1 : -1;
    }
    __syncthreads();
    for (int row0 = rpar; row0 < rows; row0 += NP * kTileBatch) {
        for (int i = lane; i < n1; i += 128) {
            double v[kTileBatch];
#pragma unroll
            for (int u = 0; u < kTileBatch; ++u) {
                const int row = row0 + NP * u;
                const long long off = row < rows ? row_off[row] : -1;
                v[u] = off >= 0 ? __ldg(Wall + off + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kTileBatch; ++u) {
                const int row = row0 + NP * u;
                if (row < rows) tile[row * n1 + i] = split_f64(v[u]);
            }
        }
    }
    if (threadIdx.x < TJ) {
        const int j = min(j0 + (int)threadIdx.x, n2 - 1);
        cj[0][threadIdx.x] = tb.ax[1].rs[j];
        cj[1][threadIdx.x] = tb.ax[1].lower[j];
        cj[2][threadIdx.x] = tb.ax[1].upper[j];
    }
    if (TS::k3 && threadIdx.x >= 64 && threadIdx.x < 64 + TS::TK) {
        const int t = threadIdx.x - 64;
        const int k = min(k0 + t, n3 - 1);
        ck[0][t] = tb.ax[2].rs[k];
        ck[1][t] = tb.ax[2].lower[k];
        ck[2][t] = tb.ax[2].upper[k];
        ck[3][t] = (GEO == GEO_BALL) ? tb.Dp[k] : 1.f;
    }
    __syncthreads();
    const int species_stride = nK * nJ * n1;
    for (int i = lane; i < n1; i += 128) {
        const StencilAxis<float>& a1 = tb.ax[0];
        const float lo1 = a1.lower[i], up1 = a1.upper[i], rs1 = a1.rs[i];
        const float dr = (GEO == GEO_SPHERE) ? 1.f : tb.Dr[i];
        const bool has_m = i > 0 || TS::periodic1, has_p = i < n1 - 1 || TS::periodic1;
        const int im = i > 0 ? i - 1 : n1 - 1, ip = i < n1 - 1 ? i + 1 : 0;
        for (int line = rpar; line < TS::TK * TJ; line += NP) {
            const int kl = line / TJ, jl = line - kl * TJ;
            const int j = j0 + jl, k = k0 + kl;
            if (j >= n2 || k >= n3) continue;
            const int cidx = ((kl + TS::KH) * nJ + (jl + 1)) * n1 + i;
            float w[kMaxSpecies];
#pragma unroll
            for (int r = 0; r < kMaxSpecies; ++r) {
                if (r < S) {
                    const float2 c = tile[r * species_stride + cidx];
                    w[r] = c.x + c.y;
                } else {
                    w[r] = 0.f;
                }
            }
            const long long idx = (long long)k * n12 + (long long)j * n1 + i;
#pragma unroll
            for (int s = 0; s < kMaxSpecies; ++s) {
                if (s >= S) break;
                const float2* row = tile + s * species_stride + cidx - i;
                const float2 c = row[i];
                float t0 = rs1 * (c.x + c.y);
                if (has_m) t0 += lo1 * sdiff(row[im], c);
                if (has_p) t0 += up1 * sdiff(row[ip], c);
                float t1 = cj[0][jl] * (c.x + c.y);
                if (j > 0 || TS::periodic2) t1 += cj[1][jl] * sdiff(row[i - n1], c);
                if (j < n2 - 1 || TS::periodic2) t1 += cj[2][jl] * sdiff(row[i + n1], c);
                float lap;
                if constexpr (GEO == GEO_DISK) {
                    lap = t0 + dr * t1;
                } else if constexpr (GEO == GEO_SPHERE) {
                    lap = tb.Dp[j] * t0 + t1;
                } else {
                    float t2 = ck[0][kl] * (c.x + c.y);
                    if (k > 0) t2 += ck[1][kl] * sdiff(row[i - nJ * n1], c);
                    if (k < n3 - 1) t2 += ck[2][kl] * sdiff(row[i + nJ * n1], c);
                    if constexpr (GEO == GEO_BALL) lap = t0 + dr * (ck[3][kl] * t1 + t2);
                    else lap = t0 + dr * t1 + t2;
                }
                F[s * ys + ((long long)k * n2 + j) * n1q + i] = tb.d[s] * lap + reaction<float>(tb.reac, w, s);
            }
        }
    }
}

// ------------------------------------------------------------------------------
// mode-3 pass: rows = 128 consecutive points of the padded (i, j) plane
// (row index j * n1q + i), columns = the k fibre; reads F from Y and overwrites
// the same entries with the result.  The TMA warp stages every chunk's F rows
// (16 k-planes x 128 points) and, for the ball, the Phi rows next to the
// matrix chunk, so the producers read shared memory only.
template <int GEO>
__global__ void __launch_bounds__(kBlock, 1)
    k_tc_mode3(SplitTables T, uint32_t stage_bytes, uint32_t nst, uint32_t raw_bytes,
                                              uint32_t tmem_cols) {
    extern __shared__ char smem_raw[];
    CtaRes R = cta_begin(smem_raw, stage_bytes, nst, raw_bytes, tmem_cols, T.err);
    const int s = blockIdx.y;
    const int n3 = T.n3, n1q = T.n1q;
    const int n3p = (n3 + 15) & ~15;
    const long long plane = (long long)T.n2 * n1q;          // floats per k-plane of Y
    const long long row0 = (long long)blockIdx.x * kRows;
    const int tile_rows = (int)(plane - row0 < kRows ? plane - row0 : kRows);
    float* Ys = T.Y + (long long)s * T.ys;
    GemmSpec gs[2] = {{GEO == GEO_BALL ? T.M3a : T.M3b[s], 0, kRows, 1, n3p, n3p / kKC, R.tmem,
                       AuxCopy{Ys + row0, plane, tile_rows, n3}},
                      {T.M3b[0], 0, kRows, 1, n3p, n3p / kKC, R.tmem + (uint32_t)n3p,
                       AuxCopy{T.had_phi + (long long)s * n3 * n1q, n1q, n1q, n3}}};
    if (threadIdx.x >= kThreads + 32) {
        mma_issuer(R.P, gs, GEO == GEO_BALL ? 2 : 1);
    } else if (threadIdx.x >= kThreads) {
        tma_issuer(R.P, gs, GEO == GEO_BALL ? 2 : 1);
    } else {
        const int tid = threadIdx.x;
        const int r = tid & (kRows - 1), h = tid >> 7;
        const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
        const bool valid = r < tile_rows;
        const int i = (int)((row0 + r) % n1q);
        run_gemm(R.P, gs[0], [&](int c, char* hi, char* lo, const float* raw) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int kk = h * 8 + q;
                v[q] = (valid && c * 16 + kk < n3) ? raw[kk * tile_rows + r] : 0.f;
            }
            store_row8(hi, lo, r, h, v);
        });
        uint32_t last = 0;
        if constexpr (GEO == GEO_BALL) {
            run_gemm(R.P, gs[1], [&](int c, char* hi, char* lo, const float* raw) {
                float v[8];
                tmem_ld8(R.tmem + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int kk = h * 8 + q;
                    v[q] = (valid && c * 16 + kk < n3) ? v[q] * raw[kk * n1q + i] : 0.f;
                }
                store_row8(hi, lo, r, h, v);
            });
            last = (uint32_t)n3p;
        }
        for (int c = 0; c < n3p / 16; ++c) {
            float v[8];
            tmem_ld8(R.tmem + lane_base + last + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = c * 16 + h * 8 + q;
                if (valid && k < n3) Ys[k * plane + row0 + r] = v[q];
            }
        }
    }
    cta_end(R, tmem_cols);
}

// ------------------------------------------------------------------------------
// slab pass: one k-slab (n2 x n1 matrix, rho contiguous) of one species.
struct SlabJob {
    int n1, n2, n1q;      // n1q: row pitch of Y and of the Phi table (n1 rounded up to 4)
    const float* Y;       // F after the earlier directions, slab base (null: F from the state)
    const double* Win;    // state slab base read by the update (== W for an in-place step)
    double* W;            // state slab base written by the update
    Image QT, Q, P;
    const float* had;     // Phi of the theta direction for this slab, [j'][n1q]
    float tau_f;
};

// The three products of a slab and their tensor-memory columns within an
// allocation of T columns: G1 [0, n2p); G2 [T - m2 n1p, T); G3 [0, m2 n1p),
// reusing G1's columns, which are dead once G2's operands are written.
// Valid when n2p + m2 n1p <= T and 2 m2 n1p <= T (slab_tmem_cols).
__device__ __forceinline__ void slab_specs(const SlabJob& J, uint32_t tmem, uint32_t T, GemmSpec* gs,
                                           uint32_t* cols) {
    const int n1p = (J.n1 + 15) & ~15, n2p = (J.n2 + 15) & ~15, m2 = (J.n2 + 127) / 128;
    cols[0] = 0;
    cols[1] = T - (uint32_t)(m2 * n1p);
    cols[2] = 0;
    gs[0] = GemmSpec{J.QT, 0, kRows, 1, n2p, n2p / kKC, tmem + cols[0], AuxCopy{J.Y, J.n1q, J.n1q, J.n2}};
    gs[1] = GemmSpec{J.Q, 1, n1p, m2, n1p, n2p / kKC, tmem + cols[1], AuxCopy{J.had, J.n1q, J.n1q, J.n2}};
    gs[2] = GemmSpec{J.P, 0, kRows * m2, m2, n1p, n1p / kKC, tmem + cols[2], AuxCopy{nullptr, 0, 0, 0}};
}

// F of one disk species at (i, j0 + q), q < 8, from FP64-accurate differences of
// the state (both species of the instance at `inst_base`), 0 outside the grid.
__device__ __forceinline__ void disk_F8(const BatchInstance& I, const double* inst_base, int s, int i, int j0,
                                        float* v) {
    const int n1 = I.n1, n2 = I.n2;
    const long long n12 = (long long)n1 * n2;
    const double* Ws = inst_base + s * n12;
    const double* Wo = inst_base + (1 - s) * n12;
    const bool iv = i < n1;
    const int ii = iv ? i : 0;
    double c[8], m1[8], p1[8], m2[8], p2[8], o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = j0 + q;
        const int jj = j < n2 ? j : 0;
        const long long idx = (long long)jj * n1 + ii;
        c[q] = Ws[idx];
        m1[q] = ii > 0 ? Ws[idx - 1] : 0.0;
        p1[q] = ii < n1 - 1 ? Ws[idx + 1] : 0.0;
        m2[q] = Ws[(long long)(jj > 0 ? jj - 1 : n2 - 1) * n1 + ii];
        p2[q] = Ws[(long long)(jj < n2 - 1 ? jj + 1 : 0) * n1 + ii];
        o[q] = Wo[idx];
    }
    const float lo1 = I.ax_rho.lower[ii], up1 = I.ax_rho.upper[ii], rs1 = I.ax_rho.rs[ii], dr = I.Dr[ii];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = j0 + q;
        const int jj = j < n2 ? j : 0;
        const float2 cc = split_f64(c[q]);
        float t0 = rs1 * (cc.x + cc.y);
        if (ii > 0) t0 += lo1 * sdiff(split_f64(m1[q]), cc);
        if (ii < n1 - 1) t0 += up1 * sdiff(split_f64(p1[q]), cc);
        float t1 = I.ax_theta.rs[jj] * (cc.x + cc.y) + I.ax_theta.lower[jj] * sdiff(split_f64(m2[q]), cc) +
                   I.ax_theta.upper[jj] * sdiff(split_f64(p2[q]), cc);
        const float2 oo = split_f64(o[q]);
        float w[kMaxSpecies] = {0.f, 0.f, 0.f, 0.f};
        w[s] = cc.x + cc.y;
        w[1 - s] = oo.x + oo.y;
        const float f = I.d[s] * (t0 + dr * t1) + reaction<float>(I.reac, w, s);
        v[q] = (iv && j < n2) ? f : 0.f;
    }
}

__device__ __forceinline__ void slab_compute(const SlabJob& J, const GemmSpec* gs, const uint32_t* cols, Pipe& P,
                                             uint32_t tmem, char* epi, const BatchInstance* BI = nullptr,
                                             const double* inst_base = nullptr, int species = 0) {
    const int tid = threadIdx.x;
    const int r = tid & (kRows - 1), h = tid >> 7;
    const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
    const int n1 = J.n1, n2 = J.n2;
    const int n1p = (n1 + 15) & ~15, m2 = (n2 + 127) / 128;
    const uint32_t c1 = cols[0], c2 = cols[1], c3 = cols[2];

    // G1: X[i][j'] = sum_j Y[i][j] Q[j][j']          (Y x_2 Q_theta^T), rows i
    const int n1q = J.n1q;
    if (BI) {
        run_gemm(P, gs[0], [&](int c, char* hi, char* lo, const float*) {
            float v[8];
            disk_F8(*BI, inst_base, species, r, c * 16 + h * 8, v);
            store_row8(hi, lo, r, h, v);
        });
    } else {
        run_gemm(P, gs[0], [&](int c, char* hi, char* lo, const float* raw) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int jl = h * 8 + q;
                v[q] = (r < n1 && c * 16 + jl < n2) ? raw[jl * n1q + r] : 0.f;
            }
            store_row8(hi, lo, r, h, v);
        });
    }
    // G2: Z^T[j][i] = sum_j' Q[j][j'] (Phi o X)[i][j']   (x_2 Q_theta), data in B, rows j
    run_gemm(P, gs[1], [&](int c, char* hi, char* lo, const float* raw) {
        float v[8];
        tmem_ld8(tmem + lane_base + c1 + (uint32_t)(c * 16 + h * 8), v);
        if (r < n1p) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int jl = h * 8 + q;
                v[q] = (r < n1 && c * 16 + jl < n2) ? v[q] * raw[jl * n1q + r] : 0.f;
            }
            store_row8(hi, lo, r, h, v);
        }
    });
    // G3: R^T[j][i'] = sum_i Z^T[j][i] P[i'][i]      (x_1 phi_1(tau d A_rho)), rows j
    run_gemm(P, gs[2], [&](int c, char* hi, char* lo, const float*) {
        for (int mt = 0; mt < m2; ++mt) {
            float v[8];
            tmem_ld8(tmem + lane_base + c2 + (uint32_t)(mt * n1p + c * 16 + h * 8), v);
            const int j = mt * kRows + r;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = c * 16 + h * 8 + q;
                if (!(j < n2 && i < n1)) v[q] = 0.f;
            }
            store_row8(hi, lo, mt * kRows + r, h, v);
        }
    });
    // w[k][j][i'] += tau R^T[j][i'], staged through shared memory for coalesced FP64 RMW.
    float* E = reinterpret_cast<float*>(epi);
    const int pitch = n1p + 1;
    for (int mt = 0; mt < m2; ++mt) {
        for (int c = 0; c < n1p / 16; ++c) {
            float v[8];
            tmem_ld8(tmem + lane_base + c3 + (uint32_t)(mt * n1p + c * 16 + h * 8), v);
#pragma unroll
            for (int q = 0; q < 8; ++q) E[r * pitch + c * 16 + h * 8 + q] = v[q];
        }
        compute_sync();
        const int rows = min(kRows, n2 - mt * kRows);
        const int count = rows * n1;
        double* Wt = J.W + (long long)mt * kRows * n1;
        const double* Wi = J.Win + (long long)mt * kRows * n1;
        // increment rounded to FP32, widened exactly by integer operations: one FP64 add per
        // point; eight independent read-modify-writes in flight per thread
        for (int f0 = tid; f0 < count; f0 += kThreads * 8) {
            double w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int f = f0 + u * kThreads;
                w[u] = f < count ? Wi[f] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int f = f0 + u * kThreads;
                if (f < count) {
                    const int jl = f / n1, i = f - jl * n1;
                    Wt[f] = w[u] + f32_to_f64(J.tau_f * E[jl * pitch + i]);
                }
            }
        }
        compute_sync();
    }
}

__global__ void __launch_bounds__(kBlock, 1)
    k_tc_slab(SplitTables T, uint32_t stage_bytes, uint32_t nst, uint32_t raw_bytes,
                                              uint32_t tmem_cols) {
    extern __shared__ char smem_raw[];
    CtaRes R = cta_begin(smem_raw, stage_bytes, nst, raw_bytes, tmem_cols, T.err);
    const int k = blockIdx.x, s = blockIdx.y;
    const long long n12 = (long long)T.n1 * T.n2;
    const long long plane = (long long)T.n2 * T.n1q;
    SlabJob J;
    J.n1 = T.n1;
    J.n2 = T.n2;
    J.n1q = T.n1q;
    J.Y = T.Y + (long long)s * T.ys + k * plane;
    J.W = T.state_upd + (long long)s * T.npts + k * n12;
    J.Win = J.W;
    J.QT = T.QT;
    J.Q = T.Q;
    J.P = T.P[s];
    J.had = T.had_theta + (long long)s * T.had_theta_sp + (T.geometry == GEO_BALL ? k * plane : 0);
    J.tau_f = T.tau;
    if (threadIdx.x == kThreads) l2_prefetch(J.W, (unsigned long long)n12 * 8);
    GemmSpec gs[3];
    uint32_t cols[3];
    slab_specs(J, R.tmem, tmem_cols, gs, cols);
    if (threadIdx.x >= kThreads + 32) mma_issuer(R.P, gs, 3);
    else if (threadIdx.x >= kThreads) tma_issuer(R.P, gs, 3);
    else slab_compute(J, gs, cols, R.P, R.tmem, R.P.stages);
    cta_end(R, tmem_cols);
}

// ------------------------------------------------------------------------------
// Batched disks: a persistent CTA per SM takes (instance, species) items from the
// LPT-ordered work list and runs the whole disk chain of eq. ee_disk for it --
// F from the previous state, x_2 Q_theta^T, Hadamard, x_2 Q_theta, x_1
// phi_1(tau d A_rho) -- writing the updated species into the other state buffer.
__global__ void __launch_bounds__(kBlock, 1)
    k_tc_batch(BatchTables B, uint32_t stage_bytes, uint32_t nst, uint32_t raw_bytes,
                                              uint32_t tmem_cols) {
    extern __shared__ char smem_raw[];
    __shared__ int s_item;
    CtaRes R = cta_begin(smem_raw, stage_bytes, nst, raw_bytes, tmem_cols, B.err);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(B.counter, 1);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const int it = s_item;
        __syncthreads();
        if (it >= B.n_items) break;
        const int2 item = B.items[it];
        const BatchInstance& I = B.inst[item.x];
        const int s = item.y;
        const long long n12 = (long long)I.n1 * I.n2;
        SlabJob J;
        J.n1 = I.n1;
        J.n2 = I.n2;
        J.n1q = (I.n1 + 3) & ~3;
        J.Y = nullptr;
        J.Win = B.W_in + I.w_off + s * n12;
        J.W = B.W_out + I.w_off + s * n12;
        J.QT = I.QT;
        J.Q = I.Q;
        J.P = I.P[s];
        J.had = I.had + s * (long long)I.n2 * J.n1q;
        J.tau_f = B.tau;
        if (threadIdx.x == kThreads) l2_prefetch(J.Win, (unsigned long long)n12 * 8);
        GemmSpec gs[3];
        uint32_t cols[3];
        slab_specs(J, R.tmem, tmem_cols, gs, cols);
        if (threadIdx.x >= kThreads + 32) mma_issuer(R.P, gs, 3);
        else if (threadIdx.x >= kThreads) tma_issuer(R.P, gs, 3);
        else slab_compute(J, gs, cols, R.P, R.tmem, R.P.stages, &I, B.W_in + I.w_off, s);
    }
    cta_end(R, tmem_cols);
}

// ------------------------------------------------------------------------------
// Host-side shape logic.

static uint32_t round_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

static uint32_t pow2_cols(uint32_t c) {
    uint32_t p = 32;
    while (p < c) p <<= 1;
    return p;
}

// Stage-ring depth and shared-memory size: three stages when two CTAs still fit
// on one SM (228 KB per SM, 1 KB reserved per CTA), else two.
static void ring(TcShape& sh, uint32_t min_body) {
    const uint32_t pair_limit = 228 * 1024 / 2 - 1024 - 128;   // 128: alignment slack of the ring
    sh.nst = 3;
    if (kHeaderBytes + 3 * sh.stage_bytes > pair_limit && kHeaderBytes + 2 * sh.stage_bytes >= min_body) sh.nst = 2;
    uint32_t body = sh.nst * sh.stage_bytes;
    if (body < min_body) body = min_body;
    sh.smem_bytes = 128 + kHeaderBytes + body;
}

TcShape tc_mode3_shape(int geometry, int n1, int n2, int n3) {
    (void)n1;
    (void)n2;
    TcShape sh{};
    const uint32_t n3p = round_up(n3, 16);
    sh.raw_bytes = raw_bytes_for(kRows);
    sh.stage_bytes = round_up(2u * kRows * kTileRowBytes + 2u * n3p * kTileRowBytes + sh.raw_bytes, 128);
    sh.tmem_cols = pow2_cols(geometry == GEO_BALL ? 2 * n3p : n3p);
    ring(sh, 0);
    return sh;
}

// Tensor-memory columns of a slab (see slab_specs): a power of two holding G1
// and G2 side by side and G2 and G3 side by side.
uint32_t slab_tmem_cols(int n1, int n2) {
    const uint32_t n1p = round_up(n1, 16), n2p = round_up(n2, 16), m2 = (n2 + 127) / 128;
    const uint32_t need = std::max(n2p + m2 * n1p, 2 * m2 * n1p);
    return pow2_cols(need);
}

TcShape tc_slab_shape(int n1, int n2) {
    TcShape sh{};
    const uint32_t n1p = round_up(n1, 16), n2p = round_up(n2, 16), m2 = (n2 + 127) / 128;
    const uint32_t rows1 = kRows + n2p;                 // G1: data 128 rows, matrix n2p rows
    const uint32_t rows2 = n1p + kRows * m2;            // G2: data n1p rows, matrix 128 m2 rows
    const uint32_t rows3 = kRows * m2 + n1p;            // G3
    uint32_t rows = rows1 > rows2 ? rows1 : rows2;
    rows = rows > rows3 ? rows : rows3;
    sh.raw_bytes = raw_bytes_for((int)round_up(n1, 4));
    sh.stage_bytes = round_up(2u * rows * kTileRowBytes + sh.raw_bytes, 128);
    const uint32_t epi = kRows * (n1p + 1) * 4u;       // epilogue staging reuses the ring
    sh.tmem_cols = slab_tmem_cols(n1, n2);
    ring(sh, epi);
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
    if (e != cudaSuccess) return e;
    const int big = 212 * 1024;   // stencil tiles (all species) are sized to at most 212 KB
    e = cudaFuncSetAttribute(k_rhs_tile<GEO_DISK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_tile<GEO_SPHERE>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_tile<GEO_BALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_tile<GEO_CYLINDER>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    return e;
}

cudaError_t launch_tc_mode3(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    dim3 grid((unsigned)((T.n1q * (long long)T.n2 + kRows - 1) / kRows), T.S);
    if (T.geometry == GEO_BALL)
        k_tc_mode3<GEO_BALL><<<grid, kBlock, sh.smem_bytes, st>>>(T, sh.stage_bytes, sh.nst, sh.raw_bytes, sh.tmem_cols);
    else
        k_tc_mode3<GEO_CYLINDER><<<grid, kBlock, sh.smem_bytes, st>>>(T, sh.stage_bytes, sh.nst, sh.raw_bytes, sh.tmem_cols);
    return cudaGetLastError();
}

cudaError_t launch_tc_slab(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    dim3 grid(T.geometry == GEO_DISK ? 1 : T.n3, T.S);
    k_tc_slab<<<grid, kBlock, sh.smem_bytes, st>>>(T, sh.stage_bytes, sh.nst, sh.raw_bytes, sh.tmem_cols);
    return cudaGetLastError();
}

// j-tile of the stencil pass: among the sizes whose all-species tile fits in
// 200 KB, the one with the least (waves x lines per CTA), i.e. the shortest
// critical path when CTAs are spread over the 152 SMs.
template <int GEO>
static int rhs_tile_tj(const SplitTables& T) {
    using TS = TileShape<GEO>;
    const size_t per_line = sizeof(float2) * (size_t)T.S * (TS::TK + 2 * TS::KH) * T.n1;
    const long long ktiles = (T.n3 + TS::TK - 1) / TS::TK;
    int best = 1;
    double best_cost = 1e300;
    for (int tj = 1; tj <= (TS::k3 ? 16 : 32); ++tj) {
        const size_t smem = per_line * (tj + 2) + 8 * 1024;
        if (smem > 220 * 1024) break;
        const long long per_sm = std::min<long long>(228 * 1024 / smem, 2048 / kRhsThreads);
        const long long ctas = (T.n2 + tj - 1) / tj * ktiles;
        const long long waves = (ctas + 152 * per_sm - 1) / (152 * per_sm);
        const double cost = (double)waves * tj * (1.0 + 2.0 / tj * 0.25);   // halo rows cost a quarter line
        if (cost < best_cost) {
            best_cost = cost;
            best = tj;
        }
    }
    return best;
}

template <int GEO>
static cudaError_t launch_rhs_tile_geo(const SplitTables& T, cudaStream_t st) {
    using TS = TileShape<GEO>;
    const int tj = rhs_tile_tj<GEO>(T);
    const size_t smem = sizeof(float2) * (size_t)T.S * (TS::TK + 2 * TS::KH) * (tj + 2) * T.n1;
    dim3 grid((T.n2 + tj - 1) / tj, (T.n3 + TS::TK - 1) / TS::TK, 1);
    k_rhs_tile<GEO><<<grid, kRhsThreads, smem, st>>>(T.rhs, T.state, T.Y, tj, T.n1q, T.ys);
    return cudaGetLastError();
}

TcShape tc_batch_shape(int max_n1, int max_n2, uint32_t tmem_cols) {
    TcShape sh = tc_slab_shape(max_n1, max_n2);
    sh.tmem_cols = std::max(sh.tmem_cols, tmem_cols);
    return sh;
}

cudaError_t tc_prepare_batch(uint32_t smem) {
    return cudaFuncSetAttribute(k_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_tc_batch(const BatchTables& B, const TcShape& sh, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(B.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_tc_batch<<<152, kBlock, sh.smem_bytes, st>>>(B, sh.stage_bytes, sh.nst, sh.raw_bytes, sh.tmem_cols);
    return cudaGetLastError();
}

cudaError_t launch_rhs_split(const SplitTables& T, cudaStream_t st) {
    switch (T.geometry) {
    case GEO_DISK: return launch_rhs_tile_geo<GEO_DISK>(T, st);
    case GEO_SPHERE: return launch_rhs_tile_geo<GEO_SPHERE>(T, st);
    case GEO_BALL: return launch_rhs_tile_geo<GEO_BALL>(T, st);
    default: return launch_rhs_tile_geo<GEO_CYLINDER>(T, st);
    }
}

}  // namespace sexpe
