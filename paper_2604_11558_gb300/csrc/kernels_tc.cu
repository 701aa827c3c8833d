// Split-TF32 tensor-core kernels (tcgen05 + TMEM + TMA bulk copies, sm_103a)
// for the per-step chain of the split exponential Euler method:
//
//   stencil pass (all geometries, SIMT): F = d M w + g(w) in FP32 from FP64-
//       accurate differences -> Y; a tiled kernel and, for the 3-D
//       geometries, a rolling-window kernel along k (timed against each other
//       at setup).
//   mode-3 pass (ball, cylinder), in place on Y: F x_3 V_phi^{-1}, Hadamard
//       Phi_{rho,.,phi}, x_3 V_phi (ball, eq. ee_ball) or F x_3 phi_1(tau d A_z)
//       (cylinder, eq. ee_cylinder).
//   slab pass (disk, ball, cylinder), one k-slab per CTA: Y x_2 Q_theta^T,
//       Hadamard Phi (theta factor), x_2 Q_theta, x_1 phi_1(tau d A_rho),
//       w += tau * result (eqs. ee_disk, ee_ball, ee_cylinder).
//   sphere (eq. ee_sphere): Y x_2 phi_1(tau d A_phi) (N-tiled over CTAs), then
//       x_1 Q_theta^T, Hadamard, x_1 Q_theta and the update.
//   batched disks: one cooperative persistent launch per step, a stencil phase
//       over every instance, a grid barrier, then the disk chain per
//       (instance, species) item.
//
// Every mu-mode product is D = A B^T with FP32 accumulation in tensor memory
// and three TF32 MMAs per K-step (lo*hi, hi*lo, hi*hi).  The constant matrix of
// a product arrives by one TMA bulk copy per K-chunk, from an image pre-laid in
// the canonical K-major no-swizzle layout, into a matrix ring; the data operand
// is written into a data ring by 256 threads (two per row, eight K-columns
// each), split into TF32 hi/lo on the way.  Intermediates stay in tensor
// memory: a row (lane) of one product becomes the row of the next operand, so
// the slab chain swaps the row mode once (theta -> rho) by putting the data in
// the B operand of the middle product.  Kernels of a step are launched with
// programmatic stream serialization (prologues overlap the previous kernel).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"
#include "launch.h"
#include "tc_ptx.cuh"

namespace sexpe {

// Launch with programmatic stream serialization (see pdl_wait in tc_ptx.cuh):
// the kernel's prologue overlaps the tail of the previous kernel in the stream.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

constexpr int kRows = 128;                 // MMA M and tensor-memory lanes
constexpr int kThreads = 256;              // producer threads: two per row, columns 0-7 / 8-15 of a chunk
constexpr int kBlock = kThreads + 64;      // + one warp issuing TMA copies ahead, one issuing the MMAs
constexpr int kMaxMat = 4;                 // matrix-ring slots (TMA lookahead; at most the data-ring slots)
constexpr int kMaxData = 4;                // data-ring slots
constexpr uint32_t kHeaderBytes = 256;     // barriers + tensor-memory slot + abort flag

// Two rings of shared-memory slots, both indexed by the running K-chunk
// counter g of the CTA: the constant matrix of chunk g goes to matrix slot
// g % nm (written by the TMA warp), its data operand to data slot g % nd
// (written by the producers).  The MMAs of a chunk release both slots through
// tcgen05.commit, so the TMA warp can run nm chunks ahead of the MMAs while
// the producers run nd chunks ahead.
struct Pipe {
    uint64_t* mat_empty;    // MMAs reading the matrix slot completed
    uint64_t* data_full;    // chunk ready: one arrive per producer warp + the matrix copy (TMA
                            // thread's arrive and transaction count)
    uint64_t* data_empty;   // MMAs reading the data slot completed
    char* mat_slots;
    char* data_slots;
    uint32_t mat_bytes;     // bytes per matrix slot (hi + lo tiles)
    uint32_t data_bytes;    // bytes per data slot (hi + lo tiles)
    uint32_t nm, nd;
    uint32_t g;             // K-chunks this thread's role has passed so far in this CTA
    // ring position of chunk g, kept incrementally (no divisions on the hot
    // paths): slot and phase parity (the number of completed ring turns, mod 2)
    uint32_t sd, pd, sm, pm;
    int* err;
    volatile int* aborted;
    __device__ __forceinline__ void advance() {
        ++g;
        if (++sd == nd) { sd = 0; pd ^= 1u; }
        if (++sm == nm) { sm = 0; pm ^= 1u; }
    }
};

// Bounded wait on a pipeline barrier; a phase that already completed returns
// after one try_wait (the hot path of the MMA thread), and after a timeout
// anywhere in the CTA the remaining waits give up quickly.
__device__ __forceinline__ void pipe_wait(Pipe& P, uint64_t* bar, uint32_t parity, int code) {
    if (mbar_try_wait(bar, parity)) return;
    const long long lim = *P.aborted ? 2000000LL : 4000000000LL;
    if (!mbar_wait_bounded(bar, parity, P.err, code, lim)) *P.aborted = 1;
}

// Barrier of the 256 compute threads only (the TMA and MMA warps run on their own).
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

struct GemmSpec {
    Image mat;
    int mat_is_A;     // constant matrix is the A operand (data is B) or the B operand
    int data_rows;    // rows of the data tile
    int m_tiles;      // 128-row tiles of A
    int n_pad;        // N of the product (rows of B), multiple of 16
    int k_chunks;
    uint32_t tmem_d;  // tensor-memory address of the accumulator (tile mt at + mt * n_pad)
};

// Eight floats a producer thread needs from global memory for one K-chunk.
struct Pre8 {
    float v[8];
};

// Eight values of a producer thread's row at columns k0 .. k0 + 7 of a strided
// table, base[k * stride], zero where the row is invalid or k >= kmax.  Full
// groups take unpredicated loads at 32-bit offsets from one row pointer (the
// producers issue few instructions per chunk: with 8 warps on an SM their
// instruction chains are not hidden by other warps).
__device__ __forceinline__ void load8_strided(Pre8& p, const float* base, int stride, int k0, int kmax, bool valid) {
    if (valid && k0 + 8 <= kmax) {
        const float* a = base + (long long)k0 * stride;
#pragma unroll
        for (int q = 0; q < 8; ++q) p.v[q] = __ldg(a + q * stride);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            p.v[q] = (valid && k0 + q < kmax) ? __ldg(base + (long long)(k0 + q) * stride) : 0.f;
    }
}

// Producer side of one product.  `load(c, Pre8&)` issues the global loads a
// thread needs for chunk c (or nothing), `produce(c, hi, lo, const Pre8&)`
// writes the data operand of chunk c into its slot; loads run two chunks ahead
// in registers so their latency overlaps the work of the chunks in between.  A
// data slot is rewritten only after the MMAs that read it completed.  Each
// producer warp arrives on the chunk's data barrier once its part is written
// AND the chunk's matrix copy has landed, so the MMA thread waits on a single
// barrier per chunk (every wait costs the issuing thread ~100+ cycles during
// which the tensor pipe runs dry).
// `tail()` runs after the last chunk is handed over and before the wait for the
// product's completion: loads that need nothing of this product (the next
// product's first chunks, the update's first state values) overlap that wait.
// With PRE the loads of chunks 0 and 1 were issued earlier, into pre[0..1].
struct NoTail {
    __device__ void operator()() const {}
};

template <bool PRE = false, class Loader, class Producer, class Tail = NoTail>
__device__ __forceinline__ void run_gemm(Pipe& P, const GemmSpec& G, Loader&& load, Producer&& produce,
                                         Tail&& tail = Tail{}, const Pre8* pre = nullptr) {
    Pre8 p0, p1;
    if constexpr (PRE) {
        p0 = pre[0];
        p1 = pre[1];
    } else {
        load(0, p0);
        if (G.k_chunks > 1) load(1, p1);
    }
    uint32_t last_sd = 0, last_pd = 0;
    const bool lane0 = (threadIdx.x & 31) == 0;
    for (int c = 0; c < G.k_chunks; ++c) {
        Pre8 p2;
        if (c + 2 < G.k_chunks) load(c + 2, p2);
        const uint32_t s = P.sd;
        // Slot reuse: the MMAs of chunk g - nd completed.  One lane per warp waits, once per
        // pair of chunks, on the later chunk's slot: MMAs complete (and commit) in issue order,
        // so that phase implies this one.  Every barrier probe costs the warp ~200+ cycles
        // while the tensor core streams operands from shared memory.
        if (lane0 && (c & 1) == 0) {
            const bool pair = c + 1 < G.k_chunks;
            const uint32_t s1 = pair ? (s + 1 == P.nd ? 0u : s + 1) : s;
            const uint32_t p1 = pair && s + 1 == P.nd ? P.pd ^ 1u : P.pd;
            if (P.g + (pair ? 1u : 0u) >= P.nd) pipe_wait(P, &P.data_empty[s1], p1 ^ 1u, DERR_TIMEOUT_MMA);
        }
        __syncwarp();
        char* hi = P.data_slots + (size_t)s * P.data_bytes;
        produce(c, hi, hi + G.data_rows * kTileRowBytes, p0);
        fence_async_smem();
        __syncwarp();
        if (lane0) mbar_arrive(&P.data_full[s]);
        last_sd = s;
        last_pd = P.pd;
        P.advance();
        p0 = p1;
        p1 = p2;
    }
    tail();
    // the product is complete in tensor memory once the last chunk's MMAs are
    if (lane0) pipe_wait(P, &P.data_empty[last_sd], last_pd, DERR_TIMEOUT_MMA);
    __syncwarp();
    tc_fence_after();
}

template <class Producer>
__device__ __forceinline__ void run_gemm(Pipe& P, const GemmSpec& G, Producer&& produce) {
    run_gemm(P, G, [](int, Pre8&) {}, produce);
}

// MMA side: one lane of the MMA warp walks the K-chunks of every product in
// order; once a chunk's data barrier completes (data operand written, matrix
// copy landed) it issues the three TF32 MMAs per K-step and commits them to
// both slots' empty barriers.
//
// The issuing thread is the only producer of work for the tensor pipe, and a
// few scalar instructions per MMA already cost more than an MMA of N = 112
// takes to execute (~60 cycles), so the loop is kept lean: descriptors of
// slot 0 are formed once per product and moved by constant offsets (in the
// descriptor's 16-byte address units, which cannot carry out of the 14-bit
// field below 256 KB), and the usual one-tile product is fully unrolled.
//
// The NG products are walked in an unrolled loop (NG is a compile-time constant at
// every call site), so the specs stay in registers instead of a local-memory array
// indexed at run time.
template <int NG>
__device__ __forceinline__ void mma_issuer(Pipe& P, const GemmSpec* gs) {
    if ((threadIdx.x & 31) != 0) return;
    const uint32_t mat16 = P.mat_bytes >> 4, data16 = P.data_bytes >> 4;
    constexpr uint64_t kKStep = (2 * kLBO) >> 4;       // next 8 K-columns: two core matrices
    const uint32_t mslot0 = smem_u32(P.mat_slots), dslot0 = smem_u32(P.data_slots);
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        const GemmSpec& G = gs[q];
        const int nsub = G.n_pad < 256 ? G.n_pad : 256;
        const int n_halves = G.n_pad / nsub;
        const uint32_t idesc = idesc_tf32(128, nsub);
        // hi tile at the slot start, lo tile right after it
        const uint32_t mtile = (uint32_t)G.mat.rows_pad * kTileRowBytes, dtile = (uint32_t)G.data_rows * kTileRowBytes;
        const uint64_t dmh = smem_desc(mslot0, kLBO, kSBO), dml = smem_desc(mslot0 + mtile, kLBO, kSBO);
        const uint64_t ddh = smem_desc(dslot0, kLBO, kSBO), ddl = smem_desc(dslot0 + dtile, kLBO, kSBO);
        const uint32_t d = G.tmem_d;
        const bool one_tile = G.m_tiles == 1 && n_halves == 1;
        const bool two_tiles = G.m_tiles == 2 && n_halves == 1;
        for (int c = 0; c < G.k_chunks; ++c, P.advance()) {
            const uint32_t sm = P.sm, sd = P.sd;
            pipe_wait(P, &P.data_full[sd], P.pd, DERR_TIMEOUT_MMA);     // data written, matrix landed
            tc_fence_after();
            const uint64_t om = (uint64_t)sm * mat16, od = (uint64_t)sd * data16;
            const uint64_t mh = dmh + om, ml = dml + om, dh = ddh + od, dl = ddl + od;
            const uint64_t ah = G.mat_is_A ? mh : dh, al = G.mat_is_A ? ml : dl;
            const uint64_t bh = G.mat_is_A ? dh : mh, bl = G.mat_is_A ? dl : ml;
            if (one_tile) {
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {       // lo*hi, hi*lo, hi*hi per K-step
                    const uint64_t k = (uint64_t)ks * kKStep;
                    mma_tf32(d, al + k, bh + k, idesc, (c | ks) != 0);
                    mma_tf32(d, ah + k, bl + k, idesc, 1u);
                    mma_tf32(d, ah + k, bh + k, idesc, 1u);
                }
            } else if (two_tiles) {
                // two 128-row tiles of A, one N range: the general loop's order, unrolled (the
                // issuing thread's per-MMA overhead otherwise doubles the chunk's issue time)
                constexpr uint64_t kTile = (16 * kSBO) >> 4;  // next 128 rows of A
                const uint32_t d1 = d + (uint32_t)G.n_pad;
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint64_t k = (uint64_t)ks * kKStep;
                    const uint32_t acc = (c | ks) != 0;
                    mma_tf32(d, al + k, bh + k, idesc, acc);
                    mma_tf32(d1, al + kTile + k, bh + k, idesc, acc);
                    mma_tf32(d, ah + k, bl + k, idesc, 1u);
                    mma_tf32(d1, ah + kTile + k, bl + k, idesc, 1u);
                    mma_tf32(d, ah + k, bh + k, idesc, 1u);
                    mma_tf32(d1, ah + kTile + k, bh + k, idesc, 1u);
                }
            } else {
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
#pragma unroll
                    for (int pass = 0; pass < 3; ++pass) {
                        const uint64_t a = ((pass == 0) ? al : ah) + (uint64_t)ks * kKStep;
                        const uint64_t b = ((pass == 1) ? bl : bh) + (uint64_t)ks * kKStep;
                        const uint32_t acc = (c | ks | pass) != 0;
                        for (int mt = 0; mt < G.m_tiles; ++mt) {
                            const uint64_t am = a + (uint64_t)mt * ((16 * kSBO) >> 4);
                            for (int nh = 0; nh < n_halves; ++nh)
                                mma_tf32(d + (uint32_t)(mt * G.n_pad + nh * nsub), am,
                                         b + (uint64_t)nh * (((nsub / 8) * kSBO) >> 4), idesc, acc);
                        }
                    }
                }
            }
            mma_commit(&P.data_empty[sd]);
            mma_commit(&P.mat_empty[sm]);
        }
    }
    // No MMA of this CTA may be in flight when its tensor memory is freed, also
    // after a timed-out wait made the chain run ahead: wait (bounded) for the
    // last commit.  In a healthy run it completes within the MMAs' latency.
    if (P.g > 0) {
        const uint32_t sd = P.sd ? P.sd - 1 : P.nd - 1, pd = P.sd ? P.pd : P.pd ^ 1u;
        pipe_wait(P, &P.data_empty[sd], pd, DERR_TIMEOUT_MMA);
    }
}

// TMA side: one lane of the extra warp walks the K-chunks of every product of
// the CTA in order and copies each chunk's matrix image (hi tile then lo tile,
// one bulk copy) into its slot as soon as the slot is free, up to nm chunks ahead
// of the MMAs.
template <int NG>
__device__ __forceinline__ void tma_issuer(Pipe& P, const GemmSpec* gs) {
    if ((threadIdx.x & 31) != 0) return;
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        const GemmSpec& G = gs[q];
        const uint32_t tile = (uint32_t)G.mat.rows_pad * kTileRowBytes;
        for (int c = 0; c < G.k_chunks; ++c, P.advance()) {
            const uint32_t s = P.sm;
            if (P.g >= P.nm) pipe_wait(P, &P.mat_empty[s], P.pm ^ 1u, DERR_TIMEOUT_MMA);
            char* slot = P.mat_slots + (size_t)s * P.mat_bytes;
            const float* src = G.mat.ptr + (long long)c * G.mat.chunk_floats;
            // the copy completes on the chunk's data barrier; its previous phase (chunk
            // g - nd <= g - nm, consumed by the MMA thread before it issued the MMAs whose
            // completion freed this matrix slot) is over, as nm <= nd
            mbar_arrive_expect_tx(&P.data_full[P.sd], 2 * tile);
            tma_bulk_g2s(slot, src, 2 * tile, &P.data_full[P.sd]);
        }
    }
    // No copy of this CTA may still be landing when the CTA exits or its shared
    // memory is reused, also after a timed-out wait: wait (bounded) for the
    // data barriers of the last nd chunks.  In a healthy run these phases
    // completed long ago.
    const uint32_t last = P.g < P.nd ? P.g : P.nd;
    for (uint32_t b = 1; b <= last; ++b) {
        const uint32_t sd = (P.sd + P.nd - b) % P.nd;
        const uint32_t pd = b > P.sd ? P.pd ^ 1u : P.pd;
        pipe_wait(P, &P.data_full[sd], pd, DERR_TIMEOUT_TMA);
    }
}

// Kernel prologue/epilogue: carve shared memory, init barriers, allocate TMEM.
struct CtaRes {
    Pipe P;
    uint32_t tmem;
};

__device__ __forceinline__ CtaRes cta_begin(char* smem_raw, const TcShape& rs, int* err) {
    const uint32_t tmem_cols = rs.tmem_cols;
    const uint32_t base = smem_u32(smem_raw);
    char* smem = smem_raw + (((base + 127u) & ~127u) - base);   // 128-byte aligned rings
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + (kMaxMat + 2 * kMaxData) * sizeof(uint64_t));
    int* aborted = reinterpret_cast<int*>(tslot + 4);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxMat; ++s) mbar_init(&bars[s], 1);   // mat_empty: tcgen05.commit
        for (int s = 0; s < kMaxData; ++s) {
            mbar_init(&bars[kMaxMat + s], kThreads / 32 + 1);              // data_full: producer warps + TMA
            mbar_init(&bars[kMaxMat + kMaxData + s], 1);                   // data_empty: tcgen05.commit
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
    r.P.mat_empty = bars;
    r.P.data_full = bars + kMaxMat;
    r.P.data_empty = bars + kMaxMat + kMaxData;
    r.P.mat_slots = smem + kHeaderBytes;
    r.P.data_slots = r.P.mat_slots + (size_t)rs.nm * rs.mat_bytes;
    r.P.mat_bytes = rs.mat_bytes;
    r.P.data_bytes = rs.data_bytes;
    r.P.nm = rs.nm;
    r.P.nd = rs.nd;
    r.P.g = r.P.sd = r.P.pd = r.P.sm = r.P.pm = 0;
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

constexpr int kRhsThreads = 512;   // threads of a stencil CTA, spread over (line, i) items

// Coefficients of the stencil at one point: axis 1 at i, axis 2 at j, axis 3 at k.
struct PointCoef {
    float lo1, up1, rs1, dr;     // A_rho row i (A_theta row i on the sphere), rho_i^-2
    float rs2, lo2, up2;         // axis-2 row j
    float rs3, lo3, up3, dp3;    // axis-3 row k, sin^-2 phi_k (ball)
};

// F of species s at one point from split (hi, lo) pairs: centre c, neighbours
// along mode 1 (m, p), mode 2 (jm, jp) and mode 3 (km, kp), each used only when
// its flag is set; g is the species' reaction term at the point.  Differences
// of pairs keep FP32 relative accuracy of the difference (Section 2 Kronecker
// sums, applied in difference form).  Every operation is pinned, so all
// stencil kernels form bit-identical F.
template <int GEO>
__device__ __forceinline__ float point_F(const RhsTables<float>& tb, int s, float g, float2 c, float2 m,
                                         float2 p, float2 jm, float2 jp, float2 km, float2 kp, bool has_m,
                                         bool has_p, bool has_jm, bool has_jp, bool has_km, bool has_kp,
                                         const PointCoef& cf, float dpj) {
    const float cv = c.x + c.y;
    float t0 = __fmul_rn(cf.rs1, cv);
    if (has_m) t0 = __fmaf_rn(cf.lo1, sdiff(m, c), t0);
    if (has_p) t0 = __fmaf_rn(cf.up1, sdiff(p, c), t0);
    float t1 = __fmul_rn(cf.rs2, cv);
    if (has_jm) t1 = __fmaf_rn(cf.lo2, sdiff(jm, c), t1);
    if (has_jp) t1 = __fmaf_rn(cf.up2, sdiff(jp, c), t1);
    float lap;
    if constexpr (GEO == GEO_DISK) {
        lap = __fmaf_rn(cf.dr, t1, t0);
    } else if constexpr (GEO == GEO_SPHERE) {
        lap = __fmaf_rn(dpj, t0, t1);
    } else {
        float t2 = __fmul_rn(cf.rs3, cv);
        if (has_km) t2 = __fmaf_rn(cf.lo3, sdiff(km, c), t2);
        if (has_kp) t2 = __fmaf_rn(cf.up3, sdiff(kp, c), t2);
        if constexpr (GEO == GEO_BALL) lap = __fmaf_rn(cf.dr, __fmaf_rn(cf.dp3, t1, t2), t0);
        else lap = __fmaf_rn(cf.dr, t1, t0) + t2;
    }
    return __fmaf_rn(tb.d[s], lap, g);
}

// F of every species at one point from split pairs in shared memory: pc[s * ss]
// is the centre of species s; in-plane neighbours at -1/+1 (i, with the
// periodic wrap dm/dp) and -/+ jstride (j); the k-neighbours at km/kp
// (relative to pc).
template <int GEO>
__device__ __forceinline__ void rhs_point(const RhsTables<float>& tb, const float2* pc, int ss, int jstride,
                                          long long km, long long kp, int dm, int dp, bool has_m, bool has_p,
                                          bool has_jm, bool has_jp, bool has_km, bool has_kp, const PointCoef& cf,
                                          float* Fo, long long ys, float dpj, const float* add = nullptr) {
    const int S = tb.S;
    float w[kMaxSpecies];
#pragma unroll
    for (int r = 0; r < kMaxSpecies; ++r) {
        if (r < S) {
            const float2 c = pc[r * ss];
            w[r] = c.x + c.y;
        } else {
            w[r] = 0.f;
        }
    }
    float g[kMaxSpecies];
    reactions<float, kMaxSpecies>(tb.reac, w, g);
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        if (s >= S) break;
        const float2* q = pc + s * ss;
        const float2 c = q[0];
        const bool k3 = GEO == GEO_BALL || GEO == GEO_CYLINDER;
        const float f = point_F<GEO>(tb, s, g[s], c, has_m ? q[dm] : c, has_p ? q[dp] : c, has_jm ? q[-jstride] : c,
                                     has_jp ? q[jstride] : c, (k3 && has_km) ? q[km] : c,
                                     (k3 && has_kp) ? q[kp] : c, has_m, has_p, has_jm, has_jp, has_km, has_kp, cf,
                                     dpj);
        Fo[s * ys] = add ? f + add[s] : f;
    }
}

// floor(q / d) by a multiply-high with m = floor(2^32 / d) + 1: q m / 2^32 lies in
// [q/d, q/d + q/2^32], and the excess cannot reach the next integer while
// q < 2^20 and d < 2^12 (the fractional part of q/d is at most 1 - 1/d).  For
// d = 1 the multiplier does not fit in 32 bits; it is encoded as 0.
__host__ __device__ constexpr uint32_t div_magic(uint32_t d) { return d == 1 ? 0u : (uint32_t)((1ull << 32) / d + 1); }
__device__ __forceinline__ int div_by(int q, uint32_t m) { return m ? (int)__umulhi((uint32_t)q, m) : q; }

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
    const uint32_t m_n1 = div_magic((uint32_t)n1), m_tj = div_magic((uint32_t)TJ);
    for (int row = threadIdx.x; row < rows; row += blockDim.x) {
        const int jj = row % nJ, kk = (row / nJ) % nK, sp = row / (nJ * nK);
        int j = j0 - 1 + jj;
        const int k = k0 - TS::KH + kk;
        if (TS::periodic2) j = j < 0 ? j + n2 : (j >= n2 ? j - n2 : j);
        const bool ok = j >= 0 && j < n2 && k >= 0 && k < n3;
        row_off[row] = ok ? sp * npts + (long long)k * n12 + (long long)j * n1 : -1;
    }
    __syncthreads();
    pdl_wait();          // the state (and the step counter) are the previous step's results
    pdl_trigger();
    __shared__ float s_et;                           // e^-t of this step (manufactured sources)
    if (GEO == GEO_DISK && threadIdx.x == 0) s_et = (float)mms_time_factor(tb);
    // tile fill: (row, i) items over all threads, kTileBatch loads in flight per thread
    const int items = rows * n1;
    for (int q0 = threadIdx.x; q0 < items; q0 += kRhsThreads * kTileBatch) {
        double v[kTileBatch];
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            const int q = q0 + u * kRhsThreads;
            const int row = div_by(q, m_n1);
            const long long off = q < items ? row_off[row] : -1;
            v[u] = off >= 0 ? __ldg(Wall + off + (q - row * n1)) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            const int q = q0 + u * kRhsThreads;
            if (q < items) tile[q] = split_f64(v[u]);
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
    // stencil + reaction: (line, i) items over all threads, line = kl * TJ + jl
    const int species_stride = nK * nJ * n1;
    const StencilAxis<float>& a1 = tb.ax[0];
    const int total = TS::TK * TJ * n1;
    for (int q = threadIdx.x; q < total; q += kRhsThreads) {
        const int line = div_by(q, m_n1);
        const int i = q - line * n1;
        const int kl = TS::k3 ? div_by(line, m_tj) : 0;
        const int jl = line - kl * TJ;
        const int j = j0 + jl, k = k0 + kl;
        if (j >= n2 || k >= n3) continue;
        PointCoef cf;
        cf.lo1 = __ldg(a1.lower + i);
        cf.up1 = __ldg(a1.upper + i);
        cf.rs1 = __ldg(a1.rs + i);
        cf.dr = (GEO == GEO_SPHERE) ? 1.f : __ldg(tb.Dr + i);
        cf.rs2 = cj[0][jl];
        cf.lo2 = cj[1][jl];
        cf.up2 = cj[2][jl];
        if (TS::k3) {
            cf.rs3 = ck[0][kl];
            cf.lo3 = ck[1][kl];
            cf.up3 = ck[2][kl];
            cf.dp3 = ck[3][kl];
        }
        const int cidx = ((kl + TS::KH) * nJ + (jl + 1)) * n1 + i;
        float src[2];
        const bool mms = GEO == GEO_DISK && tb.reac.kind == R_BVAM_MMS;
        if (mms) {
            src[0] = mms_source<float>(tb, i, j, s_et, 0);
            src[1] = mms_source<float>(tb, i, j, s_et, 1);
        }
        rhs_point<GEO>(tb, tile + cidx, species_stride, n1, -(long long)nJ * n1, (long long)nJ * n1,
                       i > 0 ? -1 : n1 - 1, i < n1 - 1 ? 1 : 1 - n1, i > 0 || TS::periodic1,
                       i < n1 - 1 || TS::periodic1, j > 0 || TS::periodic2, j < n2 - 1 || TS::periodic2, k > 0,
                       k < n3 - 1, cf, F + ((long long)k * n2 + j) * n1q + i, ys,
                       GEO == GEO_SPHERE ? tb.Dp[j] : 1.f, mms ? src : nullptr);
    }
}

// Stencil pass of the 3-D geometries as a rolling window along k: the CTA owns
// TJ theta-lines x KS planes (all rho, all species) and keeps four planes
// (k - 1, k, k + 1 and the one being filled) in a shared-memory ring.  The
// loads of plane k + 2 are in flight in registers while plane k is computed,
// so HBM latency overlaps the stencil work; each plane is split once.
// RV = values per thread and plane (S (TJ + 2) n1 <= RV * 512); MINB = CTAs
// per SM the registers are capped for (2: 64 registers, two CTAs' warps hide
// each other's latency; 1: no cap, no spills).
template <int GEO, int RV, int MINB>
__global__ void __launch_bounds__(kRhsThreads, MINB) k_rhs_roll(RhsTables<float> tb, const double* __restrict__ Wall,
                                                          float* __restrict__ F, int TJ, int KS, int n1q,
                                                          long long ys) {
    extern __shared__ float2 ring[];                 // [4][S][nJ][n1]
    __shared__ float cj[3][32];
    __shared__ long long line_off[kMaxSpecies * 34];   // offset of (species, j-line) within a plane, -1 outside
    const int n1 = tb.n1, n2 = tb.n2, n3 = tb.n3, S = tb.S;
    const int j0 = blockIdx.x * TJ, k0 = blockIdx.y * KS;
    const int kend = min(k0 + KS, n3);
    const int nJ = TJ + 2;
    const int lines = S * nJ;
    const int pv = lines * n1;                       // values per plane
    const long long npts = tb.npts;
    const long long n12 = (long long)n1 * n2;
    const uint32_t m_n1 = div_magic((uint32_t)n1);
    for (int l = threadIdx.x; l < lines; l += kRhsThreads) {
        const int jj = l % nJ, sp = l / nJ;
        int j = j0 - 1 + jj;
        j = j < 0 ? j + n2 : (j >= n2 ? j - n2 : j);   // theta is periodic
        line_off[l] = (j >= 0 && j < n2) ? sp * npts + (long long)j * n1 : -1;
    }
    if (threadIdx.x < TJ) {
        const int j = min(j0 + (int)threadIdx.x, n2 - 1);
        cj[0][threadIdx.x] = tb.ax[1].rs[j];
        cj[1][threadIdx.x] = tb.ax[1].lower[j];
        cj[2][threadIdx.x] = tb.ax[1].upper[j];
    }
    __syncthreads();
    double v[RV];
    auto load_plane = [&](int k) {
#pragma unroll
        for (int u = 0; u < RV; ++u) {
            const int q = threadIdx.x + u * kRhsThreads;
            const int line = div_by(q, m_n1);
            const long long off = (q < pv && k >= 0 && k < n3) ? line_off[line] : -1;
            v[u] = off >= 0 ? __ldg(Wall + off + (long long)k * n12 + (q - line * n1)) : 0.0;
        }
    };
    auto store_plane = [&](int k) {
        float2* P = ring + (size_t)((k - k0 + 1) & 3) * pv;
#pragma unroll
        for (int u = 0; u < RV; ++u) {
            const int q = threadIdx.x + u * kRhsThreads;
            if (q < pv) P[q] = split_f64(v[u]);
        }
    };
    pdl_wait();          // the state is the previous step's result
    pdl_trigger();
    load_plane(k0 - 1);
    store_plane(k0 - 1);
    load_plane(k0);
    store_plane(k0);
    load_plane(k0 + 1);
    store_plane(k0 + 1);
    __syncthreads();
    const StencilAxis<float>& a1 = tb.ax[0];
    const int total = TJ * n1;
    for (int k = k0; k < kend; ++k) {
        if (k + 2 <= kend) load_plane(k + 2);        // lands while plane k is computed
        PointCoef cf;
        cf.rs3 = tb.ax[2].rs[k];
        cf.lo3 = tb.ax[2].lower[k];
        cf.up3 = tb.ax[2].upper[k];
        cf.dp3 = (GEO == GEO_BALL) ? tb.Dp[k] : 1.f;
        const float2* Pc = ring + (size_t)((k - k0 + 1) & 3) * pv;
        const long long km = (long long)(((k - k0) & 3) - ((k - k0 + 1) & 3)) * pv;
        const long long kp = (long long)(((k - k0 + 2) & 3) - ((k - k0 + 1) & 3)) * pv;
        for (int q = threadIdx.x; q < total; q += kRhsThreads) {
            const int jl = div_by(q, m_n1);
            const int i = q - jl * n1;
            const int j = j0 + jl;
            if (j >= n2) continue;
            cf.lo1 = __ldg(a1.lower + i);
            cf.up1 = __ldg(a1.upper + i);
            cf.rs1 = __ldg(a1.rs + i);
            cf.dr = __ldg(tb.Dr + i);
            cf.rs2 = cj[0][jl];
            cf.lo2 = cj[1][jl];
            cf.up2 = cj[2][jl];
            rhs_point<GEO>(tb, Pc + (jl + 1) * n1 + i, nJ * n1, n1, km, kp, -1, 1, i > 0, i < n1 - 1, true, true,
                           k > 0, k < n3 - 1, cf, F + ((long long)k * n2 + j) * n1q + i, ys, 1.f);
        }
        if (k + 2 <= kend) store_plane(k + 2);       // slot of plane k - 2, free since the last barrier
        __syncthreads();
    }
}

// Stencil pass of the 3-D geometries marching along k with the k-neighbours in
// registers: the CTA owns TJ theta-lines x KS planes of every species, thread t
// the column (jl, i) = (t / n1, t mod n1), jl < TJ.  Each thread keeps the
// split pairs of planes k - 1 and k of its column in registers; only plane k
// goes through shared memory (two buffers, with the halo lines j0 - 1 and
// j0 + TJ, which threads t < 2 n1 carry as well) for the in-plane neighbours:
// one FP64 load and one split per value and plane, four shared loads per
// point and species.  The FP64 values of planes k + 1 .. k + kMarchAhead are in
// flight in a shared-memory ring of asynchronous copies (each thread reads back
// only its own copies), enough bytes in flight per SM to cover the DRAM latency
// without holding them in registers; one barrier per plane.  Addresses advance
// by one plane per step (the kernel issues few instructions per point: it is
// otherwise issue-bound).  Lines past n2 of a ragged last tile are loaded with
// the periodic wrap of theta but not computed.  SM: the number of species
// (1024 threads per CTA for up to two, else 512).
constexpr int kMarchAhead = 4;

template <int GEO, int SM>
__global__ void __launch_bounds__(SM <= 2 ? 1024 : 512, 1)
    k_rhs_march(RhsTables<float> tb, const double* __restrict__ Wall, float* __restrict__ F, int TJ, int KS, int n1q,
                long long ys) {
    extern __shared__ float2 pbuf[];                 // [2][S][TJ + 2][n1] pairs, then the ring
    const int n1 = tb.n1, n2 = tb.n2, n3 = tb.n3;
    constexpr int S = SM;                            // the species count, fixed per instantiation
    const int j0 = blockIdx.x * TJ, k0 = blockIdx.y * KS;
    const int kend = min(k0 + KS, n3);
    const int lpv = (TJ + 2) * n1;                   // values per species and buffered plane
    const int rs = blockDim.x + 2 * n1;              // ring values per species and plane: own, then halo
    double* ring = reinterpret_cast<double*>(pbuf + 2 * S * lpv);   // [kMarchAhead][S][rs]
    const long long npts = tb.npts, n12 = (long long)n1 * n2;
    const int t = threadIdx.x;
    const int jl = t / n1, i = t - jl * n1;
    const int jr = j0 + jl;
    const bool ld = jl < TJ;                         // loads buffer line jl + 1
    const bool own = ld && jr < n2;                  // and computes its points
    const int jw = ld ? (jr < n2 ? jr : jr - n2) : 0;
    const bool halo = t < 2 * n1;
    const int hline = t < n1 ? 0 : TJ + 1, hi = halo ? (t < n1 ? t : t - n1) : 0;
    int hj = t < n1 ? j0 - 1 : j0 + TJ;
    hj = hj < 0 ? hj + n2 : (hj >= n2 ? hj - n2 : hj);
    const int obuf = (jl + 1) * n1 + i, hbuf = hline * n1 + hi;
    PointCoef cf{};
    if (own) {
        cf.lo1 = __ldg(tb.ax[0].lower + i);
        cf.up1 = __ldg(tb.ax[0].upper + i);
        cf.rs1 = __ldg(tb.ax[0].rs + i);
        cf.dr = __ldg(tb.Dr + i);
        cf.rs2 = __ldg(tb.ax[1].rs + jr);
        cf.lo2 = __ldg(tb.ax[1].lower + jr);
        cf.up2 = __ldg(tb.ax[1].upper + jr);
    }
    // next plane to fetch, its global sources and this thread's ring entries
    int kf = k0 + 1;
    const double* go = Wall + (long long)jw * n1 + i + (long long)kf * n12;
    const double* gh = Wall + (long long)(halo ? hj : 0) * n1 + hi + (long long)kf * n12;
    const uint32_t r_own = smem_u32(ring + t), r_halo = smem_u32(ring + blockDim.x + t);
    const uint32_t slot_b = (uint32_t)(S * rs) * 8u, sp_b = (uint32_t)rs * 8u;
    auto fetch = [&]() {
        if (kf <= kend && kf < n3) {                 // later planes are never read
            const uint32_t so = (uint32_t)(kf & (kMarchAhead - 1)) * slot_b;
#pragma unroll
            for (int s = 0; s < SM; ++s) {
                if (s < S) {
                    if (ld) cp_async8(r_own + so + s * sp_b, go + s * npts);
                    if (halo) cp_async8(r_halo + so + s * sp_b, gh + s * npts);
                }
            }
        }
        cp_async_commit();
        go += n12;
        gh += n12;
        ++kf;
    };
    float2 pm[SM], pc[SM], pn[SM];
    pdl_wait();          // the state is the previous step's result
    pdl_trigger();
    for (int q = 0; q < kMarchAhead; ++q) fetch();
    {
        const double* g0 = Wall + (long long)jw * n1 + i + (long long)k0 * n12;
        const double* h0 = Wall + (long long)(halo ? hj : 0) * n1 + hi + (long long)k0 * n12;
#pragma unroll
        for (int s = 0; s < SM; ++s) {
            const bool v = s < S && ld;
            pm[s] = split_f64(v && k0 > 0 ? __ldg(g0 + s * npts - n12) : 0.0);
            pc[s] = split_f64(v ? __ldg(g0 + s * npts) : 0.0);
            if (v) pbuf[s * lpv + obuf] = pc[s];
            if (s < S && halo) pbuf[s * lpv + hbuf] = split_f64(__ldg(h0 + s * npts));
        }
    }
    __syncthreads();
    float* Fo = F + ((long long)k0 * n2 + (own ? jr : 0)) * n1q + i;
    const long long fstep = (long long)n2 * n1q;
    const bool hm = i > 0, hp = i < n1 - 1;
    for (int k = k0; k < kend; ++k, Fo += fstep) {
        const int b = (k - k0) & 1;
        const float2* Bc = pbuf + b * S * lpv + obuf;
        float2* Bn = pbuf + (b ^ 1) * S * lpv;
        cp_async_wait<kMarchAhead - 1>();            // plane k + 1 landed (this thread's copies)
        const double* R = ring + (size_t)((k + 1) & (kMarchAhead - 1)) * S * rs + t;
#pragma unroll
        for (int s = 0; s < SM; ++s) pn[s] = split_f64(s < S && ld ? R[s * rs] : 0.0);
        if (own) {
            cf.rs3 = __ldg(tb.ax[2].rs + k);
            cf.lo3 = __ldg(tb.ax[2].lower + k);
            cf.up3 = __ldg(tb.ax[2].upper + k);
            cf.dp3 = (GEO == GEO_BALL) ? __ldg(tb.Dp + k) : 1.f;
            float w[kMaxSpecies], g[SM];
#pragma unroll
            for (int r = 0; r < kMaxSpecies; ++r) w[r] = 0.f;
#pragma unroll
            for (int r = 0; r < SM; ++r)
                if (r < S) w[r] = pc[r].x + pc[r].y;
            reactions<float, SM>(tb.reac, w, g);
            const bool hkm = k > 0, hkp = k < n3 - 1;
#pragma unroll
            for (int s = 0; s < SM; ++s) {
                if (s < S) {
                    // every neighbour lies inside the buffer (lines 0 .. TJ + 1); the flags drop the absent ones
                    const float2* q = Bc + s * lpv;
                    Fo[s * ys] = point_F<GEO>(tb, s, g[s], pc[s], q[-1], q[1], q[-n1], q[n1], pm[s], pn[s], hm, hp,
                                              true, true, hkm, hkp, cf, 1.f);
                }
            }
        }
        if (k + 1 < kend) {
#pragma unroll
            for (int s = 0; s < SM; ++s) {
                if (s < S && ld) Bn[s * lpv + obuf] = pn[s];
                if (s < S && halo) Bn[s * lpv + hbuf] = split_f64(R[s * rs + blockDim.x]);
            }
        }
        __syncthreads();
        fetch();                                     // plane k + 1 + kMarchAhead, into the slot just read
#pragma unroll
        for (int s = 0; s < SM; ++s) {
            pm[s] = pc[s];
            pc[s] = pn[s];
        }
    }
    cp_async_wait<0>();                              // no copy may land after the CTA exits
}

// The marching stencil with two adjacent columns (i, i + 1), i even, per thread
// (n1 even, state 16-byte aligned): 16-byte copies and stores, the j-neighbours
// of both columns in one shared load each, and each column's i-neighbour on
// the other side taken from the thread's own registers; half the threads of
// k_rhs_march for the same tile and the same F bit for bit (same pairs, same
// point formula).
template <int GEO, int SM, int RK = -1>
__global__ void __launch_bounds__(512, 1)
    k_rhs_march2(RhsTables<float> tb, const double* __restrict__ Wall, float* __restrict__ F, int TJ, int KS, int n1q,
                 long long ys) {
    extern __shared__ float2 pbuf[];                 // [2][S][TJ + 2][n1] pairs, then the ring
    const int n1 = tb.n1, n2 = tb.n2, n3 = tb.n3, h1 = n1 >> 1;
    constexpr int S = SM;
    const int j0 = blockIdx.x * TJ, k0 = blockIdx.y * KS;
    const int kend = min(k0 + KS, n3);
    const int lpv = (TJ + 2) * n1;
    const int rs = 2 * (blockDim.x + n1);            // ring doubles per species and plane: own pairs, halo pairs
    double* ring = reinterpret_cast<double*>(pbuf + 2 * S * lpv);   // [kMarchAhead][S][rs]
    const long long npts = tb.npts, n12 = (long long)n1 * n2;
    const int t = threadIdx.x;
    const int jl = t / h1, i = 2 * (t - jl * h1);
    const int jr = j0 + jl;
    const bool ld = jl < TJ;
    const bool own = ld && jr < n2;
    const int jw = ld ? (jr < n2 ? jr : jr - n2) : 0;
    const bool halo = t < n1;                        // h1 pairs of each halo line
    const int hline = t < h1 ? 0 : TJ + 1, hi = halo ? 2 * (t < h1 ? t : t - h1) : 0;
    int hj = t < h1 ? j0 - 1 : j0 + TJ;
    hj = hj < 0 ? hj + n2 : (hj >= n2 ? hj - n2 : hj);
    const int obuf = (jl + 1) * n1 + i, hbuf = hline * n1 + hi;
    PointCoef cf0{}, cf1{};
    if (own) {
        cf0.lo1 = __ldg(tb.ax[0].lower + i);
        cf0.up1 = __ldg(tb.ax[0].upper + i);
        cf0.rs1 = __ldg(tb.ax[0].rs + i);
        cf0.dr = __ldg(tb.Dr + i);
        cf1.lo1 = __ldg(tb.ax[0].lower + i + 1);
        cf1.up1 = __ldg(tb.ax[0].upper + i + 1);
        cf1.rs1 = __ldg(tb.ax[0].rs + i + 1);
        cf1.dr = __ldg(tb.Dr + i + 1);
        cf0.rs2 = cf1.rs2 = __ldg(tb.ax[1].rs + jr);
        cf0.lo2 = cf1.lo2 = __ldg(tb.ax[1].lower + jr);
        cf0.up2 = cf1.up2 = __ldg(tb.ax[1].upper + jr);
    }
    int kf = k0 + 1;
    const double* go = Wall + (long long)jw * n1 + i + (long long)kf * n12;
    const double* gh = Wall + (long long)(halo ? hj : 0) * n1 + hi + (long long)kf * n12;
    const uint32_t r_own = smem_u32(ring + 2 * t), r_halo = smem_u32(ring + 2 * (blockDim.x + t));
    const uint32_t slot_b = (uint32_t)(S * rs) * 8u, sp_b = (uint32_t)rs * 8u;
    auto fetch = [&]() {
        if (kf <= kend && kf < n3) {
            const uint32_t so = (uint32_t)(kf & (kMarchAhead - 1)) * slot_b;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                if (ld) cp_async16(r_own + so + s * sp_b, go + s * npts);
                if (halo) cp_async16(r_halo + so + s * sp_b, gh + s * npts);
            }
        }
        cp_async_commit();
        go += n12;
        gh += n12;
        ++kf;
    };
    float2 pm0[S], pc0[S], pn0[S], pm1[S], pc1[S], pn1[S];   // columns i and i + 1
    pdl_wait();          // the state is the previous step's result
    pdl_trigger();
    for (int q = 0; q < kMarchAhead; ++q) fetch();
    {
        const double* g0 = Wall + (long long)jw * n1 + i + (long long)k0 * n12;
        const double* h0 = Wall + (long long)(halo ? hj : 0) * n1 + hi + (long long)k0 * n12;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const double2 a = ld && k0 > 0 ? __ldg(reinterpret_cast<const double2*>(g0 + s * npts - n12)) : make_double2(0.0, 0.0);
            const double2 b = ld ? __ldg(reinterpret_cast<const double2*>(g0 + s * npts)) : make_double2(0.0, 0.0);
            pm0[s] = split_f64(a.x);
            pm1[s] = split_f64(a.y);
            pc0[s] = split_f64(b.x);
            pc1[s] = split_f64(b.y);
            if (ld) *reinterpret_cast<float4*>(pbuf + s * lpv + obuf) = make_float4(pc0[s].x, pc0[s].y, pc1[s].x, pc1[s].y);
            if (halo) {
                const double2 hv = __ldg(reinterpret_cast<const double2*>(h0 + s * npts));
                const float2 u = split_f64(hv.x), v = split_f64(hv.y);
                *reinterpret_cast<float4*>(pbuf + s * lpv + hbuf) = make_float4(u.x, u.y, v.x, v.y);
            }
        }
    }
    __syncthreads();
    float* Fo = F + ((long long)k0 * n2 + (own ? jr : 0)) * n1q + i;
    const long long fstep = (long long)n2 * n1q;
    const bool hm0 = i > 0, hp1 = i + 1 < n1 - 1;
    for (int k = k0; k < kend; ++k, Fo += fstep) {
        const int b = (k - k0) & 1;
        const float2* Bc = pbuf + b * S * lpv + obuf;
        float2* Bn = pbuf + (b ^ 1) * S * lpv;
        cp_async_wait<kMarchAhead - 1>();            // plane k + 1 landed (this thread's copies)
        const double* R = ring + (size_t)((k + 1) & (kMarchAhead - 1)) * S * rs + 2 * t;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const double2 v = ld ? *reinterpret_cast<const double2*>(R + s * rs) : make_double2(0.0, 0.0);
            pn0[s] = split_f64(v.x);
            pn1[s] = split_f64(v.y);
        }
        if (own) {
            const float rs3 = __ldg(tb.ax[2].rs + k), lo3 = __ldg(tb.ax[2].lower + k), up3 = __ldg(tb.ax[2].upper + k);
            const float dp3 = (GEO == GEO_BALL) ? __ldg(tb.Dp + k) : 1.f;
            cf0.rs3 = cf1.rs3 = rs3;
            cf0.lo3 = cf1.lo3 = lo3;
            cf0.up3 = cf1.up3 = up3;
            cf0.dp3 = cf1.dp3 = dp3;
            float w0[kMaxSpecies], w1[kMaxSpecies], g0[S], g1[S];
#pragma unroll
            for (int r = 0; r < kMaxSpecies; ++r) w0[r] = w1[r] = 0.f;
#pragma unroll
            for (int r = 0; r < S; ++r) {
                w0[r] = pc0[r].x + pc0[r].y;
                w1[r] = pc1[r].x + pc1[r].y;
            }
            reactions<float, S, RK>(tb.reac, w0, g0);
            reactions<float, S, RK>(tb.reac, w1, g1);
            const bool hkm = k > 0, hkp = k < n3 - 1;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                // every neighbour lies inside the buffer (lines 0 .. TJ + 1); the flags drop the absent ones
                const float2* q = Bc + s * lpv;
                const float4 jm = *reinterpret_cast<const float4*>(q - n1);
                const float4 jp = *reinterpret_cast<const float4*>(q + n1);
                const float2 m0 = q[-1], p1 = q[2];
                const float f0 = point_F<GEO>(tb, s, g0[s], pc0[s], m0, pc1[s], make_float2(jm.x, jm.y),
                                              make_float2(jp.x, jp.y), pm0[s], pn0[s], hm0, true, true, true, hkm, hkp,
                                              cf0, 1.f);
                const float f1 = point_F<GEO>(tb, s, g1[s], pc1[s], pc0[s], p1, make_float2(jm.z, jm.w),
                                              make_float2(jp.z, jp.w), pm1[s], pn1[s], true, hp1, true, true, hkm, hkp,
                                              cf1, 1.f);
                *reinterpret_cast<float2*>(Fo + s * ys) = make_float2(f0, f1);
            }
        }
        if (k + 1 < kend) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                if (ld)
                    *reinterpret_cast<float4*>(Bn + s * lpv + obuf) = make_float4(pn0[s].x, pn0[s].y, pn1[s].x, pn1[s].y);
                if (halo) {
                    const double2 hv = *reinterpret_cast<const double2*>(R + s * rs + 2 * blockDim.x);
                    const float2 u = split_f64(hv.x), v = split_f64(hv.y);
                    *reinterpret_cast<float4*>(Bn + s * lpv + hbuf) = make_float4(u.x, u.y, v.x, v.y);
                }
            }
        }
        __syncthreads();
        fetch();
#pragma unroll
        for (int s = 0; s < S; ++s) {
            pm0[s] = pc0[s];
            pc0[s] = pn0[s];
            pm1[s] = pc1[s];
            pc1[s] = pn1[s];
        }
    }
    cp_async_wait<0>();
}

// ------------------------------------------------------------------------------
// mode-3 pass: rows = 128 consecutive points of the padded (i, j) plane
// (row index j * n1q + i), columns = the k fibre; reads F from Y and overwrites
// the same entries with the result.  Each producer thread loads the eight F
// values (and, for the ball, Phi values) of its row and columns two chunks
// ahead of use.
template <int GEO>
__global__ void __launch_bounds__(kBlock, 1)
    k_tc_mode3(SplitTables T, TcShape sh) {
    extern __shared__ char smem_raw[];
    const uint32_t tmem_cols = sh.tmem_cols;
    CtaRes R = cta_begin(smem_raw, sh, T.err);
    const int s = blockIdx.y;
    const int n3 = T.n3, n1q = T.n1q;
    const int n3p = (n3 + 15) & ~15;
    const long long plane = (long long)T.n2 * n1q;          // floats per k-plane of Y
    const long long row0 = (long long)blockIdx.x * kRows;
    const int tile_rows = (int)(plane - row0 < kRows ? plane - row0 : kRows);
    float* Ys = T.Y + (long long)s * T.ys;
    GemmSpec gs[2] = {{GEO == GEO_BALL ? T.M3a : T.M3b[s], 0, kRows, 1, n3p, n3p / kKC, R.tmem},
                      {T.M3b[0], 0, kRows, 1, n3p, n3p / kKC, R.tmem + (uint32_t)n3p}};
    if (threadIdx.x >= kThreads + 32) {
        pdl_trigger();
        mma_issuer<GEO == GEO_BALL ? 2 : 1>(R.P, gs);
    } else if (threadIdx.x >= kThreads) {
        pdl_trigger();
        tma_issuer<GEO == GEO_BALL ? 2 : 1>(R.P, gs);     // constant matrices only
    } else {
        pdl_wait();      // F from the stencil pass
        pdl_trigger();
        const int tid = threadIdx.x;
        const int r = tid & (kRows - 1), h = tid >> 7;
        const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
        const bool valid = r < tile_rows;
        const int i = (int)((row0 + r) % n1q);
        float* Yr = Ys + row0 + r;
        const float* hp = T.had_phi + (long long)s * n3 * n1q + i;     // ball only
        auto load_h = [&](int c, Pre8& p) { load8_strided(p, hp, n1q, c * 16 + h * 8, n3, valid); };
        Pre8 hpre[2] = {};                   // the ball's G2: first two chunks of Hadamard factors
        auto g1_tail = [&] {
            if constexpr (GEO == GEO_BALL) {
                load_h(0, hpre[0]);
                if (gs[1].k_chunks > 1) load_h(1, hpre[1]);
            }
        };
        run_gemm(
            R.P, gs[0],
            [&](int c, Pre8& p) { load8_strided(p, Yr, (int)plane, c * 16 + h * 8, n3, valid); },
            [&](int, char* hi, char* lo, const Pre8& p) { store_row8(hi, lo, r, h, p.v); }, g1_tail);
        uint32_t last = 0;
        if constexpr (GEO == GEO_BALL) {
            run_gemm<true>(
                R.P, gs[1], load_h,
                [&](int c, char* hi, char* lo, const Pre8& p) {
                    float v[8];
                    tmem_ld8(R.tmem + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] *= p.v[q];
                    store_row8(hi, lo, r, h, v);
                },
                NoTail{}, hpre);
            last = (uint32_t)n3p;
        }
        for (int c = 0; c < n3p / 16; ++c) {
            float v[8];
            tmem_ld8(R.tmem + lane_base + last + (uint32_t)(c * 16 + h * 8), v);
            const int k0 = c * 16 + h * 8;
            float* o = Yr + (long long)k0 * plane;
            if (valid && k0 + 8 <= n3) {
#pragma unroll
                for (int q = 0; q < 8; ++q) o[q * (int)plane] = v[q];
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (valid && k0 + q < n3) o[q * (int)plane] = v[q];
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
    gs[0] = GemmSpec{J.QT, 0, kRows, 1, n2p, n2p / kKC, tmem + cols[0]};
    gs[1] = GemmSpec{J.Q, 1, n1p, m2, n1p, n2p / kKC, tmem + cols[1]};
    gs[2] = GemmSpec{J.P, 0, kRows * m2, m2, n1p, n1p / kKC, tmem + cols[2]};
}

// Update of up to 128 state rows from an FP32 accumulator in tensor memory:
// W[row * stride + i] = Win[...] + tau * D[row][i] for row < rows, i < n1, with D
// at tensor-memory columns [dcol, dcol + n1p) of lane `row`.  The accumulator is
// staged through shared memory (`epi`, 128 (n1p + 1) floats) so the FP64
// read-modify-write is coalesced; the increment is rounded to FP32 and widened
// exactly by integer operations: one FP64 add per point, kUpdBatch independent
// read-modify-writes in flight per thread.  Called by the 256 producer threads.
constexpr int kUpdBatch = 16;   // FP64 read-modify-writes in flight per thread in update_rows

// The first batch of state values update_rows reads (same rows, n1, stride), loaded ahead of it.
__device__ __forceinline__ void update_prefetch(double (&w)[kUpdBatch], int rows, int n1, const double* Win,
                                                int stride = 0) {
    if (stride == 0) stride = n1;
    const int count = rows * n1;
    const uint32_t m_n1 = div_magic((uint32_t)n1);
#pragma unroll
    for (int u = 0; u < kUpdBatch; ++u) {
        const int f = (int)threadIdx.x + u * kThreads;
        const int jl = div_by(f, m_n1);
        w[u] = f < count ? Win[jl * stride + (f - jl * n1)] : 0.0;
    }
}

// With PRE the first batch comes from `wpre` (update_prefetch with the same arguments).
template <bool PRE = false>
__device__ __forceinline__ void update_rows(uint32_t dcol, int rows, int n1, int n1p, const double* Win,
                                            double* W, float tau_f, char* epi, int stride = 0,
                                            const double* wpre = nullptr) {
    if (stride == 0) stride = n1;
    const int tid = threadIdx.x;
    const int r = tid & (kRows - 1), h = tid >> 7;
    const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
    float* E = reinterpret_cast<float*>(epi);
    const int pitch = n1p + 1;
    for (int c = 0; c < n1p / 16; ++c) {
        float v[8];
        tmem_ld8(dcol + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
        for (int q = 0; q < 8; ++q) E[r * pitch + c * 16 + h * 8 + q] = v[q];
    }
    compute_sync();
    const int count = rows * n1;
    const uint32_t m_n1 = div_magic((uint32_t)n1);
    for (int f0 = tid; f0 < count; f0 += kThreads * kUpdBatch) {
        double w[kUpdBatch];
        if (PRE && f0 == tid) {
#pragma unroll
            for (int u = 0; u < kUpdBatch; ++u) w[u] = wpre[u];
        } else {
#pragma unroll
            for (int u = 0; u < kUpdBatch; ++u) {
                const int f = f0 + u * kThreads;
                const int jl = div_by(f, m_n1);
                w[u] = f < count ? Win[jl * stride + (f - jl * n1)] : 0.0;     // offsets < 2^31
            }
        }
#pragma unroll
        for (int u = 0; u < kUpdBatch; ++u) {
            const int f = f0 + u * kThreads;
            if (f < count) {
                const int jl = div_by(f, m_n1), i = f - jl * n1;
                W[jl * stride + i] = w[u] + f32_to_f64(tau_f * E[jl * pitch + i]);
            }
        }
    }
    compute_sync();
}

// COMP: also form the theta-mean coefficient X[i][0] by compensated summation (see below).
template <bool COMP>
__device__ __forceinline__ void slab_compute(const SlabJob& J, const GemmSpec* gs, const uint32_t* cols, Pipe& P,
                                             uint32_t tmem, char* epi) {
    const int tid = threadIdx.x;
    const int r = tid & (kRows - 1), h = tid >> 7;
    const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
    const int n1 = J.n1, n2 = J.n2;
    const int n1p = (n1 + 15) & ~15, m2 = (n2 + 127) / 128;
    const uint32_t c1 = cols[0], c2 = cols[1], c3 = cols[2];

    // G1: X[i][j'] = sum_j Y[i][j] Q[j][j']          (Y x_2 Q_theta^T), rows i
    const int n1q = J.n1q;
    // eight values of row r, columns 16c + 8h + q, of a [j][n1q] table, 0 outside the slab
    auto load_rows = [&](const float* base) {
        return [=](int c, Pre8& p) { load8_strided(p, base + r, n1q, c * 16 + h * 8, n2, r < n1); };
    };
    // The theta-mean coefficient X[i][0] = (1/sqrt(n2)) sum_j Y[i][j] (Q's first column is the
    // constant vector) is also summed by the producers with compensation (Neumaier's variant of
    // Kahan summation): near the axis Y is dominated by the theta-Laplacian, values ~1e4 whose
    // theta-mean is ~0, and the tensor cores' truncating FP32 accumulation of that cancelling sum
    // leaves a coherent bias in the one coefficient that no Phi damps (Phi_0 = 1).
    // The compensation costs ~4% of the slab on the 100^3 ball and is compiled in where the setup
    // enables it (SplitTables::theta_comp: disks and the grids of coupled plans).
    float rs_s = 0.f, rs_c = 0.f;
    const auto load_had = load_rows(J.had);
    Pre8 hpre[2] = {};                       // G2's first two chunks of Hadamard factors
    auto g1_tail = [&] {
        load_had(0, hpre[0]);
        if (gs[1].k_chunks > 1) load_had(1, hpre[1]);
    };
    run_gemm(P, gs[0], load_rows(J.Y), [&](int, char* hi, char* lo, const Pre8& p) {
        store_row8(hi, lo, r, h, p.v);
        if constexpr (COMP) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float t = rs_s + p.v[q];
                rs_c += fabsf(rs_s) >= fabsf(p.v[q]) ? (rs_s - t) + p.v[q] : (p.v[q] - t) + rs_s;
                rs_s = t;
            }
        }
    }, g1_tail);
    // the two halves of a row meet in the data slot of G1's last chunk (free once G1 completed;
    // the next chunk to reuse it comes nd - 1 chunks into G2, after the second barrier)
    float x0 = 0.f;
    if constexpr (COMP) {
        const uint32_t last = P.sd == 0 ? P.nd - 1 : P.sd - 1;
        float2* xch = reinterpret_cast<float2*>(P.data_slots + (size_t)last * P.data_bytes);
        if (h == 1) xch[r] = make_float2(rs_s, rs_c);
        compute_sync();
        if (h == 0) {
            const float2 o = xch[r];
            const float t = rs_s + o.x;
            const float c = (fabsf(rs_s) >= fabsf(o.x) ? (rs_s - t) + o.x : (o.x - t) + rs_s) + (rs_c + o.y);
            x0 = (float)((double)(t + c) / sqrt((double)n2));
        }
        compute_sync();
    }
    // G2: Z^T[j][i] = sum_j' Q[j][j'] (Phi o X)[i][j']   (x_2 Q_theta), data in B, rows j
    run_gemm<true>(P, gs[1], load_had, [&](int c, char* hi, char* lo, const Pre8& p) {
        float v[8];
        tmem_ld8(tmem + lane_base + c1 + (uint32_t)(c * 16 + h * 8), v);
        if (COMP && c == 0 && h == 0) v[0] = x0;        // the compensated theta-mean coefficient
        if (r < n1p) {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] *= p.v[q];
            store_row8(hi, lo, r, h, v);
        }
    }, NoTail{}, hpre);
    // G3: R^T[j][i'] = sum_i Z^T[j][i] P[i'][i]      (x_1 phi_1(tau d A_rho)), rows j
    double wpre[kUpdBatch];                 // the update's first state values, read during G3's last wait
    auto g3_tail = [&] { update_prefetch(wpre, min(kRows, n2), n1, J.Win); };
    run_gemm(P, gs[2], [](int, Pre8&) {}, [&](int c, char* hi, char* lo, const Pre8&) {
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
    }, g3_tail);
    // w[k][j][i'] += tau R^T[j][i']
    update_rows<true>(tmem + c3, min(kRows, n2), n1, n1p, J.Win, J.W, J.tau_f, epi, 0, wpre);
    for (int mt = 1; mt < m2; ++mt)
        update_rows(tmem + c3 + (uint32_t)(mt * n1p), min(kRows, n2 - mt * kRows), n1, n1p,
                    J.Win + (long long)mt * kRows * n1, J.W + (long long)mt * kRows * n1, J.tau_f, epi);
}

template <bool COMP>
__global__ void __launch_bounds__(kBlock, 2)
    k_tc_slab(SplitTables T, TcShape sh) {
    extern __shared__ char smem_raw[];
    const uint32_t tmem_cols = sh.tmem_cols;
    CtaRes R = cta_begin(smem_raw, sh, T.err);
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
    if (threadIdx.x >= kThreads + 32) {
        pdl_trigger();
        mma_issuer<3>(R.P, gs);
    } else if (threadIdx.x >= kThreads) {
        pdl_trigger();
        tma_issuer<3>(R.P, gs);             // constant matrices only
    } else {
        pdl_wait();                         // Y from the earlier directions
        pdl_trigger();
        slab_compute<COMP>(J, gs, cols, R.P, R.tmem, R.P.mat_slots);
    }
    cta_end(R, tmem_cols);
}

// ------------------------------------------------------------------------------
// Sphere (eq. ee_sphere; mode 1 = theta, contiguous; mode 2 = phi).
//
// phi direction (plain): Y2[s][j'][i] = sum_j phi_1(tau d_s A_phi)[j'][j] Y[s][j][i].
// CTA = 128 consecutive theta points (rows) x phi_nt output phi rows (the B
// operand's N-tile blockIdx.y) of species blockIdx.z; K runs over all phi.
// With phi_ks > 1 the K range (phi) of each output tile is split over a cluster of phi_ks CTAs
// (consecutive blockIdx.z = z phi_ks + cluster rank): each accumulates its 1/phi_ks of the
// K-chunks and stages its partial product in its shared memory; after a cluster barrier each CTA
// adds the phi_ks partials of its share of the output columns, in rank order (a fixed order), from
// the cluster's shared memory, and a second cluster barrier keeps every partial in place until the
// peers have read it.
__global__ void __launch_bounds__(kBlock, 1) k_tc_sphere_phi(SplitTables T, TcShape sh) {
    extern __shared__ char smem_raw[];
    const uint32_t tmem_cols = sh.tmem_cols;
    CtaRes R = cta_begin(smem_raw, sh, T.err);
    const int ks = T.phi_ks > 1 ? T.phi_ks : 1;
    const int kz = ks > 1 ? (int)cluster_ctarank() : 0, zz = (int)blockIdx.z / ks;
    const bool second = zz >= T.S;                         // phi_pair: the second image set into Y3
    const int s = second ? zz - T.S : zz, nt = blockIdx.y;
    const int n1 = T.n1, n2 = T.n2, n1q = T.n1q, NT = T.phi_nt;
    const int i0 = blockIdx.x * kRows;
    Image mat = second ? T.Pphi2[s] : T.Pphi[s];
    const int kc = mat.k_chunks / ks, kc0 = kz * kc;       // this CTA's K-chunks
    mat.ptr += (long long)nt * mat.k_chunks * mat.chunk_floats + (long long)kc0 * mat.chunk_floats;
    GemmSpec gs[1] = {{mat, 0, kRows, 1, NT, kc, R.tmem}};
    if (threadIdx.x >= kThreads + 32) {
        pdl_trigger();
        mma_issuer<1>(R.P, gs);
    } else if (threadIdx.x >= kThreads) {
        pdl_trigger();
        tma_issuer<1>(R.P, gs);
    } else {
        pdl_wait();
        pdl_trigger();
        const int tid = threadIdx.x;
        const int r = tid & (kRows - 1), h = tid >> 7;
        const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
        const int i = i0 + r;
        const bool valid = i < n1;
        const float* Yi = T.Y + (long long)s * T.ys + i;
        run_gemm(
            R.P, gs[0],
            [&](int c, Pre8& p) { load8_strided(p, Yi, n1q, (kc0 + c) * 16 + h * 8, n2, valid); },
            [&](int, char* hi, char* lo, const Pre8& p) { store_row8(hi, lo, r, h, p.v); });
        if (ks == 1) {
            float* Yo = (second ? T.Y3 : T.Y2) + (long long)s * T.ys + i;
            for (int c = 0; c < NT / 16; ++c) {
                float v[8];
                tmem_ld8(R.tmem + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = nt * NT + c * 16 + h * 8 + q;
                    if (valid && j < n2) Yo[(long long)j * n1q] = v[q];
                }
            }
        } else {
            // the partial product, [column][row], in the rings (free: the product completed)
            float* Pm = reinterpret_cast<float*>(R.P.mat_slots);
            for (int c = 0; c < NT / 16; ++c) {
                float v[8];
                tmem_ld8(R.tmem + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
                for (int q = 0; q < 8; ++q) Pm[(c * 16 + h * 8 + q) * kRows + r] = v[q];
            }
        }
    }
    if (ks > 1) {
        __syncwarp();
        cluster_sync_all();                              // every CTA's partial is staged
        if (threadIdx.x < kThreads) {
            const int r = threadIdx.x & (kRows - 1), g = threadIdx.x >> 7;
            const int cw = NT / ks;                      // this CTA's output columns: [kz cw, (kz + 1) cw)
            const uint32_t base = smem_u32(R.P.mat_slots);
            const int i = i0 + r;
            float* Yo = (second ? T.Y3 : T.Y2) + (long long)s * T.ys + i;
            for (int cc = g; cc < cw; cc += 2) {
                const int col = kz * cw + cc;
                const uint32_t off = base + (uint32_t)(col * kRows + r) * 4u;
                float acc = ld_dsmem(dsmem_addr(off, 0));
                for (int k = 1; k < ks; ++k) acc += ld_dsmem(dsmem_addr(off, (uint32_t)k));
                const int j = nt * NT + col;
                if (i < n1 && j < n2) Yo[(long long)j * n1q] = acc;
            }
        }
        __syncwarp();
        cluster_sync_all();                              // the peers have read this CTA's partial
    }
    cta_end(R, tmem_cols);
}

// theta direction (scaled) + update: rows = 128 phi rows j of species blockIdx.y,
// output theta columns [z th_nt, (z + 1) th_nt) with z = blockIdx.z.
// G1: X = Y2 x_1 Q_theta^T (all theta', the K of G2), Hadamard Phi(j, theta'),
// G2: x_1 Q_theta for this column group, then w[s][j][i] += tau * result.
// Splitting the columns over CTAs repeats G1 in each but multiplies the CTAs of
// a grid of only (n_phi / 128) x species row tiles.  Accumulators: G1 at
// [0, n1p), G2 at [n1p, n1p + th_nt).
__global__ void __launch_bounds__(kBlock, 1) k_tc_sphere_theta(SplitTables T, TcShape sh) {
    extern __shared__ char smem_raw[];
    const uint32_t tmem_cols = sh.tmem_cols;
    CtaRes R = cta_begin(smem_raw, sh, T.err);
    const int s = blockIdx.y, z = blockIdx.z;
    const int n1 = T.n1, n2 = T.n2, n1q = T.n1q, NT = T.th_nt;
    const int n1p = (n1 + 15) & ~15;
    const int j0 = blockIdx.x * kRows;
    Image qz = T.Qsph;
    qz.ptr += (long long)z * qz.k_chunks * qz.chunk_floats;
    GemmSpec gs[2] = {{T.QT, 0, kRows, 1, n1p, n1p / kKC, R.tmem},
                      {qz, 0, kRows, 1, NT, n1p / kKC, R.tmem + (uint32_t)n1p}};
    if (threadIdx.x >= kThreads + 32) {
        pdl_trigger();
        mma_issuer<2>(R.P, gs);
    } else if (threadIdx.x >= kThreads) {
        pdl_trigger();
        tma_issuer<2>(R.P, gs);
    } else {
        pdl_wait();
        pdl_trigger();
        const int tid = threadIdx.x;
        const int r = tid & (kRows - 1), h = tid >> 7;
        const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
        const int j = j0 + r;
        const bool valid = j < n2;
        // eight consecutive theta values of row j (16-byte aligned: n1q and 8-column groups)
        auto load_row8 = [&](const float* row) {
            return [=](int c, Pre8& p) {
                const int i = c * 16 + h * 8;
                if (valid && i + 8 <= n1q) {
                    const float4 a = __ldg(reinterpret_cast<const float4*>(row + i));
                    const float4 b = __ldg(reinterpret_cast<const float4*>(row + i + 4));
                    p.v[0] = a.x; p.v[1] = a.y; p.v[2] = a.z; p.v[3] = a.w;
                    p.v[4] = b.x; p.v[5] = b.y; p.v[6] = b.z; p.v[7] = b.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) p.v[q] = (valid && i + q < n1q) ? __ldg(row + i + q) : 0.f;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (i + q >= n1) p.v[q] = 0.f;
            };
        };
        const long long roff = (long long)s * T.ys + (long long)(valid ? j : 0) * n1q;
        const auto load_had = load_row8(T.had_sph + roff);
        Pre8 hpre[2] = {};                   // G2's first two chunks of Hadamard factors, read during G1's last wait
        auto g1_tail = [&] {
            load_had(0, hpre[0]);
            if (gs[1].k_chunks > 1) load_had(1, hpre[1]);
        };
        run_gemm(R.P, gs[0], load_row8(T.Y2 + roff),
                 [&](int, char* hi, char* lo, const Pre8& p) { store_row8(hi, lo, r, h, p.v); }, g1_tail);
        const long long n12 = (long long)n1 * n2;
        const int i0 = z * NT;
        double* W = T.state_upd + (long long)s * n12 + (long long)j0 * n1 + i0;
        const int rows = min(kRows, n2 - j0), cols = min(NT, n1 - i0);
        double wpre[kUpdBatch];              // the update's first state values, read during G2's last wait
        auto g2_tail = [&] { update_prefetch(wpre, rows, cols, W, n1); };
        run_gemm<true>(R.P, gs[1], load_had, [&](int c, char* hi, char* lo, const Pre8& p) {
            float v[8];
            tmem_ld8(R.tmem + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] *= p.v[q];
            store_row8(hi, lo, r, h, v);
        }, g2_tail, hpre);
        update_rows<true>(R.tmem + (uint32_t)n1p, rows, cols, NT, W, W, T.tau, R.P.mat_slots, n1, wpre);
    }
    cta_end(R, tmem_cols);
}

// Adjoint theta step of the split sphere (the transposed eq. ee_sphere): rows = 128 phi rows j of
// species blockIdx.y, output theta columns [z th_nt, (z + 1) th_nt).  G1: X = lambda x_1 Q_theta^T
// (lambda rounded to FP32, chain layout); G2a: Za = (Phi o X) x_1 Q_theta and G2b: Zb =
// (dPhi/dd o X) x_1 Q_theta for the group's columns.  Epilogue: tau Za (= tau P_theta lambda, P_theta
// symmetric) into A.tpl, and <tau Zb, Y2> + <tau Za, Y3> into A.acc_d[s].  Accumulators: G1 at
// [0, n1p), G2a at [n1p, n1p + th_nt), G2b after it.
__global__ void __launch_bounds__(kBlock, 1) k_tc_sphere_theta_adj(SplitTables T, TcShape sh, SphereAdjArgs A) {
    extern __shared__ char smem_raw[];
    __shared__ double red[kThreads / 32];
    const uint32_t tmem_cols = sh.tmem_cols;
    CtaRes R = cta_begin(smem_raw, sh, T.err);
    const int s = blockIdx.y, z = blockIdx.z;
    const int n1 = T.n1, n2 = T.n2, n1q = T.n1q, NT = T.th_nt;
    const int n1p = (n1 + 15) & ~15;
    const int j0 = blockIdx.x * kRows;
    Image qz = T.Qsph;
    qz.ptr += (long long)z * qz.k_chunks * qz.chunk_floats;
    GemmSpec gs[3] = {{T.QT, 0, kRows, 1, n1p, n1p / kKC, R.tmem},
                      {qz, 0, kRows, 1, NT, n1p / kKC, R.tmem + (uint32_t)n1p},
                      {qz, 0, kRows, 1, NT, n1p / kKC, R.tmem + (uint32_t)(n1p + NT)}};
    if (threadIdx.x >= kThreads + 32) {
        pdl_trigger();
        mma_issuer<3>(R.P, gs);
    } else if (threadIdx.x >= kThreads) {
        pdl_trigger();
        tma_issuer<3>(R.P, gs);
    } else {
        pdl_wait();
        pdl_trigger();
        const int tid = threadIdx.x;
        const int r = tid & (kRows - 1), h = tid >> 7;
        const uint32_t lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
        const int j = j0 + r;
        const bool valid = j < n2;
        const long long roff = (long long)s * T.ys + (long long)(valid ? j : 0) * n1q;
        // lambda rounded to FP32 in the chain layout: eight consecutive theta values of row j in two
        // 16-byte loads (n1q and the 8-column groups keep them aligned)
        const float* lrow = A.lam32 + roff;
        auto load_had = [&](const float* row) {
            return [=](int c, Pre8& p) {
                const int i = c * 16 + h * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) p.v[q] = (valid && i + q < n1) ? __ldg(row + i + q) : 0.f;
            };
        };
        const auto load_had1 = load_had(T.had_sph + roff), load_had2 = load_had(A.had_d + roff);
        // each product's first two chunks of Hadamard factors, read during the previous product's last wait
        Pre8 hpre1[2] = {}, hpre2[2] = {};
        auto g1_tail = [&] {
            load_had1(0, hpre1[0]);
            if (gs[1].k_chunks > 1) load_had1(1, hpre1[1]);
        };
        auto g2_tail = [&] {
            load_had2(0, hpre2[0]);
            if (gs[2].k_chunks > 1) load_had2(1, hpre2[1]);
        };
        run_gemm(
            R.P, gs[0],
            [&](int c, Pre8& p) {
                const int i = c * 16 + h * 8;
                if (valid && i + 8 <= n1q) {
                    const float4 a = __ldg(reinterpret_cast<const float4*>(lrow + i));
                    const float4 b = __ldg(reinterpret_cast<const float4*>(lrow + i + 4));
                    p.v[0] = a.x; p.v[1] = a.y; p.v[2] = a.z; p.v[3] = a.w;
                    p.v[4] = b.x; p.v[5] = b.y; p.v[6] = b.z; p.v[7] = b.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) p.v[q] = (valid && i + q < n1q) ? __ldg(lrow + i + q) : 0.f;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (i + q >= n1) p.v[q] = 0.f;
            },
            [&](int, char* hi, char* lo, const Pre8& p) { store_row8(hi, lo, r, h, p.v); }, g1_tail);
        auto hadamard = [&](int c, char* hi, char* lo, const Pre8& p) {
            float v[8];
            tmem_ld8(R.tmem + lane_base + (uint32_t)(c * 16 + h * 8), v);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] *= p.v[q];
            store_row8(hi, lo, r, h, v);
        };
        run_gemm<true>(R.P, gs[1], load_had1, hadamard, g2_tail, hpre1);
        run_gemm<true>(R.P, gs[2], load_had2, hadamard, NoTail{}, hpre2);
        const int i0 = z * NT;
        double dot = 0.0;
        for (int c = 0; c < NT / 16; ++c) {
            float va[8], vb[8];
            tmem_ld8(R.tmem + lane_base + (uint32_t)(n1p + c * 16 + h * 8), va);
            tmem_ld8(R.tmem + lane_base + (uint32_t)(n1p + NT + c * 16 + h * 8), vb);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = i0 + c * 16 + h * 8 + q;
                if (valid && i < n1) {
                    const float ta = T.tau * va[q], tb = T.tau * vb[q];
                    A.tpl[roff + i] = ta;
                    dot += (double)tb * (double)__ldg(A.Y2 + roff + i) + (double)ta * (double)__ldg(A.Y3 + roff + i);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if ((tid & 31) == 0) red[tid >> 5] = dot;
        compute_sync();
        if (tid == 0) {
            double t = 0.0;
            for (int w8 = 0; w8 < kThreads / 32; ++w8) t += red[w8];
            atomicAdd(A.acc_d + s, t);
        }
    }
    cta_end(R, tmem_cols);
}

// ------------------------------------------------------------------------------
// Batched disks: one persistent CTA per SM, launched cooperatively (all CTAs
// resident).  Phase 1: the CTAs take (instance, 16 theta-lines) tiles from a
// work list and evaluate F = d M w + g(w) of both species (eq. disk_discr, the
// Schnakenberg or other reaction) into an FP32 buffer, each FP64 value split
// once into an FP32 pair in shared memory.  A grid-wide barrier (bounded wait)
// separates the phases.  Phase 2: the CTAs take (instance, species) items from
// the LPT-ordered work list and run the disk chain of eq. ee_disk on F --
// x_2 Q_theta^T, Hadamard, x_2 Q_theta, x_1 phi_1(tau d A_rho) -- writing the
// updated species into the other state buffer.
// Phase-1 tiles are tj theta-lines of one instance (tj measured at setup: BatchTables.tj), both
// species, with a one-line halo in theta: values [s][jj][i], jj = 0 .. lines + 1 for the lines
// j0 - 1 .. j0 + lines (periodic), as split pairs.  A tile's raw FP64 values arrive by
// asynchronous copies (batch_tile_issue) while the CTA computes the previous tile, are split in
// place (batch_tile_convert) and then used (batch_tile_compute).
struct FTileGeom {
    int n1, n2, lines, per_sp, items;
};
__device__ __forceinline__ FTileGeom ftile_geom(const BatchInstance& I, int j0, int tj) {
    FTileGeom g;
    g.n1 = I.n1;
    g.n2 = I.n2;
    g.lines = min(tj, g.n2 - j0);
    g.per_sp = (g.lines + 2) * g.n1;                    // lines j0 - 1 .. j0 + lines: one wrap at most
    g.items = 2 * g.per_sp;
    return g;
}

__device__ __forceinline__ void batch_tile_issue(const BatchInstance& I, const double* Win, int j0, int tj,
                                                 double* raw) {
    const FTileGeom g = ftile_geom(I, j0, tj);
    const long long n12 = (long long)g.n1 * g.n2;
    const uint32_t m_n1 = div_magic((uint32_t)g.n1);
    for (int q = threadIdx.x; q < g.items; q += kBlock) {
        const int sp = q >= g.per_sp;
        const int qq = q - sp * g.per_sp;
        const int jj = div_by(qq, m_n1), i = qq - jj * g.n1;
        int j = j0 - 1 + jj;
        j = j < 0 ? j + g.n2 : (j >= g.n2 ? j - g.n2 : j);   // theta is periodic
        cp_async8(smem_u32(raw + q), Win + sp * n12 + (long long)j * g.n1 + i);
    }
    cp_async_commit();
}

// Each thread splits the values it copied (its own copies are complete after cp_async_wait).
__device__ __forceinline__ void batch_tile_convert(const BatchInstance& I, int j0, int tj, float2* tile) {
    const FTileGeom g = ftile_geom(I, j0, tj);
    const double* raw = reinterpret_cast<const double*>(tile);
    for (int q = threadIdx.x; q < g.items; q += kBlock) {
        const double v = raw[q];
        tile[q] = split_f64(v);
    }
}

__device__ __forceinline__ void batch_tile_compute(const BatchInstance& I, float* Fout, int j0, int tj,
                                                   const float2* tile) {
    const FTileGeom g = ftile_geom(I, j0, tj);
    const int n1 = g.n1, n2 = g.n2, n1q = (n1 + 3) & ~3, per_sp = g.per_sp;
    const uint32_t m_n1 = div_magic((uint32_t)n1);
    const int total = g.lines * n1;
    for (int q = threadIdx.x; q < total; q += kBlock) {
        const int jl = div_by(q, m_n1), i = q - jl * n1;
        const int j = j0 + jl;
        const float lo1 = __ldg(I.ax_rho.lower + i), up1 = __ldg(I.ax_rho.upper + i), rs1 = __ldg(I.ax_rho.rs + i);
        const float dr = __ldg(I.Dr + i);
        const float rs2 = __ldg(I.ax_theta.rs + j), lo2 = __ldg(I.ax_theta.lower + j), up2 = __ldg(I.ax_theta.upper + j);
        const int c0 = (jl + 1) * n1 + i;
        float w[kMaxSpecies] = {0.f, 0.f, 0.f, 0.f};
        w[0] = tile[c0].x + tile[c0].y;
        w[1] = tile[per_sp + c0].x + tile[per_sp + c0].y;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float2* pc = tile + s * per_sp + c0;
            const float2 c = pc[0];
            float t0 = rs1 * (c.x + c.y);
            if (i > 0) t0 += lo1 * sdiff(pc[-1], c);
            if (i < n1 - 1) t0 += up1 * sdiff(pc[1], c);
            const float t1 = rs2 * (c.x + c.y) + lo2 * sdiff(pc[-n1], c) + up2 * sdiff(pc[n1], c);
            Fout[(long long)s * n2 * n1q + (long long)j * n1q + i] = I.d[s] * (t0 + dr * t1) + reaction<float>(I.reac, w, s);
        }
    }
    __syncthreads();
}

// Grid-wide barrier of a cooperative launch, bounded: after ~2 s the waiting
// thread records a timeout and the CTA goes on (the results are then invalid
// and sexpe_synchronize reports SEXPE_ETIMEOUT).
__device__ __forceinline__ void grid_barrier(int* bar, int nblocks, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1);
        const long long t0 = clock64();
        for (long long it = 0; it < (1LL << 32); ++it) {
            if (*reinterpret_cast<volatile int*>(bar) >= nblocks) break;
            if (clock64() - t0 > 4000000000LL) {
                atomicCAS(err, 0, DERR_TIMEOUT_MMA);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBlock, 1) k_tc_batch(BatchTables B, TcShape sh) {
    extern __shared__ char smem_raw[];
    __shared__ int s_item;
    const uint32_t tmem_cols = sh.tmem_cols;
    CtaRes R = cta_begin(smem_raw, sh, B.err);
    // phase 1: F of every instance, two tiles in flight: while the CTA computes one tile, the raw
    // values of the next arrive by asynchronous copies into the other buffer.  Each tile's instance
    // record is copied to shared memory once: read through a global reference, its fields (sizes,
    // table pointers, reaction parameters) are reloaded after every store of the tile loops, which
    // may alias it.
    float2* tbuf0 = reinterpret_cast<float2*>(R.P.mat_slots);
    float2* tbuf1 = tbuf0 + B.tile_f2;
    __shared__ __align__(16) BatchInstance s_inst[2];
    __shared__ int2 s_tile[2];
    constexpr int kInstWords = (int)(sizeof(BatchInstance) / sizeof(int));
    static_assert(sizeof(BatchInstance) % sizeof(int) == 0, "instance record copied as words");
    // claims the next tile into slot b (false when none is left); uniform across the CTA
    auto fetch = [&](int b) -> bool {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(B.counter + 2, 1);
            s_tile[b] = it < B.n_ftiles ? B.ftiles[it] : make_int2(-1, 0);
        }
        __syncthreads();
        if (s_tile[b].x < 0) return false;
        const int* src = reinterpret_cast<const int*>(B.inst + s_tile[b].x);
        for (int q = threadIdx.x; q < kInstWords; q += kBlock) reinterpret_cast<int*>(&s_inst[b])[q] = src[q];
        __syncthreads();
        return true;
    };
    int cb = 0;
    bool have = fetch(0);
    if (have) batch_tile_issue(s_inst[0], B.W_in + s_inst[0].w_off, s_tile[0].y, B.tj, reinterpret_cast<double*>(tbuf0));
    while (have) {
        float2* cur = cb ? tbuf1 : tbuf0;
        cp_async_wait<0>();
        batch_tile_convert(s_inst[cb], s_tile[cb].y, B.tj, cur);
        __syncthreads();
        const bool next = fetch(cb ^ 1);
        if (next)
            batch_tile_issue(s_inst[cb ^ 1], B.W_in + s_inst[cb ^ 1].w_off, s_tile[cb ^ 1].y, B.tj,
                             reinterpret_cast<double*>(cb ? tbuf0 : tbuf1));
        batch_tile_compute(s_inst[cb], B.F + s_inst[cb].f_off, s_tile[cb].y, B.tj, cur);
        have = next;
        cb ^= 1;
    }
    grid_barrier(B.counter + 1, gridDim.x, B.err);
    // phase 2: the chains
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
        J.Y = B.F + I.f_off + (long long)s * I.n2 * J.n1q;
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
        if (threadIdx.x >= kThreads + 32) mma_issuer<3>(R.P, gs);
        else if (threadIdx.x >= kThreads) tma_issuer<3>(R.P, gs);
        else slab_compute<true>(J, gs, cols, R.P, R.tmem, R.P.mat_slots);
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

// Ring depths and shared-memory size.  With `pair`, the rings are sized so
// that two CTAs share an SM (228 KB per SM, 1 KB reserved per CTA): up to four
// data slots and as many matrix slots as fit, at most as many as data slots
// (the matrix copies complete on the data barriers), fewer data slots only if
// three matrix slots would not fit; otherwise (or if even two and two do not
// fit) one CTA takes the SM's 227 KB.
static void rings(TcShape& sh, uint32_t min_body, bool pair) {
    const uint32_t slack = 128 + kHeaderBytes;                 // ring alignment + barriers
    const uint32_t pair_limit = 228 * 1024 / 2 - 1024 - slack;
    const uint32_t solo_limit = 227 * 1024 - slack;
    auto fit = [&](uint32_t limit) {
        for (uint32_t nd = kMaxData; nd >= 2; --nd) {
            if (nd * sh.data_bytes >= limit) continue;
            uint32_t nm = (limit - nd * sh.data_bytes) / sh.mat_bytes;
            nm = nm > nd ? nd : nm;            // the matrix copies signal the data barriers: nm <= nd
            if (nm >= 3 || (nd == 2 && nm >= 2)) {
                sh.nd = nd;
                sh.nm = nm;
                return true;
            }
        }
        return false;
    };
    if (!(pair && fit(pair_limit)) && !fit(solo_limit)) {
        sh.nd = sh.nm = 2;                                     // reported as too large by the caller
    }
    uint32_t body = sh.nm * sh.mat_bytes + sh.nd * sh.data_bytes;
    if (body < min_body) body = min_body;
    sh.smem_bytes = slack + body;
}

TcShape tc_mode3_shape(int geometry, int n1, int n2, int n3) {
    (void)n1;
    (void)n2;
    TcShape sh{};
    const uint32_t n3p = round_up(n3, 16);
    sh.data_bytes = 2u * kRows * kTileRowBytes;
    sh.mat_bytes = 2u * n3p * kTileRowBytes;
    sh.tmem_cols = pow2_cols(geometry == GEO_BALL ? 2 * n3p : n3p);
    rings(sh, 0, true);
    return sh;
}

// Tensor-memory columns of a slab (see slab_specs): a power of two holding G1
// and G2 side by side and G2 and G3 side by side.
uint32_t slab_tmem_cols(int n1, int n2) {
    const uint32_t n1p = round_up(n1, 16), n2p = round_up(n2, 16), m2 = (n2 + 127) / 128;
    const uint32_t need = std::max(n2p + m2 * n1p, 2 * m2 * n1p);
    return pow2_cols(need);
}

// Slots of the three slab products: matrix rows n2p (G1), 128 m2 (G2, A operand),
// n1p (G3); data rows 128 (G1), n1p (G2, B operand), 128 m2 (G3).
static TcShape slab_shape(int n1, int n2, bool pair) {
    TcShape sh{};
    const uint32_t n1p = round_up(n1, 16), n2p = round_up(n2, 16), m2 = (n2 + 127) / 128;
    const uint32_t mat_rows = std::max(std::max(n2p, kRows * m2), n1p);
    const uint32_t data_rows = std::max(kRows * m2, n1p);
    sh.mat_bytes = 2u * mat_rows * kTileRowBytes;
    sh.data_bytes = 2u * data_rows * kTileRowBytes;
    const uint32_t epi = kRows * (n1p + 1) * 4u;       // epilogue staging reuses the rings
    sh.tmem_cols = slab_tmem_cols(n1, n2);
    rings(sh, epi, pair);
    return sh;
}

TcShape tc_slab_shape(int n1, int n2) { return slab_shape(n1, n2, true); }

// Sphere phi product: data tile 128 rows, matrix N-tile nt rows, accumulator nt columns.
TcShape tc_sphere_phi_shape(int nt) {
    TcShape sh{};
    sh.data_bytes = 2u * kRows * kTileRowBytes;
    sh.mat_bytes = 2u * (uint32_t)nt * kTileRowBytes;
    sh.tmem_cols = pow2_cols((uint32_t)nt);
    rings(sh, 0, sh.tmem_cols <= 256);
    return sh;
}

// Sphere theta product pair: matrices n1p rows, accumulators n1p + nt columns,
// update staging of nt columns.
TcShape tc_sphere_theta_shape(int n1, int nt) {
    TcShape sh{};
    const uint32_t n1p = round_up(n1, 16);
    sh.data_bytes = 2u * kRows * kTileRowBytes;
    sh.mat_bytes = 2u * n1p * kTileRowBytes;
    sh.tmem_cols = pow2_cols(n1p + (uint32_t)nt);
    rings(sh, kRows * ((uint32_t)nt + 1) * 4u, sh.tmem_cols <= 256);
    return sh;
}

// Adjoint theta kernel: matrices n1p rows, accumulators n1p + 2 nt columns, no update staging.
TcShape tc_sphere_theta_adj_shape(int n1, int nt) {
    TcShape sh{};
    const uint32_t n1p = round_up(n1, 16);
    sh.data_bytes = 2u * kRows * kTileRowBytes;
    sh.mat_bytes = 2u * n1p * kTileRowBytes;
    sh.tmem_cols = pow2_cols(n1p + 2u * (uint32_t)nt);
    rings(sh, 0, sh.tmem_cols <= 256);
    return sh;
}

cudaError_t launch_tc_sphere_theta_adj(const SplitTables& T, const TcShape& sh, const SphereAdjArgs& A,
                                       cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_sphere_theta_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sh.smem_bytes);
    if (e != cudaSuccess) return e;
    const int n1p = (T.n1 + 15) & ~15;
    dim3 grid((T.n2 + kRows - 1) / kRows, T.S, (n1p + T.th_nt - 1) / T.th_nt);
    return launch_pdl(k_tc_sphere_theta_adj, grid, dim3(kBlock), sh.smem_bytes, st, T, sh, A);
}

cudaError_t tc_prepare_sphere(uint32_t smem_phi, uint32_t smem_theta) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_sphere_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_phi);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tc_sphere_theta, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_theta);
    return e;
}

cudaError_t launch_tc_sphere_phi(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    const int n2p = (T.n2 + 15) & ~15;
    const int ks = T.phi_ks > 1 ? T.phi_ks : 1;
    dim3 grid((T.n1 + kRows - 1) / kRows, (n2p + T.phi_nt - 1) / T.phi_nt, (T.phi_pair ? 2 * T.S : T.S) * ks);
    if (ks == 1) return launch_pdl(k_tc_sphere_phi, grid, dim3(kBlock), sh.smem_bytes, st, T, sh);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = sh.smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = (unsigned)ks;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_tc_sphere_phi, T, sh);
}

cudaError_t launch_tc_sphere_theta(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    const int n1p = (T.n1 + 15) & ~15;
    dim3 grid((T.n2 + kRows - 1) / kRows, T.S, (n1p + T.th_nt - 1) / T.th_nt);
    return launch_pdl(k_tc_sphere_theta, grid, dim3(kBlock), sh.smem_bytes, st, T, sh);
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
    if (smem_slab) {
        e = cudaFuncSetAttribute(k_tc_slab<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_slab);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_slab<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_slab);
    }
    if (e != cudaSuccess) return e;
    const int big = 212 * 1024;   // stencil tiles (all species) are sized to at most 212 KB
    e = cudaFuncSetAttribute(k_rhs_tile<GEO_DISK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_tile<GEO_SPHERE>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_tile<GEO_BALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_tile<GEO_CYLINDER>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    const int ring = 4 * 8 * kRhsThreads * (int)sizeof(float2);    // four planes of at most 8 values per thread
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_BALL, 4, 1>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_BALL, 8, 1>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_BALL, 4, 2>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_BALL, 8, 2>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_CYLINDER, 4, 1>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_CYLINDER, 8, 1>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_CYLINDER, 4, 2>, A, ring);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_roll<GEO_CYLINDER, 8, 2>, A, ring);
    const int march = 200 * 1024;   // the marching kernels: candidates and launcher keep march_smem within this
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_BALL, 1>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_BALL, 2>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_BALL, 3>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_BALL, 4>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_CYLINDER, 1>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_CYLINDER, 2>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_CYLINDER, 3>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march<GEO_CYLINDER, 4>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_BALL, 1>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_BALL, 2>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_BALL, 3>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_BALL, 4>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_CYLINDER, 1>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_CYLINDER, 2>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_CYLINDER, 3>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_CYLINDER, 4>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_BALL, 2, R_GRAY_SCOTT>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_BALL, 2, R_SCHNAKENBERG>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_CYLINDER, 2, R_GRAY_SCOTT>, A, march);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rhs_march2<GEO_CYLINDER, 2, R_SCHNAKENBERG>, A, march);
    return e;
}

cudaError_t launch_tc_mode3(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    dim3 grid((unsigned)((T.n1q * (long long)T.n2 + kRows - 1) / kRows), T.S);
    if (T.geometry == GEO_BALL)
        return launch_pdl(k_tc_mode3<GEO_BALL>, grid, dim3(kBlock), sh.smem_bytes, st, T, sh);
    return launch_pdl(k_tc_mode3<GEO_CYLINDER>, grid, dim3(kBlock), sh.smem_bytes, st, T, sh);
}

cudaError_t launch_tc_slab(const SplitTables& T, const TcShape& sh, cudaStream_t st) {
    dim3 grid(T.geometry == GEO_DISK ? 1 : T.n3, T.S);
    if (T.theta_comp) return launch_pdl(k_tc_slab<true>, grid, dim3(kBlock), sh.smem_bytes, st, T, sh);
    return launch_pdl(k_tc_slab<false>, grid, dim3(kBlock), sh.smem_bytes, st, T, sh);
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
    if (T.n1 >= 4096) return cudaErrorInvalidValue;      // exactness bound of div_by
    const int tj = T.rhs_tj > 0 ? T.rhs_tj : rhs_tile_tj<GEO>(T);
    const size_t smem = sizeof(float2) * (size_t)T.S * (TS::TK + 2 * TS::KH) * (tj + 2) * T.n1;
    dim3 grid((T.n2 + tj - 1) / tj, (T.n3 + TS::TK - 1) / TS::TK, 1);
    cudaError_t e = launch_pdl(k_rhs_tile<GEO>, grid, dim3(kRhsThreads), smem, st, T.rhs, T.state, T.Y, tj, T.n1q, T.ys);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Stencil configurations the autotuner times: (tile height, 0, 1) for the tiled
// kernel whose all-species tile fits 220 KB, and, for the 3-D geometries,
// (tile height, planes per CTA, register cap for 1 or 2 CTAs per SM) for the
// rolling-window kernel whose plane holds at most 8 values per thread.
// The marching stencil's launch: two columns per thread when n1 is even and the
// state 16-byte aligned (then 16-byte copies apply), else one; threads and
// shared memory (two planes of pairs and the ring of FP64 values).
static bool march_pairs(const SplitTables& T) { return T.n1 % 2 == 0 && ((uintptr_t)T.state & 15u) == 0; }
static int march_threads(int tj, int n1, bool pairs) {
    return (std::max(tj, 2) * (pairs ? n1 / 2 : n1) + 31) / 32 * 32;
}
static size_t march_smem(int S, int tj, int n1, bool pairs) {
    const int threads = march_threads(tj, n1, pairs);
    const size_t ring_vals = pairs ? 2 * (size_t)(threads + n1) : (size_t)(threads + 2 * n1);
    return 2 * sizeof(float2) * (size_t)S * (tj + 2) * n1 + sizeof(double) * kMarchAhead * S * ring_vals;
}
constexpr size_t kMarchSmemMax = 200 * 1024;

int rhs_candidates(const SplitTables& T, int3* out, int max_out) {
    const bool k3 = T.geometry == GEO_BALL || T.geometry == GEO_CYLINDER;
    const size_t per_line = sizeof(float2) * (size_t)T.S * (k3 ? 10 : 1) * T.n1;
    int n = 0;
    for (int tj = 1; tj <= (k3 ? 16 : 32) && tj <= T.n2 && n < max_out; ++tj)
        if (per_line * (tj + 2) + 8 * 1024 <= 220 * 1024) out[n++] = make_int3(tj, 0, 1);
    if (k3) {
        // marching kernel: one thread per column of TJ lines (at least 2 n1 for the halo lines)
        const int maxt = T.S <= 2 ? 1024 : 512;
        const int tjs[] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 16, 20, 24, 28, 32};
        for (int tj : tjs) {
            if (tj > T.n2 || T.S > 4 || std::max(tj, 2) * T.n1 > maxt) break;
            if (march_smem(T.S, tj, T.n1, false) > kMarchSmemMax ||
                (T.n1 % 2 == 0 && march_smem(T.S, tj, T.n1, true) > kMarchSmemMax))
                continue;
            const int kss[] = {2, 3, 4, 6, 8, 12, 16};
            for (int ks : kss)
                if (ks <= T.n3 && n < max_out) out[n++] = make_int3(tj, ks, 0);
        }
        for (int tj = 2; tj <= 24 && tj <= T.n2 + 1; tj += 2) {
            if ((long long)T.S * (tj + 2) * T.n1 > 8 * kRhsThreads) break;
            for (int ks = 2; ks <= 16 && ks <= T.n3; ks *= 2)
                for (int mb = 1; mb <= 2 && n < max_out; ++mb) out[n++] = make_int3(tj, ks, mb);
        }
    }
    return n;
}


template <int GEO>
static cudaError_t launch_rhs_march_geo(const SplitTables& T, cudaStream_t st) {
    const int tj = T.rhs_tj, ks = T.rhs_ks;
    if (tj < 1 || tj > T.n2 || ks < 1 || T.S < 1 || T.S > kMaxSpecies ||
        std::max(tj, 2) * T.n1 > (T.S <= 2 ? 1024 : 512))
        return cudaErrorInvalidValue;
    const bool pairs = march_pairs(T);
    const int threads = march_threads(tj, T.n1, pairs);
    const size_t smem = march_smem(T.S, tj, T.n1, pairs);
    if (smem > kMarchSmemMax) return cudaErrorInvalidValue;
    dim3 grid((T.n2 + tj - 1) / tj, (T.n3 + ks - 1) / ks, 1);
    cudaError_t e;
    if (pairs) {
        // two-species Gray-Scott / Schnakenberg: the reaction kind compiled in (same arithmetic)
        const int kind = T.rhs.reac.kind;
        auto kern = T.S == 1 ? k_rhs_march2<GEO, 1>
                  : T.S == 2 ? (kind == R_GRAY_SCOTT ? k_rhs_march2<GEO, 2, R_GRAY_SCOTT>
                                : kind == R_SCHNAKENBERG ? k_rhs_march2<GEO, 2, R_SCHNAKENBERG> : k_rhs_march2<GEO, 2>)
                  : T.S == 3 ? k_rhs_march2<GEO, 3> : k_rhs_march2<GEO, 4>;
        e = launch_pdl(kern, grid, dim3(threads), smem, st, T.rhs, T.state, T.Y, tj, ks, T.n1q, T.ys);
    } else {
        auto kern = T.S == 1 ? k_rhs_march<GEO, 1>
                  : T.S == 2 ? k_rhs_march<GEO, 2> : T.S == 3 ? k_rhs_march<GEO, 3> : k_rhs_march<GEO, 4>;
        e = launch_pdl(kern, grid, dim3(threads), smem, st, T.rhs, T.state, T.Y, tj, ks, T.n1q, T.ys);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int GEO>
static cudaError_t launch_rhs_roll_geo(const SplitTables& T, cudaStream_t st) {
    const int tj = T.rhs_tj, ks = T.rhs_ks;
    const long long pv = (long long)T.S * (tj + 2) * T.n1;
    if (tj < 1 || tj > 32 || pv > 8 * kRhsThreads) return cudaErrorInvalidValue;
    const size_t smem = 4 * sizeof(float2) * (size_t)pv;
    dim3 grid((T.n2 + tj - 1) / tj, (T.n3 + ks - 1) / ks, 1);
    const bool small = pv <= 4 * kRhsThreads;
    auto kern = T.rhs_mb == 2 ? (small ? k_rhs_roll<GEO, 4, 2> : k_rhs_roll<GEO, 8, 2>)
                              : (small ? k_rhs_roll<GEO, 4, 1> : k_rhs_roll<GEO, 8, 1>);
    cudaError_t e = launch_pdl(kern, grid, dim3(kRhsThreads), smem, st, T.rhs, T.state, T.Y, tj, ks, T.n1q, T.ys);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

TcShape tc_batch_shape(int max_n1, int max_n2, uint32_t tmem_cols) {
    TcShape sh = slab_shape(max_n1, max_n2, false);        // one persistent CTA per SM
    sh.tmem_cols = std::max(sh.tmem_cols, tmem_cols);
    return sh;
}

// Every ring configuration of the batch kernel that fits one CTA per SM: nd data slots and
// nm <= nd matrix slots (the matrix copies complete on the data barriers), with room for the
// epilogue staging and for a phase-1 stencil tile of max_tj + 2 lines of both species.
int tc_batch_shapes(int max_n1, int max_n2, uint32_t tmem_cols, int max_tj, TcShape* out, int cap) {
    const TcShape base = tc_batch_shape(max_n1, max_n2, tmem_cols);
    const uint32_t slack = 128 + kHeaderBytes;
    const uint32_t n1p = round_up(max_n1, 16);
    const uint32_t epi = kRows * (n1p + 1) * 4u;
    // two phase-1 tile buffers (the next tile's copies land while the current one is computed)
    const uint32_t tile = 2u * (uint32_t)(max_tj + 2) * (uint32_t)max_n1 * 2u * (uint32_t)sizeof(float2);
    int n = 0;
    for (uint32_t nd = 2; nd <= (uint32_t)kMaxData; ++nd)
        for (uint32_t nm = 2; nm <= nd && nm <= (uint32_t)kMaxMat; ++nm) {
            TcShape sh = base;
            sh.nd = nd;
            sh.nm = nm;
            const uint32_t body = std::max(std::max(nm * sh.mat_bytes + nd * sh.data_bytes, epi), tile);
            sh.smem_bytes = slack + body;
            if (sh.smem_bytes > 227u * 1024u || n >= cap) continue;
            out[n++] = sh;
        }
    return n;
}

cudaError_t tc_prepare_batch(uint32_t smem) {
    return cudaFuncSetAttribute(k_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// Cooperative launch: every CTA resident, as the grid barrier between the phases requires.
cudaError_t launch_tc_batch(const BatchTables& B, const TcShape& sh, int grid, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(B.counter, 0, 3 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = sh.smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tc_batch, B, sh);
}

// CTAs of the batch kernel that can be resident at once (the cooperative grid).
int batch_grid(const TcShape& sh) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_batch, kBlock, sh.smem_bytes) != cudaSuccess)
        return 0;
    return sms * per_sm;
}

// Self-test of the bounded-wait path every pipeline wait uses: one thread waits
// on an mbarrier nobody arrives on; after `limit_cycles` the wait gives up,
// records DERR_TIMEOUT_MMA in *err and the kernel returns normally.
__global__ void k_wait_selftest(int* err, long long limit_cycles) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, err, DERR_TIMEOUT_MMA, limit_cycles);
}

cudaError_t launch_wait_selftest(int* err, long long limit_cycles, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, limit_cycles);
    return cudaGetLastError();
}

cudaError_t launch_rhs_split(const SplitTables& T, cudaStream_t st) {
    if (T.rhs_ks > 0 && T.rhs_mb == 0) {
        if (T.geometry == GEO_BALL) return launch_rhs_march_geo<GEO_BALL>(T, st);
        if (T.geometry == GEO_CYLINDER) return launch_rhs_march_geo<GEO_CYLINDER>(T, st);
        return cudaErrorInvalidValue;
    }
    if (T.rhs_ks > 0) {
        if (T.geometry == GEO_BALL) return launch_rhs_roll_geo<GEO_BALL>(T, st);
        if (T.geometry == GEO_CYLINDER) return launch_rhs_roll_geo<GEO_CYLINDER>(T, st);
        return cudaErrorInvalidValue;
    }
    switch (T.geometry) {
    case GEO_DISK: return launch_rhs_tile_geo<GEO_DISK>(T, st);
    case GEO_SPHERE: return launch_rhs_tile_geo<GEO_SPHERE>(T, st);
    case GEO_BALL: return launch_rhs_tile_geo<GEO_BALL>(T, st);
    default: return launch_rhs_tile_geo<GEO_CYLINDER>(T, st);
    }
}

}  // namespace sexpe
