// C ABI of libsexpe: plan construction (FP64 host setup + one upload), the
// per-step launch sequence of both arithmetic paths, CUDA-graph replay and
// error reporting.  See include/sexpe.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "couple_terms.cuh"
#include "plan_internal.h"

using namespace sexpe;

namespace {

sexpe_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SEXPE_OK;
    if (e == cudaErrorMemoryAllocation) return SEXPE_ENOMEM;
    return SEXPE_ECUDA;
}

#define SX_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_status(e_);  \
    } while (0)

template <class T>
sexpe_status upload(sexpe_plan* p, const std::vector<T>& h, const T** out, cudaStream_t st) {
    void* dptr = nullptr;
    const size_t bytes = h.size() * sizeof(T);
    SX_CUDA(cudaMalloc(&dptr, bytes > 0 ? bytes : 16));
    p->allocs.push_back(dptr);
    p->bytes += bytes;
    if (bytes) SX_CUDA(cudaMemcpyAsync(dptr, h.data(), bytes, cudaMemcpyHostToDevice, st));
    *out = static_cast<const T*>(dptr);
    return SEXPE_OK;
}

template <class T>
sexpe_status alloc_dev(sexpe_plan* p, size_t count, T** out) {
    void* dptr = nullptr;
    SX_CUDA(cudaMalloc(&dptr, count * sizeof(T) > 0 ? count * sizeof(T) : 16));
    p->allocs.push_back(dptr);
    p->bytes += count * sizeof(T);
    *out = static_cast<T*>(dptr);
    return SEXPE_OK;
}

#define SX_TRY(call)                         \
    do {                                     \
        sexpe_status s_ = (call);            \
        if (s_ != SEXPE_OK) return s_;       \
    } while (0)

// Scale factor of direction mu at grid point (i, j, k): the diagonal factors of
// the other modes in the Kronecker term M_mu (Section 2).
double dir_scale(const sexpe_plan* p, int mu, int i, int j, int k) {
    auto Dr = [&](int ii) { return std::pow(p->ax[0].pts[ii], p->rho_pow); };
    auto Dp = [&](int m, int kk) { double s = std::sin(p->ax[m].pts[kk]); return 1.0 / (s * s); };
    switch (p->geometry) {
    case SEXPE_DISK: return mu == 2 ? Dr(i) : 1.0;
    case SEXPE_SPHERE: return mu == 1 ? Dp(1, j) : 1.0;
    case SEXPE_BALL: return mu == 2 ? Dr(i) * Dp(2, k) : (mu == 3 ? Dr(i) : 1.0);
    default: return mu == 2 ? Dr(i) : 1.0;
    }
}

bool dir_is_eigen(int geometry, int mu) {
    switch (geometry) {
    case SEXPE_DISK: return mu == 2;
    case SEXPE_SPHERE: return mu == 1;
    case SEXPE_BALL: return mu >= 2;
    default: return mu == 2;
    }
}

bool all_finite(const std::vector<double>& v) {
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

bool all_finite(const std::vector<float>& v) {
    for (float x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

// TF32 rounding to nearest (ties away from zero) of an FP32 value, on the host.
float tf32_rna_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return x;
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Pre-laid operand image of a constant matrix: for each 16-wide K-chunk, a hi
// tile then a lo tile of rows_pad rows in the K-major no-swizzle core-matrix
// layout the kernels' shared-memory descriptors describe.
std::vector<float> make_image(int rows_valid, int k_valid, int rows_pad, int k_pad,
                              const std::function<double(int, int)>& f) {
    const int chunks = k_pad / kKC;
    const size_t tile = (size_t)rows_pad * kKC;
    std::vector<float> img((size_t)chunks * 2 * tile, 0.0f);
    for (int c = 0; c < chunks; ++c) {
        float* hi = img.data() + (size_t)c * 2 * tile;
        float* lo = hi + tile;
        for (int r = 0; r < rows_valid; ++r) {
            for (int kk = 0; kk < kKC; ++kk) {
                const int k = c * kKC + kk;
                if (k >= k_valid) continue;
                const double x = f(r, k);
                const float h = tf32_rna_host((float)x);
                const float l = tf32_rna_host((float)(x - (double)h));
                const size_t off = ((size_t)(r >> 3) * kSBO + (size_t)(kk >> 2) * kLBO + (size_t)(r & 7) * 16 +
                                    (size_t)(kk & 3) * 4) / 4;
                hi[off] = h;
                lo[off] = l;
            }
        }
    }
    return img;
}

sexpe_status upload_image(sexpe_plan* p, int rows_valid, int k_valid, int rows_pad, int k_pad,
                          const std::function<double(int, int)>& f, Image* out, cudaStream_t st) {
    std::vector<float> img = make_image(rows_valid, k_valid, rows_pad, k_pad, f);
    const float* dptr = nullptr;
    SX_TRY(upload(p, img, &dptr, st));
    out->ptr = dptr;
    out->rows_pad = rows_pad;
    out->k_chunks = k_pad / kKC;
    out->chunk_floats = 2LL * rows_pad * kKC;
    return SEXPE_OK;
}

int rup16(int x) { return (x + 15) / 16 * 16; }

template <class T>
sexpe_status build_rhs_tables(sexpe_plan* p, RhsTables<T>* tb, cudaStream_t st) {
    tb->geometry = p->geometry;
    tb->S = p->S;
    tb->n1 = p->n[0];
    tb->n2 = p->n[1];
    tb->n3 = p->n[2];
    tb->npts = p->npts;
    for (int m = 0; m < 3; ++m) {
        const Axis& a = p->ax[m];
        if (m >= p->ndim) {
            tb->ax[m] = StencilAxis<T>{nullptr, nullptr, nullptr, 1, 0};
            continue;
        }
        std::vector<T> lo(a.n), up(a.n), rs(a.n);
        for (int r = 0; r < a.n; ++r) {
            lo[r] = (T)a.lower[r];
            up[r] = (T)a.upper[r];
            // Row sums are zero for every Neumann/periodic row; only a Dirichlet
            // end (A_z as printed) leaves a nonzero residual.
            const double l = (r > 0 || a.periodic) ? a.lower[r] : 0.0;
            const double u = (r < a.n - 1 || a.periodic) ? a.upper[r] : 0.0;
            const double sum = a.diag[r] + l + u;
            rs[r] = (T)(std::fabs(sum) <= 1e-9 * std::fabs(a.diag[r]) ? 0.0 : sum);
        }
        StencilAxis<T> sa{};
        SX_TRY(upload(p, lo, &sa.lower, st));
        SX_TRY(upload(p, up, &sa.upper, st));
        SX_TRY(upload(p, rs, &sa.rs, st));
        sa.n = a.n;
        sa.periodic = a.periodic ? 1 : 0;
        tb->ax[m] = sa;
    }
    tb->Dr = nullptr;
    tb->Dp = nullptr;
    if (p->geometry != SEXPE_SPHERE) {
        std::vector<T> dr(p->n[0]);
        for (int i = 0; i < p->n[0]; ++i) dr[i] = (T)std::pow(p->ax[0].pts[i], p->rho_pow);
        SX_TRY(upload(p, dr, &tb->Dr, st));
    }
    if (p->geometry == SEXPE_SPHERE || p->geometry == SEXPE_BALL) {
        const int m = p->geometry == SEXPE_SPHERE ? 1 : 2;
        std::vector<T> dp(p->n[m]);
        for (int k = 0; k < p->n[m]; ++k) {
            const double s = std::sin(p->ax[m].pts[k]);
            dp[k] = (T)(1.0 / (s * s));
        }
        SX_TRY(upload(p, dp, &tb->Dp, st));
    }
    for (int s = 0; s < kMaxSpecies; ++s) tb->d[s] = (T)(s < p->S ? p->d[s] : 0.0);
    tb->mms_rho = tb->mms_theta = nullptr;
    tb->step = nullptr;
    tb->t0 = 0.0;
    tb->tau_t = p->tau;
    if (p->reaction == SEXPE_BVAM_MANUFACTURED) {        // Section 5.1, disk: tables of the exact solution
        const int n1 = p->n[0], n2 = p->n[1];
        std::vector<T> mr(3 * (size_t)n1), mt(4 * (size_t)n2);
        for (int i = 0; i < n1; ++i) {
            const double r = p->ax[0].pts[i];
            const double R = (1.0 - r) * (1.0 - r), dR = -2.0 * (1.0 - r), d2R = 2.0;
            mr[i] = (T)R;
            mr[n1 + i] = (T)(d2R + dR / r);
            mr[2 * n1 + i] = (T)(R / (r * r));
        }
        for (int j = 0; j < n2; ++j) {
            const double th = p->ax[1].pts[j], c = std::cos(th), s = std::sin(th);
            const double Tt = std::exp(c / 10.0), Sv = std::exp(s / 10.0);
            mt[j] = (T)Tt;
            mt[n2 + j] = (T)(Tt * (s * s / 100.0 - c / 10.0));
            mt[2 * n2 + j] = (T)Sv;
            mt[3 * n2 + j] = (T)(Sv * (c * c / 100.0 - s / 10.0));
        }
        SX_TRY(upload(p, mr, &tb->mms_rho, st));
        SX_TRY(upload(p, mt, &tb->mms_theta, st));
        if (!p->d_step) {
            SX_TRY(alloc_dev(p, 1, &p->d_step));
            SX_CUDA(cudaMemsetAsync(p->d_step, 0, sizeof(long long), st));
        }
        tb->step = p->d_step;
        tb->t0 = p->t0;
    }
    tb->reac.kind = p->reaction;
    tb->reac.S = p->S;
    for (int s = 0; s < kMaxSpecies; ++s) tb->reac.off[s] = (T)(s < (int)p->offset.size() ? p->offset[s] : 0.0);
    tb->reac.lifted = 0;
    for (int q = 0; q < 6; ++q) tb->reac.q[q] = (T)0;
    if (p->reaction == SEXPE_SCHNAKENBERG && !p->offset.empty()) {
        // b(c), c(c) are differences of O(1) terms that nearly cancel at a steady state and are
        // then multiplied by gamma: formed in extended precision, rounded once
        const long double cu = p->offset[0], cv = p->offset[1], a = p->params[1], b = p->params[2];
        tb->reac.lifted = 1;
        tb->reac.q[0] = (T)(double)(a - cu + cu * cu * cv);
        tb->reac.q[1] = (T)(double)(b - cu * cu * cv);
        tb->reac.q[2] = (T)(double)(2.0L * cu * cv);
        tb->reac.q[3] = (T)(double)(cu * cu);
        tb->reac.q[4] = (T)(double)cv;
        tb->reac.q[5] = (T)(double)(2.0L * cu);
    }
    for (int q = 0; q < 16; ++q) tb->reac.p[q] = (T)(q < (int)p->params.size() ? p->params[q] : 0.0);
    return SEXPE_OK;
}

sexpe_status build_fp64(sexpe_plan* p, cudaStream_t st) {
    SX_TRY(build_rhs_tables<double>(p, &p->rhs64, st));
    for (int b = 0; b < 3; ++b) SX_TRY(alloc_dev(p, (size_t)p->S * p->npts, &p->buf64[b]));
    for (int mu = p->ndim; mu >= 1; --mu) {
        const Axis& a = p->ax[mu - 1];
        const int n = a.n;
        Dir64 dir;
        dir.mu = mu;
        dir.eigen = dir_is_eigen(p->geometry, mu);
        if (dir.eigen) {
            Eigen e = a.periodic ? theta_eigen(a) : tridiag_eigen(a);
            if (!all_finite(e.V.a) || !all_finite(e.Vinv.a)) return SEXPE_ENUMERIC;
            SX_TRY(upload(p, e.V.a, &dir.V, st));
            SX_TRY(upload(p, e.Vinv.a, &dir.Vinv, st));
            std::vector<double> had((size_t)p->S * p->npts);
            for (int s = 0; s < p->S; ++s)
                for (int k = 0; k < p->n[2]; ++k)
                    for (int j = 0; j < p->n[1]; ++j)
                        for (int i = 0; i < p->n[0]; ++i) {
                            const int m = mu == 1 ? i : (mu == 2 ? j : k);
                            const long long idx = i + (long long)p->n[0] * (j + (long long)p->n[1] * k);
                            had[(size_t)s * p->npts + idx] =
                                phi1_scalar(p->tau * p->d[s] * dir_scale(p, mu, i, j, k) * e.lam[m]);
                        }
            if (!all_finite(had)) return SEXPE_ENUMERIC;
            SX_TRY(upload(p, had, &dir.had, st));
        } else {
            const Mat A = a.dense();
            std::vector<double> P((size_t)p->S * n * n);
            for (int s = 0; s < p->S; ++s) {
                Mat X(n);
                for (size_t q = 0; q < X.a.size(); ++q) X.a[q] = p->tau * p->d[s] * A.a[q];
                const Mat R = phi1_pade(X);
                std::memcpy(&P[(size_t)s * n * n], R.a.data(), sizeof(double) * n * n);
            }
            if (!all_finite(P)) return SEXPE_ENUMERIC;
            SX_TRY(upload(p, P, &dir.P, st));
        }
        p->dirs64.push_back(dir);
    }
    p->kernels_per_step = 1;
    for (const Dir64& d : p->dirs64) p->kernels_per_step += d.eigen ? 2 : 1;
    return SEXPE_OK;
}

// Unsplit exponential Euler (the accuracy baseline of the splitting, eq. ee with
// phi_1 of the whole operator): M = M_1 + ... + M_d assembled densely from the
// same 1-D axes and diagonal factors as the split chain (each point's row gets
// s * A_mu along every mode mu, s the direction's scale at the point), then
// P_s = phi_1(tau d_s M) by Pade scaling and squaring.  N_pts <= 2048.
constexpr long long kUnsplitMaxPts = 2048;

sexpe_status build_unsplit(sexpe_plan* p, cudaStream_t st) {
    if (p->npts > kUnsplitMaxPts) return SEXPE_EUNSUPPORTED;
    const int N = (int)p->npts;
    SX_TRY(build_rhs_tables<double>(p, &p->rhs64, st));
    SX_TRY(alloc_dev(p, (size_t)p->S * p->npts, &p->buf64[0]));
    Mat M(N);
    for (int k = 0; k < p->n[2]; ++k)
        for (int j = 0; j < p->n[1]; ++j)
            for (int i = 0; i < p->n[0]; ++i) {
                const int c[3] = {i, j, k};
                const int row = i + p->n[0] * (j + p->n[1] * k);
                for (int mu = 1; mu <= p->ndim; ++mu) {
                    const Axis& a = p->ax[mu - 1];
                    const int r = c[mu - 1], n = a.n;
                    const int stride = mu == 1 ? 1 : (mu == 2 ? p->n[0] : p->n[0] * p->n[1]);
                    const double sc = dir_scale(p, mu, i, j, k);
                    M(row, row) += sc * a.diag[r];
                    if (r > 0) M(row, row - stride) += sc * a.lower[r];
                    else if (a.periodic) M(row, row + (n - 1) * stride) += sc * a.lower[r];
                    if (r < n - 1) M(row, row + stride) += sc * a.upper[r];
                    else if (a.periodic) M(row, row - (n - 1) * stride) += sc * a.upper[r];
                }
            }
    std::vector<double> P((size_t)p->S * N * N);
    for (int s = 0; s < p->S; ++s) {
        Mat X(N);
        for (size_t q = 0; q < X.a.size(); ++q) X.a[q] = p->tau * p->d[s] * M.a[q];
        const Mat R = phi1_pade(X);
        std::memcpy(&P[(size_t)s * N * N], R.a.data(), sizeof(double) * (size_t)N * N);
    }
    if (!all_finite(P)) return SEXPE_ENUMERIC;
    SX_TRY(upload(p, P, &p->unsplit_P, st));
    p->kernels_per_step = 2;
    return SEXPE_OK;
}

// Measured choice of the stencil tile height (the autotuner of the split path):
// every feasible height is timed with CUDA events -- one warm-up launch, then
// three launches -- on a zeroed scratch state of the plan's shape, and the
// fastest is kept.  The model in the launcher ranks heights by waves and halo
// rows, but the halo's real cost (each halo line is loaded and split again)
// and the overlap of co-resident CTAs are only known by running them.  Runs
// once at setup, before any graph capture; the scratch state is freed here.
static sexpe_status tune_stencil(sexpe_plan* p, cudaStream_t st) {
    SplitTables T = p->tabs;
    int3 cand[256];
    const int nc = rhs_candidates(T, cand, 256);
    if (nc == 0) return SEXPE_EUNSUPPORTED;
    double* scratch = nullptr;
    const size_t bytes = sizeof(double) * (size_t)p->S * p->npts;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SEXPE_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sexpe_status rc = SEXPE_OK;
    float best_ms = 1e30f;
    int3 best = cand[0];
    if (cudaMemsetAsync(scratch, 0, bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = SEXPE_ECUDA;
    } else {
        T.state = scratch;
        for (int c = 0; c < nc && rc == SEXPE_OK; ++c) {
            T.rhs_tj = cand[c].x;
            T.rhs_ks = cand[c].y;
            T.rhs_mb = cand[c].z;
            bool ok = launch_rhs_split(T, st) == cudaSuccess && cudaEventRecord(e0, st) == cudaSuccess;
            for (int r = 0; r < 3 && ok; ++r) ok = launch_rhs_split(T, st) == cudaSuccess;
            float ms = 0.f;
            ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (!ok) rc = SEXPE_ECUDA;
            else if (ms < best_ms) {
                best_ms = ms;
                best = cand[c];
            }
        }
    }
    if (rc != SEXPE_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    p->tabs.rhs_tj = best.x;
    p->tabs.rhs_ks = best.y;
    p->tabs.rhs_mb = best.z;
    p->rhs_tj_us = best_ms * 1000.f / 3.f;
    return rc;
}

// Measured K-split of the sphere's phi product: one output tile's product runs over all n_phi / 16
// K-chunks in one CTA, and with few tiles (16 CTAs on the 256 x 512 sphere) that serial chain sets
// the kernel's time.  Split over a cluster of ks CTAs, each runs 1/ks of the chunks and the
// partials are added through distributed shared memory.  Every ks in {1, 2, 4, 8} that divides
// the chunk count (at least two chunks per CTA) and the tile's columns, and whose partial tile
// fits in the rings, is timed like the theta splits (a configuration the device cannot launch is
// skipped), and the fastest is kept.
static sexpe_status tune_sphere_phi(sexpe_plan* p, cudaStream_t st) {
    SplitTables& T = p->tabs;
    T.phi_ks = 1;
    const int kc = rup16(p->n[1]) / kKC;
    const uint32_t rings_bytes = p->sh3.nm * p->sh3.mat_bytes + p->sh3.nd * p->sh3.data_bytes;
    std::vector<int> cands{1};
    for (int ks = 2; ks <= 8; ks *= 2)
        if (kc % ks == 0 && kc / ks >= 2 && T.phi_nt % ks == 0 &&
            (uint32_t)T.phi_nt * 128u * sizeof(float) <= rings_bytes)   // 128-row partial tile
            cands.push_back(ks);
    if (cands.size() == 1) return SEXPE_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sexpe_status rc = SEXPE_OK;
    float best_ms = 1e30f;
    int best = 1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = SEXPE_ECUDA;
    } else {
        SplitTables Tt = T;
        for (size_t c = 0; c < cands.size() && rc == SEXPE_OK; ++c) {
            Tt.phi_ks = cands[c];
            if (launch_tc_sphere_phi(Tt, p->sh3, st) != cudaSuccess) {   // e.g. no room for the cluster
                cudaGetLastError();
                if (cands[c] == 1) rc = SEXPE_ECUDA;
                continue;
            }
            bool ok = cudaEventRecord(e0, st) == cudaSuccess;
            for (int r = 0; r < 3 && ok; ++r) ok = launch_tc_sphere_phi(Tt, p->sh3, st) == cudaSuccess;
            float ms = 0.f;
            ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (!ok) rc = SEXPE_ECUDA;
            else if (ms < best_ms) {
                best_ms = ms;
                best = cands[c];
            }
        }
    }
    if (rc != SEXPE_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    T.phi_ks = best;
    return rc;
}

// Times the theta kernel of the sphere at every column split (one warm-up launch,
// then three, CUDA events) on a zeroed scratch state and keeps the fastest.
static sexpe_status tune_sphere_theta(sexpe_plan* p, const std::vector<int>& splits, const std::vector<Image>& qimg,
                                      cudaStream_t st) {
    SplitTables T = p->tabs;
    const int n1p = rup16(p->n[0]);
    double* scratch = nullptr;
    const size_t bytes = sizeof(double) * (size_t)p->S * p->npts;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SEXPE_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sexpe_status rc = SEXPE_OK;
    float best_ms = 1e30f;
    size_t best = 0;
    if (cudaMemsetAsync(scratch, 0, bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = SEXPE_ECUDA;
    } else {
        T.state = T.state_upd = scratch;
        for (size_t c = 0; c < splits.size() && rc == SEXPE_OK; ++c) {
            T.Qsph = qimg[c];
            T.th_nt = n1p / splits[c];
            const TcShape sh = tc_sphere_theta_shape(p->n[0], T.th_nt);
            bool ok = launch_tc_sphere_theta(T, sh, st) == cudaSuccess && cudaEventRecord(e0, st) == cudaSuccess;
            for (int r = 0; r < 3 && ok; ++r) ok = launch_tc_sphere_theta(T, sh, st) == cudaSuccess;
            float ms = 0.f;
            ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (!ok) rc = SEXPE_ECUDA;
            else if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    if (rc != SEXPE_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    p->th_splits = splits;
    p->th_imgs = qimg;
    p->tabs.Qsph = qimg[best];
    p->tabs.th_nt = n1p / splits[best];
    p->shs = tc_sphere_theta_shape(p->n[0], p->tabs.th_nt);
    return rc;
}

// Split-TF32 sphere (eq. ee_sphere): mode 1 theta (scaled by sin^-2 phi_j),
// mode 2 phi (plain); phi first, then theta with the update.
sexpe_status build_split_sphere(sexpe_plan* p, cudaStream_t st) {
    const int n1 = p->n[0], n2 = p->n[1];
    if (n1 > 256) return SEXPE_EUNSUPPORTED;
    SplitTables& T = p->tabs;
    T.geometry = p->geometry;
    T.S = p->S;
    T.n1 = n1;
    T.n2 = n2;
    T.n3 = 1;
    T.npts = p->npts;
    T.tau = (float)p->tau;
    T.tau_d = p->tau;
    SX_TRY(build_rhs_tables<float>(p, &T.rhs, st));
    T.n1q = (n1 + 3) & ~3;
    T.ys = (long long)n2 * T.n1q;
    SX_TRY(alloc_dev(p, (size_t)p->S * T.ys, &T.Y));
    SX_TRY(alloc_dev(p, (size_t)p->S * T.ys, &T.Y2));
    SX_CUDA(cudaMemsetAsync(T.Y, 0, sizeof(float) * (size_t)p->S * T.ys, st));
    SX_CUDA(cudaMemsetAsync(T.Y2, 0, sizeof(float) * (size_t)p->S * T.ys, st));
    T.err = p->d_err;
    const int n1p = rup16(n1), n2p = rup16(n2);
    // theta: Q_theta (closed form), as B operands of both products
    Eigen th = theta_eigen(p->ax[0]);
    SX_TRY(upload_image(p, n1, n1, n1p, n1p, [&](int r, int k) { return th.V(k, r); }, &T.QT, st));
    SX_TRY(upload_image(p, n1, n1, n1p, n1p, [&](int r, int k) { return th.V(r, k); }, &T.Q, st));
    std::vector<float> hs((size_t)p->S * T.ys, 0.f);
    for (int s = 0; s < p->S; ++s)
        for (int j = 0; j < n2; ++j)
            for (int ip = 0; ip < n1; ++ip)
                hs[(size_t)s * T.ys + (size_t)j * T.n1q + ip] =
                    (float)phi1_scalar(p->tau * p->d[s] * dir_scale(p, 1, 0, j, 0) * th.lam[ip]);
    SX_TRY(upload(p, hs, &T.had_sph, st));
    // phi: phi_1(tau d_s A_phi), N-tiled so several CTAs share the product of one theta tile
    T.phi_nt = n2p <= 128 ? n2p : 128;
    const int ntiles = (n2p + T.phi_nt - 1) / T.phi_nt;
    const Mat Aphi = p->ax[1].dense();
    for (int s = 0; s < p->S; ++s) {
        Mat X(n2);
        for (size_t q = 0; q < X.a.size(); ++q) X.a[q] = p->tau * p->d[s] * Aphi.a[q];
        const Mat Ps = phi1_pade(X);
        if (!all_finite(Ps.a)) return SEXPE_ENUMERIC;
        std::vector<float> img;
        for (int t = 0; t < ntiles; ++t) {
            const int r0 = t * T.phi_nt;
            const std::vector<float> part = make_image(std::min(T.phi_nt, n2 - r0), n2, T.phi_nt, n2p,
                                                       [&](int r, int k) { return Ps(r0 + r, k); });
            img.insert(img.end(), part.begin(), part.end());
        }
        const float* dptr = nullptr;
        SX_TRY(upload(p, img, &dptr, st));
        T.Pphi[s] = Image{dptr, T.phi_nt, n2p / kKC, 2LL * T.phi_nt * kKC};
    }
    p->sh3 = tc_sphere_phi_shape(T.phi_nt);
    if (p->sh3.smem_bytes > 227 * 1024 || p->sh3.tmem_cols > 512) return SEXPE_EUNSUPPORTED;
    // theta kernel: output columns split over 1, 2, 4 or 8 CTAs per row tile, each split timed
    // (the splits repeat the first product in every CTA, so the best one depends on the grid)
    std::vector<int> splits;
    std::vector<Image> qimg;
    uint32_t smem_max = 0;
    for (int sp = 1; sp <= 8; sp *= 2) {
        const int nt = n1p / sp;
        if (nt < 16 || nt % 16 != 0 || (sp > 1 && nt * sp != n1p)) continue;
        const TcShape sh = tc_sphere_theta_shape(n1, nt);
        if (sh.smem_bytes > 227 * 1024 || sh.tmem_cols > 512) continue;
        std::vector<float> img;
        for (int t = 0; t < sp; ++t) {
            const int r0 = t * nt;
            const std::vector<float> part = make_image(std::max(0, std::min(nt, n1 - r0)), n1, nt, n1p,
                                                       [&](int r, int k) { return th.V(r0 + r, k); });
            img.insert(img.end(), part.begin(), part.end());
        }
        const float* dptr = nullptr;
        SX_TRY(upload(p, img, &dptr, st));
        splits.push_back(sp);
        qimg.push_back(Image{dptr, nt, n1p / kKC, 2LL * nt * kKC});
        smem_max = std::max(smem_max, sh.smem_bytes);
    }
    if (splits.empty()) return SEXPE_EUNSUPPORTED;
    SX_CUDA(tc_prepare(0, 0));
    SX_CUDA(tc_prepare_sphere(p->sh3.smem_bytes, smem_max));
    p->kernels_per_step = 3;
    SX_TRY(tune_sphere_theta(p, splits, qimg, st));
    SX_TRY(tune_sphere_phi(p, st));
    return tune_stencil(p, st);
}

sexpe_status build_split(sexpe_plan* p, cudaStream_t st) {
    if (p->geometry == SEXPE_SPHERE) return build_split_sphere(p, st);
    const int n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
    if (n1 > 128 || n2 > 256 || (p->ndim == 3 && n3 > 256)) return SEXPE_EUNSUPPORTED;
    SplitTables& T = p->tabs;
    T.geometry = p->geometry;
    T.S = p->S;
    T.n1 = n1;
    T.n2 = n2;
    T.n3 = n3;
    T.npts = p->npts;
    T.tau = (float)p->tau;
    T.tau_d = p->tau;
    SX_TRY(build_rhs_tables<float>(p, &T.rhs, st));
    T.n1q = (n1 + 3) & ~3;
    T.ys = (long long)n3 * n2 * T.n1q;
    SX_TRY(alloc_dev(p, (size_t)p->S * T.ys, &T.Y));
    SX_CUDA(cudaMemsetAsync(T.Y, 0, sizeof(float) * (size_t)p->S * T.ys, st));   // padding columns stay zero
    T.err = p->d_err;
    // theta direction (mode 2): Q_theta, eigenvalues, Hadamard coefficients
    const int n1p = rup16(n1), n2p = rup16(n2), m2 = (n2 + 127) / 128;
    Eigen th = theta_eigen(p->ax[1]);
    SX_TRY(upload_image(p, n2, n2, n2p, n2p, [&](int r, int k) { return th.V(k, r); }, &T.QT, st));
    SX_TRY(upload_image(p, n2, n2, 128 * m2, n2p, [&](int r, int k) { return th.V(r, k); }, &T.Q, st));
    // Phi of the theta direction: phi_1(tau d_s s(i, k) lambda_theta_j'), one FP64 evaluation rounded once.
    const bool ball = p->geometry == SEXPE_BALL;
    const long long plane = (long long)n2 * T.n1q;
    T.had_theta_sp = ball ? (long long)n3 * plane : plane;
    std::vector<float> hc((size_t)p->S * T.had_theta_sp, 0.f);
    for (int s = 0; s < p->S; ++s)
        for (int k = 0; k < (ball ? n3 : 1); ++k)
            for (int jp = 0; jp < n2; ++jp)
                for (int i = 0; i < n1; ++i)
                    hc[(size_t)s * T.had_theta_sp + (size_t)k * plane + (size_t)jp * T.n1q + i] =
                        (float)phi1_scalar(p->tau * p->d[s] * dir_scale(p, 2, i, 0, k) * th.lam[jp]);
    SX_TRY(upload(p, hc, &T.had_theta, st));
    // rho direction (mode 1): phi_1(tau d_s A_rho) per species
    const Mat Arho = p->ax[0].dense();
    for (int s = 0; s < p->S; ++s) {
        Mat X(n1);
        for (size_t q = 0; q < X.a.size(); ++q) X.a[q] = p->tau * p->d[s] * Arho.a[q];
        const Mat Ps = phi1_pade(X);
        if (!all_finite(Ps.a)) return SEXPE_ENUMERIC;
        SX_TRY(upload_image(p, n1, n1, n1p, n1p, [&](int r, int k) { return Ps(r, k); }, &T.P[s], st));
    }
    // mode 3
    if (p->ndim == 3) {
        const int n3p = rup16(n3);
        if (ball) {
            Eigen ph = tridiag_eigen(p->ax[2]);
            if (!all_finite(ph.V.a) || !all_finite(ph.Vinv.a)) return SEXPE_ENUMERIC;
            SX_TRY(upload_image(p, n3, n3, n3p, n3p, [&](int r, int k) { return ph.Vinv(r, k); }, &T.M3a, st));
            SX_TRY(upload_image(p, n3, n3, n3p, n3p, [&](int r, int k) { return ph.V(r, k); }, &T.M3b[0], st));
            std::vector<float> hp((size_t)p->S * n3 * T.n1q, 0.f);
            for (int s = 0; s < p->S; ++s)
                for (int kp = 0; kp < n3; ++kp)
                    for (int i = 0; i < n1; ++i)
                        hp[((size_t)s * n3 + kp) * T.n1q + i] =
                            (float)phi1_scalar(p->tau * p->d[s] * dir_scale(p, 3, i, 0, 0) * ph.lam[kp]);
            SX_TRY(upload(p, hp, &T.had_phi, st));
        } else {
            const Mat Az = p->ax[2].dense();
            for (int s = 0; s < p->S; ++s) {
                Mat X(n3);
                for (size_t q = 0; q < X.a.size(); ++q) X.a[q] = p->tau * p->d[s] * Az.a[q];
                const Mat Pz = phi1_pade(X);
                if (!all_finite(Pz.a)) return SEXPE_ENUMERIC;
                SX_TRY(upload_image(p, n3, n3, n3p, n3p, [&](int r, int k) { return Pz(r, k); }, &T.M3b[s], st));
            }
        }
        p->sh3 = tc_mode3_shape(p->geometry, n1, n2, n3);
    }
    p->shs = tc_slab_shape(n1, n2);
    if (p->shs.smem_bytes > 227 * 1024 || p->sh3.smem_bytes > 227 * 1024) return SEXPE_EUNSUPPORTED;
    if (p->shs.tmem_cols > 512 || (p->ndim == 3 && p->sh3.tmem_cols > 512)) return SEXPE_EUNSUPPORTED;
    SX_CUDA(tc_prepare(p->ndim == 3 ? p->sh3.smem_bytes : 0, p->shs.smem_bytes));
    p->kernels_per_step = p->ndim == 3 ? 3 : 2;
    // the theta-mean coefficient by compensated summation on disks (whose F near the axis is the
    // cancelling theta-Laplacian of the whole field); coupled plans turn it on for both grids
    T.theta_comp = p->geometry == SEXPE_DISK ? 1 : 0;
    return tune_stencil(p, st);
}

// Mode-mu product of all species: out = X x_mu L (L row-major n_mu x n_mu,
// per-species stride L_sp), with optional Hadamard table and fused update.
Gemm64 mode_gemm(const sexpe_plan* p, int mu, const double* L, long long L_sp, const double* X, double* out,
                 const double* had, double* upd) {
    const long long n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
    Gemm64 g{};
    if (mu == 1) {          // Y[p][i'] = sum_i X[p][i] L[i'][i]
        g.R = (int)(n2 * n3); g.C = (int)n1; g.K = (int)n1; g.batch = 1;
        g.A = X; g.a_b = 0; g.a_r = n1; g.a_k = 1; g.A_sp = p->npts;
        g.B = L; g.b_b = 0; g.b_k = 1; g.b_c = n1; g.B_sp = L_sp;
        g.o_b = 0; g.o_r = n1; g.o_c = 1;
    } else if (mu == 2) {   // Y[k][j'][i] = sum_j L[j'][j] X[k][j][i]
        g.R = (int)n2; g.C = (int)n1; g.K = (int)n2; g.batch = (int)n3;
        g.A = L; g.a_b = 0; g.a_r = n2; g.a_k = 1; g.A_sp = L_sp;
        g.B = X; g.b_b = n1 * n2; g.b_k = n1; g.b_c = 1; g.B_sp = p->npts;
        g.o_b = n1 * n2; g.o_r = n1; g.o_c = 1;
    } else {                // Y[k'][q] = sum_k L[k'][k] X[k][q]
        g.R = (int)n3; g.C = (int)(n1 * n2); g.K = (int)n3; g.batch = 1;
        g.A = L; g.a_b = 0; g.a_r = n3; g.a_k = 1; g.A_sp = L_sp;
        g.B = X; g.b_b = 0; g.b_k = n1 * n2; g.b_c = 1; g.B_sp = p->npts;
        g.o_b = 0; g.o_r = n1 * n2; g.o_c = 1;
    }
    g.out = out;
    g.out_sp = p->npts;
    g.had = had;
    g.had_sp = p->npts;
    g.upd = upd;
    g.upd_sp = p->npts;
    g.tau = p->tau;
    return g;
}

// Record the profiling event of the next kernel slot (no-op unless profiling).
cudaError_t prof_mark(sexpe_plan* p, cudaStream_t st) {
    if (!p->profiling || p->prof_steps >= p->prof_max_steps) return cudaSuccess;
    const int per = p->kernels_per_step + 1;
    return cudaEventRecord(p->prof_ev[(size_t)p->prof_steps * per + p->prof_slot++], st);
}

sexpe_status enqueue_step_body(sexpe_plan* p, double* state, cudaStream_t st);

// FP64 direction chain of plan q on F in q->buf64[0], the last product fused with the update of
// `state` (profiling marks recorded on plan `prof`).
sexpe_status enqueue_fp64_chain(sexpe_plan* q, sexpe_plan* prof, double* state, cudaStream_t st) {
    int x = 0;                                  // buffer holding the current operand
    for (const Dir64& d : q->dirs64) {
        const bool last = d.mu == 1;
        const int nmu = q->n[d.mu - 1];
        const int t = (x + 1) % 3, y = (x + 2) % 3;
        if (d.eigen) {
            SX_CUDA(prof_mark(prof, st));
            SX_CUDA(launch_gemm64(mode_gemm(q, d.mu, d.Vinv, 0, q->buf64[x], q->buf64[t], d.had, nullptr), q->S, st));
            SX_CUDA(prof_mark(prof, st));
            SX_CUDA(launch_gemm64(mode_gemm(q, d.mu, d.V, 0, q->buf64[t], q->buf64[y], nullptr,
                                            last ? state : nullptr), q->S, st));
            x = y;
        } else {
            SX_CUDA(prof_mark(prof, st));
            SX_CUDA(launch_gemm64(mode_gemm(q, d.mu, d.P, (long long)nmu * nmu, q->buf64[x], q->buf64[t],
                                            nullptr, last ? state : nullptr), q->S, st));
            x = t;
        }
    }
    return SEXPE_OK;
}

// Split-TF32 products of plan q on the FP32 F in T.Y, the last fused with the update of
// T.state_upd (profiling marks recorded on plan `prof`).
sexpe_status enqueue_split_products(sexpe_plan* q, sexpe_plan* prof, const SplitTables& T, cudaStream_t st) {
    if (q->geometry == SEXPE_SPHERE) {
        SX_CUDA(prof_mark(prof, st));
        SX_CUDA(launch_tc_sphere_phi(T, q->sh3, st));
        SX_CUDA(prof_mark(prof, st));
        SX_CUDA(launch_tc_sphere_theta(T, q->shs, st));
        return SEXPE_OK;
    }
    if (q->ndim == 3) {
        SX_CUDA(prof_mark(prof, st));
        SX_CUDA(launch_tc_mode3(T, q->sh3, st));
    }
    SX_CUDA(prof_mark(prof, st));
    SX_CUDA(launch_tc_slab(T, q->shs, st));
    return SEXPE_OK;
}

// Bulk-surface step (Sections 5.5, 5.6): both stencil+reaction passes, the boundary coupling
// added to their F (explicit at t_n), then each component's own split chain (eqs. ee_ball and
// ee_sphere, or ee_cylinder and ee_disk).  State: [bulk species][surface species].
sexpe_status enqueue_coupled_step(sexpe_plan* p, double* state, cudaStream_t st) {
    sexpe_plan* b = p->sub[0];
    sexpe_plan* s = p->sub[1];
    double* Wb = state;
    double* Ws = state + 2 * b->npts;
    if (p->precision == SEXPE_SPLIT_TF32) {
        SplitTables Tb = b->tabs, Ts = s->tabs;
        Tb.state = Tb.state_upd = Wb;
        Ts.state = Ts.state_upd = Ws;
        Tb.err = Ts.err = p->d_err;                    // bounded-wait timeouts reported by sexpe_synchronize
        // The surface component runs on a second stream beside the bulk one: its stencil beside
        // the bulk stencil, its chain beside the bulk chain; the coupling kernel, which reads and
        // writes both, joins them (profiled steps keep one stream, in the order of their slots).
        const bool fork = p->cpl_stream && !p->profiling;
        cudaStream_t s2 = fork ? p->cpl_stream : st;
        if (fork) {
            SX_CUDA(cudaEventRecord(p->cpl_ev[0], st));
            SX_CUDA(cudaStreamWaitEvent(s2, p->cpl_ev[0], 0));
        }
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_rhs_split(Tb, st));
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_rhs_split(Ts, s2));
        if (fork) {
            SX_CUDA(cudaEventRecord(p->cpl_ev[1], s2));
            SX_CUDA(cudaStreamWaitEvent(st, p->cpl_ev[1], 0));
        }
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_couple_split(p->cpl, Wb, Ws, Tb.Y, Ts.Y, Tb.n1q, Tb.ys, Ts.n1q, Ts.ys, st));
        if (fork) {
            SX_CUDA(cudaEventRecord(p->cpl_ev[2], st));
            SX_CUDA(cudaStreamWaitEvent(s2, p->cpl_ev[2], 0));
        }
        SX_TRY(enqueue_split_products(b, p, Tb, st));
        SX_TRY(enqueue_split_products(s, p, Ts, s2));
        if (fork) {
            SX_CUDA(cudaEventRecord(p->cpl_ev[3], s2));
            SX_CUDA(cudaStreamWaitEvent(st, p->cpl_ev[3], 0));
        }
        return SEXPE_OK;
    }
    SX_CUDA(prof_mark(p, st));
    SX_CUDA(launch_rhs64(b->geometry, b->rhs64, Wb, b->buf64[0], st));
    SX_CUDA(prof_mark(p, st));
    SX_CUDA(launch_rhs64(s->geometry, s->rhs64, Ws, s->buf64[0], st));
    SX_CUDA(prof_mark(p, st));
    SX_CUDA(launch_couple64(p->cpl, Wb, Ws, b->buf64[0], s->buf64[0], st));
    SX_TRY(enqueue_fp64_chain(b, p, Wb, st));
    SX_TRY(enqueue_fp64_chain(s, p, Ws, st));
    return SEXPE_OK;
}

sexpe_status enqueue_step(sexpe_plan* p, double* state, cudaStream_t st) {
    p->prof_slot = 0;
    SX_TRY(enqueue_step_body(p, state, st));
    if (p->profiling && p->prof_steps < p->prof_max_steps) {
        SX_CUDA(prof_mark(p, st));
        ++p->prof_steps;
    }
    return SEXPE_OK;
}

sexpe_status enqueue_step_body(sexpe_plan* p, double* state, cudaStream_t st) {
    if (p->batch) {
        BatchTables B = p->btab;
        B.W_in = p->bparity ? p->bstate : state;
        B.W_out = p->bparity ? state : p->bstate;
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_tc_batch(B, p->bsh, p->batch_grid, st));
        p->bparity ^= 1;
        return SEXPE_OK;
    }
    if (p->precision == SEXPE_UNSPLIT_FP64) {
        // w_s += tau P_s F_s: one dense matrix-vector product per species, update fused
        const long long N = p->npts;
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_rhs64(p->geometry, p->rhs64, state, p->buf64[0], st));
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_matvec64(p->unsplit_P, p->buf64[0], state, (int)N, p->S, p->tau, st));
        if (p->d_step) SX_CUDA(launch_tick(p->d_step, st));
        return SEXPE_OK;
    }
    if (p->coupled) return enqueue_coupled_step(p, state, st);
    if (p->precision == SEXPE_FP64) {
        SX_CUDA(prof_mark(p, st));
        SX_CUDA(launch_rhs64(p->geometry, p->rhs64, state, p->buf64[0], st));
        SX_TRY(enqueue_fp64_chain(p, p, state, st));
        if (p->d_step) SX_CUDA(launch_tick(p->d_step, st));
        return SEXPE_OK;
    }
    SplitTables T = p->tabs;
    T.state = state;
    T.state_upd = state;
    SX_CUDA(prof_mark(p, st));
    SX_CUDA(launch_rhs_split(T, st));
    SX_TRY(enqueue_split_products(p, p, T, st));
    if (p->d_step && p->geometry != SEXPE_SPHERE) SX_CUDA(launch_tick(p->d_step, st));
    return SEXPE_OK;
}

// FP64 elements of a plan's whole state.
long long state_elems(const sexpe_plan* p) {
    if (p->batch) return p->inst_off.back();
    if (p->coupled) return 2 * (p->sub[0]->npts + p->sub[1]->npts);
    return (long long)p->S * p->npts;
}

sexpe_status validate(const sexpe_grid* g, const sexpe_species* sp, double tau, int32_t precision) {
    if (!g || !sp) return SEXPE_EINVAL;
    if (g->geometry < SEXPE_DISK || g->geometry > SEXPE_CYLINDER) return SEXPE_EINVAL;
    if (precision != SEXPE_FP64 && precision != SEXPE_SPLIT_TF32 && precision != SEXPE_UNSPLIT_FP64) return SEXPE_EINVAL;
    if (!(tau > 0.0) || !std::isfinite(tau)) return SEXPE_EINVAL;
    const int ndim = (g->geometry == SEXPE_BALL || g->geometry == SEXPE_CYLINDER) ? 3 : 2;
    for (int m = 0; m < ndim; ++m)
        if (g->n[m] < 3 || g->n[m] > kMaxN) return SEXPE_EINVAL;
    if (g->geometry != SEXPE_SPHERE && !(g->rho_star > 0.0 && std::isfinite(g->rho_star))) return SEXPE_EINVAL;
    if (g->geometry == SEXPE_CYLINDER) {
        if (!(g->z_star > 0.0 && std::isfinite(g->z_star))) return SEXPE_EINVAL;
        if (g->z_bc != SEXPE_Z_NEUMANN && g->z_bc != SEXPE_Z_PAPER) return SEXPE_EINVAL;
    }
    if (sp->n_species < 1 || sp->n_species > kMaxSpecies || !sp->d_host) return SEXPE_EINVAL;
    for (int s = 0; s < sp->n_species; ++s)
        if (!(sp->d_host[s] > 0.0) || !std::isfinite(sp->d_host[s])) return SEXPE_EINVAL;
    if (sp->n_params < 0 || sp->n_params > 16 || (sp->n_params > 0 && !sp->params_host)) return SEXPE_EINVAL;
    if (g->rho_op != 0 && g->rho_op != 1) return SEXPE_EINVAL;
    if (g->rho_op == 1 && (g->geometry != SEXPE_DISK || !(g->lambda > -3.0 && g->lambda < 1.0))) return SEXPE_EINVAL;
    if (sp->offset_host)
        for (int s = 0; s < sp->n_species; ++s)
            if (!std::isfinite(sp->offset_host[s])) return SEXPE_EINVAL;
    switch (sp->reaction) {
    case SEXPE_REACTION_NONE: break;
    case SEXPE_SCHNAKENBERG: if (sp->n_species != 2 || sp->n_params != 3) return SEXPE_EINVAL; break;
    case SEXPE_GRAY_SCOTT: if (sp->n_species != 2 || sp->n_params != 2) return SEXPE_EINVAL; break;
    case SEXPE_LINEAR_CUBIC:
    case SEXPE_LINEAR:
        if (sp->n_params != sp->n_species * sp->n_species) return SEXPE_EINVAL;
        break;
    case SEXPE_BVAM: if (sp->n_species != 2 || sp->n_params != 5 || sp->params_host[3] == 0.0) return SEXPE_EINVAL; break;
    case SEXPE_BVAM_MANUFACTURED:
        if (sp->n_species != 2 || sp->n_params != 5 || sp->params_host[3] == 0.0) return SEXPE_EINVAL;
        if (g->geometry != SEXPE_DISK) return SEXPE_EINVAL;
        break;
    default: return SEXPE_EINVAL;
    }
    for (int q = 0; q < sp->n_params; ++q)
        if (!std::isfinite(sp->params_host[q])) return SEXPE_EINVAL;
    return SEXPE_OK;
}

void free_profile(sexpe_plan* p) {
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    p->profiling = false;
    p->prof_steps = p->prof_max_steps = 0;
}

void free_plan(sexpe_plan* p) {
    if (!p) return;
    free_plan(p->sub[0]);
    free_plan(p->sub[1]);
    free_profile(p);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->sadj_stream) {
        cudaStreamSynchronize(p->sadj_stream);
        cudaStreamDestroy(p->sadj_stream);
    }
    for (int b = 0; b < 2; ++b) {
        if (p->sadj_ev_replayed[b]) cudaEventDestroy(p->sadj_ev_replayed[b]);
        if (p->sadj_ev_swept[b]) cudaEventDestroy(p->sadj_ev_swept[b]);
    }
    if (p->cpl_stream) {
        cudaStreamSynchronize(p->cpl_stream);
        cudaStreamDestroy(p->cpl_stream);
    }
    for (cudaEvent_t e : p->cpl_ev)
        if (e) cudaEventDestroy(e);
    for (void* a : p->allocs) cudaFree(a);
    if (p->h_err) cudaFreeHost(p->h_err);
    delete p;
}

// The plan's device error word (zeroed on `st`) and its pinned host copy.
static sexpe_status alloc_err_word(sexpe_plan* p, cudaStream_t st) {
    SX_TRY(alloc_dev(p, 4, &p->d_err));
    SX_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int) * 4, st));
    if (cudaHostAlloc((void**)&p->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        p->h_err = nullptr;       // sexpe_synchronize then reads the word with a blocking copy
    }
    return SEXPE_OK;
}

sexpe_status build_plan(sexpe_plan* p, const sexpe_grid* g, const sexpe_species* sp, double tau, int32_t precision,
                        cudaStream_t st) {
    SX_CUDA(cudaGetDevice(&p->device));
    p->geometry = g->geometry;
    p->precision = precision;
    p->S = sp->n_species;
    p->ndim = (g->geometry == SEXPE_BALL || g->geometry == SEXPE_CYLINDER) ? 3 : 2;
    for (int m = 0; m < 3; ++m) p->n[m] = m < p->ndim ? g->n[m] : 1;
    p->npts = (long long)p->n[0] * p->n[1] * p->n[2];
    p->tau = tau;
    p->d.assign(sp->d_host, sp->d_host + sp->n_species);
    p->params.assign(sp->params_host, sp->params_host + sp->n_params);
    p->reaction = sp->reaction;
    if (sp->offset_host) p->offset.assign(sp->offset_host, sp->offset_host + sp->n_species);
    switch (g->geometry) {
    case SEXPE_DISK:
        if (g->rho_op == 1) {
            p->ax[0] = build_axis(AX_RHO_LAMBDA, p->n[0], g->rho_star, g->lambda);
            p->rho_pow = -2.0 - g->lambda;
        } else {
            p->ax[0] = build_axis(AX_RHO2, p->n[0], g->rho_star);
        }
        p->ax[1] = build_axis(AX_THETA, p->n[1], 0.0);
        break;
    case SEXPE_SPHERE:
        p->ax[0] = build_axis(AX_THETA, p->n[0], 0.0);
        p->ax[1] = build_axis(AX_PHI, p->n[1], 0.0);
        break;
    case SEXPE_BALL:
        p->ax[0] = build_axis(AX_RHO3, p->n[0], g->rho_star);
        p->ax[1] = build_axis(AX_THETA, p->n[1], 0.0);
        p->ax[2] = build_axis(AX_PHI, p->n[2], 0.0);
        break;
    default:
        p->ax[0] = build_axis(AX_RHO2, p->n[0], g->rho_star);
        p->ax[1] = build_axis(AX_THETA, p->n[1], 0.0);
        p->ax[2] = build_axis(g->z_bc == SEXPE_Z_PAPER ? AX_Z_PAPER : AX_Z_NEUMANN, p->n[2], g->z_star);
        break;
    }
    SX_TRY(alloc_err_word(p, st));
    SX_TRY(alloc_dev(p, (size_t)p->S * p->npts, &p->d_host_state));
    if (precision == SEXPE_FP64) SX_TRY(build_fp64(p, st));
    else if (precision == SEXPE_UNSPLIT_FP64) SX_TRY(build_unsplit(p, st));
    else SX_TRY(build_split(p, st));
    SX_CUDA(cudaStreamSynchronize(st));   // host vectors of the uploads go out of scope
    return SEXPE_OK;
}

// ---------------------------------------------------------------------------
// Batched independent disks.

// Candidate phase-1 tile heights of the batch kernel and launches timed per candidate.
const std::vector<int> kBatchTileLines = {8, 16, 32};
constexpr int kBatchTuneReps = 3;

sexpe_status build_batch(sexpe_plan* p, int count, const sexpe_grid* grids, const sexpe_species* species,
                         double tau, cudaStream_t st) {
    p->batch = true;
    p->n_instances = count;
    p->geometry = SEXPE_DISK;
    p->precision = SEXPE_SPLIT_TF32;
    p->S = 2;
    p->ndim = 2;
    p->tau = tau;
    // one float pool for every per-instance table, uploaded once
    std::vector<float> pool;
    auto put = [&](const std::vector<float>& v) {
        while (pool.size() % 64) pool.push_back(0.f);            // 256-byte alignment of every table
        const size_t off = pool.size();
        pool.insert(pool.end(), v.begin(), v.end());
        return off;
    };
    struct Offs { size_t qt, q, p0, p1, had, rl, ru, rr, tl, tu, tr, dr; };
    std::vector<Offs> offs(count);
    std::vector<BatchInstance> inst(count);
    p->inst_off.assign(count + 1, 0);
    long long f_total = 0;
    int max_n1 = 0, max_n2 = 0;
    uint32_t tmem_cols = 32;
    for (int q = 0; q < count; ++q) {
        const int n1 = grids[q].n[0], n2 = grids[q].n[1];
        max_n1 = std::max(max_n1, n1);
        max_n2 = std::max(max_n2, n2);
        tmem_cols = std::max(tmem_cols, slab_tmem_cols(n1, n2));
        const Axis ar = build_axis(AX_RHO2, n1, grids[q].rho_star);
        const Axis at = build_axis(AX_THETA, n2, 0.0);
        const Eigen th = theta_eigen(at);
        const int n1p = rup16(n1), n2p = rup16(n2), m2 = (n2 + 127) / 128;
        Offs& o = offs[q];
        o.qt = put(make_image(n2, n2, n2p, n2p, [&](int r, int k) { return th.V(k, r); }));
        o.q = put(make_image(n2, n2, 128 * m2, n2p, [&](int r, int k) { return th.V(r, k); }));
        const double* dsp = species[q].d_host;
        const Mat A = ar.dense();
        size_t pofs[2];
        for (int sp = 0; sp < 2; ++sp) {
            Mat X(n1);
            for (size_t t = 0; t < X.a.size(); ++t) X.a[t] = tau * dsp[sp] * A.a[t];
            const Mat Ps = phi1_pade(X);
            if (!all_finite(Ps.a)) return SEXPE_ENUMERIC;
            pofs[sp] = put(make_image(n1, n1, n1p, n1p, [&](int r, int k) { return Ps(r, k); }));
        }
        o.p0 = pofs[0];
        o.p1 = pofs[1];
        const int n1q = (n1 + 3) & ~3;
        std::vector<float> had((size_t)2 * n1q * n2, 0.f);
        for (int sp = 0; sp < 2; ++sp)
            for (int jp = 0; jp < n2; ++jp)
                for (int i = 0; i < n1; ++i)
                    had[(size_t)sp * n1q * n2 + (size_t)jp * n1q + i] =
                        (float)phi1_scalar(tau * dsp[sp] * th.lam[jp] / (ar.pts[i] * ar.pts[i]));
        o.had = put(had);
        auto axis_f = [&](const Axis& a, size_t& lo, size_t& up, size_t& rs) {
            std::vector<float> vl(a.n), vu(a.n), vr(a.n);
            for (int r = 0; r < a.n; ++r) {
                vl[r] = (float)a.lower[r];
                vu[r] = (float)a.upper[r];
                vr[r] = 0.f;   // every row of A_rho2 and A_theta sums to zero
            }
            lo = put(vl);
            up = put(vu);
            rs = put(vr);
        };
        axis_f(ar, o.rl, o.ru, o.rr);
        axis_f(at, o.tl, o.tu, o.tr);
        std::vector<float> dr(n1);
        for (int i = 0; i < n1; ++i) dr[i] = (float)(1.0 / (ar.pts[i] * ar.pts[i]));
        o.dr = put(dr);
        BatchInstance& I = inst[q];
        I.n1 = n1;
        I.n2 = n2;
        I.w_off = p->inst_off[q];
        I.d[0] = (float)dsp[0];
        I.d[1] = (float)dsp[1];
        I.reac.kind = species[q].reaction;
        I.reac.S = 2;
        for (int t = 0; t < 16; ++t)
            I.reac.p[t] = t < species[q].n_params ? (float)species[q].params_host[t] : 0.f;
        I.QT = Image{nullptr, n2p, n2p / kKC, 2LL * n2p * kKC};
        I.Q = Image{nullptr, 128 * m2, n2p / kKC, 2LL * 128 * m2 * kKC};
        I.P[0] = Image{nullptr, n1p, n1p / kKC, 2LL * n1p * kKC};
        I.P[1] = I.P[0];
        I.ax_rho.n = n1;
        I.ax_rho.periodic = 0;
        I.ax_theta.n = n2;
        I.ax_theta.periodic = 1;
        p->inst_off[q + 1] = p->inst_off[q] + 2LL * n1 * n2;
        I.f_off = f_total;
        f_total += 2LL * n2 * ((n1 + 3) & ~3);
    }
    const float* base = nullptr;
    SX_TRY(upload(p, pool, &base, st));
    for (int q = 0; q < count; ++q) {
        BatchInstance& I = inst[q];
        const Offs& o = offs[q];
        I.QT.ptr = base + o.qt;
        I.Q.ptr = base + o.q;
        I.P[0].ptr = base + o.p0;
        I.P[1].ptr = base + o.p1;
        I.had = base + o.had;
        I.ax_rho.lower = base + o.rl;
        I.ax_rho.upper = base + o.ru;
        I.ax_rho.rs = base + o.rr;
        I.ax_theta.lower = base + o.tl;
        I.ax_theta.upper = base + o.tu;
        I.ax_theta.rs = base + o.tr;
        I.Dr = base + o.dr;
    }
    // Work lists of (instance, species) chain items, two orders the setup times against each other:
    // 0 = longest item first (LPT over items); 1 = instances longest first with their two species
    // adjacent (the pair shares the instance's Q images in L2).
    auto cost = [&](int q) {
        const double n1 = inst[q].n1, n2 = inst[q].n2;
        return n1 * n2 * (2.0 * n2 + n1);
    };
    std::vector<int2> items;
    for (int q = 0; q < count; ++q)
        for (int sp = 0; sp < 2; ++sp) items.push_back(make_int2(q, sp));
    std::stable_sort(items.begin(), items.end(), [&](const int2& a, const int2& b) { return cost(a.x) > cost(b.x); });
    std::vector<int> order(count);
    for (int q = 0; q < count; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<int2> items_pairs;
    for (int q : order) {
        items_pairs.push_back(make_int2(q, 0));
        items_pairs.push_back(make_int2(q, 1));
    }
    // the instance descriptors go up as raw bytes
    std::vector<char> ibytes(sizeof(BatchInstance) * count);
    std::memcpy(ibytes.data(), inst.data(), ibytes.size());
    const char* dinst = nullptr;
    SX_TRY(upload(p, ibytes, &dinst, st));
    const int2* ditems[2] = {nullptr, nullptr};
    SX_TRY(upload(p, items, &ditems[0], st));
    SX_TRY(upload(p, items_pairs, &ditems[1], st));
    // phase-1 stencil tiles of tj theta-lines of one instance each, one list per candidate tj
    std::vector<const int2*> dftiles(kBatchTileLines.size(), nullptr);
    std::vector<int> nftiles(kBatchTileLines.size(), 0);
    for (size_t c = 0; c < kBatchTileLines.size(); ++c) {
        std::vector<int2> ftiles;
        for (int q = 0; q < count; ++q)
            for (int j0 = 0; j0 < inst[q].n2; j0 += kBatchTileLines[c]) ftiles.push_back(make_int2(q, j0));
        SX_TRY(upload(p, ftiles, &dftiles[c], st));
        nftiles[c] = (int)ftiles.size();
    }
    float* dF = nullptr;
    SX_TRY(alloc_dev(p, (size_t)f_total, &dF));
    SX_CUDA(cudaMemsetAsync(dF, 0, sizeof(float) * (size_t)f_total, st));   // padding columns stay zero
    SX_TRY(alloc_err_word(p, st));
    int* counter = nullptr;
    SX_TRY(alloc_dev(p, 4, &counter));
    SX_TRY(alloc_dev(p, (size_t)p->inst_off.back(), &p->bstate));
    SX_TRY(alloc_dev(p, (size_t)p->inst_off.back(), &p->d_host_state));
    p->btab.inst = reinterpret_cast<const BatchInstance*>(dinst);
    p->btab.n_items = (int)items.size();
    p->btab.counter = counter;
    p->btab.F = dF;
    p->btab.tau = (float)tau;
    p->btab.err = p->d_err;
    // Autotuner: time every (ring configuration, phase-1 tile height, work-list order) on the
    // plan's own buffers (a zero state; the arithmetic is data-independent) and keep the fastest.
    TcShape shapes[16];
    const int max_tj = *std::max_element(kBatchTileLines.begin(), kBatchTileLines.end());
    p->btab.tile_f2 = (max_tj + 2) * max_n1 * 2;
    const int nsh = tc_batch_shapes(max_n1, max_n2, tmem_cols, max_tj, shapes, 16);
    if (nsh < 1 || shapes[0].tmem_cols > 512) return SEXPE_EUNSUPPORTED;
    uint32_t smem_max = 0;
    for (int c = 0; c < nsh; ++c) smem_max = std::max(smem_max, shapes[c].smem_bytes);
    SX_CUDA(tc_prepare_batch(smem_max));
    SX_CUDA(cudaMemsetAsync(p->bstate, 0, sizeof(double) * (size_t)p->inst_off.back(), st));
    cudaEvent_t ev[2];
    SX_CUDA(cudaEventCreate(&ev[0]));
    SX_CUDA(cudaEventCreate(&ev[1]));
    float best = 1e30f;
    sexpe_status ts = SEXPE_OK;
    for (int c = 0; c < nsh && ts == SEXPE_OK; ++c) {
        const int grid = batch_grid(shapes[c]);
        if (grid < 1) continue;
        for (size_t t = 0; t < kBatchTileLines.size() && ts == SEXPE_OK; ++t)
            for (int o = 0; o < 2 && ts == SEXPE_OK; ++o) {
                BatchTables B = p->btab;
                B.items = ditems[o];
                B.ftiles = dftiles[t];
                B.n_ftiles = nftiles[t];
                B.tj = kBatchTileLines[t];
                B.W_in = p->bstate;
                B.W_out = p->d_host_state;
                float ms = 0.f;
                cudaError_t e = launch_tc_batch(B, shapes[c], grid, st);                   // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
                for (int r = 0; r < kBatchTuneReps && e == cudaSuccess; ++r) e = launch_tc_batch(B, shapes[c], grid, st);
                if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
                if (e != cudaSuccess) {
                    ts = cuda_status(e);
                    break;
                }
                ms /= kBatchTuneReps;
                if (ms < best) {
                    best = ms;
                    p->bsh = shapes[c];
                    p->batch_grid = grid;
                    p->btab.items = ditems[o];
                    p->btab.ftiles = dftiles[t];
                    p->btab.n_ftiles = nftiles[t];
                    p->btab.tj = kBatchTileLines[t];
                    p->batch_order = o;
                }
            }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    SX_TRY(ts);
    if (best >= 1e30f) return SEXPE_EUNSUPPORTED;
    p->batch_step_us = best * 1e3f;
    // the timing runs left a timeout flag only if a bounded wait ran out: report it now
    int herr = 0;
    SX_CUDA(cudaMemcpyAsync(&herr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SX_CUDA(cudaStreamSynchronize(st));
    if (herr != 0) return SEXPE_ETIMEOUT;
    p->npts = p->inst_off.back() / 2;
    p->n[0] = max_n1;
    p->n[1] = max_n2;
    p->kernels_per_step = 1;
    SX_CUDA(cudaStreamSynchronize(st));
    return SEXPE_OK;
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the FP64 step (see include/sexpe.h, sexpe_adjoint).

Mat transpose(const Mat& A) {
    Mat T(A.n);
    for (int r = 0; r < A.n; ++r)
        for (int c = 0; c < A.n; ++c) T(c, r) = A(r, c);
    return T;
}

constexpr int kAdjBuffers = 12;   // F, X1..X3, H0..H2, Y0, Y1, HA, Z, MU

sexpe_status build_adjoint(sexpe_plan* p, cudaStream_t st) {
    if (!p->adj.empty()) return SEXPE_OK;
    // M^T: same off-diagonals, the full diagonal a_l in the rs slot
    p->adj_diag = p->rhs64;
    for (int m = 0; m < p->ndim; ++m) {
        const double* dg = nullptr;
        SX_TRY(upload(p, p->ax[m].diag, &dg, st));
        p->adj_diag.ax[m].rs = dg;
    }
    std::vector<DirAdj> adj;
    for (const Dir64& d : p->dirs64) {
        const Axis& a = p->ax[d.mu - 1];
        const int n = a.n;
        DirAdj q;
        if (d.eigen) {
            const Eigen e = a.periodic ? theta_eigen(a) : tridiag_eigen(a);
            SX_TRY(upload(p, transpose(e.V).a, &q.VT, st));
            SX_TRY(upload(p, transpose(e.Vinv).a, &q.VinvT, st));
            // weight Phi' / Phi^2 with Phi' = d Phi / d d_s = tau s lambda phi_1'(tau d_s s lambda)
            std::vector<double> wt((size_t)p->S * p->npts);
            for (int s = 0; s < p->S; ++s)
                for (int k = 0; k < p->n[2]; ++k)
                    for (int j = 0; j < p->n[1]; ++j)
                        for (int i = 0; i < p->n[0]; ++i) {
                            const int m = d.mu == 1 ? i : (d.mu == 2 ? j : k);
                            const double sl = dir_scale(p, d.mu, i, j, k) * e.lam[m];
                            const double x = p->tau * p->d[s] * sl;
                            const double ph = phi1_scalar(x);
                            wt[(size_t)s * p->npts + i + (size_t)p->n[0] * (j + (size_t)p->n[1] * k)] =
                                p->tau * sl * dphi1_scalar(x) / (ph * ph);
                        }
            if (!all_finite(wt)) return SEXPE_ENUMERIC;
            SX_TRY(upload(p, wt, &q.dhad, st));
        } else {
            const Mat A = a.dense();
            const Eigen e = tridiag_eigen(a);
            std::vector<double> PT((size_t)p->S * n * n), dP((size_t)p->S * n * n);
            for (int s = 0; s < p->S; ++s) {
                Mat X(n);
                for (size_t t = 0; t < X.a.size(); ++t) X.a[t] = p->tau * p->d[s] * A.a[t];
                const Mat Pt = transpose(phi1_pade(X));
                std::memcpy(&PT[(size_t)s * n * n], Pt.a.data(), sizeof(double) * n * n);
                // d phi_1(tau d A)/d d = V diag(tau lambda phi_1'(tau d lambda)) V^{-1}
                std::vector<double> wm(n);
                for (int m = 0; m < n; ++m) wm[m] = p->tau * e.lam[m] * dphi1_scalar(p->tau * p->d[s] * e.lam[m]);
                double* out = &dP[(size_t)s * n * n];
                for (int r = 0; r < n; ++r) {
                    double* row = out + (size_t)r * n;
                    for (int c = 0; c < n; ++c) row[c] = 0.0;
                    for (int m = 0; m < n; ++m) {
                        const double vm = e.V(r, m) * wm[m];
                        const double* vi = &e.Vinv.a[(size_t)m * n];
                        for (int c = 0; c < n; ++c) row[c] += vm * vi[c];
                    }
                }
            }
            if (!all_finite(PT) || !all_finite(dP)) return SEXPE_ENUMERIC;
            SX_TRY(upload(p, PT, &q.PT, st));
            SX_TRY(upload(p, dP, &q.dP, st));
        }
        adj.push_back(q);
    }
    SX_TRY(alloc_dev(p, (size_t)kAdjBuffers * p->S * p->npts, &p->adj_buf));
    SX_TRY(alloc_dev(p, 32, &p->adj_red));
    SX_CUDA(cudaStreamSynchronize(st));
    p->adj = adj;
    return SEXPE_OK;
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the split-TF32 sphere step (eq. ee_sphere): the step is
//     W_{n+1} = W_n + tau P_theta P_phi F(W_n),   P_theta = Q diag(Phi) Q^T,  P_phi = phi_1(tau d A_phi)
// so, with lambda = dL/dW_{n+1} and mu = tau P^T lambda = P_phi^T (tau P_theta lambda) (P_theta is
// symmetric: Q orthogonal, Phi diagonal),
//     dL/dW_n = lambda + (d M + J_g(W_n))^T mu,
//     dL/dd_s += <mu_s, M w_s> + tau <lambda_s, (dP_theta/dd_s) P_phi F_s> + tau <P_theta lambda_s, (dP_phi/dd_s) F_s>,
// dP_theta/dd_s = Q diag(tau s lambda_theta phi_1'(tau d_s s lambda_theta)) Q^T (symmetric),
// dP_phi/dd_s = V diag(tau lambda_phi phi_1'(tau d_s lambda_phi)) V^{-1}, phi_1' = phi_1 - phi_2.
// Every product runs on the forward's tensor-core kernels (split TF32, FP32 accumulation) with
// the transposed / differentiated operand images; lambda and the parameter sums stay FP64.

// FP32 tables of M^T in difference form: per axis the transpose's off-diagonals,
// (A^T)_{r,r-1} = A_{r-1,r} and (A^T)_{r,r+1} = A_{r+1,r} (with the periodic wrap), and its column
// sums in the rs slot (zero where they vanish, as for the symmetric circulant A_theta); the
// diagonal factors, diffusion and reaction as in the forward tables `base`.
sexpe_status build_transposed_tables_f32(sexpe_plan* p, const RhsTables<float>& base, RhsTables<float>* out,
                                         cudaStream_t st) {
    *out = base;
    for (int m = 0; m < p->ndim; ++m) {
        const Axis& a = p->ax[m];
        const int n = a.n;
        std::vector<float> lo(n), up(n), cs(n);
        for (int r = 0; r < n; ++r) {
            const bool has_m = r > 0 || a.periodic, has_p = r < n - 1 || a.periodic;
            const double l = has_m ? a.upper[(r + n - 1) % n] : 0.0;
            const double u = has_p ? a.lower[(r + 1) % n] : 0.0;
            const double sum = a.diag[r] + l + u;
            lo[r] = (float)l;
            up[r] = (float)u;
            cs[r] = (float)(std::fabs(sum) <= 1e-9 * std::fabs(a.diag[r]) ? 0.0 : sum);
        }
        StencilAxis<float> sa{};
        SX_TRY(upload(p, lo, &sa.lower, st));
        SX_TRY(upload(p, up, &sa.upper, st));
        SX_TRY(upload(p, cs, &sa.rs, st));
        sa.n = n;
        sa.periodic = a.periodic ? 1 : 0;
        out->ax[m] = sa;
    }
    return SEXPE_OK;
}

sexpe_status build_adjoint_split(sexpe_plan* p, cudaStream_t st) {
    if (p->sadj_built) return SEXPE_OK;
    SX_TRY(build_transposed_tables_f32(p, p->tabs.rhs, &p->sadj_rhsT, st));
    SX_TRY(build_rhs_tables<double>(p, &p->rhs64, st));
    p->adj_diag = p->rhs64;                      // M^T: same off-diagonals, the full diagonal in rs
    for (int m = 0; m < p->ndim; ++m) {
        const double* dg = nullptr;
        SX_TRY(upload(p, p->ax[m].diag, &dg, st));
        p->adj_diag.ax[m].rs = dg;
    }
    SplitTables& T = p->tabs;
    const int n1 = p->n[0], n2 = p->n[1], n2p = rup16(n2);
    const int ntiles = (n2p + T.phi_nt - 1) / T.phi_nt;
    const Mat Aphi = p->ax[1].dense();
    const Eigen e = tridiag_eigen(p->ax[1]);
    for (int s = 0; s < p->S; ++s) {
        Mat X(n2);
        for (size_t q = 0; q < X.a.size(); ++q) X.a[q] = p->tau * p->d[s] * Aphi.a[q];
        const Mat Ps = phi1_pade(X);
        Mat dP(n2);
        for (int r = 0; r < n2; ++r)
            for (int c = 0; c < n2; ++c) {
                double acc = 0.0;
                for (int m = 0; m < n2; ++m)
                    acc += e.V(r, m) * p->tau * e.lam[m] * dphi1_scalar(p->tau * p->d[s] * e.lam[m]) * e.Vinv(m, c);
                dP(r, c) = acc;
            }
        if (!all_finite(Ps.a) || !all_finite(dP.a)) return SEXPE_ENUMERIC;
        std::vector<float> imgT, imgD;
        for (int t = 0; t < ntiles; ++t) {
            const int r0 = t * T.phi_nt, rows = std::min(T.phi_nt, n2 - r0);
            const std::vector<float> a = make_image(rows, n2, T.phi_nt, n2p, [&](int r, int k) { return Ps(k, r0 + r); });
            const std::vector<float> b = make_image(rows, n2, T.phi_nt, n2p, [&](int r, int k) { return dP(r0 + r, k); });
            imgT.insert(imgT.end(), a.begin(), a.end());
            imgD.insert(imgD.end(), b.begin(), b.end());
        }
        const float* pt = nullptr;
        const float* pd = nullptr;
        SX_TRY(upload(p, imgT, &pt, st));
        SX_TRY(upload(p, imgD, &pd, st));
        p->sadj_PphiT[s] = Image{pt, T.phi_nt, n2p / kKC, 2LL * T.phi_nt * kKC};
        p->sadj_dPphi[s] = Image{pd, T.phi_nt, n2p / kKC, 2LL * T.phi_nt * kKC};
    }
    const Eigen th = theta_eigen(p->ax[0]);
    std::vector<float> hd((size_t)p->S * T.ys, 0.f);
    for (int s = 0; s < p->S; ++s)
        for (int j = 0; j < n2; ++j)
            for (int ip = 0; ip < n1; ++ip) {
                const double sl = dir_scale(p, 1, 0, j, 0) * th.lam[ip];
                hd[(size_t)s * T.ys + (size_t)j * T.n1q + ip] = (float)(p->tau * sl * dphi1_scalar(p->tau * p->d[s] * sl));
            }
    if (!all_finite(hd)) return SEXPE_ENUMERIC;
    SX_TRY(upload(p, hd, &p->sadj_had_d, st));
    const size_t yf = (size_t)p->S * T.ys, e64 = (size_t)p->S * p->npts;
    SX_TRY(alloc_dev(p, yf, &p->sadj_Yl));
    SX_TRY(alloc_dev(p, yf, &p->sadj_Y3));
    SX_TRY(alloc_dev(p, yf, &p->sadj_Ymu));
    SX_CUDA(cudaMemsetAsync(p->sadj_Yl, 0, sizeof(float) * yf, st));    // padding columns stay zero
    SX_CUDA(cudaMemsetAsync(p->sadj_Y3, 0, sizeof(float) * yf, st));
    SX_CUDA(cudaMemsetAsync(p->sadj_Ymu, 0, sizeof(float) * yf, st));
    SX_TRY(alloc_dev(p, e64, &p->sadj_T64[0]));
    SX_TRY(alloc_dev(p, e64, &p->sadj_T64[1]));
    SX_TRY(alloc_dev(p, e64, &p->sadj_MU));
    if (!p->adj_red) SX_TRY(alloc_dev(p, 32, &p->adj_red));
    // The merged adjoint theta kernel holds three accumulators (n1p + 2 nt columns): time it at every
    // column split the setup built whose shape fits, on the (zeroed) work buffers, and keep the fastest.
    SX_CUDA(cudaMemsetAsync(p->sadj_T64[0], 0, sizeof(double) * 32, st));
    float* zchain = p->sadj_Y3;                 // zeroed chain buffer: lambda, P_phi F, dP_phi F inputs
    cudaEvent_t ev[2];
    SX_CUDA(cudaEventCreate(&ev[0]));
    SX_CUDA(cudaEventCreate(&ev[1]));
    float best = 1e30f;
    cudaError_t te = cudaSuccess;
    for (size_t c = 0; c < p->th_splits.size() && te == cudaSuccess; ++c) {
        const int nt = rup16(n1) / p->th_splits[c];
        const TcShape sh = tc_sphere_theta_adj_shape(n1, nt);
        if (sh.tmem_cols > 512 || sh.smem_bytes > 227u * 1024u) continue;
        SplitTables Ta = T;
        Ta.th_nt = nt;
        Ta.Qsph = p->th_imgs[c];
        const SphereAdjArgs A{zchain, p->sadj_had_d, p->sadj_Ymu, zchain, zchain, p->sadj_T64[0]};
        float ms = 0.f;
        te = launch_tc_sphere_theta_adj(Ta, sh, A, st);
        if (te == cudaSuccess) te = cudaEventRecord(ev[0], st);
        for (int r = 0; r < 3 && te == cudaSuccess; ++r) te = launch_tc_sphere_theta_adj(Ta, sh, A, st);
        if (te == cudaSuccess) te = cudaEventRecord(ev[1], st);
        if (te == cudaSuccess) te = cudaEventSynchronize(ev[1]);
        if (te == cudaSuccess) te = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (te == cudaSuccess && ms < best) {
            best = ms;
            p->sadj_shape = sh;
            p->sadj_nt = nt;
            p->sadj_Q = p->th_imgs[c];
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    SX_CUDA(te);
    p->sadj_merged = best < 1e30f;
    SX_CUDA(cudaMemsetAsync(p->sadj_Ymu, 0, sizeof(float) * yf, st));
    SX_CUDA(cudaStreamSynchronize(st));
    p->sadj_built = true;
    return SEXPE_OK;
}

// The forward quantities an adjoint step of the split sphere plan reads at the state W: F into
// Y (chain layout), P_phi F into Y2 and (dP_phi/dd) F into Y3; with `upd`, the theta kernel then
// completes the forward step into upd (which holds a copy of W), as sexpe_step would.
sexpe_status split_forward_parts(sexpe_plan* p, const double* W, float* Y, float* Y2, float* Y3, double* upd,
                                 cudaStream_t st) {
    SplitTables T = p->tabs;
    T.state = W;
    T.Y = Y;
    T.Y2 = Y2;
    SX_CUDA(launch_rhs_split(T, st));
    SplitTables Td = T;                           // P_phi F and (dP_phi/dd) F in one launch
    Td.Y3 = Y3;
    for (int s = 0; s < p->S; ++s) Td.Pphi2[s] = p->sadj_dPphi[s];
    Td.phi_pair = 1;
    SX_CUDA(launch_tc_sphere_phi(Td, p->sh3, st));
    if (upd) {
        T.state_upd = upd;
        SX_CUDA(launch_tc_sphere_theta(T, p->shs, st));
    }
    return SEXPE_OK;
}

// One adjoint step of the split sphere plan at the state W_n: lam (FP64, state layout) goes from
// lambda_{n+1} to lambda_n; the parameter gradient accumulates in p->adj_red.  Y2 = P_phi F and
// Y3 = (dP_phi/dd) F at W_n come from the segment replay.
sexpe_status adjoint_step_split(sexpe_plan* p, const double* Wn, const float* Y2, const float* Y3, double* lam,
                                cudaStream_t st) {
    const SplitTables& T0 = p->tabs;
    const size_t e64 = (size_t)p->S * p->npts;
    const int n1 = p->n[0];
    double* acc_d = p->adj_red + 16;
    if (p->sadj_merged) {
        // one kernel: tau P_theta lambda into the chain buffer and both d-derivative dots
        SX_CUDA(launch_to_chain_f32(lam, p->sadj_Yl, n1, T0.n1q, T0.ys, p->npts, p->S, st));
        SplitTables Ta = T0;
        Ta.th_nt = p->sadj_nt;
        Ta.Qsph = p->sadj_Q;
        const SphereAdjArgs A{p->sadj_Yl, p->sadj_had_d, p->sadj_Ymu, Y2, Y3, acc_d};
        SX_CUDA(launch_tc_sphere_theta_adj(Ta, p->sadj_shape, A, st));
    } else {
        // tau P_theta lambda and tau (dP_theta/dd) lambda: the theta kernel's update adds tau x its
        // product to a zeroed FP64 buffer
        SX_CUDA(launch_to_chain_f32(lam, p->sadj_Yl, n1, T0.n1q, T0.ys, p->npts, p->S, st));
        for (int q = 0; q < 2; ++q) {
            SplitTables Tt = T0;
            Tt.Y2 = p->sadj_Yl;
            if (q == 1) Tt.had_sph = p->sadj_had_d;
            Tt.state_upd = p->sadj_T64[q];
            SX_CUDA(cudaMemsetAsync(p->sadj_T64[q], 0, sizeof(double) * e64, st));
            SX_CUDA(launch_tc_sphere_theta(Tt, p->shs, st));
        }
        // d-derivative terms: <tau dP_theta lambda, P_phi F> + <tau P_theta lambda, dP_phi F>
        SX_CUDA(launch_dot_state_chain(p->sadj_T64[1], Y2, n1, T0.n1q, T0.ys, p->npts, p->S, acc_d, st));
        SX_CUDA(launch_dot_state_chain(p->sadj_T64[0], Y3, n1, T0.n1q, T0.ys, p->npts, p->S, acc_d, st));
        SX_CUDA(launch_to_chain_f32(p->sadj_T64[0], p->sadj_Yl, n1, T0.n1q, T0.ys, p->npts, p->S, st));
    }
    // mu = P_phi^T (tau P_theta lambda)
    SplitTables Tm = T0;
    Tm.Y = p->sadj_merged ? p->sadj_Ymu : p->sadj_Yl;
    Tm.Y2 = p->sadj_merged ? p->sadj_Yl : p->sadj_Ymu;
    for (int s = 0; s < p->S; ++s) Tm.Pphi[s] = p->sadj_PphiT[s];
    SX_CUDA(launch_tc_sphere_phi(Tm, p->sh3, st));
    // reaction-parameter and <mu, M w> sums, and lambda += (d M + J_g)^T mu, in one pass
    const int np = (int)p->params.size();
    if (np + p->S <= 8 && p->tabs.rhs.reac.lifted == 0) {
        SX_CUDA(launch_adj_fused_split(p->geometry, p->tabs.rhs, p->sadj_rhsT, Wn, Tm.Y2, T0.n1q, T0.ys, lam,
                                       p->adj_red, np, st));
        return SEXPE_OK;
    }
    SX_CUDA(launch_from_chain_f32(Tm.Y2, p->sadj_MU, n1, T0.n1q, T0.ys, p->npts, p->S, st));
    if (np + p->S <= 8) {
        SX_CUDA(launch_adj_fused(p->geometry, p->rhs64, p->adj_diag, Wn, p->sadj_MU, lam, p->adj_red, np, st));
    } else {
        SX_CUDA(launch_adj_params(p->geometry, p->rhs64, Wn, p->sadj_MU, p->adj_red, st));
        SX_CUDA(launch_adj_lambda(p->geometry, p->adj_diag, Wn, p->sadj_MU, lam, st));
    }
    return SEXPE_OK;
}

// sexpe_adjoint for a split-TF32 sphere plan.  Per checkpoint segment the states are replayed by
// the split forward step (keeping each step's F, P_phi F and (dP_phi/dd) F), then the adjoint steps
// run backwards over them.  The replay of segment c - 1 does not depend on the adjoint variable, so
// it runs on a second stream into the other half of double-buffered segment storage while the
// adjoint steps of segment c run on `st` (both are chains of small, latency-bound launches that
// leave most SMs idle); events order each buffer's reuse.
sexpe_status adjoint_split(sexpe_plan* p, const double* checkpoints, int n_ckpt, int every, const double* dL_dWT,
                           double* dL_dW0, double* dL_dparams, cudaStream_t st) {
    try {
        SX_TRY(build_adjoint_split(p, st));
    } catch (const std::bad_alloc&) {
        return SEXPE_ENOMEM;
    } catch (...) {
        return SEXPE_ENUMERIC;
    }
    const size_t E = (size_t)p->S * p->npts;
    const size_t yf = (size_t)p->S * p->tabs.ys;
    if (p->sadj_seg_cap < every) {
        double* seg = nullptr;
        float* parts = nullptr;
        SX_TRY(alloc_dev(p, (size_t)2 * every * E, &seg));
        SX_TRY(alloc_dev(p, (size_t)2 * 3 * every * yf, &parts));
        SX_CUDA(cudaMemsetAsync(parts, 0, sizeof(float) * (size_t)2 * 3 * every * yf, st));   // padding stays zero
        p->sadj_states = seg;
        p->sadj_seg = parts;
        p->sadj_seg_cap = every;
    }
    if (!p->sadj_stream) {
        SX_CUDA(cudaStreamCreateWithFlags(&p->sadj_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            SX_CUDA(cudaEventCreateWithFlags(&p->sadj_ev_replayed[b], cudaEventDisableTiming));
            SX_CUDA(cudaEventCreateWithFlags(&p->sadj_ev_swept[b], cudaEventDisableTiming));
        }
    }
    cudaStream_t st2 = p->sadj_stream;
    auto state = [&](int b, int j) { return p->sadj_states + ((size_t)b * every + j) * E; };
    auto part = [&](int b, int j, int q) { return p->sadj_seg + (((size_t)b * every + j) * 3 + q) * yf; };
    auto replay = [&](int c, int b, cudaStream_t s) -> sexpe_status {
        SX_CUDA(cudaMemcpyAsync(state(b, 0), checkpoints + (size_t)c * E, E * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
        for (int j = 0; j < every; ++j) {
            double* next = j + 1 < every ? state(b, j + 1) : nullptr;
            if (next) SX_CUDA(cudaMemcpyAsync(next, state(b, j), E * sizeof(double), cudaMemcpyDeviceToDevice, s));
            SX_TRY(split_forward_parts(p, state(b, j), part(b, j, 0), part(b, j, 1), part(b, j, 2), next, s));
        }
        return SEXPE_OK;
    };
    double* lam = dL_dW0;                      // the adjoint variable lives in the output buffer
    if (lam != dL_dWT) SX_CUDA(cudaMemcpyAsync(lam, dL_dWT, E * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SX_CUDA(cudaMemsetAsync(p->adj_red, 0, 32 * sizeof(double), st));
    // the second stream starts after everything enqueued on `st` so far (the checkpoints included)
    SX_CUDA(cudaEventRecord(p->sadj_ev_swept[0], st));
    SX_CUDA(cudaEventRecord(p->sadj_ev_swept[1], st));
    SX_CUDA(cudaStreamWaitEvent(st2, p->sadj_ev_swept[0], 0));
    SX_TRY(replay(n_ckpt - 1, 0, st2));
    SX_CUDA(cudaEventRecord(p->sadj_ev_replayed[0], st2));
    for (int c = n_ckpt - 1; c >= 0; --c) {
        const int b = (n_ckpt - 1 - c) & 1;
        if (c > 0) {                           // next segment's replay into the other buffer
            SX_CUDA(cudaStreamWaitEvent(st2, p->sadj_ev_swept[b ^ 1], 0));
            SX_TRY(replay(c - 1, b ^ 1, st2));
            SX_CUDA(cudaEventRecord(p->sadj_ev_replayed[b ^ 1], st2));
        }
        SX_CUDA(cudaStreamWaitEvent(st, p->sadj_ev_replayed[b], 0));
        for (int j = every - 1; j >= 0; --j)
            SX_TRY(adjoint_step_split(p, state(b, j), part(b, j, 1), part(b, j, 2), lam, st));
        SX_CUDA(cudaEventRecord(p->sadj_ev_swept[b], st));
    }
    if (dL_dparams) {
        double red[32];
        SX_CUDA(cudaMemcpyAsync(red, p->adj_red, sizeof(red), cudaMemcpyDeviceToHost, st));
        SX_CUDA(cudaStreamSynchronize(st));
        const int np = (int)p->params.size();
        for (int q = 0; q < np; ++q) dL_dparams[q] = red[q];
        for (int s = 0; s < p->S; ++s) dL_dparams[np + s] = red[16 + s];
    }
    return SEXPE_OK;
}

// Forward chain of the FP64 step at state W: X[0] = F, then every direction in
// order -- X[q] its input, H[q] = Phi o (V^{-1} X[q]) for a direction in an
// eigenbasis, X[q + 1] its output.  With `upd`, the last direction's output is
// added (times tau) to upd, which completes the step when upd == W; without it
// the chain stops once every quantity the adjoint step reads is formed (the
// last direction's input, and its H for an eigen direction).
sexpe_status forward_chain(sexpe_plan* p, const double* W, double* const* X, double* const* H, double* upd,
                           cudaStream_t st) {
    SX_CUDA(launch_rhs64(p->geometry, p->rhs64, W, X[0], st));
    const int nd = (int)p->dirs64.size();
    for (int q = 0; q < nd; ++q) {
        const Dir64& d = p->dirs64[q];
        const long long nmu = p->n[d.mu - 1];
        const bool last = q + 1 == nd;
        if (last && !upd && !d.eigen) break;
        if (d.eigen) {
            SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, d.Vinv, 0, X[q], H[q], d.had, nullptr), p->S, st));
            if (!last || upd)
                SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, d.V, 0, H[q], last ? nullptr : X[q + 1], nullptr,
                                                last ? upd : nullptr), p->S, st));
        } else {
            SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, d.P, nmu * nmu, X[q], last ? nullptr : X[q + 1], nullptr,
                                            last ? upd : nullptr), p->S, st));
        }
    }
    return SEXPE_OK;
}

// Buffers of one step's saved forward chain: nd inputs X[q], then one H per
// eigen direction (indexed by direction; unused entries left null).
int saved_slots(const sexpe_plan* p) {
    int n = (int)p->dirs64.size();
    for (const Dir64& d : p->dirs64) n += d.eigen ? 1 : 0;
    return n;
}

void chain_views(const sexpe_plan* p, double* base, size_t E, double** X, double** H) {
    const int nd = (int)p->dirs64.size();
    int slot = 0;
    for (int q = 0; q < nd; ++q) X[q] = base + (size_t)slot++ * E;
    for (int q = 0; q < nd; ++q) H[q] = p->dirs64[q].eigen ? base + (size_t)slot++ * E : nullptr;
}

// One adjoint step: lam <- lam_n from lam_{n+1} at the state W_n, accumulating
// the parameter gradient in p->adj_red.  `saved` holds the forward chain at W_n
// (from the replay of the checkpoint segment), or is null and the chain is
// formed here.
sexpe_status adjoint_step(sexpe_plan* p, const double* Wn, double* lam, double* saved, cudaStream_t st) {
    const size_t E = (size_t)p->S * p->npts;
    double* B = p->adj_buf;
    double* X[4];
    double* H[4];
    chain_views(p, saved ? saved : B, E, X, H);          // work buffers: slots 0..6 of adj_buf
    double* Y[2] = {B + 7 * E, B + 8 * E};
    double* HA = B + 9 * E;
    double* Z = B + 10 * E;
    double* MU = B + 11 * E;
    const int nd = (int)p->dirs64.size();
    if (!saved) SX_TRY(forward_chain(p, Wn, X, H, nullptr, st));
    // transposed chain: phi_1(tau d M_1)^T first, with the d-derivative terms
    double* acc_d = p->adj_red + 16;
    const double* y = lam;
    int yi = 0;
    for (int q = nd - 1; q >= 0; --q) {
        const Dir64& d = p->dirs64[q];
        const DirAdj& a = p->adj[q];
        const long long nmu = p->n[d.mu - 1];
        double* yo = Y[yi];
        if (d.eigen) {
            SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, a.VT, 0, y, HA, d.had, nullptr), p->S, st));
            SX_CUDA(launch_wdot(HA, H[q], a.dhad, p->npts, p->S, p->tau, acc_d, st));
            SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, a.VinvT, 0, HA, yo, nullptr, nullptr), p->S, st));
        } else {
            SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, a.dP, nmu * nmu, X[q], Z, nullptr, nullptr), p->S, st));
            SX_CUDA(launch_wdot(Z, y, nullptr, p->npts, p->S, p->tau, acc_d, st));
            SX_CUDA(launch_gemm64(mode_gemm(p, d.mu, a.PT, nmu * nmu, y, yo, nullptr, nullptr), p->S, st));
        }
        y = yo;
        yi ^= 1;
    }
    // mu = tau P^T lam
    SX_CUDA(cudaMemcpyAsync(MU, y, E * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SX_CUDA(launch_scale(MU, p->tau, (long long)E, st));
    SX_CUDA(launch_adj_params(p->geometry, p->rhs64, Wn, MU, p->adj_red, st));
    SX_CUDA(launch_adj_lambda(p->geometry, p->adj_diag, Wn, MU, lam, st));
    return SEXPE_OK;
}

}  // namespace

namespace sexpe {

// True when the plan was made on the device that is current now (its tables live there).
bool plan_on_current_device(const sexpe_plan* p) {
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && dev == p->device;
}

// Checks of a split step into caller-provided scratch: a split-TF32 single-grid plan made on the
// current device, an 8-byte-aligned state and scratch that holds the plan's FP32 intermediate.
sexpe_status check_split_step_with_scratch(const sexpe_plan* p, const double* state, const float* Y,
                                           long long y_floats) {
    if (!p || !state || !Y) return SEXPE_EINVAL;
    if (((uintptr_t)state & 7u) != 0 || ((uintptr_t)Y & 15u) != 0) return SEXPE_EINVAL;
    if (p->precision != SEXPE_SPLIT_TF32 || p->batch || p->coupled) return SEXPE_EINVAL;
    if ((long long)p->S * p->tabs.ys > y_floats) return SEXPE_EINVAL;
    if (!plan_on_current_device(p)) return SEXPE_EINVAL;
    return SEXPE_OK;
}

// Zero the padding columns (rho slots n1 .. n1q - 1 of every line) of the plan's FP32
// intermediate laid out in `Y`: the kernels never write them, and the plan's own buffer is
// zeroed once at setup, so scratch shared with other plans gets the same start.  A 2-D
// memset; no allocation.
sexpe_status zero_scratch_padding(const sexpe_plan* p, float* Y, cudaStream_t st) {
    const SplitTables& T = p->tabs;
    if (T.n1q == T.n1) return SEXPE_OK;
    const size_t lines = (size_t)p->S * (size_t)(T.ys / T.n1q);
    SX_CUDA(cudaMemset2DAsync(Y + T.n1, sizeof(float) * (size_t)T.n1q, 0, sizeof(float) * (size_t)(T.n1q - T.n1),
                              lines, st));
    return SEXPE_OK;
}

// Enqueue one split-TF32 step of plan `p` with the FP32 intermediate of the
// chain in caller-provided device memory `Y` (capacity `y_floats`) instead of
// the plan's own buffer.  Used by the no-allocation entry point, which checks the
// arguments with check_split_step_with_scratch first.
sexpe_status enqueue_split_step_with_scratch(sexpe_plan* p, double* state, float* Y, long long y_floats,
                                             cudaStream_t st) {
    SX_TRY(check_split_step_with_scratch(p, state, Y, y_floats));
    SplitTables T = p->tabs;
    T.state = state;
    T.state_upd = state;
    T.Y = Y;
    SX_CUDA(launch_rhs_split(T, st));
    if (p->geometry == SEXPE_SPHERE) {        // the phi product's output stays in the plan's own buffer
        SX_CUDA(launch_tc_sphere_phi(T, p->sh3, st));
        SX_CUDA(launch_tc_sphere_theta(T, p->shs, st));
        return SEXPE_OK;
    }
    if (p->ndim == 3) SX_CUDA(launch_tc_mode3(T, p->sh3, st));
    SX_CUDA(launch_tc_slab(T, p->shs, st));
    if (p->d_step) SX_CUDA(launch_tick(p->d_step, st));
    return SEXPE_OK;
}

}  // namespace sexpe

namespace {

// The coupling kernel's arguments for a bulk grid, its bulk diffusion and the coupling constants
// (sexpe_coupled_setup and sexpe_coupling_terms): the surface is the ball's outer shell
// (theta x phi) or the cylinder's bottom disk (rho x theta); the virtual-point factor of the
// boundary row is 2/h + 2/rho_* with the ball's radial step h = rho_*/n_rho (eq. ball_discr) or
// 2/h_z with the cylinder's h_z = z_*/n_z (eq. A_z).
CoupleArgs make_couple_args(const sexpe_grid* bg, const double* d_bulk, const sexpe_coupling* cp) {
    CoupleArgs a{};
    const bool dib = cp->kind == SEXPE_COUPLING_DIB_CYLINDER;
    a.kind = cp->kind;
    a.bn1 = bg->n[0];
    a.bn2 = bg->n[1];
    a.sn1 = dib ? bg->n[0] : bg->n[1];
    a.nb = (long long)bg->n[0] * bg->n[1] * bg->n[2];
    a.ns = dib ? (long long)bg->n[0] * bg->n[1] : (long long)bg->n[1] * bg->n[2];
    a.coef = dib ? 2.0 / (bg->z_star / bg->n[2]) : 2.0 / (bg->rho_star / bg->n[0]) + 2.0 / bg->rho_star;
    a.d0 = d_bulk[0];
    a.d1 = d_bulk[1];
    for (int q = 0; q < 5; ++q) {
        a.z[q] = cp->zeta[q];
        a.e[q] = cp->eta[q];
    }
    a.a3 = cp->alpha3;
    a.b3 = cp->beta3;
    a.u_top = cp->u_top;
    a.v_top = cp->v_top;
    return a;
}

// Arguments of sexpe_coupled_setup / sexpe_coupling_terms that need no GPU to check.
sexpe_status validate_coupling(const sexpe_grid* bg, const sexpe_species* bulk, const sexpe_coupling* cp) {
    if (!bg || !bulk || !cp) return SEXPE_EINVAL;
    if (cp->kind != SEXPE_COUPLING_SCHNAKENBERG_BALL && cp->kind != SEXPE_COUPLING_DIB_CYLINDER) return SEXPE_EINVAL;
    const bool dib = cp->kind == SEXPE_COUPLING_DIB_CYLINDER;
    if (bg->geometry != (dib ? SEXPE_CYLINDER : SEXPE_BALL)) return SEXPE_EINVAL;
    if (dib && bg->z_bc != SEXPE_Z_PAPER) return SEXPE_EINVAL;
    if (bulk->n_species != 2) return SEXPE_EINVAL;
    for (int q = 0; q < 5; ++q)
        if (!std::isfinite(cp->zeta[q]) || !std::isfinite(cp->eta[q])) return SEXPE_EINVAL;
    const double extra[4] = {cp->alpha3, cp->beta3, cp->u_top, cp->v_top};
    for (double x : extra)
        if (!std::isfinite(x)) return SEXPE_EINVAL;
    return SEXPE_OK;
}

}  // namespace

extern "C" {

const char* sexpe_status_string(int32_t status) {
    switch (status) {
    case SEXPE_OK: return "ok";
    case SEXPE_EINVAL: return "invalid argument";
    case SEXPE_ENOMEM: return "out of memory";
    case SEXPE_ECUDA: return "CUDA runtime error";
    case SEXPE_ETIMEOUT: return "bounded device wait timed out";
    case SEXPE_EUNSUPPORTED: return "unsupported configuration";
    case SEXPE_ENUMERIC: return "non-finite setup table";
    default: return "unknown status";
    }
}

sexpe_status sexpe_setup(const sexpe_grid* grid, const sexpe_species* species, double tau, int32_t precision,
                         void* stream, sexpe_plan** out) {
    if (!out) return SEXPE_EINVAL;
    *out = nullptr;
    sexpe_status v = validate(grid, species, tau, precision);
    if (v != SEXPE_OK) return v;
    auto t0 = std::chrono::steady_clock::now();
    sexpe_plan* p = new (std::nothrow) sexpe_plan();
    if (!p) return SEXPE_ENOMEM;
    sexpe_status s;
    try {
        s = build_plan(p, grid, species, tau, precision, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        s = SEXPE_ENOMEM;
    } catch (...) {
        s = SEXPE_ENUMERIC;
    }
    if (s != SEXPE_OK) {
        free_plan(p);
        return s;
    }
    p->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SEXPE_OK;
}

sexpe_status sexpe_coupled_setup(const sexpe_grid* bg, const sexpe_species* bulk, const sexpe_species* surface,
                                 const sexpe_coupling* cp, double tau, int32_t precision, void* stream,
                                 sexpe_plan** out) {
    if (!out) return SEXPE_EINVAL;
    *out = nullptr;
    if (!surface) return SEXPE_EINVAL;
    const sexpe_status vc = validate_coupling(bg, bulk, cp);
    if (vc != SEXPE_OK) return vc;
    const bool dib = cp->kind == SEXPE_COUPLING_DIB_CYLINDER;
    if (surface->n_species != 2) return SEXPE_EINVAL;
    if (bulk->offset_host || surface->offset_host) return SEXPE_EINVAL;
    if (bulk->reaction == SEXPE_BVAM_MANUFACTURED || surface->reaction == SEXPE_BVAM_MANUFACTURED) return SEXPE_EINVAL;
    sexpe_grid sg = *bg;                               // the surface grid: part of the bulk grid's boundary
    sg.n[2] = 0;
    if (dib) {                                         // bottom disk: the cylinder's rho x theta grid
        sg.geometry = SEXPE_DISK;
        sg.rho_op = 0;
        sg.z_bc = 0;
    } else {                                           // boundary sphere: the ball's theta x phi grid
        sg.geometry = SEXPE_SPHERE;
        sg.n[0] = bg->n[1];
        sg.n[1] = bg->n[2];
    }
    sexpe_status v = validate(bg, bulk, tau, precision);
    if (v == SEXPE_OK) v = validate(&sg, surface, tau, precision);
    if (v != SEXPE_OK) return v;
    if (precision != SEXPE_FP64 && precision != SEXPE_SPLIT_TF32) return SEXPE_EUNSUPPORTED;
    auto t0 = std::chrono::steady_clock::now();
    sexpe_plan* p = new (std::nothrow) sexpe_plan();
    if (!p) return SEXPE_ENOMEM;
    sexpe_status s = SEXPE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    try {
        p->sub[0] = new sexpe_plan();
        p->sub[1] = new sexpe_plan();
        s = build_plan(p->sub[0], bg, bulk, tau, precision, st);
        if (s == SEXPE_OK) s = build_plan(p->sub[1], &sg, surface, tau, precision, st);
        if (s == SEXPE_OK) {
            for (int q = 0; q < 2; ++q) p->sub[q]->tabs.theta_comp = 1;
            p->device = p->sub[0]->device;
            p->coupled = true;
            p->geometry = bg->geometry;
            p->precision = precision;
            p->S = 4;
            p->ndim = 3;
            for (int m = 0; m < 3; ++m) p->n[m] = bg->n[m];
            p->npts = p->sub[0]->npts;
            p->tau = tau;
            p->cpl = make_couple_args(bg, p->sub[0]->d.data(), cp);
            p->kernels_per_step = 1 + p->sub[0]->kernels_per_step + p->sub[1]->kernels_per_step;
            s = alloc_err_word(p, st);
            if (s == SEXPE_OK && precision == SEXPE_SPLIT_TF32) {
                if (cudaStreamCreateWithFlags(&p->cpl_stream, cudaStreamNonBlocking) != cudaSuccess) s = SEXPE_ECUDA;
                for (int e = 0; e < 4 && s == SEXPE_OK; ++e)
                    if (cudaEventCreateWithFlags(&p->cpl_ev[e], cudaEventDisableTiming) != cudaSuccess) s = SEXPE_ECUDA;
            }
            if (s == SEXPE_OK) s = alloc_dev(p, (size_t)state_elems(p), &p->d_host_state);
            if (s == SEXPE_OK && cudaStreamSynchronize(st) != cudaSuccess) s = SEXPE_ECUDA;
        }
    } catch (const std::bad_alloc&) {
        s = SEXPE_ENOMEM;
    } catch (...) {
        s = SEXPE_ENUMERIC;
    }
    if (s != SEXPE_OK) {
        free_plan(p);
        return s;
    }
    p->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SEXPE_OK;
}

sexpe_status sexpe_coupling_terms(const sexpe_grid* bulk_grid, const sexpe_species* bulk, const sexpe_coupling* cp,
                                  int64_t n, const double* ub, const double* vb, const double* r, const double* s,
                                  double* add_b0, double* add_b1, double* add_s0, double* add_s1) {
    const sexpe_status v = validate_coupling(bulk_grid, bulk, cp);
    if (v != SEXPE_OK) return v;
    if (n < 0 || !bulk->d_host) return SEXPE_EINVAL;
    if (n > 0 && (!ub || !vb || !r || !s || !add_b0 || !add_b1 || !add_s0 || !add_s1)) return SEXPE_EINVAL;
    const int ndim = 3;
    for (int m = 0; m < ndim; ++m)
        if (bulk_grid->n[m] < 3 || bulk_grid->n[m] > kMaxN) return SEXPE_EINVAL;
    if (!(bulk_grid->rho_star > 0.0 && std::isfinite(bulk_grid->rho_star))) return SEXPE_EINVAL;
    if (bulk_grid->geometry == SEXPE_CYLINDER && !(bulk_grid->z_star > 0.0 && std::isfinite(bulk_grid->z_star)))
        return SEXPE_EINVAL;
    const CoupleArgs a = make_couple_args(bulk_grid, bulk->d_host, cp);
    for (int64_t q = 0; q < n; ++q) {
        double add[4];
        couple_terms(a, ub[q], vb[q], r[q], s[q], add);
        add_b0[q] = add[0];
        add_b1[q] = add[1];
        add_s0[q] = add[2];
        add_s1[q] = add[3];
    }
    return SEXPE_OK;
}

sexpe_status sexpe_batch_setup(int32_t count, const sexpe_grid* grids, const sexpe_species* species, double tau,
                               int32_t precision, void* stream, sexpe_plan** out) {
    if (!out) return SEXPE_EINVAL;
    *out = nullptr;
    if (count < 1 || count > 65536 || !grids || !species) return SEXPE_EINVAL;
    for (int q = 0; q < count; ++q) {
        const sexpe_status v = validate(&grids[q], &species[q], tau, precision);
        if (v != SEXPE_OK) return v;
        if (grids[q].geometry != SEXPE_DISK || species[q].n_species != 2) return SEXPE_EINVAL;
        if (species[q].reaction == SEXPE_LINEAR_CUBIC || species[q].reaction == SEXPE_BVAM_MANUFACTURED ||
            species[q].reaction == SEXPE_LINEAR)
            return SEXPE_EUNSUPPORTED;
        if (grids[q].rho_op != 0 || species[q].offset_host) return SEXPE_EUNSUPPORTED;
        if (grids[q].n[0] > 128 || grids[q].n[1] > 256) return SEXPE_EUNSUPPORTED;
    }
    if (precision != SEXPE_SPLIT_TF32) return SEXPE_EUNSUPPORTED;
    auto t0 = std::chrono::steady_clock::now();
    sexpe_plan* p = new (std::nothrow) sexpe_plan();
    if (!p) return SEXPE_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    sexpe_status status = SEXPE_OK;
    try {
        if (cudaGetDevice(&p->device) != cudaSuccess) status = SEXPE_ECUDA;
        if (status == SEXPE_OK) status = build_batch(p, count, grids, species, tau, st);
    } catch (const std::bad_alloc&) {
        status = SEXPE_ENOMEM;
    } catch (...) {
        status = SEXPE_ENUMERIC;
    }
    if (status != SEXPE_OK) {
        free_plan(p);
        return status;
    }
    p->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SEXPE_OK;
}

sexpe_status sexpe_state_offsets(const sexpe_plan* plan, int64_t* offsets_host) {
    if (!plan || !offsets_host) return SEXPE_EINVAL;
    if (plan->batch) {
        for (size_t q = 0; q < plan->inst_off.size(); ++q) offsets_host[q] = plan->inst_off[q];
        return SEXPE_OK;
    }
    offsets_host[0] = 0;
    offsets_host[1] = state_elems(plan);
    return SEXPE_OK;
}

sexpe_status sexpe_set_time(sexpe_plan* p, double t, void* stream) {
    if (!p || !std::isfinite(t)) return SEXPE_EINVAL;
    if (p->reaction != SEXPE_BVAM_MANUFACTURED || !p->d_step) return SEXPE_OK;
    p->t0 = t;
    p->rhs64.t0 = t;
    p->tabs.rhs.t0 = t;
    SX_CUDA(cudaMemsetAsync(p->d_step, 0, sizeof(long long), (cudaStream_t)stream));
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_set_stencil(sexpe_plan* p, int32_t tile_j, int32_t planes, int32_t ctas_per_sm) {
    if (!p) return SEXPE_EINVAL;
    if (p->batch || p->coupled || p->precision != SEXPE_SPLIT_TF32) return SEXPE_EUNSUPPORTED;
    int3 cand[256];
    const int nc = rhs_candidates(p->tabs, cand, 256);
    bool ok = false;
    for (int c = 0; c < nc; ++c) ok = ok || (cand[c].x == tile_j && cand[c].y == planes && cand[c].z == ctas_per_sm);
    if (!ok) return SEXPE_EINVAL;
    p->tabs.rhs_tj = tile_j;
    p->tabs.rhs_ks = planes;
    p->tabs.rhs_mb = ctas_per_sm;
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_set_theta_split(sexpe_plan* p, int32_t split) {
    if (!p) return SEXPE_EINVAL;
    if (p->th_splits.empty()) return SEXPE_EUNSUPPORTED;
    size_t c = 0;
    while (c < p->th_splits.size() && p->th_splits[c] != split) ++c;
    if (c == p->th_splits.size()) return SEXPE_EINVAL;
    const int n1p = rup16(p->n[0]);
    p->tabs.Qsph = p->th_imgs[c];
    p->tabs.th_nt = n1p / split;
    p->shs = tc_sphere_theta_shape(p->n[0], p->tabs.th_nt);
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_step(sexpe_plan* p, double* state, int64_t n_steps, void* stream) {
    if (!p || !state || n_steps < 0) return SEXPE_EINVAL;
    if (((uintptr_t)state & 7u) != 0) return SEXPE_EINVAL;
    if (!sexpe::plan_on_current_device(p)) return SEXPE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t done = 0;
    p->bparity = 0;
    if (n_steps >= kGraphSteps && !p->profiling) {
        if (!p->gexec || p->g_state != state) {
            if (p->gexec) {
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
            cudaStream_t cs;
            SX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            sexpe_status s = SEXPE_OK;
            if (e == cudaSuccess) {
                for (int k = 0; k < kGraphSteps && s == SEXPE_OK; ++k) s = enqueue_step(p, state, cs);
                cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess && s == SEXPE_OK) e = cudaGraphInstantiate(&p->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cs);
            if (s != SEXPE_OK) return s;
            if (e != cudaSuccess) {
                p->gexec = nullptr;
                return cuda_status(e);
            }
            p->g_state = state;
        }
        for (; done + kGraphSteps <= n_steps; done += kGraphSteps) SX_CUDA(cudaGraphLaunch(p->gexec, st));
    }
    for (; done < n_steps; ++done) SX_TRY(enqueue_step(p, state, st));
    if (p->batch && p->bparity) {   // odd number of ping-pong steps: the result is in the plan's buffer
        SX_CUDA(cudaMemcpyAsync(state, p->bstate, sizeof(double) * (size_t)p->inst_off.back(),
                                cudaMemcpyDeviceToDevice, st));
        p->bparity = 0;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_step_host(sexpe_plan* p, double* state_host, int64_t n_steps, void* stream) {
    if (!p || !state_host || n_steps < 0) return SEXPE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)state_elems(p);
    SX_CUDA(cudaMemcpyAsync(p->d_host_state, state_host, bytes, cudaMemcpyHostToDevice, st));
    SX_TRY(sexpe_step(p, p->d_host_state, n_steps, stream));
    SX_CUDA(cudaMemcpyAsync(state_host, p->d_host_state, bytes, cudaMemcpyDeviceToHost, st));
    return sexpe_synchronize(p, stream);
}

sexpe_status sexpe_selftest_wait_timeout(void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SEXPE_ENOMEM;
    }
    int host = -1;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_wait_selftest(err, 2000000LL, st);   // ~1 ms at 2 GHz
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&host, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_status(e);
    return host == DERR_TIMEOUT_MMA ? SEXPE_ETIMEOUT : SEXPE_ECUDA;
}

sexpe_status sexpe_synchronize(sexpe_plan* p, void* stream) {
    if (!p) return SEXPE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int err = 0;
    if (p->h_err) {
        // the error word is copied on the stream behind the plan's work: one synchronisation
        SX_CUDA(cudaMemcpyAsync(p->h_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SX_CUDA(cudaStreamSynchronize(st));
        err = *p->h_err;
    } else {
        SX_CUDA(cudaStreamSynchronize(st));
        SX_CUDA(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    }
    if (err != 0) {
        SX_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
        return SEXPE_ETIMEOUT;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_plan_get_info(const sexpe_plan* p, sexpe_plan_info* info) {
    if (!p || !info) return SEXPE_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->geometry = p->geometry;
    info->precision = p->precision;
    info->n_species = p->S;
    info->ndim = p->ndim;
    for (int m = 0; m < 3; ++m) info->n[m] = p->n[m];
    info->n_instances = p->n_instances;
    info->kernels_per_step = p->kernels_per_step;
    info->npts = p->npts;
    info->state_elems = state_elems(p);
    info->workspace_bytes = (int64_t)p->bytes;
    if (p->coupled) info->workspace_bytes += (int64_t)(p->sub[0]->bytes + p->sub[1]->bytes);
    info->setup_ms = p->setup_ms;
    const sexpe_plan* t = p->coupled ? p->sub[0] : p;   // a coupled plan reports its bulk grid's tiling
    if (!p->batch && p->precision == SEXPE_SPLIT_TF32) {
        info->stencil_tile_j = t->tabs.rhs_tj;
        info->ring_slots[0] = (int32_t)t->shs.nm;
        info->ring_slots[1] = (int32_t)t->shs.nd;
        info->stencil_tile_us = t->rhs_tj_us;
        info->stencil_planes = t->tabs.rhs_ks;
        info->stencil_ctas_per_sm = t->tabs.rhs_mb;
        if (!t->th_splits.empty()) info->theta_split = rup16(t->n[0]) / t->tabs.th_nt;
    } else if (p->batch) {
        info->ring_slots[0] = (int32_t)p->bsh.nm;
        info->ring_slots[1] = (int32_t)p->bsh.nd;
        info->stencil_tile_j = p->btab.tj;
        info->batch_order = p->batch_order;
        info->batch_step_us = p->batch_step_us;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_step_checkpointed(sexpe_plan* p, double* state, int64_t n_steps, int32_t every,
                                     double* checkpoints, void* stream) {
    if (!p || !state || !checkpoints || n_steps < 0 || every < 1) return SEXPE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t E = (size_t)state_elems(p);
    for (int64_t k = 0; k < n_steps; ++k) {
        if (k % every == 0)
            SX_CUDA(cudaMemcpyAsync(checkpoints + (size_t)(k / every) * E, state, E * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
        SX_TRY(enqueue_step(p, state, st));
    }
    return SEXPE_OK;
}

sexpe_status sexpe_adjoint(sexpe_plan* p, const double* checkpoints, int32_t n_ckpt, int32_t every,
                           const double* dL_dWT, double* dL_dW0, double* dL_dparams, void* stream) {
    if (!p || !checkpoints || !dL_dWT || !dL_dW0 || n_ckpt < 1 || every < 1) return SEXPE_EINVAL;
    const bool split = p->precision == SEXPE_SPLIT_TF32 && p->geometry == SEXPE_SPHERE && !p->batch && !p->coupled;
    if ((p->precision != SEXPE_FP64 && !split) || p->coupled) return SEXPE_EUNSUPPORTED;
    if (p->reaction == SEXPE_BVAM || p->reaction == SEXPE_BVAM_MANUFACTURED || p->reaction == SEXPE_LINEAR)
        return SEXPE_EUNSUPPORTED;
    for (double c : p->offset)
        if (c != 0.0) return SEXPE_EUNSUPPORTED;
    if (!plan_on_current_device(p)) return SEXPE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (split) return adjoint_split(p, checkpoints, n_ckpt, every, dL_dWT, dL_dW0, dL_dparams, st);
    try {
        SX_TRY(build_adjoint(p, st));
    } catch (const std::bad_alloc&) {
        return SEXPE_ENOMEM;
    } catch (...) {
        return SEXPE_ENUMERIC;
    }
    const size_t E = (size_t)p->S * p->npts;
    if (p->adj_seg_cap < every) {
        double* seg = nullptr;
        SX_TRY(alloc_dev(p, (size_t)every * E, &seg));
        p->adj_seg = seg;
        p->adj_seg_cap = every;
    }
    // The replay of a segment keeps each step's forward chain, so the adjoint
    // steps do not form it again; without room for it they do.
    const int ns = saved_slots(p);
    if (every > 1 && p->adj_save_cap < every) {
        double* sv = nullptr;
        if (alloc_dev(p, (size_t)(every - 1) * ns * E, &sv) == SEXPE_OK) {
            p->adj_save = sv;
            p->adj_save_cap = every;
        } else {
            cudaGetLastError();
        }
    }
    const bool keep = every > 1 && p->adj_save_cap >= every;
    double* lam = dL_dW0;                      // the adjoint variable lives in the output buffer
    if (lam != dL_dWT) SX_CUDA(cudaMemcpyAsync(lam, dL_dWT, E * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SX_CUDA(cudaMemsetAsync(p->adj_red, 0, 32 * sizeof(double), st));
    for (int c = n_ckpt - 1; c >= 0; --c) {
        SX_CUDA(cudaMemcpyAsync(p->adj_seg, checkpoints + (size_t)c * E, E * sizeof(double), cudaMemcpyDeviceToDevice,
                                st));
        for (int j = 1; j < every; ++j) {
            double* w = p->adj_seg + (size_t)j * E;
            SX_CUDA(cudaMemcpyAsync(w, w - E, E * sizeof(double), cudaMemcpyDeviceToDevice, st));
            if (keep) {
                double* X[4];
                double* H[4];
                chain_views(p, p->adj_save + (size_t)(j - 1) * ns * E, E, X, H);
                SX_TRY(forward_chain(p, w, X, H, w, st));     // chain at W_{j-1}, then W_j in place
            } else {
                SX_TRY(enqueue_step(p, w, st));
            }
        }
        for (int j = every - 1; j >= 0; --j)
            SX_TRY(adjoint_step(p, p->adj_seg + (size_t)j * E, lam,
                                keep && j < every - 1 ? p->adj_save + (size_t)j * ns * E : nullptr, st));
    }
    if (dL_dparams) {
        double red[32];
        SX_CUDA(cudaMemcpyAsync(red, p->adj_red, sizeof(red), cudaMemcpyDeviceToHost, st));
        SX_CUDA(cudaStreamSynchronize(st));
        const int np = (int)p->params.size();
        for (int q = 0; q < np; ++q) dL_dparams[q] = red[q];
        for (int s = 0; s < p->S; ++s) dL_dparams[np + s] = red[16 + s];
    }
    return SEXPE_OK;
}

sexpe_status sexpe_profile_begin(sexpe_plan* p, int32_t max_steps) {
    if (!p || max_steps < 1 || max_steps > 100000) return SEXPE_EINVAL;
    free_profile(p);
    const size_t n = (size_t)max_steps * (p->kernels_per_step + 1);
    p->prof_ev.resize(n);
    for (size_t i = 0; i < n; ++i) {
        cudaError_t e = cudaEventCreate(&p->prof_ev[i]);
        if (e != cudaSuccess) {
            p->prof_ev.resize(i);
            free_profile(p);
            return cuda_status(e);
        }
    }
    p->prof_max_steps = max_steps;
    p->prof_steps = 0;
    p->profiling = true;
    return SEXPE_OK;
}

sexpe_status sexpe_profile_end(sexpe_plan* p, double* kernel_ms, int32_t* n_kernels, int32_t cap) {
    if (!p || !kernel_ms || !n_kernels || cap < 0 || !p->profiling) return SEXPE_EINVAL;
    const int per = p->kernels_per_step + 1;
    const int k = p->kernels_per_step < cap ? p->kernels_per_step : cap;
    *n_kernels = k;
    sexpe_status st = SEXPE_OK;
    if (p->prof_steps > 0) {
        cudaError_t e = cudaEventSynchronize(p->prof_ev[(size_t)(p->prof_steps - 1) * per + per - 1]);
        if (e != cudaSuccess) st = cuda_status(e);
        for (int q = 0; q < k && st == SEXPE_OK; ++q) {
            double acc = 0.0;
            for (int s = 0; s < p->prof_steps; ++s) {
                float ms = 0.f;
                e = cudaEventElapsedTime(&ms, p->prof_ev[(size_t)s * per + q], p->prof_ev[(size_t)s * per + q + 1]);
                if (e != cudaSuccess) { st = cuda_status(e); break; }
                acc += ms;
            }
            kernel_ms[q] = acc / p->prof_steps;
        }
    } else {
        for (int q = 0; q < k; ++q) kernel_ms[q] = 0.0;
    }
    free_profile(p);
    return st;
}

static bool axis_args(int32_t axis, int32_t n, double extent, AxisKind* kind) {
    static const AxisKind kinds[6] = {AX_THETA, AX_RHO2, AX_RHO3, AX_PHI, AX_Z_NEUMANN, AX_Z_PAPER};
    if (axis < 0 || axis > 5 || n < 3 || n > kMaxN) return false;
    if ((axis == 1 || axis == 2 || axis == 4 || axis == 5) && !(extent > 0.0 && std::isfinite(extent))) return false;
    *kind = kinds[axis];
    return true;
}

sexpe_status sexpe_axis_matrix(int32_t axis, int32_t n, double extent, double* A_host) {
    AxisKind kind;
    if (!A_host || !axis_args(axis, n, extent, &kind)) return SEXPE_EINVAL;
    const Mat A = build_axis(kind, n, extent).dense();
    std::memcpy(A_host, A.a.data(), sizeof(double) * n * n);
    return SEXPE_OK;
}

sexpe_status sexpe_axis_phi1(int32_t axis, int32_t n, double extent, double t, double* out_host) {
    AxisKind kind;
    if (!out_host || !std::isfinite(t) || !axis_args(axis, n, extent, &kind)) return SEXPE_EINVAL;
    try {
        Mat X = build_axis(kind, n, extent).dense();
        for (double& v : X.a) v *= t;
        const Mat R = phi1_pade(X);
        std::memcpy(out_host, R.a.data(), sizeof(double) * n * n);
    } catch (...) {
        return SEXPE_ENUMERIC;
    }
    return SEXPE_OK;
}

sexpe_status sexpe_axis_eigen(int32_t axis, int32_t n, double extent, double* lam_host, double* V_host,
                              double* Vinv_host) {
    AxisKind kind;
    if (!axis_args(axis, n, extent, &kind)) return SEXPE_EINVAL;
    const Axis a = build_axis(kind, n, extent);
    const Eigen e = a.periodic ? theta_eigen(a) : tridiag_eigen(a);
    if (lam_host) std::memcpy(lam_host, e.lam.data(), sizeof(double) * n);
    if (V_host) std::memcpy(V_host, e.V.a.data(), sizeof(double) * n * n);
    if (Vinv_host) std::memcpy(Vinv_host, e.Vinv.a.data(), sizeof(double) * n * n);
    return SEXPE_OK;
}

sexpe_status sexpe_destroy(sexpe_plan* p) {
    if (!p) return SEXPE_EINVAL;
    cudaDeviceSynchronize();
    free_plan(p);
    return SEXPE_OK;
}

}  // extern "C"
