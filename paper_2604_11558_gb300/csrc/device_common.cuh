// Stencil + reaction evaluation shared by the FP64 and split-TF32 kernels:
// F_s = d_s (M w_s) + g_s(w) at one grid point (first line of eqs. ee_disk,
// ee_sphere, ee_ball, ee_cylinder), with M applied in difference form
// (A w)_r = lower_r (w_{r-1} - w_r) + upper_r (w_{r+1} - w_r) + rs_r w_r.
#pragma once
#include <cstdint>

#include "internal.h"

namespace sexpe {

// Split an FP64 value into FP32 (hi, lo) with hi = w truncated to 24 significant
// bits and lo = the truncated remainder (rounded to 24 bits), using integer
// operations only.  Differences of nearby values, (hi_a - hi_b) + (lo_a - lo_b),
// then carry FP32 relative accuracy of the *difference* (hi_a - hi_b is exact
// when a and b are within a factor 2), which the stencil needs: its
// coefficients reach ~1e7 near the coordinate singularities, where rounding w
// itself to FP32 would leave errors far above the difference.
__device__ __forceinline__ float2 split_f64(double w) {
    const unsigned hi32 = (unsigned)__double2hiint(w), lo32 = (unsigned)__double2loint(w);
    const unsigned sign = hi32 & 0x80000000u;
    const unsigned e = (hi32 >> 20) & 0x7FFu;           // biased FP64 exponent
    // hi: a funnel shift brings the low 8 exponent bits and the top 23 fraction bits into
    // FP32 position; flipping exponent bit 7 rebiases e to e - 896 for every FP32-normal e.
    // |w| < 2^-126 (below FP32 normals) -> signed zero; beyond FP32 range -> infinity.
    const unsigned f = __funnelshift_l(lo32, hi32, 3);
    unsigned fb = ((f & 0x7FFFFFFFu) ^ 0x40000000u) | sign;
    fb = (e - 897u <= 253u) ? fb : (e < 897u ? sign : (sign | 0x7F800000u));
    // lo: the 29 truncated bits, weight 2^(e - 1075) each (zero below |w| = 2^-74)
    const float lo = (float)(lo32 & 0x1FFFFFFFu) * __uint_as_float(sign | ((e - 948u) << 23));
    return make_float2(__uint_as_float(fb), (e - 949u <= 201u) ? lo : 0.f);
}

// Exact FP32 -> FP64 conversion with integer operations only (FP32 denormals
// flush to zero); keeps the conversion off the FP64 pipe.
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned m = u & 0x7FFFFFu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    hi = (e == 0u) ? sign : hi;
    lo = (e == 0u) ? 0u : lo;
    hi = (e == 0xFFu) ? (sign | 0x7FF00000u | (m >> 3)) : hi;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

struct F64Acc {
    using V = double;
    using T = double;
    __device__ static V load(const double* p) { return __ldg(p); }
    __device__ static T diff(V a, V b) { return a - b; }
    __device__ static T value(V a) { return a; }
};

struct SplitAcc {
    using V = float2;
    using T = float;
    __device__ static V load(const double* p) { return split_f64(__ldg(p)); }
    __device__ static T diff(V a, V b) { return (a.x - b.x) + (a.y - b.y); }
    __device__ static T value(V a) { return a.x + a.y; }
};

template <class Acc>
__device__ __forceinline__ typename Acc::T axis_term(const StencilAxis<typename Acc::T>& ax, const double* W,
                                                     long long idx, int r, long long st, typename Acc::V c) {
    using T = typename Acc::T;
    T acc = ax.rs[r] * Acc::value(c);
    long long im = -1, ip = -1;
    if (r > 0) im = idx - st;
    else if (ax.periodic) im = idx + (long long)(ax.n - 1) * st;
    if (r < ax.n - 1) ip = idx + st;
    else if (ax.periodic) ip = idx - (long long)(ax.n - 1) * st;
    if (im >= 0) acc += ax.lower[r] * Acc::diff(Acc::load(W + im), c);
    if (ip >= 0) acc += ax.upper[r] * Acc::diff(Acc::load(W + ip), c);
    return acc;
}

// (M w)(i, j, k) for one species, Kronecker sums of Section 2:
//  disk     M = I (x) A_rho2 + A_theta (x) D_rho
//  sphere   M = D_phi (x) A_theta + A_phi (x) I          (mode 1 theta, mode 2 phi)
//  ball     M = I (x) I (x) A_rho3 + D_phi (x) A_theta (x) D_rho + A_phi (x) I (x) D_rho
//  cylinder M = I (x) I (x) A_rho2 + I (x) A_theta (x) D_rho + A_z (x) I (x) I
template <class Acc, int GEO>
__device__ __forceinline__ typename Acc::T laplacian(const RhsTables<typename Acc::T>& tb, const double* W,
                                                     long long idx, int i, int j, int k, typename Acc::V c) {
    using T = typename Acc::T;
    const T t0 = axis_term<Acc>(tb.ax[0], W, idx, i, 1, c);
    const T t1 = axis_term<Acc>(tb.ax[1], W, idx, j, tb.n1, c);
    if constexpr (GEO == GEO_DISK) return t0 + tb.Dr[i] * t1;
    if constexpr (GEO == GEO_SPHERE) return tb.Dp[j] * t0 + t1;
    const T t2 = axis_term<Acc>(tb.ax[2], W, idx, k, (long long)tb.n1 * tb.n2, c);
    if constexpr (GEO == GEO_BALL) return t0 + tb.Dr[i] * (tb.Dp[k] * t1 + t2);
    return t0 + tb.Dr[i] * t1 + t2;   // cylinder
}

// a * b + c with one rounding, spelled out so that every kernel that inlines
// the reaction or the stencil forms the same value (the compiler's own choice of
// which products to fuse may differ between instantiations)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_t(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_t(double a, double b) { return __dmul_rn(a, b); }

template <class T>
__device__ __forceinline__ T reaction(const ReactionParams<T>& rp, const T* w_state, int s) {
    if (rp.lifted) {
        // Schnakenberg about the lifting constants c (the polynomial expanded exactly, so that
        // every term is small when w is and keeps the arithmetic's relative accuracy):
        // b(c + w) = b(c) - w_u + N + Q, c(c + w) = c(c) - N - Q with
        // N = 2 c_u c_v w_u + c_u^2 w_v, Q = w_u (c_v w_u + 2 c_u w_v + w_u w_v)
        const T wu = w_state[0], wv = w_state[1];
        const T N = fma_t(rp.q[2], wu, mul_t(rp.q[3], wv));
        const T Q = mul_t(wu, fma_t(rp.q[4], wu, fma_t(rp.q[5], wv, mul_t(wu, wv))));
        return s == 0 ? mul_t(rp.p[0], (N + Q - wu) + rp.q[0]) : mul_t(rp.p[0], rp.q[1] - (N + Q));
    }
    T w[kMaxSpecies];
#pragma unroll
    for (int r = 0; r < kMaxSpecies; ++r) w[r] = w_state[r] + rp.off[r];    // lifted boundary values
    switch (rp.kind) {
    case R_SCHNAKENBERG: {   // f = gamma(a - u + u^2 v), g = gamma(b - u^2 v)
        const T u2v = mul_t(mul_t(w[0], w[0]), w[1]);
        return s == 0 ? mul_t(rp.p[0], (rp.p[1] - w[0]) + u2v) : mul_t(rp.p[0], rp.p[2] - u2v);
    }
    case R_GRAY_SCOTT: {     // f = -u v^2 + F(1 - u), g = u v^2 - (F + k) v
        const T uv2 = mul_t(mul_t(w[0], w[1]), w[1]);
        return s == 0 ? fma_t(rp.p[0], (T)1 - w[0], -uv2) : fma_t(-(rp.p[0] + rp.p[1]), w[1], uv2);
    }
    case R_BVAM:
    case R_BVAM_MMS: {       // eq. BVAMnl: b = a1 u (1 - a2 v^2) + v (1 - a3 u), c = b1 v (1 + a1 a2/b1 u v) + u (b2 + a3 v)
        const T u = w[0], v = w[1];
        if (s == 0)
            return fma_t(mul_t(rp.p[0], u), fma_t(-rp.p[1], mul_t(v, v), (T)1), mul_t(v, fma_t(-rp.p[2], u, (T)1)));
        const T q = mul_t(rp.p[0], rp.p[1]) / rp.p[3];
        return fma_t(mul_t(rp.p[3], v), fma_t(q, mul_t(u, v), (T)1), mul_t(u, fma_t(rp.p[2], v, rp.p[4])));
    }
    case R_LINEAR_CUBIC: {   // f_i = sum_j K_ij u_j - u_i^3
        T acc = -mul_t(mul_t(w[s], w[s]), w[s]);
#pragma unroll
        for (int r = 0; r < kMaxSpecies; ++r)
            if (r < rp.S) acc = fma_t(rp.p[s * rp.S + r], w[r], acc);
        return acc;
    }
    case R_LINEAR: {         // f_i = sum_j K_ij u_j
        T acc = (T)0;
#pragma unroll
        for (int r = 0; r < kMaxSpecies; ++r)
            if (r < rp.S) acc = fma_t(rp.p[s * rp.S + r], w[r], acc);
        return acc;
    }
    default:
        return (T)0;
    }
}

// Reaction terms of every species at one point, g[s] equal to reaction<T>(rp, w_state, s) bit
// for bit (the same operations), with the kind tested once per point by uniform branches
// rather than once per species, and the terms two species share formed once.  KIND >= 0
// compiles only that kind (the caller knows it).
template <class T>
__device__ __forceinline__ void reac_gray_scott(const ReactionParams<T>& rp, const T* w, T* g) {
    const T uv2 = mul_t(mul_t(w[0], w[1]), w[1]);
    g[0] = fma_t(rp.p[0], (T)1 - w[0], -uv2);
    g[1] = fma_t(-(rp.p[0] + rp.p[1]), w[1], uv2);
}
template <class T>
__device__ __forceinline__ void reac_schnakenberg(const ReactionParams<T>& rp, const T* w, T* g) {
    const T u2v = mul_t(mul_t(w[0], w[0]), w[1]);
    g[0] = mul_t(rp.p[0], (rp.p[1] - w[0]) + u2v);
    g[1] = mul_t(rp.p[0], rp.p[2] - u2v);
}
template <class T>
__device__ __forceinline__ void reac_schnakenberg_lifted(const ReactionParams<T>& rp, const T* w_state, T* g) {
    const T wu = w_state[0], wv = w_state[1];
    const T N = fma_t(rp.q[2], wu, mul_t(rp.q[3], wv));
    const T Q = mul_t(wu, fma_t(rp.q[4], wu, fma_t(rp.q[5], wv, mul_t(wu, wv))));
    g[0] = mul_t(rp.p[0], (N + Q - wu) + rp.q[0]);
    g[1] = mul_t(rp.p[0], rp.q[1] - (N + Q));
}

template <class T, int NS, int KIND = -1>
__device__ __forceinline__ void reactions(const ReactionParams<T>& rp, const T* w_state, T* g) {
#pragma unroll
    for (int r = 0; r < NS; ++r) g[r] = (T)0;
    T w[kMaxSpecies];
#pragma unroll
    for (int r = 0; r < kMaxSpecies; ++r) w[r] = r < NS ? w_state[r] + rp.off[r] : (T)0;
    if constexpr (NS >= 2 && KIND == R_GRAY_SCOTT) {
        reac_gray_scott(rp, w, g);
        return;
    }
    if constexpr (NS >= 2 && KIND == R_SCHNAKENBERG) {
        if (rp.lifted) reac_schnakenberg_lifted(rp, w_state, g);
        else reac_schnakenberg(rp, w, g);
        return;
    }
    if constexpr (NS >= 2 && KIND < 0) {     // the two-species kinds
        if (rp.lifted) {
            reac_schnakenberg_lifted(rp, w_state, g);
            return;
        }
        if (rp.kind == R_GRAY_SCOTT) {
            reac_gray_scott(rp, w, g);
            return;
        }
        if (rp.kind == R_SCHNAKENBERG) {
            reac_schnakenberg(rp, w, g);
            return;
        }
        if (rp.kind == R_BVAM || rp.kind == R_BVAM_MMS) {
            const T u = w[0], v = w[1];
            g[0] = fma_t(mul_t(rp.p[0], u), fma_t(-rp.p[1], mul_t(v, v), (T)1), mul_t(v, fma_t(-rp.p[2], u, (T)1)));
            const T q = mul_t(rp.p[0], rp.p[1]) / rp.p[3];
            g[1] = fma_t(mul_t(rp.p[3], v), fma_t(q, mul_t(u, v), (T)1), mul_t(u, fma_t(rp.p[2], v, rp.p[4])));
            return;
        }
    }
    if constexpr (KIND < 0) {
        if (rp.kind == R_LINEAR_CUBIC || rp.kind == R_LINEAR) {
            const bool cubic = rp.kind == R_LINEAR_CUBIC;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (s < rp.S) {
                    T acc = cubic ? -mul_t(mul_t(w[s], w[s]), w[s]) : (T)0;
#pragma unroll
                    for (int r = 0; r < NS; ++r)
                        if (r < rp.S) acc = fma_t(rp.p[s * rp.S + r], w[r], acc);
                    g[s] = acc;
                }
            }
        }
    }
}

// Manufactured source of species s at disk point (rho_i, theta_j) (Section 5.1):
// u_t - d_s Lap u - g_s(u, v) at the exact solution, whose time factor is et = e^-t.
template <class T>
__device__ __forceinline__ T mms_source(const RhsTables<T>& tb, int i, int j, T et, int s) {
    const int n1 = tb.n1, n2 = tb.n2;
    const T R = tb.mms_rho[i], LR = tb.mms_rho[n1 + i], IR2 = tb.mms_rho[2 * n1 + i];
    const T Tt = tb.mms_theta[j], T2 = tb.mms_theta[n2 + j], Sv = tb.mms_theta[2 * n2 + j],
            S2 = tb.mms_theta[3 * n2 + j];
    const T eR = mul_t(et, R);
    T w[kMaxSpecies] = {mul_t(eR, Tt), mul_t(eR, Sv), (T)0, (T)0};
    const T lap = s == 0 ? mul_t(et, fma_t(LR, Tt, mul_t(IR2, T2))) : mul_t(et, fma_t(LR, Sv, mul_t(IR2, S2)));
    return fma_t(-tb.d[s], lap, -w[s]) - reaction<T>(tb.reac, w, s);
}

// e^-t of the current step of a plan with manufactured sources (1 otherwise).
template <class T>
__device__ __forceinline__ double mms_time_factor(const RhsTables<T>& tb) {
    return tb.reac.kind == R_BVAM_MMS ? exp(-(tb.t0 + (double)(*tb.step) * tb.tau_t)) : 1.0;
}

// F_s at flat index idx = i + n1 (j + n2 k) of species s; Wall = all species.
template <class Acc, int GEO>
__device__ __forceinline__ typename Acc::T rhs_point(const RhsTables<typename Acc::T>& tb, const double* Wall,
                                                     int s, long long idx, int i, int j, int k) {
    using T = typename Acc::T;
    const double* W = Wall + (long long)s * tb.npts;
    const typename Acc::V c = Acc::load(W + idx);
    const T lap = laplacian<Acc, GEO>(tb, W, idx, i, j, k, c);
    T w[kMaxSpecies];
#pragma unroll
    for (int r = 0; r < kMaxSpecies; ++r) {
        if (r < tb.S) w[r] = (r == s) ? Acc::value(c) : Acc::value(Acc::load(Wall + (long long)r * tb.npts + idx));
        else w[r] = (T)0;
    }
    return tb.d[s] * lap + reaction<T>(tb.reac, w, s);
}

}  // namespace sexpe
