// Internal types shared by the plan (host) and the kernels of libsexpe.
#pragma once
#include <cstdint>

namespace sexpe {

enum Geo { GEO_DISK = 0, GEO_SPHERE = 1, GEO_BALL = 2, GEO_CYLINDER = 3 };
enum Reac { R_NONE = 0, R_SCHNAKENBERG = 1, R_GRAY_SCOTT = 2, R_LINEAR_CUBIC = 3, R_BVAM = 4, R_BVAM_MMS = 5, R_LINEAR = 6 };

constexpr int kMaxSpecies = 4;
constexpr int kMaxN = 512;

// Device error word values (first error wins).
enum DevErr { DERR_NONE = 0, DERR_TIMEOUT_TMA = 1, DERR_TIMEOUT_MMA = 2, DERR_BAD_TILE = 3 };

// One axis of the stencil: (A w)_r = lower[r](w_{r-1} - w_r) + upper[r](w_{r+1} - w_r) + rs[r] w_r,
// rs = row sum (zero for Neumann/periodic rows).  Periodic axes wrap r-1 / r+1.
template <class T>
struct StencilAxis {
    const T* lower;
    const T* upper;
    const T* rs;
    int n;
    int periodic;
};

// Bulk-surface coupling terms, one thread per surface point q (Sections 5.5 and 5.6).
// kind 0: ball + boundary sphere, q = j + n_theta k, bulk node (n_rho - 1, j, k);
// kind 1: cylinder + bottom disk, q = i + n_rho j, bulk node (i, j, 0).
struct CoupleArgs {
    int kind;
    int bn1, bn2;            // bulk points along modes 1 and 2
    int sn1;                 // surface points along its mode 1
    long long nb, ns;        // points per species of the bulk and of the surface
    double coef;             // ball: 2/h + 2/rho_*; cylinder: 2/h_z (the virtual-point factor)
    double d0, d1;           // bulk diffusion
    double z[5], e[5];       // zeta1..5, eta1..5
    double a3, b3;           // flux scalings (kind 1)
    double u_top, v_top;     // lifting of the bulk state (kind 1)
};

template <class T>
struct ReactionParams {
    int kind;
    int S;
    T p[16];     // in the arithmetic type of the kernels that read them (no conversions on the device)
    T off[kMaxSpecies];   // lifting offsets: the reaction sees w_s + off_s
    int lifted;           // Schnakenberg with offsets: evaluated in the exact expansion about off
    T q[6];               // its coefficients (FP64 on the host): g_u(c)/gamma, g_v(c)/gamma, 2 c_u c_v,
                          // c_u^2, c_v, 2 c_u
};

// Everything the stencil+reaction evaluation needs (values of type T).
template <class T>
struct RhsTables {
    int geometry;
    int S;
    int n1, n2, n3;
    long long npts;
    StencilAxis<T> ax[3];
    const T* Dr;   // rho_i^-2 (mode-1 index), disk/ball/cylinder
    const T* Dp;   // sin^-2 phi_k (phi-mode index), sphere/ball
    T d[kMaxSpecies];
    ReactionParams<T> reac;
    // manufactured sources (R_BVAM_MMS, disk): per rho_i {R, R'' + R'/rho, R/rho^2} with
    // R = (1 - rho)^2, per theta_j {T, T'', S, S''} with T = e^{cos/10}, S = e^{sin/10};
    // time t0 + (*step) tau
    const T* mms_rho;
    const T* mms_theta;
    const long long* step;
    double t0, tau_t;
};

// ---------------- FP64 SIMT path ------------------------------------------
// C(b, r, c) = sum_k A(b, r, k) B(b, k, c); element strides given per operand.
struct Gemm64 {
    int R, C, K, batch;
    const double* A; long long a_b, a_r, a_k;
    const double* B; long long b_b, b_k, b_c;
    double* out;     long long o_b, o_r, o_c;
    const double* had;      // Hadamard factor at the output index (or null)
    double* upd;            // if set: upd[idx] += tau * value (out ignored)
    double tau;
    // per-species offsets (blockIdx.z)
    long long A_sp, B_sp, out_sp, had_sp, upd_sp;
};

// ---------------- split TF32 tensor-core path -----------------------------
// Shared-memory operand tiles: K-major, no swizzle, core matrices of 8 rows x 16 B.
// Within a tile of R rows and kKC (=16) K-columns: byte offset of (r, k) is
// (r/8)*kSBO + (k/4)*kLBO + (r%8)*16 + (k%4)*4.
constexpr int kKC = 16;               // K elements per pipeline chunk
constexpr int kLBO = 128;             // bytes between K-adjacent core matrices
constexpr int kSBO = 512;             // bytes between M/N-adjacent 8-row groups
constexpr int kTileRowBytes = 64;     // bytes per row of one tile (16 fp32)

// Pre-laid matrix image: for every K-chunk c: [hi tile (rows_pad x 16)][lo tile].
struct Image {
    const float* ptr;
    int rows_pad;        // multiple of 16 (B operand) or of 128 (A operand)
    int k_chunks;
    long long chunk_floats;   // 2 * rows_pad * 16
};

struct SplitTables {
    int geometry, S;
    int n1, n2, n3;
    long long npts;
    RhsTables<float> rhs;     // FP32 coefficients (differences are formed at FP64 accuracy)
    const double* state;      // read by the stencil pass
    double* state_upd;        // updated in the slab epilogue
    float* Y;                 // FP32 chain buffer: F from the stencil pass, overwritten in place
                              // by the mode-3 pass, read by the slab pass; layout [s][k][j][n1q]
    int n1q;                  // n1 rounded up to a multiple of 4 (16-byte rows for bulk copies)
    long long ys;             // floats per species of Y: n3 * n2 * n1q
    float tau;
    double tau_d;
    // slab pass (theta then rho)
    Image QT, Q, P[kMaxSpecies];
    const float* had_theta;   // Phi table of the theta direction, [s][k][j'][n1q] (ball) or [s][j'][n1q]
    long long had_theta_sp;   // floats per species
    // mode-3 pass
    Image M3a, M3b[kMaxSpecies];   // ball: Vinv (M3a) and V (M3b[0]); cylinder: Pz_s in M3b[s]
    const float* had_phi;          // ball: Phi table of the phi direction, [s][k'][n1q]
    // sphere (mode 1 theta, mode 2 phi): phi direction (plain) into Y2, then theta (scaled) + update
    Image Pphi[kMaxSpecies];       // phi_1(tau d_s A_phi) as B operand, N-tiled: tile t (rows
                                   // [t phi_nt, (t + 1) phi_nt)) at ptr + t * k_chunks * chunk_floats
    int phi_nt;                    // output phi rows per CTA of the phi product
    int phi_ks;                    // CTAs (one cluster) sharing the K range of one phi output tile
    float* Y2;                     // phi product output, layout of Y
    const float* had_sph;          // phi_1(tau d_s sin^-2 phi_j lambda_theta'), [s][j][n1q]
    Image Qsph;                    // Q_theta as B operand of the second theta product, N-tiled by th_nt rows
    int th_nt;                     // output theta columns per CTA of the theta kernel
    // split sphere adjoint: a second image set and output of the phi kernel (phi_pair = 1 doubles
    // its grid: species s of the second half multiplies by Pphi2[s] into Y3)
    Image Pphi2[kMaxSpecies];
    float* Y3;
    int phi_pair;
    int* err;
    int rhs_tj;                    // j-lines per stencil tile (chosen by measurement at setup; 0 = model)
    int rhs_ks;                    // 0: tiled stencil kernel; > 0: rolling-window kernel, planes per CTA
    int rhs_mb;                    // rolling-window kernel: registers capped for this many CTAs per SM
    int theta_comp;                // slab pass: compensated theta-mean coefficient (disks, coupled plans)
};

// Arguments of the split sphere adjoint's theta kernel (see k_tc_sphere_theta_adj).
struct SphereAdjArgs {
    const float* lam32;       // adjoint variable rounded to FP32, chain layout [s][j][n1q]
    const float* had_d;       // d Phi / d d_s of the theta direction, layout of had_sph
    float* tpl;               // out: tau P_theta lambda, chain layout [s][j][n1q]
    const float* Y2;          // P_phi F at the step's state, chain layout
    const float* Y3;          // (dP_phi / dd_s) F, chain layout
    double* acc_d;            // acc_d[s] += <tau dP_theta lambda, Y2> + <tau P_theta lambda, Y3>
};

// ---------------- batched independent disks (split-TF32) -------------------
struct BatchInstance {
    int n1, n2;                     // rho, theta points
    long long w_off;                // element offset of the instance's state (species blocks of n1 n2)
    long long f_off;                // float offset of the instance's F block, [s][j][n1q]
    Image QT, Q, P[2];              // theta transforms and phi_1(tau d_s A_rho) images
    const float* had;               // Phi of the theta direction, [s][j'][n1q], n1q = n1 rounded up to 4
    StencilAxis<float> ax_rho, ax_theta;
    const float* Dr;                // rho_i^-2
    float d[2];
    ReactionParams<float> reac;
};

struct BatchTables {
    const BatchInstance* inst;
    const int2* items;              // (instance, species), longest first
    int n_items;
    int* counter;                   // [0] chain work-list cursor, [1] grid barrier, [2] stencil-tile cursor;
                                    // zeroed before every launch
    const int2* ftiles;             // phase-1 stencil tiles (instance, first theta-line)
    int n_ftiles;
    int tj;                         // theta-lines per phase-1 tile
    int tile_f2;                    // float2 slots of one phase-1 tile buffer (two buffers in the rings)
    float* F;                       // F of every instance (phase 1 -> phase 2)
    const double* W_in;             // state before the step (all instances)
    double* W_out;                  // state after the step
    float tau;
    int* err;
};

}  // namespace sexpe
