// Plan object of libsexpe (internal; shared by plan.cu and adjoint.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "host_setup.h"
#include "internal.h"
#include "launch.h"
#include "sexpe.h"

namespace sexpe {

constexpr int kGraphSteps = 10;   // steps captured per CUDA graph replay

struct Dir64 {
    int mu = 0;
    bool eigen = false;
    const double* V = nullptr;      // eigen: V and V^{-1} (row-major n x n, shared by species)
    const double* Vinv = nullptr;
    const double* P = nullptr;      // plain: phi_1(tau d_s A) per species, S x n x n
    const double* had = nullptr;    // eigen: Hadamard table per species, S x npts
};

// Tables of the discrete adjoint of one direction (built on the first adjoint call).
struct DirAdj {
    const double* VT = nullptr;      // eigen: V^T      (transform of the adjoint variable)
    const double* VinvT = nullptr;   // eigen: V^{-T}   (back-transform of the adjoint variable)
    const double* dhad = nullptr;    // eigen: d Phi / d d_s = tau s lambda phi_1'(tau d_s s lambda), S x npts
    const double* PT = nullptr;      // plain: phi_1(tau d_s A)^T per species, S x n x n
    const double* dP = nullptr;      // plain: d phi_1(tau d_s A) / d d_s per species, S x n x n
};

}  // namespace sexpe

struct sexpe_plan {
    int geometry = 0, precision = 0, S = 0, ndim = 0;
    int device = -1;                  // CUDA device current at setup; steps must run with it current
    int n[3] = {1, 1, 1};
    long long npts = 0;
    double tau = 0.0;
    std::vector<double> d, params;
    int reaction = 0;
    sexpe::Axis ax[3];
    std::vector<void*> allocs;
    size_t bytes = 0;
    int* d_err = nullptr;
    int* h_err = nullptr;             // pinned host copy of the error word (read by sexpe_synchronize)
    cudaStream_t cpl_stream = nullptr;   // split coupled plans: the surface component's stream
    cudaEvent_t cpl_ev[4] = {};          // its fork and join points within a step
    double* d_host_state = nullptr;   // staging buffer of sexpe_step_host
    // FP64 path
    sexpe::RhsTables<double> rhs64{};
    std::vector<sexpe::Dir64> dirs64;
    double* buf64[3] = {nullptr, nullptr, nullptr};
    const double* unsplit_P = nullptr;     // unsplit baseline: phi_1(tau d_s M), S x N x N
    // bulk-surface coupled plan (sexpe_coupled_setup): the bulk and surface sub-plans and the
    // arguments of the coupling kernel
    bool coupled = false;
    sexpe_plan* sub[2] = {nullptr, nullptr};
    sexpe::CoupleArgs cpl{};
    // split path
    sexpe::SplitTables tabs{};
    sexpe::TcShape sh3{}, shs{};
    // per-kernel profiling (CUDA events on the launching stream)
    std::vector<cudaEvent_t> prof_ev;
    int prof_max_steps = 0, prof_steps = 0, prof_slot = 0;
    bool profiling = false;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    double* g_state = nullptr;
    // adjoint (FP64 plans; built on the first sexpe_adjoint call)
    std::vector<sexpe::DirAdj> adj;
    sexpe::RhsTables<double> adj_diag{};   // rs slot holds the full diagonal a_l for M^T
    double* adj_buf = nullptr;              // work buffers of adjoint_step (plan.cu)
    double* adj_seg = nullptr;              // recomputed states of one checkpoint segment
    int adj_seg_cap = 0;
    double* adj_save = nullptr;             // forward chains of a segment's replayed steps
    int adj_save_cap = 0;
    double* adj_red = nullptr;              // device accumulators of the parameter gradient
    // split-TF32 sphere adjoint (built on the first sexpe_adjoint call of such a plan): the
    // transposed chain on the tensor-core kernels of the forward step with other operand images
    bool sadj_built = false;
    sexpe::Image sadj_PphiT[sexpe::kMaxSpecies] = {};   // phi_1(tau d_s A_phi)^T, N-tiled as Pphi
    sexpe::Image sadj_dPphi[sexpe::kMaxSpecies] = {};   // d phi_1(tau d_s A_phi) / d d_s, N-tiled
    const float* sadj_had_d = nullptr;     // d Phi / d d_s of the theta direction, layout of had_sph
    float* sadj_Yl = nullptr;              // adjoint variable (then tau P_theta lambda) in the chain layout
    float* sadj_Y3 = nullptr;              // (d phi_1(tau d_s A_phi) / d d_s) F in the chain layout
    float* sadj_Ymu = nullptr;             // mu in the chain layout
    double* sadj_T64[2] = {nullptr, nullptr};   // tau P_theta lambda, tau (d P_theta / d d_s) lambda
    double* sadj_MU = nullptr;             // mu in the state layout
    double* sadj_states = nullptr;         // replayed states, two segment buffers of sadj_seg_cap states
    float* sadj_seg = nullptr;             // per replayed step: F, P_phi F, (dP_phi/dd) F (chain layout), x 2
    cudaStream_t sadj_stream = nullptr;    // replay stream (overlaps the adjoint steps of the segment after)
    cudaEvent_t sadj_ev_replayed[2] = {nullptr, nullptr}, sadj_ev_swept[2] = {nullptr, nullptr};
    bool sadj_merged = false;              // the merged adjoint theta kernel fits (tensor memory, smem)
    sexpe::TcShape sadj_shape{};           // its rings and tensor-memory columns
    int sadj_nt = 0;                       // its output theta columns per CTA (measured split)
    sexpe::RhsTables<float> sadj_rhsT{};   // FP32 M^T in difference form (transposed off-diagonals, column sums)
    sexpe::Image sadj_Q{};                 // the N-tiled Q_theta image of that split
    int sadj_seg_cap = 0;                  // steps a segment buffer holds
    // batched independent disks (sexpe_batch_setup)
    bool batch = false;
    int n_instances = 1;
    std::vector<long long> inst_off;          // element offsets of the instances' states (count + 1)
    sexpe::BatchTables btab{};
    sexpe::TcShape bsh{};
    double* bstate = nullptr;                 // the other state buffer of the ping-pong
    int bparity = 0;                          // steps enqueued in the current sexpe_step call, mod 2
    int kernels_per_step = 0;
    double setup_ms = 0.0;
    float rhs_tj_us = 0.f;     // measured stencil time at the chosen tile height
    int batch_grid = 0;        // CTAs of the cooperative batch launch
    int batch_order = 0;       // work-list order the batch tuner kept (sexpe_plan_info.batch_order)
    float batch_step_us = 0.f; // measured batch step at the kept configuration
    std::vector<int> th_splits;            // split sphere: theta-kernel column splits built at setup
    std::vector<sexpe::Image> th_imgs;     // their N-tiled Q_theta images
    long long* d_step = nullptr;   // steps since setup / sexpe_set_time (time-dependent sources)
    std::vector<double> offset;    // lifting offsets of the reactions (empty = 0)
    double rho_pow = -2.0;         // D_rho = rho^rho_pow (disk: -2, or -2 - lambda for Delta_lambda)
    double t0 = 0.0;               // time of step 0 of the counter
};

