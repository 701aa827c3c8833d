/*
 * sexpe.h -- C ABI of the GB300 split exponential Euler library (libsexpe.so).
 *
 * The library integrates N-coupled diffusion-reaction systems
 *     w_s' = d_s M w_s + g_s(w),   M = M_1 + ... + M_d             (Section 2, eq. ODE)
 * on a disk (polar), sphere surface (Laplace-Beltrami), ball (spherical) or
 * cylinder (cylindrical coordinates) with the split exponential Euler method
 *     F_s     = d_s M w_s + g_s(w_n)
 *     w_s,n+1 = w_s,n + tau phi_1(tau d_s M_1) ... phi_1(tau d_s M_d) F_s
 * (Section 4, eqs. ee and splitorder), every phi_1 factor applied as mu-mode
 * products with precomputed per-direction phi_1 matrices or eigenbases and
 * Hadamard factors (eqs. ee_disk, ee_sphere, ee_ball, ee_cylinder).
 *
 * Conventions shared by every entry point
 *  - State layout: FP64, species outermost, then mode 3, mode 2, mode 1 with
 *    mode 1 contiguous (the paper's vector ordering w_{i+(j-1)n1+(k-1)n1n2},
 *    Section 2).  Modes: disk (rho, theta), sphere (theta, phi),
 *    ball (rho, theta, phi), cylinder (rho, theta, z).  No padding.
 *  - Pointers named *_dev are device pointers owned by the caller; pointers
 *    named *_host are host pointers owned by the caller.  The library never
 *    frees caller memory.  A plan owns all of its own device tables.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every call returns a sexpe_status and never aborts or prints.  Device-side
 *    waits are bounded: a wait that runs out records SEXPE_ETIMEOUT, which the
 *    next sexpe_synchronize() on the plan reports.
 *  - Calls on one plan are not thread-safe; distinct plans are independent.
 */
#ifndef SEXPE_H
#define SEXPE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SEXPE_OK = 0,
    SEXPE_EINVAL = 1,        /* bad argument (size, pointer, tau, species count, ...)        */
    SEXPE_ENOMEM = 2,        /* device or host allocation failed                             */
    SEXPE_ECUDA = 3,         /* a CUDA runtime call failed                                   */
    SEXPE_ETIMEOUT = 4,      /* a bounded device-side wait ran out                           */
    SEXPE_EUNSUPPORTED = 5,  /* valid request this build does not implement                  */
    SEXPE_ENUMERIC = 6       /* setup produced a non-finite table                            */
} sexpe_status;

typedef enum { SEXPE_DISK = 0, SEXPE_SPHERE = 1, SEXPE_BALL = 2, SEXPE_CYLINDER = 3 } sexpe_geometry;

/* Arithmetic of the per-step chain.  FP64: every operation in FP64 (SIMT).
 * SPLIT_TF32: stencil differences at FP64 accuracy, F rounded to FP32, every
 * mu-mode product on tcgen05 tensor cores as three TF32 products
 * (hi*hi + hi*lo + lo*hi, each operand split x = hi + lo with both parts
 * rounded to TF32) accumulated in FP32 in tensor memory; the state stays FP64. */
typedef enum { SEXPE_FP64 = 0, SEXPE_SPLIT_TF32 = 1, SEXPE_UNSPLIT_FP64 = 2 } sexpe_precision;
/* UNSPLIT_FP64 is not the split method: it is unsplit exponential Euler (eq. ee
 * with phi_1 of the whole operator, w_s += tau phi_1(tau d_s M) F_s,
 * M = M_1 + ... + M_d the assembled Kronecker sum), the accuracy baseline that
 * the splitting error of Section 4 is measured against.  phi_1(tau d_s M) is
 * formed densely at setup by the same [13/13] Pade scaling and squaring, so it
 * is limited to grids of at most 2048 points (larger: SEXPE_EUNSUPPORTED); a
 * step is the FP64 stencil+reaction and one dense FP64 matrix-vector product
 * per species with the update fused.  No adjoint, no batch. */

/* Reaction terms g_s(w), evaluated pointwise.
 *   SCHNAKENBERG (S=2), params {gamma, a, b}: f = gamma(a - u + u^2 v), g = gamma(b - u^2 v)
 *   GRAY_SCOTT   (S=2), params {F, k}:        f = -u v^2 + F(1-u),      g = u v^2 - (F+k) v
 *   LINEAR_CUBIC (S<=4), params K row-major S x S: f_i = sum_j K_ij u_j - u_i^3
 *   LINEAR (S<=4), params K row-major S x S: f_i = sum_j K_ij u_j (the bulk kinetics
 *       b(u) = -alpha1 (u - alpha2), c(v) = -beta1 (v - beta2) of Section 5.6 on the
 *       lifted state w = (u - alpha2, v - beta2) are K = diag(-alpha1, -beta1))
 *   BVAM (S=2), params {alpha1, alpha2, alpha3, beta1, beta2} (Section 5.1, eq. BVAMnl):
 *       b = alpha1 u (1 - alpha2 v^2) + v (1 - alpha3 u),
 *       c = beta1 v (1 + alpha1 alpha2 / beta1 u v) + u (beta2 + alpha3 v)
 *   BVAM_MANUFACTURED (S=2, disk only): BVAM plus the sources of Section 5.1 that
 *       make u = e^-t (1 - rho)^2 e^{cos(theta)/10}, v = e^-t (1 - rho)^2 e^{sin(theta)/10}
 *       a solution of eq. (BVAMsys) with diffusion d = (gamma, delta): the source of u is
 *       u_t - gamma Lap u - b(u, v) at the exact solution (polar Laplacian of eq. lapdisk
 *       applied analytically), likewise for v; evaluated explicitly at t_n = t0 + n tau,
 *       n the plan's steps since setup or sexpe_set_time (t0 = 0 at setup).
 *   NONE: g = 0 (any S <= 4, no params).                                            */
typedef enum {
    SEXPE_REACTION_NONE = 0,
    SEXPE_SCHNAKENBERG = 1,
    SEXPE_GRAY_SCOTT = 2,
    SEXPE_LINEAR_CUBIC = 3,
    SEXPE_BVAM = 4,
    SEXPE_BVAM_MANUFACTURED = 5,
    SEXPE_LINEAR = 6
} sexpe_reaction;

/* Height axis of the cylinder: NEUMANN = homogeneous Neumann at both caps
 * (node-centred, h = z_star/(n-1)); PAPER = Neumann at 0 and Dirichlet at z_star
 * exactly as eq. (A_z). */
typedef enum { SEXPE_Z_NEUMANN = 0, SEXPE_Z_PAPER = 1 } sexpe_zbc;

typedef struct {
    int32_t geometry;   /* sexpe_geometry                                                 */
    int32_t n[3];       /* points per mode, mode 1 first (n[2] ignored for disk/sphere);   */
                        /* each >= 3 and <= 512 (theta >= 3, rho >= 2, phi/z >= 3)        */
    double rho_star;    /* radius of disk/ball/cylinder (> 0); sphere is the unit sphere  */
    double z_star;      /* cylinder height (> 0)                                          */
    int32_t z_bc;       /* sexpe_zbc (cylinder only)                                      */
    int32_t rho_op;     /* disk only: 0 = Laplacian, Neumann at rho_* (eq. disk_discr);     */
                        /* 1 = anomalous Delta_lambda (Section 5.3, eq. anomalous) with     */
                        /* homogeneous Dirichlet at rho_* (eq. A_lambda; lift constant      */
                        /* boundary values with sexpe_species.offset_host), D_rho = rho^(-2-lambda) */
    double lambda;      /* exponent of Delta_lambda, -3 < lambda < 1 (rho_op = 1)          */
} sexpe_grid;

typedef struct {
    int32_t n_species;      /* 1..4                                                       */
    const double* d_host;   /* n_species diffusion coefficients (> 0)                     */
    int32_t reaction;       /* sexpe_reaction                                             */
    int32_t n_params;       /* number of entries in params_host                           */
    const double* params_host;
    const double* offset_host;   /* n_species values c_s or NULL (= 0): the reactions see w_s + c_s,
                                    the lifting of constant Dirichlet boundary values c_s (the
                                    state is w = u - c); FP64 adjoint and batches need NULL   */
} sexpe_species;

typedef struct sexpe_plan sexpe_plan;

typedef struct {
    int32_t geometry, precision, n_species, ndim;
    int32_t n[3];
    int32_t n_instances;        /* 1, or the count given to sexpe_batch_setup               */
    int32_t kernels_per_step;   /* kernel launches of one step                              */
    int64_t npts;               /* grid points per species (sum over instances for a batch) */
    int64_t state_elems;        /* FP64 elements of the whole state                         */
    int64_t workspace_bytes;    /* device bytes owned by the plan                           */
    double setup_ms;            /* host wall time of the FP64 setup                         */
    int32_t stencil_tile_j;     /* split path: j-lines per stencil tile (measured at setup)  */
    int32_t ring_slots[2];      /* split path: matrix and data slots of the slab pass ring   */
    float stencil_tile_us;      /* split path: measured stencil time at that tile height     */
    int32_t stencil_planes;     /* split path: 0 = tiled stencil kernel, else k-planes per CTA
                                   of the rolling-window kernel (measured at setup)          */
    int32_t stencil_ctas_per_sm; /* split path: CTAs per SM the rolling-window stencil's
                                   registers allow (1 or 2); 0 with stencil_planes > 0 = the
                                   k-marching kernel                                          */
    int32_t theta_split;        /* split sphere: CTAs sharing one row tile of the theta kernel,
                                   each with n_theta_pad / theta_split output columns
                                   (measured at setup); 0 elsewhere                         */
    int32_t batch_order;        /* batch plans: work-list order the setup's tuner kept:
                                   0 = (instance, species) items longest first,
                                   1 = instances longest first, both species adjacent;
                                   for batch plans stencil_tile_j is the theta-lines per
                                   stencil tile and ring_slots the ring depths it kept       */
    float batch_step_us;        /* batch plans: measured step time at that configuration     */
} sexpe_plan_info;

/* Build a plan: FP64 host setup of the 1-D axes (Section 3: eqs. A_theta,
 * disk_discr, ball_discr, syscn/A_phi, A_z), phi_1(tau d_s A_mu) of every plain
 * direction (Pade [13/13] scaling and squaring on [[tau d A, I],[0,0]]), the
 * eigenbases of the scaled directions (closed-form real Fourier basis for
 * A_theta; Proposition 1 symmetrisation + implicit QL for A_phi), the Hadamard
 * factors phi_1(tau d_s s lambda) (Section 4), then one upload to the device.
 * The plan also owns the intermediate tensors of the chain.  `stream` orders
 * the uploads.  On error *out is set to NULL. */
sexpe_status sexpe_setup(const sexpe_grid* grid, const sexpe_species* species, double tau,
                         int32_t precision, void* stream, sexpe_plan** out);

/* Build one plan for `count` independent disk problems of uneven sizes
 * (geometry must be SEXPE_DISK for all; each instance has its own species
 * block).  Their states are concatenated instance after instance, each in the
 * single-plan layout; sexpe_state_offsets() gives the element offsets.  Steps
 * run as one persistent cooperative launch per step: a stencil phase over
 * tiles of theta-lines of every instance, a bounded grid barrier, then the
 * disk chain of eq. ee_disk per (instance, species) item from a work list.
 * The setup times every feasible combination of ring depths, stencil tile
 * height (8, 16 or 32 lines) and work-list order on `stream` and keeps the
 * fastest (sexpe_plan_info reports the choice and its time).  Split-TF32 only;
 * n_rho <= 128, n_theta <= 256. */
sexpe_status sexpe_batch_setup(int32_t count, const sexpe_grid* grids, const sexpe_species* species,
                               double tau, int32_t precision, void* stream, sexpe_plan** out);

/* offsets_host[count+1]: element offset of each instance's state (last = total). */
sexpe_status sexpe_state_offsets(const sexpe_plan* plan, int64_t* offsets_host);

/* Advance state_dev (caller-owned device FP64 array of state_elems elements,
 * layout above, 8-byte aligned) by n_steps split exponential Euler steps, in
 * place, enqueued on `stream`.  No allocation, no host synchronisation.
 * n_steps >= 0.  The device current at the call must be the one the plan was
 * made on (SEXPE_EINVAL otherwise, as for an unaligned state). */
sexpe_status sexpe_step(sexpe_plan* plan, double* state_dev, int64_t n_steps, void* stream);

/* Same as sexpe_step for a HOST state: copies state_host to the plan's device
 * buffer, steps, copies back, and synchronises `stream` before returning.
 * state_host should be page-locked for asynchronous copies. */
sexpe_status sexpe_step_host(sexpe_plan* plan, double* state_host, int64_t n_steps, void* stream);

/* The split-TF32 step without any device allocation, for callers that cannot
 * call cudaMalloc (a region captured into a CUDA graph in the global capture
 * mode, a host framework that owns all device memory through its own pool, a
 * loop under a fixed memory budget).  The paper has no counterpart: this is a
 * deployment variant of sexpe_step.
 *  - plan: a SEXPE_SPLIT_TF32 plan made earlier on the current device (its
 *    constant tables are read); state_dev as for sexpe_step (in place,
 *    8-byte aligned).  A plan made on another device, an unaligned state,
 *    FP64, batch or coupled plans give SEXPE_EINVAL before anything is
 *    enqueued.
 *  - The step's only scratch, the FP32 intermediate between its kernels,
 *    lives in a static device array of 2^21 floats (8 MiB) that every GPU
 *    loading the library holds until exit; plans with species x points above
 *    2,097,152 (rho lines padded to a multiple of 4) give SEXPE_EINVAL.  No
 *    cudaMalloc/cudaFree or allocating library routine is called.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents.
 *    Each step writes every value it later reads; the padding slots of the
 *    rho lines, which no kernel writes, are zeroed by each call (a 2-D
 *    memset on `stream`, no allocation).  Calls whose work overlaps on the
 *    GPU (other streams, other threads) race on the array: serialise them.
 *  - Results equal sexpe_step's, bit for bit, for the same plan and state
 *    (the same kernels run; only the intermediate's address differs). */
sexpe_status sexpe_step_noalloc(sexpe_plan* plan, double* state_dev, int64_t n_steps, void* stream);

/* Bulk-surface coupled systems (Sections 5.5 and 5.6): two bulk species on a 3-D
 * grid and two surface species on a 2-D grid that is part of its boundary,
 * coupled through flux boundary conditions of the bulk and through the surface
 * kinetics.  The paper omits the coupled discretisation; this one keeps each
 * bulk axis as printed and lets a normal derivative g = grad w . n enter the
 * boundary row through the same virtual point that gives the row its Neumann
 * form; all coupling terms are explicit at t_n with the reactions, and each
 * component takes its own geometry's split step.
 *
 *  SEXPE_COUPLING_SCHNAKENBERG_BALL (Section 5.5, eqs. bulkball): bulk u, v on
 *    the ball `bulk_grid` (SEXPE_BALL; `bulk`: diffusion d_u, d_v = delta and its
 *    reaction, alpha1 (b, c) by SCHNAKENBERG with params {alpha1, alpha2, beta1});
 *    surface r, s on the boundary sphere rho = rho_* whose grid is the ball's
 *    theta x phi grid (`surface`: diffusion 1/rho_*^2 and eps/rho_*^2, reaction
 *    zeta1 (b, c)).  grad u . n = zeta1 (zeta2 r - zeta3 u) and
 *    delta grad v . n = zeta1 (eta1 s - eta2 v) enter the outer radial row of
 *    eq. ball_discr as (2/h + 2/rho_*) times d_u grad u . n and delta grad v . n
 *    (h the radial step); the surface F loses zeta1 (zeta2 r - zeta3 u) and
 *    zeta1 (eta1 s - eta2 v).  Uses zeta[0..2], eta[0..1].
 *  SEXPE_COUPLING_DIB_CYLINDER (Section 5.6, eqs. bulkcyl): bulk u, v on the
 *    cylinder `bulk_grid` (SEXPE_CYLINDER with z_bc = SEXPE_Z_PAPER: Neumann at
 *    z = 0, Dirichlet at z_*), its state LIFTED by the top values,
 *    w = (u - u_top, v - v_top) (`bulk`: diffusion 1, delta and its reaction on w,
 *    e.g. LINEAR with K = diag(-alpha1, -beta1)); surface r, s on the bottom disk
 *    z = 0 whose grid is the cylinder's rho x theta grid (`surface`: diffusion 1,
 *    eps; reaction usually NONE).  With u = w_u + u_top, v = w_v + v_top on z = 0,
 *      p = zeta2 u (1 - s) r - zeta3 r^3 - zeta4 (s - zeta5),
 *      q = eta1 v (1 + eta2 r)(1 - s)(1 - eta3 (1 - s)) - eta4 (1 + eta5 r) s (1 + eta3 s),
 *    the surface F gains zeta1 p, zeta1 q, and grad u . n = -zeta1 alpha3 p,
 *    grad v . n = -zeta1 beta3 q enter the z = 0 row of eq. A_z as 2/h_z times
 *    d_u grad u . n and d_v grad v . n.  Uses zeta[0..4], eta[0..4], alpha3,
 *    beta3, u_top, v_top.
 *
 * State (device, FP64, caller-owned): [bulk species 0][1] in the bulk grid's
 * layout, then [surface 0][1] in the surface grid's layout (sphere: theta
 * fastest; disk: rho fastest), 2 (N_bulk + N_surface) elements.  Precision
 * SEXPE_FP64 (FP64 SIMT chains) or SEXPE_SPLIT_TF32 (each grid's tensor-core
 * chain, within its size limits; the coupling terms formed in FP64 and added to
 * the FP32 F); SEXPE_UNSPLIT_FP64 gives SEXPE_EUNSUPPORTED.  Both species sets
 * must have 2 species; no lifting offsets (SEXPE_EINVAL), no adjoint, no
 * sexpe_set_stencil / sexpe_set_theta_split (SEXPE_EUNSUPPORTED), no
 * sexpe_step_noalloc (SEXPE_EINVAL).  Step with sexpe_step / sexpe_step_host;
 * destroy with sexpe_destroy.  Other errors as sexpe_setup.  sexpe_plan_info
 * reports n_species = 4, npts of the bulk grid, the bulk grid's tile choices
 * and the device bytes of both sub-plans.  A SEXPE_SPLIT_TF32 plan owns a
 * second (non-blocking) CUDA stream: each step forks the surface grid's
 * kernels onto it from the caller's stream with an event and joins them back
 * with events, so the step stays ordered on the caller's stream (graph
 * capture included) while the two grids' chains overlap on the GPU. */
typedef enum { SEXPE_COUPLING_SCHNAKENBERG_BALL = 0, SEXPE_COUPLING_DIB_CYLINDER = 1 } sexpe_coupling_kind;
typedef struct {
    int32_t kind;            /* sexpe_coupling_kind                                       */
    double zeta[5];          /* zeta1 .. zeta5                                            */
    double eta[5];           /* eta1 .. eta5                                              */
    double alpha3, beta3;    /* DIB: scalings of the bulk fluxes                           */
    double u_top, v_top;     /* DIB: Dirichlet values on z = z_*, by which the bulk is lifted */
} sexpe_coupling;
sexpe_status sexpe_coupled_setup(const sexpe_grid* bulk_grid, const sexpe_species* bulk,
                                 const sexpe_species* surface, const sexpe_coupling* cp, double tau,
                                 int32_t precision, void* stream, sexpe_plan** out);

/* Host-only evaluation of the coupling terms a coupled plan adds every step (introspection and
 * testing; no device work, no plan): for n surface points with the bulk species' boundary values
 * (ub, vb; the DIB kind takes the lifted values w) and the surface values (r, s), writes what the
 * step adds to the bulk F of the boundary node (add_b0, add_b1) and to the surface F (add_s0,
 * add_s1), with the virtual-point factor and the bulk diffusion taken from bulk_grid and bulk as
 * in sexpe_coupled_setup.  All arrays host, n doubles, caller-owned.  Arguments are checked as by
 * sexpe_coupled_setup (the surface species aside); n < 0 or a NULL array with n > 0 gives
 * SEXPE_EINVAL.  The host compiles the same source as the coupling kernels, but the device
 * compiler may contract its multiply-adds into FMAs, so host and device results agree to FP64
 * rounding, not bit for bit. */
sexpe_status sexpe_coupling_terms(const sexpe_grid* bulk_grid, const sexpe_species* bulk, const sexpe_coupling* cp,
                                  int64_t n, const double* ub, const double* vb, const double* r, const double* s,
                                  double* add_b0, double* add_b1, double* add_s0, double* add_s1);

/* Wait for the plan's work on `stream` and report the device error word
 * (SEXPE_ETIMEOUT if a bounded wait ran out), clearing it. */
sexpe_status sexpe_synchronize(sexpe_plan* plan, void* stream);

sexpe_status sexpe_plan_get_info(const sexpe_plan* plan, sexpe_plan_info* info_host);

/* Override the stencil configuration that sexpe_setup measured for a split
 * plan (no counterpart in the paper: the tile shapes are this implementation's
 * own): tile_j j-lines per CTA with planes = 0 and ctas_per_sm = 1 for the
 * tiled kernel; for the 3-D geometries, planes k-planes per CTA of the
 * rolling-window kernel with its registers capped for ctas_per_sm (1 or 2)
 * CTAs per SM, or, with ctas_per_sm = 0, of the k-marching kernel (one thread
 * per (j, i) column of the tile_j lines, k-neighbours in registers).
 * The triple must be one the setup timed (sexpe_plan_info reports the chosen one);
 * others give SEXPE_EINVAL, FP64 and batch plans SEXPE_EUNSUPPORTED.  A graph
 * captured by an earlier sexpe_step is dropped and captured again.  Host-side
 * only; call it when no step of the plan is being enqueued by another thread. */
sexpe_status sexpe_set_stencil(sexpe_plan* plan, int32_t tile_j, int32_t planes, int32_t ctas_per_sm);

/* Override the theta-kernel column split that sexpe_setup measured for a split
 * sphere plan (no counterpart in the paper).  The theta step of eq. ee_sphere
 * is two products per tile of 128 phi rows, x_1 Q_theta^T, the Hadamard factor,
 * then x_1 Q_theta with the update; the second can be split by output theta
 * columns over `split` CTAs (1, 2, 4 or 8, n_theta rounded up to 16 divisible
 * by 16 * split), each repeating the first product.  A split the setup did not
 * build gives SEXPE_EINVAL, other plans SEXPE_EUNSUPPORTED.  A graph captured
 * by an earlier sexpe_step is dropped.  Host-side only, like sexpe_set_stencil. */
sexpe_status sexpe_set_theta_split(sexpe_plan* plan, int32_t split);

/* Time of the next step of a plan with time-dependent sources
 * (SEXPE_BVAM_MANUFACTURED): the next step evaluates its sources at t, the one
 * after at t + tau, and so on.  Resets the plan's device step counter (ordered on
 * `stream`); a captured step graph is dropped.  Other plans: SEXPE_OK, no effect. */
sexpe_status sexpe_set_time(sexpe_plan* plan, double t, void* stream);

/* Self-test of the failure path of every device wait (no counterpart in the
 * paper): one thread waits on a barrier nobody arrives on, with a limit of
 * about 1 ms; the wait gives up, records the timeout in a device error word
 * and the kernel returns.  Returns SEXPE_ETIMEOUT -- the status a plan's
 * sexpe_synchronize reports after such a timeout -- when that happened, and
 * the CUDA context stays usable; SEXPE_ECUDA if the word was not written.
 * Allocates and frees one int of device memory; synchronises `stream`. */
sexpe_status sexpe_selftest_wait_timeout(void* stream);

/* Free every device table of the plan (after synchronising its device). */
sexpe_status sexpe_destroy(sexpe_plan* plan);

/* Forward steps that also keep checkpoints for sexpe_adjoint: like sexpe_step,
 * and before every step k with k % every == 0 the current state is copied to
 * checkpoints_dev + (k / every) * state_elems (caller-owned device buffer of
 * ceil(n_steps / every) states).  Enqueued on `stream`. */
sexpe_status sexpe_step_checkpointed(sexpe_plan* plan, double* state_dev, int64_t n_steps, int32_t every,
                                     double* checkpoints_dev, void* stream);

/* Discrete adjoint of n_ckpt * every steps (the adjoint of the step map of
 * eqs. ee/splitorder; the paper has no adjoint).  Given checkpoints_dev from
 * sexpe_step_checkpointed (n_ckpt states, `every` steps apart) and the
 * gradient of a scalar loss with respect to the final state, dL_dWT_dev, it
 * writes the gradient with respect to the initial state to dL_dW0_dev (may
 * alias dL_dWT_dev) and, if dL_dparams_host is not NULL, the parameter
 * gradient in the order: the reaction parameters as given to sexpe_setup,
 * then d_s for every species.  Per step, with mu_s = tau P_s^T lambda_s:
 * lambda_r <- lambda_r + d_r M^T mu_r + sum_s (dg_s/dw_r) mu_s, where P_s^T is
 * the transposed phi_1 chain in reverse order; dL/dd_s adds <mu_s, M w_s> and
 * tau <lambda_s, (dP_s/dd_s) F_s> with dphi_1(tau d s A)/dd = V diag(tau s lambda
 * phi_1'(tau d s lambda)) V^{-1}, phi_1' = phi_1 - phi_2.  Each checkpoint
 * segment is recomputed forward.  FP64 plans of every geometry, and
 * SEXPE_SPLIT_TF32 sphere plans (eq. ee_sphere): there the adjoint
 * differentiates the split forward, whose replayed states it uses, and every
 * product of the transposed chain runs on the forward's tensor-core kernels
 * in split TF32 with FP32 accumulation -- tau P_theta lambda and
 * tau (dP_theta/dd_s) lambda by the theta kernel (P_theta = Q diag(Phi) Q^T is
 * symmetric), mu = phi_1(tau d_s A_phi)^T (tau P_theta lambda) and
 * (dphi_1(tau d_s A_phi)/dd_s) F by the phi kernel with transposed and
 * differentiated operand images -- while lambda, the transposed stencil with
 * the reaction Jacobian and the parameter sums stay FP64.  Other plans give
 * SEXPE_EUNSUPPORTED, a plan of another device SEXPE_EINVAL.  The first call
 * builds the adjoint tables and work buffers (device allocations); the
 * parameter gradient is copied to the host and the stream synchronised when
 * dL_dparams_host is given. */
sexpe_status sexpe_adjoint(sexpe_plan* plan, const double* checkpoints_dev, int32_t n_ckpt, int32_t every,
                           const double* dL_dWT_dev, double* dL_dW0_dev, double* dL_dparams_host, void* stream);

/* Per-kernel timing.  After sexpe_profile_begin(plan, max_steps), the next
 * steps (up to max_steps, across sexpe_step calls on one stream) launch their
 * kernels directly (no graph) with a CUDA event recorded on the launching
 * stream before each kernel and after the last.  sexpe_profile_end waits for
 * the last event and writes, for each kernel slot of a step in launch order,
 * the average duration in milliseconds to kernel_ms_host[0..n) (n = kernels
 * per step, capped at `cap`), stores n in *n_kernels_host, and turns
 * profiling off.  The events are created in begin and destroyed in end. */
sexpe_status sexpe_profile_begin(sexpe_plan* plan, int32_t max_steps);
sexpe_status sexpe_profile_end(sexpe_plan* plan, double* kernel_ms_host, int32_t* n_kernels_host, int32_t cap);

/* Setup introspection (host only, FP64, no GPU needed): the quantities the
 * plan is built from, for checking the setup stage on its own.
 * axis: 0 theta (eq. A_theta), 1 rho d=2 (eq. disk_discr), 2 rho d=3
 * (eq. ball_discr), 3 phi (eqs. syscn, A_phi), 4 z with Neumann caps,
 * 5 z as in eq. (A_z).  extent = rho_* or z_* (ignored for theta, phi).
 * sexpe_axis_matrix: A (n x n, row-major) into A_host.
 * sexpe_axis_phi1:   phi_1(t A) by the plan's Pade route into out_host (n x n).
 * sexpe_axis_eigen:  A = V diag(lam) Vinv by the plan's route (closed form for
 *                   theta, Proposition 1 + implicit QL otherwise); any output may be NULL. */
sexpe_status sexpe_axis_matrix(int32_t axis, int32_t n, double extent, double* A_host);
sexpe_status sexpe_axis_phi1(int32_t axis, int32_t n, double extent, double t, double* out_host);
sexpe_status sexpe_axis_eigen(int32_t axis, int32_t n, double extent, double* lam_host, double* V_host,
                              double* Vinv_host);

/* Static, never-NULL description of a status code. */
const char* sexpe_status_string(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* SEXPE_H */
