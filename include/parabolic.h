/*
 * parabolic.h -- C ABI of libparabolic, a GB300 (sm_103a) library that advances the
 * operator-split parabolic operators of a thermodynamic MHD model over one time step under the
 * practical time-step limit (PTL) of Caplan et al., "Advancing parabolic operators in
 * thermodynamic MHD models II" (arXiv:2403.01004).
 *
 * Operators (Sec. 2, Eq. 2):
 *   PB_TC_ANISO  field-aligned thermal conduction  F(T) = C/n div(kappa bb . grad T),
 *                kappa = T0^{5/2} lagged (frozen for the step), C = (gamma-1)/2 with
 *                gamma = 5/3 (m_p/k, kappa_0 and the f_c, f_m profiles folded to 1).
 *   PB_VISC_ISO  artificial viscosity F(v) = (1/rho) div(nu rho grad v) on each of the three
 *                staggered velocity components.
 * Schemes (Sec. 3.1, Appendix A): RKL2 / RKG2 super time stepping, and Backward Euler solved by
 * point-Jacobi (PC1) preconditioned conjugate gradients.
 * Cycling (Sec. 2, Eqs. 3-5 and the paragraph after Eq. 5): before every cycle the PTL is taken at
 * k = argmax |F| over the six orthogonal neighbours; the remaining time is split into
 * n = ceil(t_rem / max(dt_PTL, floor dt_E)) cycles and the next cycle has length t_rem / n.
 *
 * Discretisation (the paper gives none): finite volumes on a spherical shell (r, theta, phi),
 * phi periodic, zero-flux boundaries at r_min, r_max and the poles.  Conduction uses a symmetric
 * corner ("dual cell") scheme with 27-point support; viscosity a 7-point flux form.  dt_E is
 * 2 / max_i (sum_j |L_ij|) (Gershgorin bound on the spectral radius of L).
 *
 * Memory layout: every field is a dense array of n_r * n_theta * n_phi values with r fastest:
 * flat index i + n_r * (j + n_theta * k).  A conduction state is one such array (cells).
 * A viscosity state is the three components back to back: v_r on (n_r-1) x n_theta x n_phi
 * interior r faces, v_theta on n_r x (n_theta-1) x n_phi interior theta faces, v_phi on
 * n_r x n_theta x n_phi phi faces (on the periodic box all three are n_r x n_theta x n_phi).
 * parabolic_state_size() returns the total length.
 *
 * Conventions: all device pointers are CUDA device memory of the current device; all work is
 * enqueued on the stream given to parabolic_setup; every call returns after its work is done
 * (the host reads small scalars back), except where stated.  A context is not thread safe;
 * separate contexts are independent.  Every function returns a PB_* status; on failure
 * pb_last_error() describes it and the caller's arrays hold the last completed cycle.
 * There is no CPU fallback: without a usable GB300 every call fails with PB_ECUDA.
 */
#ifndef PARABOLIC_H
#define PARABOLIC_H

#include <stdint.h>

#if defined(__GNUC__)
#define PB_API __attribute__((visibility("default")))
#else
#define PB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define PB_OK            0
#define PB_EINVAL        1  /* bad argument (size, pointer, option)                        */
#define PB_ENOMEM        2  /* device or pinned host allocation failed                      */
#define PB_ECUDA         3  /* CUDA runtime / launch error                                  */
#define PB_ENOCONVERGE   4  /* PCG hit max_iter before reaching rtol                        */
#define PB_EMAXCYCLES    5  /* the PTL asked for more than max_cycles cycles                */
#define PB_ENONFINITE    6  /* a NaN / Inf appeared in F or in a PCG scalar                 */
#define PB_ETIMEOUT      7  /* a bounded device-side wait ran out                           */
#define PB_ENOTSUP       8  /* combination not supported by this build                      */

/* PB_FP64: float64 states, records and arithmetic.  PB_FP32: float32 states, records and
 * stencil arithmetic; the super-time-stepping stage recurrence is summed in double-float
 * arithmetic on the float32 pipes (float64 coefficients as float pairs), so a stage adds only
 * the rounding of its stored result; reductions and coefficients in float64.
 * PB_BF16_STORE: bfloat16 storage with float32 accumulation -- the caller's state arrays and
 * the operator's coefficient records are bfloat16; within a call the state and the stage values
 * are float32 (a context-owned working copy), with the PB_FP32 stage recurrence; the state is
 * rounded to bfloat16 once, when the call hands it back (STS, apply and PTL only).  dt_E of a
 * PB_BF16_STORE context is the Gershgorin bound of the operator on its rounded records.
 * PB_FP64_STORE: float64 states and stage recurrence, float32 records and stencil arithmetic
 * (STS only; BE + PCG needs PB_FP64 or PB_FP32). */
typedef enum { PB_FP64 = 0, PB_FP32 = 1, PB_BF16_STORE = 2, PB_FP64_STORE = 3 } pb_precision;
typedef enum { PB_TC_ANISO = 0, PB_VISC_ISO = 1 } pb_op_kind;
typedef enum { PB_RKL2 = 0, PB_RKG2 = 1 } pb_scheme;
/* Where the PTL condition is evaluated: at argmax |F| only (Eq. 5) or over every pair of face
 * neighbours (Eq. 4 without the F_max localisation; Sec. 2, the text after Eq. 4). */
typedef enum { PB_PTL_FMAX = 0, PB_PTL_FULL = 1 } pb_ptl_mode;
/* Preconditioner of the Backward Euler PCG (Sec. 3.1 names point-Jacobi PC1 and the stronger,
 * incomplete-factorisation PC2).  PB_PC_CHEBYSHEV is this library's GPU form of a stronger
 * preconditioner: z = p(D^-1 S) D^-1 r with p the degree-m Chebyshev acceleration of point-Jacobi
 * on [b/30, b], b = 1.05 x the Gershgorin bound of D^-1 S for the cycle; fewer iterations (and
 * global dot products) for m - 1 extra stencil passes per iteration. */
typedef enum { PB_PC_JACOBI = 0, PB_PC_CHEBYSHEV = 1 } pb_precond;

typedef struct pb_ctx pb_ctx;

/* Geometry of a grid.  PB_SPHERICAL: the (r, theta, phi) shell of the method (Sec. 2).
 * PB_CARTESIAN_PERIODIC: a box of unit cells (metric factors, corner and cell volumes 1), periodic
 * in all three directions, on which Fourier modes are eigenvectors of both operators -- the
 * closed-form checks of the schemes and the Fig. 1 set-up. */
typedef enum { PB_SPHERICAL = 0, PB_CARTESIAN_PERIODIC = 1 } pb_geometry;

/* Grid.  PB_SPHERICAL: faces of the shell, phi uniform with n_phi cells over 2 pi; requires
 * n_r >= 2, n_theta >= 2, n_phi >= 3, 0 < r_face increasing, 0 <= t_face <= pi increasing (host
 * arrays, read during setup only).  PB_CARTESIAN_PERIODIC: n_r, n_theta, n_phi >= 3 unit cells
 * along the three axes; r_face and t_face are not read (may be NULL).  Zero-initialise the struct:
 * geometry 0 is the shell. */
typedef struct {
    int32_t n_r, n_theta, n_phi;
    const double* r_face;   /* n_r + 1 */
    const double* t_face;   /* n_theta + 1 */
    int32_t geometry;       /* pb_geometry */
} pb_grid;

/* Operator inputs (device memory, float64, read during setup only; may be freed afterwards).
 * PB_TC_ANISO: T0 and n at cells; B (B_r, B_theta, B_phi) at corners, corner [i,j,k] being the
 *   vertex (r_face[i+1], t_face[j+1], (k+1) dphi); corners with i = n_r-1 or j = n_theta-1 are
 *   not used on the shell (on the periodic box every corner [i,j,k], the vertex between cells
 *   i..i+1, j..j+1, k..k+1 with wrap, is used).  C multiplies the divergence (1/3 for gamma = 5/3).
 * PB_VISC_ISO: rho[c] and nu[c] at the points of velocity component c (layout above). */
typedef struct {
    int32_t kind;            /* pb_op_kind */
    double C;
    const double* T0;
    const double* n;
    const double* B[3];
    const double* rho[3];
    const double* nu[3];
} pb_operator;

/* Options of an advance call.  pb_advance_opts_init() fills the defaults. */
typedef struct {
    int32_t scheme;           /* PB_RKL2 (default) or PB_RKG2; STS only                     */
    int32_t use_ptl;          /* 1 (default): cycle under the PTL; 0: one cycle of length dt */
    int32_t max_cycles;       /* default 100000                                             */
    double ptl_floor;         /* cycle-length floor in units of dt_E (default 1; 0 = none)  */
    const double* dt_cycles;  /* host; forced cycle lengths (overrides use_ptl) or NULL     */
    int32_t n_forced;
    double rtol;              /* BE: ||b - S x||_2 <= rtol ||b||_2, default 1e-10           */
    int32_t max_iter;         /* BE: PCG iteration cap per solve, default 100000            */
    int32_t fixed_iters;      /* BE: > 0 runs exactly this many iterations, no stop test    */
    int32_t check_every;      /* BE: iterations launched between host convergence checks   */
    int32_t judge_guess;      /* BE with x0: 1 (default) starts from whichever of x0 and u^n
                                 has the smaller initial residual ||b - S x||; 0 uses x0     */
    int32_t mixed_precision;  /* BE on a PB_FP64 context: 1 solves by iterative refinement --
                                 float64 residuals, float32 PCG corrections (default 0)      */
    double inner_rtol;        /* relative residual of each float32 correction (default 1e-6:
                                 two corrections reach 1e-10; the last one stops once the
                                 outer test is met)                                         */
    int32_t ptl_mode;         /* PB_PTL_FMAX (default) or PB_PTL_FULL: the PTL value that
                                 sets each cycle                                            */
    int32_t precond;          /* BE: PB_PC_JACOBI (default, PC1) or PB_PC_CHEBYSHEV          */
    int32_t pc_degree;        /* BE with PB_PC_CHEBYSHEV: polynomial degree m, 2..32 (default 3):
                                 m - 1 stencil passes per application                        */
} pb_advance_opts;

/* Statistics of an advance call (host struct).  The per-cycle arrays are optional caller-owned
 * host arrays of length cycle_capacity (records beyond the capacity are dropped). */
typedef struct {
    int32_t cycles;
    int32_t status_cycle;      /* cycle index at which a failure happened, or -1            */
    int64_t total_stages;      /* STS: sum of s over cycles                                 */
    int64_t total_iters;       /* BE: sum of PCG iterations over cycles                     */
    double dt_explicit;
    double last_dt_ptl;
    double fmax;
    int64_t k_index;
    double final_rel_residual; /* BE: recursive ||r|| / ||b|| of the last solve             */
    int32_t cycle_capacity;
    double* dt_cycle;          /* cycle lengths                                             */
    int32_t* work_cycle;       /* STS stages s, or PCG iterations, per cycle                */
    double* dt_ptl_cycle;      /* PTL value that set each cycle (NaN when not evaluated)    */
    int64_t* k_cycle;          /* argmax |F| location before each cycle (-1 when not)       */
    int32_t guess_used;        /* BE: 1 if the first solve started from x0, 0 from u^n      */
    double* dt_full_cycle;     /* Eq. 4 over every pair of face neighbours before each cycle;
                                  when non-NULL it is evaluated every cycle whatever ptl_mode
                                  (a second reduction pass over u and F), NaN when not      */
} pb_stats;

/* Fills *opts with the defaults listed above. */
PB_API void pb_advance_opts_init(pb_advance_opts* opts);

/* Human-readable text for a status code (static storage). */
PB_API const char* pb_status_string(int status);

/* Text of the last error on ctx, or of the last failed parabolic_setup when ctx is NULL
 * (thread-local).  Valid until the next call on the same context. */
PB_API const char* pb_last_error(const pb_ctx* ctx);

/* Builds a context: validates the grid, allocates its device workspace (owned by the context),
 * computes the frozen operator coefficients in float64 on the device (lagged kappa, Sec. 2) and
 * stores them in the context precision, and reduces dt_E.  precision: PB_FP64, PB_FP32 (float
 * state and arithmetic; PTL and PCG reductions in float64), PB_BF16_STORE (bfloat16 state and
 * records, float32 working state and arithmetic) or PB_FP64_STORE (see pb_precision).
 * cuda_stream is a cudaStream_t (NULL = legacy default). */
PB_API int parabolic_setup(const pb_grid* grid, const pb_operator* op, int32_t precision,
                    void* cuda_stream, pb_ctx** out);

/* Recomputes the frozen coefficients and dt_E for new operator inputs (same kind and grid; for
 * conduction a new lagged T0, density or field), in place: allocates nothing, runs on the
 * context's stream, returns when done.  This is the once-per-step set-up of Sec. 2 (lagged
 * diffusivity: kappa frozen at the previous step's temperature). */
PB_API int parabolic_update(pb_ctx* ctx, const pb_operator* op);

/* Frees the context and its device workspace.  NULL is accepted. */
PB_API int parabolic_destroy(pb_ctx* ctx);

/* Length of the state vector (elements) and the element size in bytes of the caller's state
 * arrays (8, 4 or 2). */
PB_API int parabolic_state_size(const pb_ctx* ctx, int64_t* n_elems, int32_t* elem_bytes);

/* The explicit (forward Euler) stable step dt_E of the operator (Appendix A's Delta t_Euler). */
PB_API int parabolic_dt_explicit(const pb_ctx* ctx, double* dt_e);

/* F = L u for a device state u (ctx precision); F is device memory of the same length. */
PB_API int parabolic_apply(pb_ctx* ctx, const void* u_dev, void* F_dev);

/* PTL of state u (Eq. 5): dt_ptl (+INF if no neighbour qualifies), the flat index k of
 * max |F| (ties: smallest index) and |F_k|.  Any output pointer may be NULL. */
PB_API int ptl_compute(pb_ctx* ctx, const void* u_dev, double* dt_ptl, int64_t* k_index,
                double* fmax);

/* PTL without the F_max localisation (Sec. 2, the text after Eq. 4): the smallest bound -du/dF
 * of Eq. 4 over every pair of face neighbours (i, i + e_d) of state u, each component on its own,
 * d = 0 (r), 1 (theta), 2 (phi, periodic), over the pairs with du = u_i - u_j != 0,
 * dF = F_i - F_j != 0 and du dF < 0 (F = L u, computed here; bounds in the arithmetic
 * precision).  Outputs: dt_full (+INF when no pair qualifies), the pair's flat cell index i and
 * direction d (both -1 then); equal bounds go to the smallest 3 i + d.  Any output pointer may
 * be NULL.  Returns PB_OK, PB_EINVAL, PB_ENONFINITE (non-finite F) or PB_ECUDA. */
PB_API int ptl_full_compute(pb_ctx* ctx, const void* u_dev, double* dt_full, int64_t* cell,
                            int32_t* direction);

/* Advances u (device, in place, ctx precision) over dt with RKL2 or RKG2 super time stepping
 * (opts->scheme) under PTL cycling (Appendix A stage loop).  stats may be NULL. */
PB_API int rkl2_advance(pb_ctx* ctx, void* u_dev, double dt, const pb_advance_opts* opts,
                 pb_stats* stats);

/* The graph-only form of rkl2_advance: the cycles of a forced schedule (opts->dt_cycles), or one
 * cycle of length dt when opts->use_ptl is 0, enqueued on the context's stream.  It returns
 * without waiting, reads nothing back to the host and allocates nothing, so it can be captured in
 * a CUDA graph and replayed.  The PTL is refused with PB_EINVAL: it needs a host round trip per
 * cycle.  No statistics; errors found on the device (a bounded wait that ran out) surface at the
 * next synchronous call. */
PB_API int rkl2_advance_async(pb_ctx* ctx, void* u_dev, double dt, const pb_advance_opts* opts);

/* Non-linear conduction under RKL2 / RKG2 (Sec. 3.1: super time stepping handles a non-linear
 * operator; Sec. 2: the diffusivity is lagged): before every cycle the coefficients are
 * recomputed with kappa = max(T, 0)^{5/2} from the current state T, with dt_E, and the cycle --
 * its PTL decision and its stages -- runs with that operator frozen.  The cycle rule, options and
 * statistics are those of rkl2_advance (no floor-cycle speculation; ptl_mode PB_PTL_FMAX only;
 * stats->dt_explicit is the last cycle's).  op: the conduction operator's n, B and C (device
 * float64, read every cycle; op->T0 is not read).  On return the context holds the coefficients
 * of the last cycle's operator.  Conduction contexts only (PB_EINVAL otherwise). */
PB_API int rkl2_advance_relag(pb_ctx* ctx, void* u_dev, double dt, const pb_advance_opts* opts,
                              const pb_operator* op, pb_stats* stats);

/* Advances u (device, in place) over dt with Backward Euler, each cycle solving
 * (M - dt_c A) x = M u (M = diag(1/w), F = w A u) by point-Jacobi PCG from x0 = u, or from
 * x0_dev (device, ctx precision) on the first cycle when it is not NULL.  Supported for
 * PB_FP64 and PB_FP32 (float vectors; the dot products sum the exact float products in
 * double-float, about 44 bits).  stats may be NULL.
 * With opts->mixed_precision on a PB_FP64 context each cycle is solved by iterative refinement:
 * float32 PCG corrections to opts->inner_rtol driven by outer residuals.  On a conduction
 * context those residuals are computed in double-float arithmetic (about 48 bits, on the float32
 * pipes), except the one after the correction meant to meet rtol, which is float64; a cycle
 * stops only when a float64 residual meets rtol.  Environment PB_MIXED_FP64_RESIDUAL=1 (read at
 * each call) uses float64 residuals throughout.
 * With mixed_precision the PTL decision is taken on a float32 view of the state (F in float32,
 * the arg-max compared in float), as the float32 contexts take it.
 * opts->precond = PB_PC_CHEBYSHEV preconditions the PCG polynomially (with mixed_precision, the
 * float32 inner solves); stats count its PCG iterations, each of which runs pc_degree - 1 extra
 * stencil passes. */
PB_API int be_pcg_advance(pb_ctx* ctx, void* u_dev, double dt, const pb_advance_opts* opts,
                   const void* x0_dev, pb_stats* stats);

/* ---- kernel accounting --------------------------------------------------------------------- */
/* Per kernel class of one context: launches, launches timed with CUDA events on the context's
 * stream, their summed duration, and the algorithmic bytes the launches must move (every operand
 * read once and every result written once; the per-point figures are in the library's design
 * notes).  Launch counts are always kept. */
typedef struct {
    char name[32];            /* "<tc|visc>.<class>", e.g. "tc.stage", "visc.ptl_pass"        */
    int64_t launches;
    int64_t timed_launches;
    double total_ms;
    double bytes;
} pb_kernel_stat;

/* Resets the counters; on != 0 also brackets every launch with CUDA events (harvested at the
 * library's host synchronisations) until called again with on = 0. */
PB_API int pb_profile_enable(pb_ctx* ctx, int32_t on);

/* Writes up to cap records (classes with at least one launch) and their number to *count. */
PB_API int pb_profile_read(pb_ctx* ctx, pb_kernel_stat* out, int32_t cap, int32_t* count);

/* ---- batched super time stepping ------------------------------------------------------------- */
/* Many independent conduction problems (float32 contexts of any sizes) advanced by one cycle each,
 * dt[p] with its own stage count, in ONE persistent kernel launched as a CUDA graph (a batched
 * form of the Appendix A stage loop; the batching itself has no counterpart in the paper).
 * Work items (problem, level, tile) are claimed in level-major order from a device counter; an
 * item waits (bounded) for all tiles of its problem's previous level.  The tile schedule is set
 * by pb_tune, chosen by pb_autotune from timed candidates. */
typedef struct pb_batch pb_batch;

typedef struct {
    int32_t kchunk;         /* phi planes per tile (default 16)                              */
    int32_t blocks_per_sm;  /* persistent blocks per SM (default 4)                          */
    int32_t small_tiles;    /* 1: 16 x 16 (r, theta) tiles for grids with n_r <= 16 (default) */
} pb_tune;

PB_API void pb_tune_init(pb_tune* tune);

/* ctxs: n float32 conduction contexts sharing one stream (not owned; they must outlive the
 * batch; their y0 / stage buffers are the batch's scratch).  tune may be NULL. */
PB_API int pb_batch_create(pb_ctx* const* ctxs, int32_t n, const pb_tune* tune, pb_batch** out);
PB_API int pb_batch_destroy(pb_batch* batch);
PB_API const char* pb_batch_last_error(const pb_batch* batch);

/* Advances every u_devs[p] (device, float32, in place) over dts[p] with RKL2 or RKG2 (one cycle,
 * no PTL), ordered after prior work on the contexts' stream; returns when done.
 * per_problem (n entries, or NULL) receives cycles = 1 and the stage count. */
PB_API int pb_batch_rkl2_advance(pb_batch* batch, void* const* u_devs, const double* dts, int32_t scheme,
                                 pb_stats* per_problem);

/* Times every candidate schedule (kchunk in {4, 8, 16, 32, 64} x blocks_per_sm in {2, 4, 6, 8}
 * x small_tiles in {0, 1}) on scratch copies of the states (the caller's u_devs are not
 * modified; this call allocates the copies), keeps the fastest in the batch and returns it
 * and its time (ms) in *best_ms (may be NULL). */
PB_API int pb_autotune(pb_batch* batch, void* const* u_devs, const double* dts, int32_t scheme, pb_tune* out,
                       double* best_ms);

/* ---- learned PCG initial guess ---------------------------------------------------------------- */
/* A small 3-D convolutional network (four 3 x 3 x 3 layers, 16 channels, ReLU between them,
 * bfloat16 weights and activations, float32 accumulation) predicts the Backward Euler
 * increment x - u^n from per-point features of the state; PCG (Sec. 3.1) starts from
 * x0 = u^n + S y and still converges to the requested tolerance.  The paper has no network: it
 * is an initial guess for the PC1 solve, trained on solves the library itself produces.
 * Features (pb_guess_features), 6 of 16 channels: e/S with e = dt F(u) and S = rms(e);
 * log10(1 + sigma) and sigma/(1 + sigma) with sigma = dt w |A_ii|; (u - mean u)/S;
 * log10(w)/10; the normalised r index.  Tensors are [sample][n_phi][n_theta][n_r][16] bfloat16
 * (features) and [sample][n_phi][n_theta][n_r] float32 (targets, outputs). */
typedef struct pb_model pb_model;

typedef struct {
    int32_t steps;     /* optimisation steps                                               */
    int32_t batch;     /* crops per step                                                   */
    int32_t crop;      /* crop edge (points)                                               */
    int32_t border;    /* loss excludes this many points at every crop face                */
    double lr;         /* Adam learning rate                                               */
    uint64_t seed;     /* crop sampling                                                    */
} pb_train_opts;

PB_API int pb_model_create(uint64_t seed, pb_model** out);
PB_API int pb_model_destroy(pb_model* model);
PB_API const char* pb_model_last_error(const pb_model* model);
PB_API int pb_model_num_params(void);
/* float32 parameters, per layer W[27][ci][co] (offset = 9 (dphi+1) + 3 (dtheta+1) + (dr+1)) then b[co] */
PB_API int pb_model_get_params(const pb_model* model, float* host, int64_t cap);
PB_API int pb_model_set_params(pb_model* model, const float* host, int64_t n);
PB_API int pb_model_save(const pb_model* model, const char* path);
PB_API int pb_model_load(pb_model* model, const char* path);
/* Features of state u for a BE step of length dt (device, ctx precision, conduction or
 * viscosity contexts with float64 / float32 storage), and S.  With x (the solved BE state) the
 * training target (x - u)/S is written too (float32); x and target are both NULL or both set. */
PB_API int pb_guess_features(pb_ctx* ctx, const void* u, double dt, const void* x, void* feats, void* target,
                             double* scale);
/* Network output for S_ samples of D x H x W feature points (wrap_d: periodic first axis).
 * The conv layers run on the tensor cores (tcgen05); environment PB_CONV_CUDA_CORES=1, read once
 * per process, selects the CUDA-core kernel of the same layers instead.  PB_ETIMEOUT: a layer's
 * bounded wait for its tensor-core operations ran out (the result is not valid).  The same holds
 * for pb_model_grad, pb_model_train and learned_guess, which run the same layers. */
PB_API int pb_model_forward(pb_model* model, const void* feats, int32_t S_, int32_t D, int32_t H, int32_t W,
                            int32_t wrap_d, void* out, void* stream);
/* Mean-squared-error loss over mask and its gradient (host float32, pb_model_num_params()). */
PB_API int pb_model_grad(pb_model* model, const void* feats, const void* target, const void* mask, int32_t S_,
                         int32_t D, int32_t H, int32_t W, double* loss, float* host_grad, void* stream);
/* Adam training on random crops of nsamples equally sized samples (device feats / targets). */
PB_API int pb_model_train(pb_model* model, const void* feats, const void* targets, int32_t nsamples, int32_t D,
                          int32_t H, int32_t W, const pb_train_opts* opts, double* last_loss, void* stream);
/* x0 = u + S smooth(model(features(u, dt))) for a conduction context (float64 / float32): the
 * network's output is passed through pb_guess_smooth_passes() passes of the filter below before it
 * becomes the increment (PCG's initial residual weights grid-scale error by up to dt/dt_E, so
 * only the smooth part of a prediction can shorten a solve to a tight tolerance). */
PB_API int learned_guess(pb_ctx* ctx, pb_model* model, const void* u, double dt, void* x0);

/* out = in smoothed by `passes` passes of the binomial filter (1, 2, 1)/4 along each axis of
 * S_ x D x H x W float32 fields (W fastest; the W and H ends repeat their edge value, D wraps when
 * wrap_d): the smoothing learned_guess applies to the network output, for preparing training
 * targets alike.  in, out, tmp: device float32 arrays of S_ D H W elements; out may equal in, tmp
 * must differ from both.  Runs on `stream` and returns when done. */
PB_API int pb_guess_smooth(const void* in, void* out, void* tmp, int32_t S_, int32_t D, int32_t H, int32_t W,
                           int32_t wrap_d, int32_t passes, void* stream);
/* The number of passes learned_guess applies. */
PB_API int pb_guess_smooth_passes(void);

/* ---- PTL without allocation ---------------------------------------------------------------- */
/* PTL of a state (the same result as ptl_compute) for callers that cannot allocate device
 * memory: a host code that hands the solver a fixed, pre-sized device arena for a whole run, or
 * one that cannot afford the device-wide synchronisation and failure modes of cudaMalloc /
 * cudaFree inside its time-step loop.  It needs no context and allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library call): the caller passes
 *   records  the operator's packed per-point records, n Coef4 entries in the layout the library
 *            uses (conduction: {ahat_r, ahat_t, ahat_p} of corner [i,j,k] and the cell weight w;
 *            viscosity: {c_r, c_t, c_p} of the +1 faces and w), 4 words of the type below;
 *   u        the state (n elements, type below), read only;
 *   F        output, n elements: F = L u;
 * and receives dt_ptl, k_index and fmax on the host (any may be NULL).  n is n_r*n_theta*n_phi
 * for conduction and the three-component total for viscosity.  Types per precision:
 *   PB_FP64        records, u and F float64;
 *   PB_FP32        records, u and F float32;
 *   PB_BF16_STORE  records and u bfloat16, F float32 (the precision's working type).
 * The paper has no counterpart: this is a deployment variant of the PTL pass.
 * Its only scratch (per-block partials, a flag, the result) is one file-scope device array of
 * 1 MiB that every GPU loading the library holds until exit; grids needing more than 65,520
 * partial records (more than that many 32 x 8 (r, theta) tiles) are rejected with PB_EINVAL.
 * The first call in a device's context looks up that array's device address
 * (cudaGetSymbolAddress) and later calls reuse it; after a device reset (a new context) it is
 * looked up again.  Every call shares the array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race; serialise them.  Work runs on `stream` (cudaStream_t,
 * NULL = legacy default) and the call waits for its own result (a copy to host memory and a
 * stream synchronisation), so it can never be made inside a stream capture.
 * Returns PB_OK, PB_EINVAL, PB_ENONFINITE (non-finite F) or PB_ECUDA. */
PB_API int pb_ptl_noalloc(int32_t kind, int32_t n_r, int32_t n_theta, int32_t n_phi,
                          int32_t precision, const void* records, const void* u, void* F,
                          double* dt_ptl, int64_t* k_index, double* fmax, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PARABOLIC_H */
