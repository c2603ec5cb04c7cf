/*
 * plsqr.h -- C ABI of libplsqr, a GB300 (sm_103a) implementation of the inner solve of
 * Arridge, Betcke & Harhanen's priorconditioned lagged-diffusivity method (arXiv 1308.6634):
 * the factorization-free priorconditioned LSQR iteration MLSQR (Algorithm 2) run inside each
 * step of the lagged-diffusivity fixed point (Algorithm 3) for
 *
 *      min_f  1/2 ||g - A f||^2 + tau R(f),     R(f) = sum_i r(|grad f|_i)       (eq. 1.6)
 *
 * with r one of (1.3)-(1.5).  The priorconditioner is a fixed symmetric geometric-multigrid
 * V-cycle P approximating M_f^{-1}, M_f = sum_d D_d^T diag(kappa) D_d (eq. 1.13, Sec. 4.2).
 *
 * Conventions for every entry point:
 *  - Arrays are dense, C order, x fastest: an image is [ny][nx], a volume [nz][ny][nx], a
 *    sinogram [n_angles][n_bins].  Element type is double for a PLSQR_FP64 handle and float
 *    for a PLSQR_FP32 handle; scalars of the Krylov recurrences are always double.
 *  - "device" pointers point to memory on the handle's device (cudaMalloc, or a PyTorch
 *    tensor's storage); "host" pointers to ordinary or pinned host memory.  The caller owns
 *    all of them; the library never frees or keeps a caller pointer after a call returns,
 *    except the operator mask, which set_operator copies.
 *  - All device work is enqueued on the stream given to plsqr_create (NULL = legacy default
 *    stream).  Entry points that return host results (histories, R) synchronise that stream.
 *  - Every call returns a plsqr_status and never aborts; on error plsqr_last_error(h)
 *    returns a message.  Handles are not thread safe: use one per host thread.
 *  - Numerical breakdown (a Golub-Kahan norm that is zero, tiny or not finite) stops that
 *    inner solve with the last complete iterate kept; the solve continues with the next
 *    outer step and finally returns PLSQR_E_BREAKDOWN.
 */
#ifndef PLSQR_H
#define PLSQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct plsqr_ctx* plsqr_handle;

typedef enum {
    PLSQR_OK = 0,
    PLSQR_E_INVALID = 1,   /* bad argument or size */
    PLSQR_E_NOMEM = 2,     /* device allocation failed */
    PLSQR_E_CUDA = 3,      /* a CUDA call failed */
    PLSQR_E_BREAKDOWN = 4, /* Golub-Kahan breakdown in some inner solve */
    PLSQR_E_TIMEOUT = 5,   /* a bounded device wait gave up (TMA staging, grid barrier) */
    PLSQR_E_STATE = 6      /* call out of order (e.g. solve before set_operator) */
} plsqr_status;

/* r(t) of eqs. (1.3)-(1.5); kappa(t) = r'(t)/t is the diffusivity of (1.13). */
typedef enum {
    PLSQR_R_TIKHONOV = 0, /* r = t^2/2                          kappa = 1               (1.3) */
    PLSQR_R_TV = 1,       /* r = T sqrt(1+(t/T)^2)              kappa = 1/sqrt(T^2+t^2) (1.4) */
    PLSQR_R_PM_LOG = 2,   /* r = T^2/2 log(1+(t/T)^2)           kappa = 1/(1+(t/T)^2)   (1.5) */
    PLSQR_R_PM_EXP = 3    /* r = T^2/2 (1-exp(-t^2/T^2))        kappa = exp(-t^2/T^2)   (1.5) */
} plsqr_reg;

typedef enum {
    PLSQR_OP_BLUR = 0,      /* separable Gaussian blur B, zero boundary; A = A^T = B          */
    PLSQR_OP_BLUR_MASK = 1, /* inpainting: A = D B, A^T = B D, D = diag(mask)                 */
    PLSQR_OP_JOSEPH = 2,    /* 2D parallel-beam Joseph projector, gather-form exact adjoint  */
    PLSQR_OP_IDENTITY = 3   /* A = I (denoising)                                             */
} plsqr_op_kind;

typedef enum { PLSQR_FP64 = 0, PLSQR_FP32 = 1 } plsqr_precision;

/* Problem size and priorconditioner shape. */
typedef struct {
    int32_t ndim;        /* 2 or 3 */
    int32_t precision;   /* plsqr_precision of the bulk vectors and stencils */
    int64_t n[3];        /* nx, ny, nz (nz ignored for ndim 2); each n[d] divisible by
                            2^(mg_levels-1) (cell-centred coarsening, Sec. 4.2) */
    int32_t mg_levels;   /* V-cycle levels including the finest (>= 1; 1 = exact M^{-1}) */
    int32_t mg_sweeps;   /* nu: red-black Gauss-Seidel sweeps before and after the coarse
                            correction (mirrored order keeps P symmetric, Sec. 4.2) */
    int32_t mg_cycles;   /* V-cycles per application of P (x <- x + V(b - M x)) */
    int32_t max_batch;   /* instances per batched solve (>= 1) */
    double kappa_floor;  /* kappa >= kappa_floor * kappa(0); 0 disables the floor */
} plsqr_config;

/* Forward map A (Sec. 1: matrix-free A, given by its action on a vector). */
typedef struct {
    int32_t kind;          /* plsqr_op_kind */
    int32_t n_angles;      /* Joseph: angles a*pi/n_angles, a = 0..n_angles-1 */
    int32_t n_bins;        /* Joseph: detector bins at (k-(n_bins-1)/2)*bin_spacing */
    int32_t reserved;
    double sigma[3];       /* blur: Gaussian widths along x, y, z in cells */
    int32_t radius[3];     /* blur: truncation radii (taps -R..R), normalised to unit sum */
    int32_t reserved2;
    double bin_spacing;    /* Joseph: detector spacing in pixel units (> 0) */
    const uint8_t* mask;   /* BLUR_MASK: device pointer to N bytes, nonzero = observed;
                              shared by every instance of a batch; copied by set_operator */
} plsqr_operator;

/* Optional per-solve outputs (host arrays, caller owned; NULL members are skipped). */
typedef struct {
    double* rbar_hist;     /* [n_outer][n_inner]: ||rbar_i||, the LSQR estimate of the
                              residual norm of the damped problem (Sec. 3.4) */
    double* R_hist;        /* [n_outer + 1]: R(f^0) .. R(f^n_outer) (Algorithm 3 step 5) */
    double* resid_hist;    /* [n_outer]: ||g - A f^k|| (Morozov quantity, Sec. 3.4 S4) */
    int32_t status;        /* plsqr_status of this instance */
    int32_t reserved;
} plsqr_stats;

/* Create a handle for problems of one size on the current CUDA device.  Allocates the whole
 * workspace for cfg->max_batch instances.  stream: a cudaStream_t (NULL = default stream).
 * Errors: PLSQR_E_INVALID (sizes, levels), PLSQR_E_NOMEM, PLSQR_E_CUDA. */
int plsqr_create(const plsqr_config* cfg, void* stream, plsqr_handle* out);

/* Set the forward map A (Sec. 1).  Precomputes blur taps / Joseph angle tables and copies
 * the mask.  Joseph needs ndim 2 and nx == ny.  Errors: PLSQR_E_INVALID, PLSQR_E_NOMEM. */
int plsqr_set_operator(plsqr_handle h, const plsqr_operator* op);

/* Algorithm 3: f^0 = 0; for k = 1..n_outer: kappa from f^{k-1} (eq. 1.13, kappa floored),
 * build the V-cycle P ~ M_{f^{k-1}}^{-1}, run n_inner MLSQR iterations (Algorithm 2) from
 * f = 0 on (eq. 4.3) with damping sqrt(tau) (eq. 2.3), giving f^k.
 * g: device, m values (m = N, or n_angles*n_bins for Joseph); f_out: device, N values.
 * stats may be NULL (then the call does not synchronise).  T > 0, tau >= 0. */
int plsqr_solve(plsqr_handle h, const void* g, int32_t reg, double T, double tau,
                int32_t n_outer, int32_t n_inner, void* f_out, plsqr_stats* stats);

/* plsqr_solve with host buffers: copies g host->device, solves, copies f device->host and
 * synchronises.  Pinned host memory makes the copies asynchronous with respect to the host. */
int plsqr_solve_host(plsqr_handle h, const void* g_host, int32_t reg, double T, double tau,
                     int32_t n_outer, int32_t n_inner, void* f_host_out, plsqr_stats* stats);

/* Batched Algorithm 3: `count` (<= max_batch) independent instances of the handle's size
 * and operator, solved together (every kernel launch covers all instances).  g[b], f_out[b]
 * are device pointers; reg/T/tau are per instance; stats is NULL or an array of `count`. */
int plsqr_solve_batch(plsqr_handle h, int32_t count, const void* const* g, const int32_t* reg,
                      const double* T, const double* tau, int32_t n_outer, int32_t n_inner,
                      void* const* f_out, plsqr_stats* stats);

void plsqr_destroy(plsqr_handle h);
const char* plsqr_last_error(plsqr_handle h);
/* Device bytes a handle with this config would allocate (for admission by memory).  op may be
 * NULL (data length = image size).  With a Joseph operator this includes the forward projection's
 * two-part scratch: for the first min(max_batch, floor(455 / n_angles)) instances, 2 x data length
 * elements and one 4-byte arrival counter per angle.  Host only; -1 for an invalid config. */
int64_t plsqr_workspace_bytes(const plsqr_config* cfg, const plsqr_operator* op);

/* ---- single steps of the path (for parity tests and custom loops) ---------------------- */

/* y = A x (x: device N values, y: device m values).  Sec. 1 (forward map). */
int plsqr_apply_A(plsqr_handle h, const void* x, void* y);
/* x = A^T y.  Gather form for Joseph (no atomics), B D for the masked blur. */
int plsqr_apply_At(plsqr_handle h, const void* y, void* x);
/* kappa_i = max(r'(t_i)/t_i, kappa_floor*kappa(0)) with t_i = |(D f)_i|, forward
 * differences and a ghost 0 past the high end of each axis (eqs. 1.12-1.13); *R_out =
 * sum_i r(t_i) (discrete eq. 1.2), computed on the device in double.  Synchronises. */
int plsqr_diffusivity(plsqr_handle h, const void* f, int32_t reg, double T, void* kappa_out,
                      double* R_out);
/* Build the priorconditioner hierarchy from kappa (device, N values): Galerkin coarse
 * conductances and the exact inverse of the coarsest operator (Sec. 4.2). */
int plsqr_prec_setup(plsqr_handle h, const void* kappa);
/* x = P b with the hierarchy of the last plsqr_prec_setup (b, x: device, N values). */
int plsqr_prec_apply(plsqr_handle h, const void* b, void* x);
/* y = M_f x with the kappa of the last plsqr_prec_setup (eq. 1.13). */
int plsqr_apply_M(plsqr_handle h, const void* x, void* y);
/* One MLSQR inner solve (Algorithm 2) from f = 0 with the current hierarchy:
 * n_inner iterations, damping sqrt(tau).  rbar_hist: host, n_inner values, or NULL.
 * Returns PLSQR_E_BREAKDOWN if it stopped early; *iters_done (may be NULL) counts the
 * completed iterations.  Synchronises. */
int plsqr_mlsqr(plsqr_handle h, const void* g, double tau, int32_t n_inner, void* f_out,
                double* rbar_hist, int32_t* iters_done);

/* ---- instrumentation --------------------------------------------------------------------- */

/* Kernel classes reported by plsqr_profile_read. */
typedef enum {
    PLSQR_KC_FWD = 0,      /* A with the forward Golub-Kahan epilogue and the beta norm    */
    PLSQR_KC_ADJ = 1,      /* A^T with the p~ update                                        */
    PLSQR_KC_OP_PLAIN = 2, /* A or A^T without epilogue                                     */
    PLSQR_KC_GS_FINE = 3,  /* red-black Gauss-Seidel half sweeps on the finest level         */
    PLSQR_KC_MG_OTHER = 4, /* coarser sweeps, residual + restriction, prolongation           */
    PLSQR_KC_COARSE = 5,   /* dense solve on the coarsest level                             */
    PLSQR_KC_GK = 6,       /* norms, dot product + rotations, solution update               */
    PLSQR_KC_SETUP = 7,    /* diffusivity, coarsening, band assembly, Cholesky, inverse      */
    PLSQR_KC_COUNT = 8
} plsqr_kclass;

/* enable != 0: later calls launch eagerly (no CUDA graph) and bracket every kernel (or
 * kernel group of one operator application) with CUDA events, accumulating device time per
 * class.  Resets the accumulators.  Synchronises.  Not part of any numerical result. */
int plsqr_profile(plsqr_handle h, int32_t enable);
/* Accumulated device milliseconds and timed launches per class (arrays of n entries). */
int plsqr_profile_read(plsqr_handle h, double* ms, int64_t* counts, int32_t n);
/* Number of kernel launches the last solve executed (graph replays included), or -1. */
int64_t plsqr_last_launches(plsqr_handle h);
/* Guard bands (a debugging aid for out-of-bounds writes; compute-sanitizer stands in where it
 * is available).  With the environment variable PLSQR_GUARD=1 when plsqr_create runs, every
 * workspace allocation of the handle gets 256 bytes of the pattern 0xA5 on each side of the
 * region the library uses (the regions stay 256-byte aligned; results are unchanged).  This call
 * synchronises both streams and reads the bands back: *n_checked (may be NULL) = allocations with
 * bands (0 when the handle was created without them), *n_bad (may be NULL) = allocations with a
 * changed band.  Allocations made for the duration of one call (plsqr_mlsqr_multi_tau's stored
 * vectors) and the caller's buffers are not covered. */
int plsqr_check_guards(plsqr_handle h, int64_t* n_checked, int64_t* n_bad);

/* ---- several damping parameters from one bidiagonalisation (Sec. 3.3) ---------------------------
 * The Golub-Kahan bidiagonalisation inside MLSQR does not depend on tau (the Krylov spaces are
 * shift invariant), so with its Lanczos vectors V_k stored, the projected problem (3.6)
 *     min_y || [B_k ; sqrt(tau) I] y - beta_1 e_1 ||
 * gives the MLSQR iterate f_k(tau) = V_k y(tau) for any number of values of tau.
 *
 * plsqr_mlsqr_multi_tau: one MLSQR run of n_inner steps from f = 0 with the current hierarchy
 *   (plsqr_prec_setup), storing the normalised vectors v~_1 .. v~_n_inner on the device
 *   (n_inner * N elements, allocated for the call and freed before it returns), then for each of
 *   the n_tau <= 32 values taus[t] >= 0: f_out[t] (device, N values) = V y(taus[t]), all of them in
 *   one pass over the stored vectors.  rbar_hist (host, n_tau x n_inner, may be NULL): ||rbar_i||
 *   for each tau.  *iters_done (may be NULL): completed steps.  Returns PLSQR_E_BREAKDOWN (with the
 *   iterates of the completed steps) if the bidiagonalisation stopped early, PLSQR_E_NOMEM if the
 *   vectors do not fit, PLSQR_E_STATE while slots are in use.  Synchronises.
 * plsqr_projected_solve: its host part, which needs no GPU: y (k values) and ||rbar_i|| (k values,
 *   may be NULL) of (3.6) from alpha[0..k] = alpha_1 .. alpha_{k+1} and beta[0..k] = beta_1 ..
 *   beta_{k+1}, by the rotations of Algorithm 2 (steps 8-20) applied to coefficient vectors.
 *   PLSQR_E_INVALID for k < 1, NULL arrays or tau < 0; PLSQR_E_BREAKDOWN if a rotation is
 *   undefined (rho = 0 or not finite). */
int plsqr_mlsqr_multi_tau(plsqr_handle h, const void* g, int32_t n_inner, int32_t n_tau, const double* taus,
                          void* const* f_out, double* rbar_hist, int32_t* iters_done);
int plsqr_projected_solve(int32_t k, const double* alpha, const double* beta, double tau, double* y, double* rbar);

/* ---- self-test of the bounded waits ------------------------------------------------------------
 * Every wait of a kernel on its TMA copies is bounded: when it runs out the kernel records
 * PLSQR_E_TIMEOUT (status 5) in the instance state, waits once more (bounded) and returns.
 * plsqr_selftest_wait runs that wait on a barrier that completes (complete != 0: *status_out = 0)
 * or that announces bytes no copy will bring (complete = 0: *status_out = 5 after 2 x 65536
 * polls).  No copy is issued and nothing faults or hangs.  Needs a GPU; synchronises. */
int plsqr_selftest_wait(int32_t complete, int32_t* status_out);

/* ---- V-cycle tile shapes ------------------------------------------------------------------------
 * The 2D V-cycle (Sec. 4.2 priorconditioner: red-black Gauss-Seidel smoothing, restriction,
 * prolongation on each level above the coarsest) runs each level as tiles staged in shared memory.
 * Several tile shapes are compiled in; every shape gives the same result bit for bit, only the
 * speed differs.  By default the first solve of a handle tunes them (env PLSQR_AUTOTUNE=0: keep
 * shape 0 everywhere): for each level it times CUDA-graph replays of that level's smoothing
 * launches with each shape and the handle's full batch, and keeps the fastest; choices are cached
 * per process for levels of the same size, batch, precision, sweep count and kappa storage.  The
 * timing reads the level's hierarchy as it stands and writes only V-cycle scratch, so tuning
 * between plsqr_prec_setup and plsqr_prec_apply leaves the priorconditioner unchanged.
 *
 * plsqr_autotune: tune now (fresh != 0: measure again instead of using the cache).  Uses the
 *   handle's scratch buffers: not while slots are in use (PLSQR_E_STATE).
 * 3D handles run each red-black half sweep as its own launch, one thread per cell row position;
 * there the tuned "shape" is the number of planes each thread takes (1, 2 or 4: the loads of
 * several planes in flight together), timed and cached the same way (per level extents, batch and
 * element size); the result does not depend on it.
 *
 * plsqr_set_tile_shape: level 0 .. mg_levels-2 takes shape `shape` (2D: 0 is the default, level 0
 *   has its own list; 3D: 1, 2 or 4 planes per thread); marks the handle as tuned, and keeps the
 *   shapes when plsqr_set_kappa_bf16 later changes the kappa storage (which otherwise makes the next
 *   solve tune again).  PLSQR_E_INVALID for an unknown level or shape.
 * plsqr_tile_shape: the shape of a level, its tile extents and threads per block (3D: the planes
 *   per thread as the shape, extents 1 x planes, 256 threads); -1 and zero extents for the coarsest
 *   level and for the one-launch-per-half-sweep 2D comparison path.  Any output pointer may be NULL. */
/* The autotuner's choices are kept per process; these two calls move them between processes
 * (no GPU needed).  Text format, one entry per line, eight decimal integers:
 *     nx ny batch element_size sweeps finest kappa_bf16 shape
 * (the level's extents, the handle's max_batch, 4 or 8 bytes, nu, 1 for level 0 else 0, 1 when
 * kappa is kept in bfloat16, the shape id).  A later first solve of a handle whose level matches
 * an entry uses that shape without timing (plsqr_autotune with fresh != 0 still measures).
 * plsqr_tune_cache_export: writes the entries to buf (at most cap - 1 characters and a NUL; buf may
 *   be NULL with cap 0) and returns the full text length without the NUL.
 * plsqr_tune_cache_import: merges the entries of a NUL-terminated text (blank lines skipped) and
 *   returns how many it read; -PLSQR_E_INVALID, with nothing merged, for a malformed line or an
 *   unknown shape. */
int64_t plsqr_tune_cache_export(char* buf, int64_t cap);
int32_t plsqr_tune_cache_import(const char* text);
int plsqr_autotune(plsqr_handle h, int32_t fresh);
int plsqr_set_tile_shape(plsqr_handle h, int32_t level, int32_t shape);
int plsqr_tile_shape(plsqr_handle h, int32_t level, int32_t* shape, int32_t* tx, int32_t* ty, int32_t* threads);
/* plsqr_mg_schedule (Sec. 4.2, schedule only): how the handle runs one 2D V-cycle.  *coop = 1: the
 *   levels from *first_level down (every coarser level, the coarse solve and, from level 0, alpha)
 *   in one cooperative launch of at most *max_blocks blocks (0: every block that can be resident),
 *   all resident at once and separated by bounded grid-wide barriers between the phases; the
 *   levels above first_level keep their two launches.  *coop = 0: two launches per level and one
 *   for the coarse solve (*first_level = -1).  -1: not decided yet: the autotuner times the
 *   per-level launches and the cooperative launch from every level with three block caps at the
 *   first solve and keeps the fastest (every schedule gives the same V-cycle bit for bit).  0 for
 *   3D handles, sweeps other than 2, coarse levels too large to stage, or PLSQR_MG_COOP=0 at
 *   create; PLSQR_MG_COOP=1 at create selects the cooperative launch from level
 *   PLSQR_MG_COOP_LEVEL (default 0) wherever it is supported.  first_level and max_blocks may be
 *   NULL.  A grid barrier that runs out records status 5 in every instance's state; the solve then
 *   returns PLSQR_E_TIMEOUT. */
int plsqr_mg_schedule(plsqr_handle h, int32_t* coop, int32_t* first_level, int32_t* max_blocks);

/* ---- bfloat16 kappa ----------------------------------------------------------------------------
 * on != 0: later solves keep the diffusivity kappa (eq. 1.13) only in bfloat16 (8 significant bits,
 * rounded to nearest even from the single-precision value); the finest level of the V-cycle and
 * the first coarsening read it and widen it to float.  Everything else is unchanged, so P is the
 * V-cycle of the rounded kappa.  Needs a 2D PLSQR_FP32 handle with mg_levels >= 2, 1..3 sweeps
 * and mg_cycles = 1 (further cycles would form b - M x from a float kappa that is not kept);
 * otherwise PLSQR_E_INVALID.  plsqr_prec_setup rounds the kappa it is given.  on = 0
 * returns to float kappa (the default). */
int plsqr_set_kappa_bf16(plsqr_handle h, int32_t on);

/* ---- stopping rules --------------------------------------------------------------------------
 * The paper's stopping logic for later solves, slots and batch instances (Sec. 3.4, Sec. 4.1):
 *   inner: MLSQR stops after the first iteration i with ||rbar_i|| <= eta * delta (S4, the
 *     Morozov discrepancy principle; ||rbar_i|| is the LSQR residual estimate, which equals
 *     ||g - A f_i|| at tau = 0 and bounds it from above for tau > 0), within the cap n_inner;
 *   outer: Algorithm 3 stops at f^k (k >= 2) when (R(f^k) - R(f^{k-1})) / R(f^{k-1}) > -r_rel
 *     (R did not decrease by the fraction r_rel), within the cap n_outer.
 * index: -1 = every instance, else one instance of solve_batch / one slot.  eta * delta = 0 turns
 * S4 off, r_rel = 0 the outer stop (the defaults).  eta, delta >= 0 and finite; 0 <= r_rel < 1.
 * The histories of iterations and steps not run stay NaN; f is the iterate where the solve
 * stopped.  Kernels skip a stopped instance, so a batch finishes when its slowest instance does. */
int plsqr_set_stopping(plsqr_handle h, int32_t index, double eta, double delta, double r_rel);

/* ---- slots: continuous batching ---------------------------------------------------------------
 * Algorithm 3 advanced one lagged-diffusivity step at a time (Sec. 4.1: steps 3-5 of one outer
 * iteration), with the handle's max_batch instances used as slots that requests enter and leave
 * independently.  A slot's iterates, Krylov state and histories stay on the device between
 * steps.  Each slot's arithmetic is that of plsqr_solve on a one-instance handle with the same
 * operator: the instances of a launch never mix, so a request gives the same result alone and in
 * any mix.  The first plsqr_slot_start puts the handle in slot mode, where plsqr_solve*,
 * plsqr_solve_batch, plsqr_set_operator and the single-operation entry points (plsqr_apply_A,
 * plsqr_apply_At, plsqr_diffusivity, plsqr_prec_setup, plsqr_prec_apply, plsqr_apply_M,
 * plsqr_mlsqr, plsqr_mlsqr_multi_tau: they would use the slots' state and scratch vectors) return
 * PLSQR_E_STATE.
 *
 * plsqr_slot_start: copies g (device, m values) into `slot` (0 <= slot < max_batch, not busy),
 *   sets f = 0, the slot's r, T, tau and target n_outer.  n_inner must equal, and n_outer must
 *   not exceed, those of the slots already running (history storage is shared).  sigma: NULL
 *   (the operator's blur) or, for a 2D single-precision PLSQR_OP_BLUR handle whose radius is 6, 9,
 *   12 or 15 on both axes, this slot's own sigma[0..1] (x, y): taps exp(-k^2/(2 sigma^2)) for
 *   |k| <= ceil(3 sigma) <= radius, zero beyond, unit sum.  Ordered after the work already on the
 *   caller's stream; the caller's stream then waits for the copy.
 * plsqr_step: enqueues one outer step for every running slot that has not reached its target
 *   (the others are skipped) and returns without waiting.
 * plsqr_query: 1 while the last enqueued slot operation runs, 0 when done, < 0 on a CUDA error.
 * plsqr_slot_progress: outer steps done by `slot` (host-side count) and *active: 0 empty, 1
 *   running, 2 stopped early by the outer rule of plsqr_set_stopping (R fell by less than r_rel:
 *   its f is final; reported once the step that stopped it is done).  Stopping parameters set for
 *   an index before plsqr_slot_start apply to the request started there.
 * plsqr_slot_finish: copies the slot's f (device, N values) to f_out, fills stats (histories of
 *   the steps done, R of the final f; its arrays must hold the n_outer x n_inner, n_outer + 1 and
 *   n_outer values of the slot's plsqr_slot_start), empties the slot; waits for the handle's stream.
 *   Returns PLSQR_E_BREAKDOWN when the slot broke down (f holds its last complete iterate). */
int plsqr_slot_start(plsqr_handle h, int32_t slot, const void* g, int32_t r, double T, double tau,
                     int32_t n_outer, int32_t n_inner, const double* sigma);
int plsqr_step(plsqr_handle h);
int plsqr_query(plsqr_handle h);
int plsqr_slot_progress(plsqr_handle h, int32_t slot, int32_t* outer_done, int32_t* active);
int plsqr_slot_finish(plsqr_handle h, int32_t slot, void* f_out, plsqr_stats* stats);

/* ---- checkpoint and resume of a slot ---------------------------------------------------------
 * The paper has no checkpointing.  Algorithm 3 restarts MLSQR from zero in every outer step (Sec.
 * 4.1), so between two outer steps a request is fully described by f^k, its data g, R(f^k), the
 * outer counter, status, r, T, tau and stopping rule, the histories so far and its blur taps:
 * saving these lets a request be moved to another handle or process, or resumed after a restart,
 * and continue bit for bit as if it had never stopped.
 * plsqr_slot_state_bytes: bytes of one checkpoint of this handle (its grid, data length, history
 *   sizes and taps), or -1 when the handle is not in slot mode.
 * plsqr_slot_save: waits for the handle's stream, then writes the running `slot`'s checkpoint to
 *   the host buffer buf (cap >= plsqr_slot_state_bytes).  The slot keeps running.
 * plsqr_slot_restore: starts `slot` (0 <= slot < max_batch, not busy) from a checkpoint made by
 *   plsqr_slot_save of the same library build on a handle with the same precision, grid, operator
 *   kind, data length and kappa storage (any max_batch, slot index or tile shapes); the request
 *   continues with its remaining outer steps under plsqr_step and ends with plsqr_slot_finish.
 *   n_inner must equal, and the request's n_outer not exceed, those of the slots already running.
 *   A buffer that is not a checkpoint, is too short or does not fit the handle: PLSQR_E_INVALID.
 *   Ordered after the work already on the caller's stream; returns once the copies are done. */
int64_t plsqr_slot_state_bytes(plsqr_handle h);
int plsqr_slot_save(plsqr_handle h, int32_t slot, void* buf, int64_t cap);
int plsqr_slot_restore(plsqr_handle h, int32_t slot, const void* buf, int64_t len);

/* ---- blur without device allocation ---------------------------------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that cannot allocate
 * device memory: a serving process that hands all device memory to its own pool and admits work
 * against that budget (an allocation behind its back could fail or push it over), and
 * latency-critical loops where cudaMalloc / cudaFree would synchronise the device and stall the
 * other streams.
 *
 * y = B x, the separable Gaussian blur of one image (ndim 2) or volume (ndim 3) with zero
 * boundary and taps exp(-k^2/(2 sigma_d^2)) normalised to unit sum, |k| <= radius[d] -- the same
 * operator and kernels as plsqr_apply_A with PLSQR_OP_BLUR.  n: nx, ny(, nz); sigma, radius:
 * per axis (x first), sigma > 0, 0 <= radius <= 32; precision: PLSQR_FP32 (float arrays) or
 * PLSQR_FP64 (double arrays); x, y: device pointers, N values each, not overlapping; stream: a
 * cudaStream_t (NULL = default stream).  No handle, and no cudaMalloc / cudaFree or other
 * allocating call: the taps and the intermediate volume of the 3D blur live in a file-scope
 * device array of 8 MiB that every GPU loading the library holds until exit.  N * element size
 * must not exceed 8 MiB - 2 KiB (2,096,640 floats, 1,048,320 doubles); in 3D, nz <= 65535 and
 * ny <= 524,280 (launch limits).  Larger grids, bad sizes, overlapping x and y or NULL pointers
 * return PLSQR_E_INVALID before anything is enqueued.  The first call on a device looks up the
 * array's device address (make that first call before any stream capture).  All calls share the
 * array, which keeps the last call's contents: calls that overlap on the GPU (other streams,
 * other threads) race on it.  The taps are computed on the host and handed to a kernel by value
 * (no copy from host memory).  The work is enqueued on `stream` and the call does not
 * synchronise.  The staging waits inside the kernels are bounded; should one run out (a copy
 * that never completed), the kernel goes on, y is unspecified, and this entry point has no
 * status to report it with. */
int plsqr_blur_noalloc(int32_t ndim, const int64_t* n, int32_t precision, const double* sigma,
                       const int32_t* radius, const void* x, void* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PLSQR_H */
