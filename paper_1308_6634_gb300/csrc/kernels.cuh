// kernels.cuh -- launchers of the libplsqr kernels (internal C++ interface).
#pragma once
#include "common.cuh"

#include <cuda_bf16.h>

#include <stdexcept>
#include <string>

namespace plsqr {

// Programmatic dependent launches are used unless PLSQR_PDL=0.
bool pdl_enabled();

// The largest shared-memory carveout for a kernel (once per kernel), so that its occupancy is set
// by its blocks' needs and not by the driver's default split of L1 and shared memory.
void max_carveout_set(const void* kfn);

// Launch a kernel that begins with pdl_grid_sync(), with the programmatic-serialization attribute
// so that its launch overlaps the tail of the previous kernel in the stream.
template <typename... KArgs, typename... Args>
void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (e != cudaSuccess) throw std::runtime_error(std::string("kernel launch: ") + cudaGetErrorString(e));
}


// Epilogue of an operator application out = op(in):
//  EPI_PLAIN     out = op(in)
//  EPI_FWD       u = op(v)/alpha - (alpha/beta) u_prev, and beta_new = ||u||  (Alg. 2 step 10)
//  EPI_ADJ       p = op(u)/beta_new - (beta_new/alpha) p                      (Alg. 2 step 11)
//  EPI_ADJ_INIT  p = op(g)/beta_1                                              (Alg. 2 step 3)
// The raw (unnormalised) vectors v, u, p are kept; their scales live in GkState.
enum Epi { EPI_PLAIN = 0, EPI_FWD = 1, EPI_ADJ = 2, EPI_ADJ_INIT = 3 };

enum OpKind { OPK_BLUR = 0, OPK_BLUR_MASK = 1, OPK_JOSEPH = 2, OPK_IDENTITY = 3 };

// Per-angle constants of the Joseph projector (computed in double on the host).
template <typename T>
struct JosephAngle {
    T a1, a2;      // forward: u = s*a1 + c_img - y*a2 along the stepped axis
    T c1, c2;      // gather: t = x*c1 + y*c2 + c_det (continuous bin index of a pixel)
    T hw, inv_hw;  // gather: half width of the footprint in bins, and its inverse
    T wgt;         // 1/|cos| (rows stepped) or 1/|sin| (columns stepped)
    int32_t rows;  // 1: step over rows (|cos| > |sin| by the index rule), 0: columns
};

struct OpDev {
    int kind;
    Dims d;              // image grid
    int64_t m;           // data length per instance
    const void* taps[3]; // blur taps per axis (T), 2R+1 each
    double taps_host[3][65];  // the same taps on the host (kernel-parameter variants)
    int R[3];
    int generic_blur;    // 1: always use the generic blur kernel (tests and comparisons)
    const uint8_t* mask; // [N], shared by all instances
    const void* jtab;    // JosephAngle<T>[n_angles]
    int na, nb;
    double ds;
    // Joseph forward in two row parts per (angle, instance): scratch T[2][jcap][na][nb] for the
    // parts and unsigned[jcap][na] arrival counters (zero between launches); null: one part
    void* jpart;
    unsigned* jcnt;
    int jcap;
    // per-instance blur taps (2D single precision, no mask): [B][2][2R+1] (x then y), or null when
    // every instance uses taps[] (slots of a serving handle may each have their own width)
    const float* tapt;
};

template <typename T>
void op_apply(const OpDev& op, bool adjoint, int epi, const T* in, T* out, const T* prev, T* tmp,
              int B, GkState* st, Red red, cudaStream_t s);

// u = A v / alpha - (alpha/beta) u with beta_new = ||u||, fused with the pending update
// f += cf w, w = v c_upd_v - cw w; false if not available for this operator (then nothing ran).
bool op_fwd_update(const OpDev& op, const float* v, float* u, float* f, float* w, int B, GkState* st, Red red,
                   cudaStream_t s);

// kappa = max(r'(t)/t, kfloor*kappa(0)), R = sum r(t) per instance (state reg/T).
template <typename T>
void diffusivity(const T* f, T* kappa, Dims d, int B, GkState* st, Hist hist, double kfloor, Red red,
                 cudaStream_t s, __nv_bfloat16* k16 = nullptr);

// ---- multigrid ----
template <typename T>
void mg_coarsen(const T* cf, bool fine_is_kappa, T* cc, Dims df, Dims dc, int B, cudaStream_t s,
                const __nv_bfloat16* k16 = nullptr);
// rd = 1 / diagonal of a 2D level's operator, in the smoother's summation order (once per outer
// step; the temporally blocked V-cycle kernels stage it)
template <typename T>
void mg_rdiag2d(const T* cond, bool is_kappa, T* rd, Dims d, int B, cudaStream_t s,
                const __nv_bfloat16* k16 = nullptr);
// kappa widened to bfloat16 storage (round to nearest even)
void to_bf16(const float* a, __nv_bfloat16* b, int64_t n, cudaStream_t s);
template <typename T>
void mg_gs_half(const T* cond, bool is_kappa, const T* b, T* x, Dims d, int colour, bool zero_init, int B,
                cudaStream_t s, int zc = 1);  // zc: planes per thread (1, 2 or 4; 3D)
template <typename T>
void mg_resid_restrict(const T* cond, bool is_kappa, const T* b, const T* x, T* bc, Dims df, Dims dc, int B,
                       cudaStream_t s);
template <typename T>
void mg_prolong_add(const T* xc, T* x, Dims df, Dims dc, int B, cudaStream_t s);
// r = b - M x (b may be null: r = -M x is not needed; y = M x when b == null and negate=false)
template <typename T>
void mg_apply_level(const T* cond, bool is_kappa, const T* x, const T* b, T* y, Dims d, int B, cudaStream_t s);
// The same half sweep, restriction and prolongation with x (and b) in the red-black split layout of
// a 3D level (nx even): [inst][colour][nz][ny][nx/2].  mode: 0 first half sweep of the finest level
// (b natural, copied split to bs), 1 first of a coarser level, 2 any other, 3 the last of the finest
// level (x also written in natural order to out).
template <typename T>
void mg_gs_half_split(const T* cond, bool is_kappa, const T* b, T* bs, T* xs, T* out, Dims d, int colour, int mode,
                      int B, cudaStream_t s);
template <typename T>
void mg_resid_restrict_split(const T* cond, bool is_kappa, const T* bs, const T* xs, T* bc, bool out_split, Dims df,
                             Dims dc, int B, cudaStream_t s);
template <typename T>
void mg_prolong_add_split(const T* xc, bool in_split, T* xs, Dims df, Dims dc, int B, cudaStream_t s);
template <typename T>
void mg_axpy(T* y, const T* x, int64_t n, cudaStream_t s);  // y += x
template <typename T>
void coarse_assemble(const T* cond, bool is_kappa, double* band, Dims d, int bw, int B, cudaStream_t s);
// band <- its Cholesky factor; rdiag <- 1/L(j,j)
void coarse_cholesky(double* band, double* rdiag, int nc, int bw, int B, cudaStream_t s);
void coarse_inverse(const double* band, const double* rdiag, double* X, int nc, int bw, int B, cudaStream_t s);
template <typename T>
void coarse_symv(const T* X, const T* b, T* x, int nc, int B, const GkState* st, cudaStream_t s);
void round_to_float(const double* a, float* b, int64_t n, cudaStream_t s);
// Subtraction-free coarse factorisation and inverse in float (bandwidth <= 32) or double
// (bandwidth <= 16): V is the type of the tables and of X.
int gth_stride(int bw);
bool gth_supported(int bw, int nc, size_t esz);
template <typename T, typename V>
void gth_assemble(const T* cond, bool is_kappa, V* gcol, Dims d, int bw, int B, cudaStream_t s);
// xscr: scratch of the blocked inverse (B * xblk_scratch(nc) elements), or null for the row-by-row
// kernels.
template <typename V>
void gth_factor_inverse(V* gcol, V* grow, V* X, V* xscr, int nc, int bw, int B, GkState* st, cudaStream_t s);
int64_t xblk_scratch(int nc, int bw);
// Wide bands: the float L D L^T with a window of bw + 1 columns, and the float inverse with a warp
// per column.
bool gth_wide_supported(int bw, int nc);
void gth_wide_factor_inverse(float* gcol, float* grow, float* X, float* xscr, int nc, int bw, int B, GkState* st,
                             cudaStream_t s);

// ---- the whole 2D V-cycle in one cooperative launch ----
constexpr int COOP_LEVELS = 8;
// Per-level buffers of one V-cycle application: level 0 holds the right-hand side b (p~ or a
// residual), the pre-smoothed iterate x and the result x2; levels >= 1 the restricted residual b,
// the pre-smoothed x and the post-smoothed x2; the last level is the coarsest (x2 = X b).
struct CoopLevels {
    const void* cond[COOP_LEVELS];  // level 0: kappa; levels >= 1: conductances [B][2][N_l]
    const void* rd[COOP_LEVELS];    // 1 / diagonal of the smoothed levels
    void* b[COOP_LEVELS];
    void* x[COOP_LEVELS];
    void* x2[COOP_LEVELS];
    Dims d[COOP_LEVELS];
    int L;
};
// The grid barrier's counters (zero between launches) and the abort flag, in device memory.
struct CoopSync {
    unsigned* arrive;
    unsigned* depart;
    int* abort;
};
// Whether the cooperative V-cycle can run for this level count and coarsest size (nu = 2).
bool mg2d_coop_supported(int nu, size_t elem, int L, int nc);
// Levels lc .. L-1 of one V-cycle in one launch: x2[lc] = the V-cycle of level lc applied to b[lc]
// (lc = 0: the whole V-cycle, x2[0] = P b[0]; dot as in mg2d_post: 0 none, 1 alpha_1, 2 alpha and
// the rotations, finest level only).  cap: at most this many blocks (0: as many as are resident).
template <typename T>
void mg2d_vcycle_coop(const CoopLevels& cl, int lc, int cap, int nu, const T* X, int nc, int B, int dot,
                      GkState* st, Hist hist, Red red, CoopSync sy, const __nv_bfloat16* k16, cudaStream_t s);

// ---- temporally blocked 2D V-cycle (one launch per level and direction) ----
bool mg2d_supported(int ndim, int nu);
// First level from which the coarse end of a 2D V-cycle (levels.. L-1) runs as one cluster launch
// (mg2d_tail), or L when it does not apply.
int mg2d_tail_level(const Dims* d, int L, int nu, size_t elem, int nc);
template <typename T>
void mg2d_tail(const TailLevels& tl, int nu, const T* X, int nc, int B, GkState* st, cudaStream_t s);
// x = nu red->black sweeps from 0 on M_l x = b; bc = R (b - M_l x).  rd: 1 / diagonal (mg_rdiag2d).
// shape: the tile shape (mg2d_shape), 0 the default; every shape gives the same result.
template <typename T>
void mg2d_pre(const T* cond, bool is_kappa, const T* b, const T* rd, T* x, T* bc, Dims d, Dims dc, int nu, int B,
              GkState* st, cudaStream_t s, const __nv_bfloat16* k16 = nullptr, int shape = 0);
// x = nu black->red sweeps from xi + P xc.  dot: 0 none, 1 alpha_1 (init), 2 alpha and rotations
template <typename T>
void mg2d_post(const T* cond, bool is_kappa, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d,
               Dims dc, int nu, int B, int dot, GkState* st, Hist hist, Red red, cudaStream_t s,
               const __nv_bfloat16* k16 = nullptr, int shape = 0);
// Tile shape `id` of the finest (fine) or the coarser levels: extents and threads per block; false
// past the last shape.
bool mg2d_shape(bool fine, int id, int* tx, int* ty, int* nth);

// ---- Golub-Kahan scalars and updates ----
void set_params(GkState* st, const SolveParams* prm, int B, bool reset_outer, cudaStream_t s);
void slots_state(GkState* st, const SolveParams* prm, int B, int slot, bool idle, cudaStream_t s,
                 bool keep_outer = false);
template <typename T>
void gk_init_norm(const T* g, int64_t m, int B, GkState* st, Red red, cudaStream_t s);
template <typename T>
void gk_dot_rotate(const T* v, const T* p, int64_t N, int B, bool init, GkState* st, Hist hist, Red red,
                   cudaStream_t s);
template <typename T>
void gk_update(T* f, T* w, const T* v, int64_t N, int B, bool init, const GkState* st, cudaStream_t s);
// Stored Lanczos vectors (one instance): V_j = v~ / alpha and ab = (alpha, beta) now; store_v
// false records the scalars only.
template <typename T>
void gk_store_basis(const T* v, T* Vj, int64_t N, const GkState* st, double* ab, bool store_v, cudaStream_t s);
constexpr int MT_MAX = 32;  // damping parameters per combination pass
// The bounded wait of the TMA staging on a barrier that completes, or never does (complete false:
// ST_TIMEOUT in st[0] after 2 x limit polls).  Issues no copy.
void selftest_wait(GkState* st, bool complete, uint32_t limit, cudaStream_t s);
template <typename T>
struct OutPtrs {
    T* p[MT_MAX];
};
// outs[t] = sum_{j < k} coef[t * k + j] V_j, t < n_tau (coef on the device)
template <typename T>
void combine_basis(const T* V, int k, int64_t N, const double* coef, int n_tau, const OutPtrs<T>& outs,
                   cudaStream_t s);
template <typename T>
void resid_norm(const T* g, const T* Af, int64_t m, int B, GkState* st, Hist hist, Red red, cudaStream_t s);
void fill_nan(double* p, int64_t n, cudaStream_t s);

int red_blocks(int64_t n);  // blocks per instance used by the plain reductions

// ---- launch bookkeeping ----
// Every launcher brackets its launch with kbegin/kend.  kend checks the launch error and
// counts it; when a Profiler is installed for the calling thread and enabled, the launch is
// also bracketed by CUDA events tagged with its class (eager launches only).
enum KClass {
    KC_FWD = 0,      // A with the Golub-Kahan forward epilogue (and beta reduction)
    KC_ADJ = 1,      // A^T with the p update
    KC_OP_PLAIN = 2, // A or A^T without epilogue (residual, single-step entry points)
    KC_GS_FINE = 3,  // red-black half sweeps on the finest level
    KC_MG_OTHER = 4, // coarse-level sweeps, residual/restriction, prolongation, residuals
    KC_COARSE = 5,   // dense solve on the coarsest level
    KC_GK = 6,       // norms, dot + rotations, solution update
    KC_SETUP = 7,    // diffusivity, coarsening, band assembly, Cholesky, inverse
    KC_COUNT = 8
};

struct Profiler {
    int64_t launches = 0;
    bool enabled = false;
    struct Rec { int cls; cudaEvent_t a, b; };
    Rec* recs = nullptr;
    int n_recs = 0, cap = 0;
    double ms[KC_COUNT] = {};
    int64_t count[KC_COUNT] = {};
    bool open = false;
    void begin(int cls, cudaStream_t s);
    void finish(cudaStream_t s);
    void collect();  // synchronise the recorded events and add their durations
    void release();
};

Profiler*& current_profiler();
void kbegin(int cls, cudaStream_t s);   // start event of a timed region (profiling only)
void klaunched(const char* what);      // check the launch that was just issued, count it
void kfinish(cudaStream_t s);          // end event of the timed region (profiling only)

}  // namespace plsqr
