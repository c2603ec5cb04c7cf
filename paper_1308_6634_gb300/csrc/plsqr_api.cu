// plsqr_api.cu -- host side of libplsqr: handles, workspace, the order of the kernels of
// Algorithms 2 and 3, CUDA-graph capture of one outer step, and the C ABI of plsqr.h.
//
// A solve runs on an internal non-blocking stream ordered after the caller's stream by
// events (so the caller's stream may be the legacy default stream, which cannot be
// captured).  One outer step of Algorithm 3 -- diffusivity, priorconditioner setup, MLSQR
// initialisation, n_inner MLSQR iterations and the residual norm -- is captured once per
// (batch count, n_inner, history shape) and replayed n_outer times; the outer step index
// lives in device memory, so every replay writes its own history row.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/plsqr.h"
#include "kernels.cuh"
#include "tma.cuh"

using namespace plsqr;

namespace {

const double kPi = 3.14159265358979323846;

// An NVTX range for the scope (host side: it marks when the work is enqueued, and a profiler
// relates it to the launches made inside).  With no tool attached the calls return at once.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    Range(const char* name, int64_t payload) {
        nvtxEventAttributes_t a;
        std::memset(&a, 0, sizeof a);
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
        a.payload.llValue = payload;
        nvtxRangePushEx(&a);
    }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct CudaError : std::runtime_error {
    using std::runtime_error::runtime_error;
};
struct InvalidArg : std::runtime_error {
    using std::runtime_error::runtime_error;
};
struct NoMem : std::runtime_error {
    using std::runtime_error::runtime_error;
};

void ck(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // reported through the return code: do not leave it for the caller's next CUDA call
        throw NoMem(std::string(what) + ": " + cudaGetErrorString(e));
    }
    if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

struct Level {
    Dims d;
    char* cond = nullptr;  // [B][ndim][N_l] (levels >= 1)
    char* b = nullptr;     // [B][N_l]
    char* x = nullptr;     // pre-smoothed iterate (fused path) or the V-cycle result (generic path)
    char* x2 = nullptr;    // V-cycle result of this level (fused path)
    char* rd = nullptr;    // [B][N_l] 1 / diagonal (2D levels above the coarsest)
};

// One workspace allocation.  With guard bands, kGuard bytes of kGuardByte sit on each side of
// the region the library uses; a write past either end of the region changes them.
struct Alloc {
    char* base;    // returned by cudaMalloc, freed with cudaFree
    char* user;    // the region the library uses: base, or base + kGuard
    size_t bytes;  // size of that region
};
constexpr size_t kGuard = 256;  // keeps the region 256-byte aligned
constexpr unsigned char kGuardByte = 0xA5;

}  // namespace

struct plsqr_ctx {
    plsqr_config cfg{};
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    bool fp64 = false;
    size_t esz = 4;
    Dims d{};
    int B = 1;
    int L = 1, nu = 2, cycles = 1;
    double kfloor = 1e-4;
    // operator
    bool op_set = false;
    plsqr_operator op{};
    OpDev od{};
    int64_t m = 0;
    void* taps[3] = {nullptr, nullptr, nullptr};
    void* jtab = nullptr;
    void* jpart = nullptr;  // Joseph forward: the two row parts and their arrival counters
    void* jcnt = nullptr;
    int jcap = 0;
    uint8_t* mask = nullptr;
    // workspace
    char *g = nullptr, *f = nullptr, *u = nullptr, *p = nullptr, *v = nullptr, *w = nullptr;
    char *kappa = nullptr, *tmp = nullptr, *tmpm = nullptr, *r0 = nullptr, *e0 = nullptr;
    Level lv[16];
    int nc = 0, bw = 0;
    double* band = nullptr;
    double* rdiag = nullptr;  // 1/L(j,j) of the coarse factor, [B][nc]
    double* X = nullptr;  // inverse of the coarsest operator, [B][nc][nc]
    float* Xf = nullptr;  // the same rounded to float (single-precision handles)
    // single-precision handles with a coarsest bandwidth <= 32: subtraction-free L D L^T in float
    bool gth = false;
    bool gthw = false;  // wide band: float L D L^T (windowed) and float inverse
    char* gcol = nullptr;  // [B][nc][stride] (float, or double for FP64 handles): column layout
                           // (input conductances, then l and 1/d)
    char* grow = nullptr;  // [B][nc][stride]: row layout of l
    char* xblk = nullptr;  // scratch of the blocked inverse, or null (row-by-row kernels)
    GkState* st = nullptr;
    SolveParams* prm_dev = nullptr;
    SolveParams* prm_host = nullptr;  // pinned
    GkState* st_host = nullptr;       // pinned
    Red red{};
    // histories
    double *h_rbar = nullptr, *h_R = nullptr, *h_resid = nullptr;
    int h_outer = 0, h_inner = 0;
    double* h_stage = nullptr;  // pinned staging for history download
    size_t h_stage_n = 0;
    // graphs (with the number of kernel launches each replay executes)
    std::map<std::tuple<int, int, int, int>, std::pair<cudaGraphExec_t, int64_t>> graphs;
    // slots (continuous batching): host bookkeeping, per-slot blur taps
    bool serving = false;
    bool st_after_step = false;  // st_host holds the states copied after the last plsqr_step
    std::vector<int> slot_active, slot_outer, slot_target;
    float* taps_inst = nullptr;       // device [B][2][2R+1]
    float* taps_inst_host = nullptr;  // pinned staging, same shape
    // kappa stored in bfloat16 (the diffusivity's only output; the finest-level V-cycle widens it)
    bool kbf16 = false;
    __nv_bfloat16* kappa16 = nullptr;
    bool generic_mg = false;  // PLSQR_GENERIC_MG=1: one launch per half sweep (comparisons)
    // 3D V-cycle in the red-black split layout (opt-in, PLSQR_MG_SPLIT=1; every smoothed level has
    // an even nx): the finest level's split x and b in xs0, bs0, the coarser levels' in their own b
    // and x.  Measured slower than natural order on the 192^3 workload (the half sweeps are bound by
    // the latency of their scattered loads, not by the DRAM sectors the split layout saves).
    bool split3 = false;
    char *xs0 = nullptr, *bs0 = nullptr;
    int tail_lc = 16;         // first level of the one-launch coarse end of the 2D V-cycle (>= L: none)
    // the whole 2D V-cycle in one cooperative launch: -1 undecided (the autotuner times both
    // schedules), 0 per-level launches, 1 cooperative; PLSQR_MG_COOP=0/1 fixes it
    int coop = -1;
    int coop_lc = 0;                // first level of the cooperative launch (the levels above: per-level)
    int coop_cap = 0;               // at most this many blocks (0: every resident block)
    bool coop_ok = false;           // supported for this handle (2D, nu = 2, TMA, levels, coarse size)
    unsigned* coop_sync = nullptr;  // grid barrier counters and abort flag (zero between launches)
    int tile[16] = {};        // tile shape of each 2D V-cycle level (mg2d_shape ids; 0 the default)
    int zc3[16] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};  // 3D: planes per thread of each level's half sweeps
    bool tuned = false;       // tile shapes chosen (autotuned or set)
    bool tiles_set = false;   // chosen by plsqr_set_tile_shape: kept when the kappa storage changes
    // stored Lanczos vectors of the running inner solve (plsqr_mlsqr_multi_tau): V_j, (alpha, beta)
    char* basis = nullptr;
    double* basis_ab = nullptr;
    int basis_n = 0;
    TailLevels tail{};
    bool no_fuse_update = false;  // PLSQR_FUSE_UPDATE=0: separate update kernel (comparisons)
    Profiler prof;
    int64_t last_launches = 0;
    bool use_graph = true;
    std::vector<Alloc> allocs;
    bool guard = false;  // PLSQR_GUARD=1 at create: guard bands around every workspace allocation
    std::string err;
};

namespace {

template <typename T>
T* P(char* p) { return reinterpret_cast<T*>(p); }

__nv_bfloat16* K16(plsqr_ctx* h) { return h->kbf16 ? h->kappa16 : nullptr; }

char* dalloc(plsqr_ctx* h, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    const size_t g = h->guard ? kGuard : 0;
    ck(cudaMalloc(&p, bytes + 2 * g), "cudaMalloc");
    char* base = (char*)p;
    h->allocs.push_back(Alloc{base, base + g, bytes});
    if (g) {
        ck(cudaMemset(base, kGuardByte, g), "cudaMemset");
        ck(cudaMemset(base + g + bytes, kGuardByte, g), "cudaMemset");
    }
    // zeroed once, so that no kernel (the tile-shape timing before the first plsqr_prec_setup
    // included) ever reads uninitialised memory
    ck(cudaMemset(base + g, 0, bytes), "cudaMemset");
    return base + g;
}

void dfree(plsqr_ctx* h, void* p) {
    if (!p) return;
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
        if (it->user == p) {
            cudaFree(it->base);
            h->allocs.erase(it);
            return;
        }
}

void clear_graphs(plsqr_ctx* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.first);
    h->graphs.clear();
}

// Installs the handle's profiler for the calling thread for the duration of a C-ABI call.
struct ProfScope {
    Profiler* prev;
    explicit ProfScope(plsqr_ctx* h) : prev(current_profiler()) { current_profiler() = &h->prof; }
    ~ProfScope() { current_profiler() = prev; }
};

Dims make_dims(int ndim, int64_t nx, int64_t ny, int64_t nz) {
    Dims d;
    d.ndim = ndim;
    d.nx = (int32_t)nx;
    d.ny = (int32_t)ny;
    d.nz = ndim == 3 ? (int32_t)nz : 1;
    d.N = (int64_t)d.nx * d.ny * d.nz;
    d.fx = make_fdiv(d.nx);
    d.fy = make_fdiv(d.ny);
    d.fh = make_fdiv(d.nx / 2);
    return d;
}

// The coarse inverse in 32 x 32 blocks (k_xblk_*) whatever the batch, so that an instance's
// result does not depend on how many share its handle; PLSQR_GTH_BLOCKED=0 keeps the row-by-row
// kernels (comparisons).
bool xblk_enabled(int B) {
    (void)B;
    const char* e = std::getenv("PLSQR_GTH_BLOCKED");
    return !(e && e[0] == '0');
}

// Sizes of everything create() allocates (used by plsqr_workspace_bytes too).
struct Plan {
    Dims d;
    int L, nc, bw;
    int64_t level_N[16];
    size_t bytes;
    bool gth;   // float factor and inverse (bandwidth <= 32)
    bool gthw;  // float factor and inverse of a wide band
    bool split3;  // 3D V-cycle in the red-black split layout
};

Plan make_plan(const plsqr_config* c, int64_t m) {
    if (!c) throw InvalidArg("config is NULL");
    if (c->ndim != 2 && c->ndim != 3) throw InvalidArg("ndim must be 2 or 3");
    if (c->precision != PLSQR_FP32 && c->precision != PLSQR_FP64) throw InvalidArg("bad precision");
    if (c->mg_levels < 1 || c->mg_levels > 12) throw InvalidArg("mg_levels must be in 1..12");
    if (c->mg_levels > 1 && (c->mg_sweeps < 1 || c->mg_sweeps > 16)) throw InvalidArg("mg_sweeps must be 1..16");
    if (c->mg_cycles < 1 || c->mg_cycles > 16) throw InvalidArg("mg_cycles must be 1..16");
    if (c->max_batch < 1 || c->max_batch > 4096) throw InvalidArg("max_batch must be 1..4096");
    if (!(c->kappa_floor >= 0.0)) throw InvalidArg("kappa_floor must be >= 0");
    const int64_t div = (int64_t)1 << (c->mg_levels - 1);
    for (int dd = 0; dd < c->ndim; ++dd) {
        if (c->n[dd] < 1 || c->n[dd] > (1 << 20)) throw InvalidArg("extent out of range");
        if (c->n[dd] % div) throw InvalidArg("each extent must be divisible by 2^(mg_levels-1)");
    }
    Plan pl;
    pl.d = make_dims(c->ndim, c->n[0], c->n[1], c->n[2]);
    if (pl.d.N > ((int64_t)1 << 31)) throw InvalidArg("grid too large");
    pl.L = c->mg_levels;
    Dims dc = pl.d;
    for (int l = 0; l < pl.L; ++l) {
        if (l > 0) dc = make_dims(c->ndim, dc.nx / 2, dc.ny / 2, dc.nz / 2);
        pl.level_N[l] = dc.N;
    }
    pl.nc = (int)dc.N;
    pl.bw = c->ndim == 3 ? dc.nx * dc.ny : dc.nx;
    if (pl.nc > 16384) throw InvalidArg("coarsest level has more than 16384 cells: add levels");
    const char* e64 = std::getenv("PLSQR_COARSE64");
    const size_t vsz = c->precision == PLSQR_FP64 ? 8 : 4;  // the GTH tables in the handle's type
    pl.gth = gth_supported(pl.bw, pl.nc, vsz) && !(e64 && e64[0] == '1');
    pl.gthw = c->precision == PLSQR_FP32 && !pl.gth && gth_wide_supported(pl.bw, pl.nc) && !(e64 && e64[0] == '1');
    if (!pl.gth && !pl.gthw &&
        (size_t)(pl.bw + 4) * (pl.bw + 1) * sizeof(double) + (size_t)pl.bw * (pl.bw + 1) * 2 + pl.bw * 8 >
            227 * 1024)
        throw InvalidArg("coarsest level too wide for the banded factorisation: add levels");
    const size_t esz = c->precision == PLSQR_FP64 ? 8 : 4;
    const int64_t B = c->max_batch, N = pl.d.N;
    if (m <= 0) m = N;
    size_t b = 0;
    b += esz * B * (2 * m + 5 * N);  // g, u, f, p, v, w, kappa
    b += esz * B * (N + m);          // tmp (N), tmpm (m)
    if (c->mg_cycles > 1) b += esz * B * 2 * N;
    {  // PLSQR_MG_SPLIT=1 (3D, every smoothed level with an even nx): split x and b of level 0
        const char* es = std::getenv("PLSQR_MG_SPLIT");
        pl.split3 = c->ndim == 3 && pl.L >= 2 && c->mg_sweeps >= 1 && es && es[0] == '1';
        for (int l = 0, nx = c->n[0]; l + 1 < pl.L; ++l, nx /= 2) pl.split3 = pl.split3 && nx % 2 == 0;
        if (pl.split3) b += esz * B * 2 * N;
    }
    for (int l = 1; l < pl.L; ++l) b += esz * B * pl.level_N[l] * (c->ndim + 3);
    if (c->ndim == 2)
        for (int l = 0; l + 1 < pl.L; ++l) b += esz * B * pl.level_N[l];  // reciprocal diagonals
    if (pl.gth || pl.gthw) {
        b += (pl.gth ? vsz : sizeof(float)) * B * (size_t)pl.nc * (2 * gth_stride(pl.bw) + pl.nc);
        if (xblk_enabled((int)B)) b += (pl.gth ? vsz : sizeof(float)) * B * (size_t)xblk_scratch(pl.nc, pl.bw);
    } else {
        b += sizeof(double) * B * (size_t)pl.nc * (pl.bw + 2);
        b += (sizeof(double) + (c->precision == PLSQR_FP64 ? 0 : sizeof(float))) * B * (size_t)pl.nc * pl.nc;
    }
    b += (sizeof(GkState) + sizeof(SolveParams) + sizeof(unsigned)) * B;
    b += sizeof(double) * B * std::max<int64_t>(8192, (int64_t)((pl.d.ny + 15) / 16) * ((pl.d.nx + 31) / 32));
    pl.bytes = b;
    return pl;
}

// Instances (at most B) for which the Joseph forward may run in two row parts per (angle,
// instance): those with n_angles x instances below 3 x 152.
int joseph_parts_cap(int64_t B, int na) {
    return na < 1 ? 0 : (int)std::min<int64_t>(B, (3 * 152 - 1) / na);
}

int64_t op_data_len(const plsqr_operator* op, const Dims& d) {
    if (op && op->kind == PLSQR_OP_JOSEPH) return (int64_t)op->n_angles * op->n_bins;
    return d.N;
}

void alloc_data_buffers(plsqr_ctx* h) {
    const int64_t B = h->B, m = h->m;
    dfree(h, h->g);
    dfree(h, h->u);
    dfree(h, h->tmpm);
    h->g = dalloc(h, h->esz * B * m);
    h->u = dalloc(h, h->esz * B * m);
    h->tmpm = dalloc(h, h->esz * B * m);
}

// ---- the order of the kernels ----------------------------------------------------------------

// Inverse of the coarsest operator in the handle's element type.
template <typename T>
const T* coarse_inverse_of(plsqr_ctx* h);
template <>
const double* coarse_inverse_of<double>(plsqr_ctx* h) { return h->X; }
template <>
const float* coarse_inverse_of<float>(plsqr_ctx* h) { return h->Xf; }

Hist hist_of(plsqr_ctx* h) {
    Hist hs;
    hs.rbar = h->h_rbar;
    hs.R = h->h_R;
    hs.resid = h->h_resid;
    hs.n_outer = h->h_outer;
    hs.n_inner = h->h_inner;
    return hs;
}


// The 3D V-cycle in the split layout: level 0 takes b and gives x in natural order; the smoothed
// levels below it keep b and x split; the coarsest is in natural order.  The same half sweeps in
// the same order as vcycle below.
template <typename T>
void vcycle_split(plsqr_ctx* h, int l, const T* b, T* x, int B, cudaStream_t s) {
    const Level& Lv = h->lv[l];
    const T* cond = l == 0 ? P<T>(h->kappa) : P<T>(Lv.cond);
    const bool isk = l == 0;
    T* xs = l == 0 ? P<T>(h->xs0) : x;
    T* bs = l == 0 ? P<T>(h->bs0) : const_cast<T*>(b);
    const Level& C = h->lv[l + 1];
    const bool c_split = l + 1 < h->L - 1;
    for (int k = 0; k < h->nu; ++k) {
        mg_gs_half_split<T>(cond, isk, k == 0 ? b : bs, bs, xs, nullptr, Lv.d, 0, k > 0 ? 2 : (l == 0 ? 0 : 1), B, s);
        mg_gs_half_split<T>(cond, isk, bs, bs, xs, nullptr, Lv.d, 1, 2, B, s);
    }
    mg_resid_restrict_split<T>(cond, isk, bs, xs, P<T>(C.b), c_split, Lv.d, C.d, B, s);
    if (c_split) vcycle_split<T>(h, l + 1, P<T>(C.b), P<T>(C.x), B, s);
    else coarse_symv<T>(coarse_inverse_of<T>(h), P<T>(C.b), P<T>(C.x), h->nc, B, h->st, s);
    mg_prolong_add_split<T>(P<T>(C.x), c_split, xs, Lv.d, C.d, B, s);
    for (int k = 0; k < h->nu; ++k) {
        mg_gs_half_split<T>(cond, isk, bs, bs, xs, nullptr, Lv.d, 1, 2, B, s);
        mg_gs_half_split<T>(cond, isk, bs, bs, xs, x, Lv.d, 0, (l == 0 && k == h->nu - 1) ? 3 : 2, B, s);
    }
}

template <typename T>
void vcycle(plsqr_ctx* h, int l, const T* b, T* x, int B, cudaStream_t s) {
    if (l == 0 && h->split3) {
        vcycle_split<T>(h, 0, b, x, B, s);
        return;
    }
    const Level& Lv = h->lv[l];
    const T* cond = l == 0 ? P<T>(h->kappa) : P<T>(Lv.cond);
    const bool isk = l == 0;
    if (l == h->L - 1) {
        coarse_symv<T>(coarse_inverse_of<T>(h), b, x, h->nc, B, h->st, s);
        return;
    }
    for (int k = 0; k < h->nu; ++k) {
        mg_gs_half<T>(cond, isk, b, x, Lv.d, 0, k == 0, B, s, h->zc3[l]);
        mg_gs_half<T>(cond, isk, b, x, Lv.d, 1, false, B, s, h->zc3[l]);
    }
    const Level& C = h->lv[l + 1];
    mg_resid_restrict<T>(cond, isk, b, x, P<T>(C.b), Lv.d, C.d, B, s);
    vcycle<T>(h, l + 1, P<T>(C.b), P<T>(C.x), B, s);
    mg_prolong_add<T>(P<T>(C.x), x, Lv.d, C.d, B, s);
    for (int k = 0; k < h->nu; ++k) {
        mg_gs_half<T>(cond, isk, b, x, Lv.d, 1, false, B, s, h->zc3[l]);
        mg_gs_half<T>(cond, isk, b, x, Lv.d, 0, false, B, s, h->zc3[l]);
    }
}

// Levels lc..L-1 of a V-cycle in one cooperative launch: x = the level-lc V-cycle applied to b (the
// hierarchy and scratch of vcycle_fused; level lc > 0 takes b = lv[lc].b, x = lv[lc].x2).
template <typename T>
void vcycle_coop(plsqr_ctx* h, int lc, const T* b, T* x, int B, int dot, cudaStream_t s) {
    CoopLevels cl{};
    cl.L = h->L;
    for (int l = 0; l < h->L; ++l) {
        const Level& Lv = h->lv[l];
        cl.d[l] = Lv.d;
        cl.cond[l] = l == 0 ? (const void*)h->kappa : (const void*)Lv.cond;
        cl.rd[l] = Lv.rd;
        cl.b[l] = l == lc ? (void*)b : (void*)Lv.b;
        cl.x[l] = l == 0 ? (void*)h->tmp : (void*)Lv.x;
        cl.x2[l] = l == lc ? (void*)x : (void*)Lv.x2;
    }
    CoopSync sy;
    sy.arrive = h->coop_sync;
    sy.depart = h->coop_sync + 1;
    sy.abort = reinterpret_cast<int*>(h->coop_sync + 2);
    mg2d_vcycle_coop<T>(cl, lc, h->coop_cap, h->nu, coarse_inverse_of<T>(h), h->nc, B, dot, h->st, hist_of(h),
                        h->red, sy, lc == 0 ? K16(h) : nullptr, s);
}

// Temporally blocked V-cycle (2D): one pre and one post launch per level.  dot (finest level
// only): 0 none, 1 alpha_1, 2 alpha and the rotations fused into the last post launch.
template <typename T>
void vcycle_fused(plsqr_ctx* h, int l, const T* b, T* x, int B, int dot, cudaStream_t s) {
    const Level& Lv = h->lv[l];
    if (l == h->L - 1) {
        coarse_symv<T>(coarse_inverse_of<T>(h), b, x, h->nc, B, h->st, s);
        return;
    }
    if (h->coop == 1 && l == h->coop_lc) {  // levels l..L-1 in one cooperative launch
        vcycle_coop<T>(h, l, b, x, B, dot, s);
        return;
    }
    if (l == h->tail_lc) {  // levels l..L-1 in one cluster launch (x is lv[l].x2 here)
        mg2d_tail<T>(h->tail, h->nu, coarse_inverse_of<T>(h), h->nc, B, h->st, s);
        return;
    }
    const T* cond = l == 0 ? P<T>(h->kappa) : P<T>(Lv.cond);
    const bool isk = l == 0;
    T* xpre = l == 0 ? P<T>(h->tmp) : P<T>(Lv.x);
    const Level& C = h->lv[l + 1];
    mg2d_pre<T>(cond, isk, b, P<T>(Lv.rd), xpre, P<T>(C.b), Lv.d, C.d, h->nu, B, h->st, s, isk ? K16(h) : nullptr,
                h->tile[l]);
    vcycle_fused<T>(h, l + 1, P<T>(C.b), P<T>(C.x2), B, 0, s);
    mg2d_post<T>(cond, isk, b, P<T>(Lv.rd), xpre, x, P<T>(C.x2), Lv.d, C.d, h->nu, B, dot, h->st, hist_of(h), h->red, s,
                 isk ? K16(h) : nullptr, h->tile[l]);
}

bool use_fused_mg(const plsqr_ctx* h) { return mg2d_supported(h->d.ndim, h->nu) && h->L > 1 && !h->generic_mg; }

// One V-cycle on level 0 with the handle's schedule (dot: see vcycle_fused).
template <typename T>
void vcycle_2d(plsqr_ctx* h, const T* b, T* x, int B, int dot, cudaStream_t s) {
    vcycle_fused<T>(h, 0, b, x, B, dot, s);
}

// x = P b: `cycles` V-cycles from zero, x <- x + V(b - M x).  Returns true when alpha and the
// rotations were fused into the last launch (dot: 1 init, 2 iteration; 0 = not requested).
template <typename T>
bool prec_apply(plsqr_ctx* h, const T* b, T* x, int B, cudaStream_t s, int dot = 0) {
    const bool fused = use_fused_mg(h);
    const bool fuse_dot = fused && dot != 0 && h->cycles == 1;
    if (fused) vcycle_2d<T>(h, b, x, B, fuse_dot ? dot : 0, s);
    else vcycle<T>(h, 0, b, x, B, s);
    for (int c = 1; c < h->cycles; ++c) {
        mg_apply_level<T>(P<T>(h->kappa), true, x, b, P<T>(h->r0), h->d, B, s);
        if (fused) vcycle_2d<T>(h, P<T>(h->r0), P<T>(h->e0), B, 0, s);
        else vcycle<T>(h, 0, P<T>(h->r0), P<T>(h->e0), B, s);
        mg_axpy<T>(x, P<T>(h->e0), (int64_t)B * h->d.N, s);
    }
    return fuse_dot;
}

// Coarse conductances, band of the coarsest operator, its Cholesky factor and inverse.
template <typename T>
void prec_setup(plsqr_ctx* h, int B, cudaStream_t s) {
    for (int l = 0; l + 1 < h->L; ++l)
        mg_coarsen<T>(l == 0 ? P<T>(h->kappa) : P<T>(h->lv[l].cond), l == 0, P<T>(h->lv[l + 1].cond), h->lv[l].d,
                      h->lv[l + 1].d, B, s, l == 0 ? K16(h) : nullptr);
    if (use_fused_mg(h))
        for (int l = 0; l + 1 < h->L; ++l)
            mg_rdiag2d<T>(l == 0 ? P<T>(h->kappa) : P<T>(h->lv[l].cond), l == 0, P<T>(h->lv[l].rd), h->lv[l].d, B, s,
                          l == 0 ? K16(h) : nullptr);
    const int lc = h->L - 1;
    const T* cc = lc == 0 ? P<T>(h->kappa) : P<T>(h->lv[lc].cond);
    if (h->gth) {  // tables and inverse in the handle's type
        gth_assemble<T, T>(cc, lc == 0, P<T>(h->gcol), h->lv[lc].d, h->bw, B, s);
        gth_factor_inverse<T>(P<T>(h->gcol), P<T>(h->grow), const_cast<T*>(coarse_inverse_of<T>(h)), P<T>(h->xblk),
                              h->nc, h->bw, B, h->st, s);
        return;
    }
    if (h->gthw) {
        gth_assemble<T, float>(cc, lc == 0, P<float>(h->gcol), h->lv[lc].d, h->bw, B, s);
        gth_wide_factor_inverse(P<float>(h->gcol), P<float>(h->grow), h->Xf, P<float>(h->xblk), h->nc, h->bw, B,
                                h->st, s);
        return;
    }
    coarse_assemble<T>(cc, lc == 0, h->band, h->lv[lc].d, h->bw, B, s);
    coarse_cholesky(h->band, h->rdiag, h->nc, h->bw, B, s);
    coarse_inverse(h->band, h->rdiag, h->X, h->nc, h->bw, B, s);
    if (!h->fp64) round_to_float(h->X, h->Xf, (int64_t)B * h->nc * h->nc, s);
}


// MLSQR (Algorithm 2) from f = 0 with the current priorconditioner.
template <typename T>
void mlsqr_seq(plsqr_ctx* h, int B, int n_inner, cudaStream_t s) {
    const int64_t N = h->d.N;
    Hist hs = hist_of(h);
    T *g = P<T>(h->g), *u = P<T>(h->u), *p = P<T>(h->p), *v = P<T>(h->v), *w = P<T>(h->w), *f = P<T>(h->f);
    T* tmp = P<T>(h->tmp);
    gk_init_norm<T>(g, h->m, B, h->st, h->red, s);                                  // steps 2, 7
    op_apply<T>(h->od, true, EPI_ADJ_INIT, g, p, nullptr, tmp, B, h->st, h->red, s);  // step 3
    if (!prec_apply<T>(h, p, v, B, s, 1))                                           // step 4
        gk_dot_rotate<T>(v, p, N, B, true, h->st, hs, h->red, s);                   // steps 5-6
    if (h->basis) gk_store_basis<T>(v, P<T>(h->basis), N, h->st, h->basis_ab, h->basis_n > 0, s);
    gk_update<T>(f, w, v, N, B, true, h->st, s);                                    // step 7
    bool pending = false;  // update (steps 19-20) of the previous iteration not yet applied
    for (int i = 1; i <= n_inner; ++i) {
        bool fused = false;
        if (pending) {
            if constexpr (std::is_same<T, float>::value)
                fused = !h->no_fuse_update && op_fwd_update(h->od, v, u, f, w, B, h->st, h->red, s);
            if (!fused) gk_update<T>(f, w, v, N, B, false, h->st, s);                        // 19-20
        }
        if (!fused) op_apply<T>(h->od, false, EPI_FWD, v, u, i == 1 ? g : u, tmp, B, h->st, h->red, s);  // 10
        op_apply<T>(h->od, true, EPI_ADJ, u, p, p, tmp, B, h->st, h->red, s);                // step 11
        if (!prec_apply<T>(h, p, v, B, s, 2))                                                // step 12
            gk_dot_rotate<T>(v, p, N, B, false, h->st, hs, h->red, s);                       // 13-17
        if (h->basis)
            gk_store_basis<T>(v, P<T>(h->basis) + (int64_t)std::min(i, h->basis_n - 1) * N, N, h->st,
                              h->basis_ab + 2 * i, i < h->basis_n, s);
        pending = true;
    }
    if (pending) gk_update<T>(f, w, v, N, B, false, h->st, s);                               // 19-20
}

// One outer step of Algorithm 3.
template <typename T>
void outer_step(plsqr_ctx* h, int B, int n_inner, cudaStream_t s) {
    Hist hs = hist_of(h);
    diffusivity<T>(P<T>(h->f), P<T>(h->kappa), h->d, B, h->st, hs, h->kfloor, h->red, s, K16(h));  // step 3
    prec_setup<T>(h, B, s);
    mlsqr_seq<T>(h, B, n_inner, s);  // step 4
    op_apply<T>(h->od, false, EPI_PLAIN, P<T>(h->f), P<T>(h->tmpm), nullptr, P<T>(h->tmp), B, h->st, h->red, s);
    resid_norm<T>(P<T>(h->g), P<T>(h->tmpm), h->m, B, h->st, hs, h->red, s);
}

void ensure_hist(plsqr_ctx* h, int n_outer, int n_inner) {
    if (n_outer <= h->h_outer && n_inner == h->h_inner && h->h_rbar) return;
    clear_graphs(h);
    dfree(h, h->h_rbar);
    dfree(h, h->h_R);
    dfree(h, h->h_resid);
    const int64_t B = h->B;
    h->h_outer = std::max(n_outer, 1);
    h->h_inner = std::max(n_inner, 1);
    h->h_rbar = (double*)dalloc(h, sizeof(double) * B * h->h_outer * h->h_inner);
    h->h_R = (double*)dalloc(h, sizeof(double) * B * (h->h_outer + 1));
    h->h_resid = (double*)dalloc(h, sizeof(double) * B * h->h_outer);
    size_t need = (size_t)B * h->h_outer * h->h_inner + (size_t)B * (h->h_outer + 1) + (size_t)B * h->h_outer;
    if (need > h->h_stage_n) {
        if (h->h_stage) cudaFreeHost(h->h_stage);
        h->h_stage = nullptr;
        ck(cudaMallocHost((void**)&h->h_stage, need * sizeof(double)), "cudaMallocHost");
        h->h_stage_n = need;
    }
}

// ---- tile-shape autotuner ----------------------------------------------------------------------
//
// Every tile shape gives the same V-cycle bit for bit, so the choice is free: for each 2D level
// above the coarsest the tuner captures a CUDA graph of 8 pre/post-smoothing pairs of that level
// with each shape (the handle's full batch, scratch buffers, a zeroed instance state), replays it,
// and keeps the fastest.  The kernels do the same work whatever the values they read.  Choices
// are cached per process by the level's size, the batch, the element size, nu and the kappa
// storage, so handles of the same layout tune once.

std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}
std::map<std::tuple<int, int, int, int, int, int, int>, int>& tune_cache() {
    static std::map<std::tuple<int, int, int, int, int, int, int>, int> c;
    return c;
}

bool coop_forced() {
    const char* e = std::getenv("PLSQR_MG_COOP");
    return e && (e[0] == '0' || e[0] == '1');
}

std::map<std::tuple<int, int, int, int, int, int>, std::array<int, 3>>& schedule_cache() {
    static std::map<std::tuple<int, int, int, int, int, int>, std::array<int, 3>> c;
    return c;
}

// Per-level launches or one cooperative launch for the whole V-cycle: a CUDA graph of 8 V-cycles
// of each, with the handle's batch and tile shapes, replayed and timed; the faster one is kept
// (cached per process by grid, batch, element size, levels and kappa storage).  Both give the same
// V-cycle bit for bit.  st0: a zeroed state for the timing (the handle's own is left alone).
template <typename T>
void choose_schedule(plsqr_ctx* h, GkState* st0, cudaEvent_t e0, cudaEvent_t e1, bool fresh) {
    const int B = h->B;
    cudaStream_t s = h->stream;
    const auto key = std::make_tuple(h->d.nx, h->d.ny, B, (int)h->esz, h->L, h->kbf16 ? 1 : 0);
    if (!fresh) {
        std::lock_guard<std::mutex> lk(tune_mutex());
        auto it = schedule_cache().find(key);
        if (it != schedule_cache().end()) {
            h->coop = it->second[0];
            h->coop_lc = it->second[1];
            h->coop_cap = it->second[2];
            return;
        }
    }
    int dev = 0, sms = 0;
    ck(cudaGetDevice(&dev), "cudaGetDevice");
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    // candidates: per-level launches, and the cooperative launch from each level with three caps
    std::vector<std::array<int, 3>> cand{{0, 0, 0}};
    for (int lc = 0; lc + 1 < h->L; ++lc)
        for (int cap : {sms, 2 * sms, 0}) cand.push_back({1, lc, cap});
    GkState* keep = h->st;
    h->st = st0;
    std::vector<float> ms(cand.size(), 0.f);
    try {
        ck(cudaMemsetAsync(h->p, 0, h->esz * B * h->d.N, s), "memset");
        for (size_t c = 0; c < cand.size(); ++c) {
            h->coop = cand[c][0];
            h->coop_lc = cand[c][1];
            h->coop_cap = cand[c][2];
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
            try {
                for (int r = 0; r < 8; ++r) vcycle_2d<T>(h, P<T>(h->p), P<T>(h->v), B, 0, s);
            } catch (...) {
                cudaStreamEndCapture(s, &graph);
                if (graph) cudaGraphDestroy(graph);
                throw;
            }
            ck(cudaStreamEndCapture(s, &graph), "cudaStreamEndCapture");
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            ck(ie, "cudaGraphInstantiate");
            cudaError_t e = cudaGraphLaunch(exec, s);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[c], e0, e1);
            cudaGraphExecDestroy(exec);
            ck(e, "autotune schedule");
        }
    } catch (...) {
        h->st = keep;
        h->coop = 0;
        throw;
    }
    h->st = keep;
    size_t best = 0;
    for (size_t c = 1; c < cand.size(); ++c)
        if (ms[c] < ms[best]) best = c;
    const char* lg = std::getenv("PLSQR_TUNE_LOG");
    if (lg && lg[0] == '1')
        for (size_t c = 0; c < cand.size(); ++c)
            std::fprintf(stderr, "plsqr schedule %dx%d batch %d: coop %d first level %d cap %d: %.2f us per V-cycle%s\n",
                         h->d.nx, h->d.ny, B, cand[c][0], cand[c][1], cand[c][2], 1e3f * ms[c] / 24.f,
                         c == best ? " (chosen)" : "");
    h->coop = cand[best][0];
    h->coop_lc = cand[best][1];
    h->coop_cap = cand[best][2];
    std::lock_guard<std::mutex> lk(tune_mutex());
    schedule_cache()[key] = cand[best];
}

// 3D levels: the planes per thread of the half sweeps (1, 2 or 4), timed like the 2D tile shapes
// (a CUDA graph of 8 red-black sweeps per candidate on the level's own hierarchy, writing only its
// V-cycle scratch) and cached per process by level extents, batch and element size.
std::map<std::tuple<int, int, int, int, int>, int>& tune3_cache() {
    static std::map<std::tuple<int, int, int, int, int>, int> m;
    return m;
}

template <typename T>
void autotune3(plsqr_ctx* h, bool fresh) {
    const int B = h->B;
    cudaStream_t s = h->stream;
    Profiler* prev = current_profiler();
    current_profiler() = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        current_profiler() = prev;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    try {
        ck(cudaStreamSynchronize(h->user_stream), "autotune");
        ck(cudaEventCreate(&e0), "cudaEventCreate");
        ck(cudaEventCreate(&e1), "cudaEventCreate");
        for (int l = 0; l + 1 < h->L; ++l) {
            const Level& Lv = h->lv[l];
            const bool isk = l == 0;
            const auto key = std::make_tuple(Lv.d.nx, Lv.d.ny, Lv.d.nz, B, (int)h->esz);
            if (!fresh) {
                std::lock_guard<std::mutex> lk(tune_mutex());
                auto it = tune3_cache().find(key);
                if (it != tune3_cache().end()) {
                    h->zc3[l] = it->second;
                    continue;
                }
            }
            const T* cond = isk ? P<T>(h->kappa) : P<T>(Lv.cond);
            T* b = isk ? P<T>(h->p) : P<T>(Lv.b);
            T* x = isk ? P<T>(h->tmp) : P<T>(Lv.x);
            const int64_t n = (int64_t)B * Lv.d.N;
            ck(cudaMemsetAsync(b, 0, sizeof(T) * n, s), "memset");
            ck(cudaMemsetAsync(x, 0, sizeof(T) * n, s), "memset");
            int best = 1;
            float best_ms = 0.f;
            const int cand[3] = {1, 2, 4};
            for (int q = 0; q < 3; ++q) {
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
                try {
                    for (int r = 0; r < 8; ++r) {
                        mg_gs_half<T>(cond, isk, b, x, Lv.d, 0, false, B, s, cand[q]);
                        mg_gs_half<T>(cond, isk, b, x, Lv.d, 1, false, B, s, cand[q]);
                    }
                } catch (...) {
                    cudaStreamEndCapture(s, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    throw;
                }
                ck(cudaStreamEndCapture(s, &graph), "cudaStreamEndCapture");
                const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                ck(ie, "cudaGraphInstantiate");
                float ms = 0.f;
                cudaError_t e = cudaGraphLaunch(exec, s);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                cudaGraphExecDestroy(exec);
                ck(e, "autotune");
                const char* lg = std::getenv("PLSQR_TUNE_LOG");
                if (lg && lg[0] == '1')
                    std::fprintf(stderr, "plsqr planes level %d (%dx%dx%d) batch %d: %d per thread: %.2f us per sweep\n",
                                 l, Lv.d.nx, Lv.d.ny, Lv.d.nz, B, cand[q], 1e3f * ms / 24.f);
                if (q == 0 || ms < best_ms) {
                    best = cand[q];
                    best_ms = ms;
                }
            }
            h->zc3[l] = best;
            std::lock_guard<std::mutex> lk(tune_mutex());
            tune3_cache()[key] = best;
        }
        ck(cudaStreamSynchronize(s), "autotune");
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

template <typename T>
void autotune(plsqr_ctx* h, bool fresh = false) {
    h->tuned = true;
    if (h->d.ndim == 3 && !h->generic_mg && !h->split3 && h->L > 1) {
        Range range("plsqr_autotune");
        autotune3<T>(h, fresh);
        return;
    }
    if (!use_fused_mg(h) || !tma_enabled()) return;
    Range range("plsqr_autotune");
    const int B = h->B;
    cudaStream_t s = h->stream;
    Profiler* prev = current_profiler();
    current_profiler() = nullptr;  // tuning launches are neither profiled nor counted
    GkState* st0 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        current_profiler() = prev;
        if (st0) cudaFree(st0);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    try {
        ck(cudaStreamSynchronize(h->user_stream), "autotune");
        ck(cudaMalloc(&st0, sizeof(GkState) * B), "cudaMalloc");
        ck(cudaMemsetAsync(st0, 0, sizeof(GkState) * B, s), "memset");
        ck(cudaEventCreate(&e0), "cudaEventCreate");
        ck(cudaEventCreate(&e1), "cudaEventCreate");
        for (int l = 0; l + 1 < h->L; ++l) {
            const Level& Lv = h->lv[l];
            const Level& C = h->lv[l + 1];
            const bool isk = l == 0;
            const auto key = std::make_tuple(Lv.d.nx, Lv.d.ny, B, (int)h->esz, h->nu, isk ? 1 : 0, h->kbf16 ? 1 : 0);
            if (!fresh) {
                std::lock_guard<std::mutex> lk(tune_mutex());
                auto it = tune_cache().find(key);
                if (it != tune_cache().end()) {
                    h->tile[l] = it->second;
                    continue;
                }
            }
            const T* cond = isk ? P<T>(h->kappa) : P<T>(Lv.cond);
            T* b = isk ? P<T>(h->p) : P<T>(Lv.b);
            T* xpre = isk ? P<T>(h->tmp) : P<T>(Lv.x);
            T* x = isk ? P<T>(h->v) : P<T>(Lv.x2);
            // the kernels read the hierarchy (kappa / conductances, 1/diagonal) as it is, so a tuning
            // between plsqr_prec_setup and plsqr_prec_apply leaves it intact; they write only V-cycle
            // scratch (the level's iterates and the coarse right-hand side), zeroed with its inputs
            const int64_t n = (int64_t)B * Lv.d.N, nc = (int64_t)B * C.d.N;
            ck(cudaMemsetAsync(b, 0, sizeof(T) * n, s), "memset");
            ck(cudaMemsetAsync(C.x2, 0, sizeof(T) * nc, s), "memset");
            int best = 0;
            float best_ms = 0.f;
            for (int id = 0;; ++id) {
                int tx, ty, nth;
                if (!mg2d_shape(isk, id, &tx, &ty, &nth)) break;
                // finest-level tiles narrower than 32 x 16 cannot carry the fused alpha (it would
                // fall back to the default shape): candidates only when alpha is a separate kernel
                if (isk && (tx % 32 != 0 || ty % 16 != 0) && h->cycles == 1) continue;
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
                try {
                    for (int r = 0; r < 8; ++r) {
                        mg2d_pre<T>(cond, isk, b, P<T>(Lv.rd), xpre, P<T>(C.b), Lv.d, C.d, h->nu, B, st0, s,
                                    isk ? K16(h) : nullptr, id);
                        mg2d_post<T>(cond, isk, b, P<T>(Lv.rd), xpre, x, P<T>(C.x2), Lv.d, C.d, h->nu, B, 0, st0,
                                     hist_of(h), h->red, s, isk ? K16(h) : nullptr, id);
                    }
                } catch (...) {
                    cudaStreamEndCapture(s, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    throw;
                }
                ck(cudaStreamEndCapture(s, &graph), "cudaStreamEndCapture");
                const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                ck(ie, "cudaGraphInstantiate");
                float ms = 0.f;
                cudaError_t e = cudaGraphLaunch(exec, s);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                cudaGraphExecDestroy(exec);
                ck(e, "autotune");
                const char* lg = std::getenv("PLSQR_TUNE_LOG");
                if (lg && lg[0] == '1')
                    std::fprintf(stderr, "plsqr tiles level %d (%dx%d) batch %d: shape %d (%dx%d/%d): %.2f us per pre+post\n",
                                 l, Lv.d.nx, Lv.d.ny, B, id, tx, ty, nth, 1e3f * ms / 24.f);
                if (id == 0 || ms < best_ms) {
                    best = id;
                    best_ms = ms;
                }
            }
            h->tile[l] = best;
            std::lock_guard<std::mutex> lk(tune_mutex());
            tune_cache()[key] = best;
        }
        if (h->coop_ok && h->coop < 0) choose_schedule<T>(h, st0, e0, e1, fresh);
        ck(cudaStreamSynchronize(s), "autotune");
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

bool autotune_enabled() {
    const char* e = std::getenv("PLSQR_AUTOTUNE");
    return !(e && e[0] == '0');
}

template <typename T>
void maybe_autotune(plsqr_ctx* h) {
    if (!h->tuned && autotune_enabled()) autotune<T>(h);
}

template <typename T>
void run_outer_steps(plsqr_ctx* h, int B, int n_outer, int n_inner) {
    maybe_autotune<T>(h);
    cudaStream_t s = h->stream;
    if (!h->use_graph || h->prof.enabled) {
        for (int k = 0; k < n_outer; ++k) {
            Range r("outer step", k + 1);
            outer_step<T>(h, B, n_inner, s);
        }
        return;
    }
    auto key = std::make_tuple(B, n_inner, h->h_outer, h->h_inner);
    auto it = h->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    int64_t per_replay = 0;
    if (it == h->graphs.end()) {
        Range r("capture outer step");
        const int64_t before = h->prof.launches;
        cudaGraph_t graph = nullptr;
        ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
        try {
            outer_step<T>(h, B, n_inner, s);
        } catch (...) {
            cudaStreamEndCapture(s, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        ck(cudaStreamEndCapture(s, &graph), "cudaStreamEndCapture");
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        ck(e, "cudaGraphInstantiate");
        per_replay = h->prof.launches - before;  // captured, not yet executed
        h->prof.launches = before;
        h->graphs[key] = std::make_pair(exec, per_replay);
    } else {
        exec = it->second.first;
        per_replay = it->second.second;
    }
    for (int k = 0; k < n_outer; ++k) {
        Range r("outer step", k + 1);
        ck(cudaGraphLaunch(exec, s), "cudaGraphLaunch");
    }
    h->prof.launches += per_replay * n_outer;
}

void validate_solve(plsqr_ctx* h, int count, const int32_t* reg, const double* T, const double* tau, int n_outer,
                    int n_inner) {
    if (!h->op_set) throw std::logic_error("set_operator must be called before a solve");
    if (count < 1 || count > h->B) throw InvalidArg("count must be in 1..max_batch");
    if (n_outer < 1 || n_outer > 100000 || n_inner < 1 || n_inner > 100000) throw InvalidArg("bad iteration counts");
    for (int b = 0; b < count; ++b) {
        if (reg[b] < 0 || reg[b] > 3) throw InvalidArg("bad regulariser");
        if (!(T[b] > 0.0) || !std::isfinite(T[b])) throw InvalidArg("T must be positive and finite");
        if (!(tau[b] >= 0.0) || !std::isfinite(tau[b])) throw InvalidArg("tau must be >= 0 and finite");
    }
}

template <typename T>
int solve_impl(plsqr_ctx* h, int count, const void* const* g, bool g_host, const int32_t* reg, const double* Tp,
               const double* tau, int n_outer, int n_inner, void* const* f_out, bool f_host, plsqr_stats* stats) {
    Range range("plsqr_solve");
    validate_solve(h, count, reg, Tp, tau, n_outer, n_inner);
    ensure_hist(h, n_outer, n_inner);
    cudaStream_t s = h->stream;
    const int64_t launches0 = h->prof.launches;
    ck(cudaEventRecord(h->ev_in, h->user_stream), "cudaEventRecord");
    ck(cudaStreamWaitEvent(s, h->ev_in, 0), "cudaStreamWaitEvent");
    const size_t mb = h->esz * h->m, nb = h->esz * h->d.N;
    for (int b = 0; b < count; ++b) {
        if (!g[b]) throw InvalidArg("g is NULL");
        ck(cudaMemcpyAsync(h->g + b * mb, g[b], mb, g_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s),
           "copy g");
    }
    for (int b = 0; b < count; ++b) {
        h->prm_host[b].reg = reg[b];
        h->prm_host[b].T = Tp[b];
        h->prm_host[b].tau = tau[b];
    }
    ck(cudaMemcpyAsync(h->prm_dev, h->prm_host, sizeof(SolveParams) * count, cudaMemcpyHostToDevice, s), "params");
    set_params(h->st, h->prm_dev, count, true, s);
    ck(cudaMemsetAsync(h->f, 0, nb * count, s), "f0");  // f^0 = 0
    const int64_t hb = (int64_t)h->B;
    fill_nan(h->h_rbar, hb * h->h_outer * h->h_inner, s);
    fill_nan(h->h_R, hb * (h->h_outer + 1), s);
    fill_nan(h->h_resid, hb * h->h_outer, s);
    run_outer_steps<T>(h, count, n_outer, n_inner);
    // R(f^n_outer) (the outer counter now equals n_outer)
    diffusivity<T>(P<T>(h->f), P<T>(h->kappa), h->d, count, h->st, hist_of(h), h->kfloor, h->red, s, K16(h));
    for (int b = 0; b < count; ++b) {
        if (!f_out[b]) throw InvalidArg("f_out is NULL");
        ck(cudaMemcpyAsync(f_out[b], h->f + b * nb, nb, f_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s),
           "copy f");
    }
    ck(cudaMemcpyAsync(h->st_host, h->st, sizeof(GkState) * count, cudaMemcpyDeviceToHost, s), "state");
    h->last_launches = h->prof.launches - launches0;
    ck(cudaEventRecord(h->ev_out, s), "cudaEventRecord");
    ck(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0), "cudaStreamWaitEvent");
    int ret = PLSQR_OK;
    if (stats || f_host) {
        const int64_t nr = hb * h->h_outer * h->h_inner, nR = hb * (h->h_outer + 1), ne = hb * h->h_outer;
        if (stats) {
            ck(cudaMemcpyAsync(h->h_stage, h->h_rbar, sizeof(double) * nr, cudaMemcpyDeviceToHost, s), "hist");
            ck(cudaMemcpyAsync(h->h_stage + nr, h->h_R, sizeof(double) * nR, cudaMemcpyDeviceToHost, s), "hist");
            ck(cudaMemcpyAsync(h->h_stage + nr + nR, h->h_resid, sizeof(double) * ne, cudaMemcpyDeviceToHost, s),
               "hist");
        }
        ck(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        for (int b = 0; b < count; ++b) {
            int sb = h->st_host[b].status_any;
            if (sb != 0 && ret == PLSQR_OK) ret = sb == PLSQR_E_TIMEOUT ? PLSQR_E_TIMEOUT : PLSQR_E_BREAKDOWN;
            if (!stats) continue;
            plsqr_stats& S = stats[b];
            S.status = sb;
            if (S.rbar_hist)
                for (int k = 0; k < n_outer; ++k)
                    std::memcpy(S.rbar_hist + (int64_t)k * n_inner,
                                h->h_stage + ((int64_t)b * h->h_outer + k) * h->h_inner, sizeof(double) * n_inner);
            if (S.R_hist)
                std::memcpy(S.R_hist, h->h_stage + nr + (int64_t)b * (h->h_outer + 1), sizeof(double) * (n_outer + 1));
            if (S.resid_hist)
                std::memcpy(S.resid_hist, h->h_stage + nr + nR + (int64_t)b * h->h_outer, sizeof(double) * n_outer);
        }
    }
    return ret;
}

int fail(plsqr_ctx* h, int code, const char* msg) {
    if (h) h->err = msg;
    return code;
}

template <typename F>
int guarded(plsqr_ctx* h, F&& fn) {
    ProfScope scope(h);
    try {
        return fn();
    } catch (const InvalidArg& e) {
        return fail(h, PLSQR_E_INVALID, e.what());
    } catch (const NoMem& e) {
        return fail(h, PLSQR_E_NOMEM, e.what());
    } catch (const CudaError& e) {
        return fail(h, PLSQR_E_CUDA, e.what());
    } catch (const std::logic_error& e) {
        return fail(h, PLSQR_E_STATE, e.what());
    } catch (const std::exception& e) {
        return fail(h, PLSQR_E_CUDA, e.what());
    }
}

void destroy_ctx(plsqr_ctx* h) {
    if (!h) return;
    clear_graphs(h);
    h->prof.release();
    for (const Alloc& a : h->allocs) cudaFree(a.base);
    h->allocs.clear();
    if (h->prm_host) cudaFreeHost(h->prm_host);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    if (h->taps_inst_host) cudaFreeHost(h->taps_inst_host);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

template <typename T>
void upload_taps(plsqr_ctx* h, OpDev& od, int dd, double sigma, int R) {
    std::vector<double> w(2 * R + 1);
    double s = 0.0;
    for (int k = -R; k <= R; ++k) s += (w[k + R] = std::exp(-(double)(k * k) / (2.0 * sigma * sigma)));
    std::vector<T> wt(2 * R + 1);
    for (int k = 0; k <= 2 * R; ++k) {
        wt[k] = (T)(w[k] / s);
        od.taps_host[dd][k] = w[k] / s;
    }
    dfree(h, h->taps[dd]);
    h->taps[dd] = dalloc(h, sizeof(T) * wt.size());
    ck(cudaMemcpy(h->taps[dd], wt.data(), sizeof(T) * wt.size(), cudaMemcpyHostToDevice), "taps");
}

template <typename T>
void upload_joseph(plsqr_ctx* h, int na, double ds) {
    std::vector<JosephAngle<T>> tab(na);
    for (int a = 0; a < na; ++a) {
        const double th = kPi * (double)a / (double)na;
        const double ct = std::cos(th), st = std::sin(th);
        const bool rows = (4 * a < na) || (4 * a > 3 * na);
        const double hh = rows ? std::fabs(ct) : std::fabs(st);
        JosephAngle<T>& J = tab[a];
        J.a1 = (T)(rows ? 1.0 / ct : 1.0 / st);
        J.a2 = (T)(rows ? st / ct : ct / st);
        J.c1 = (T)(ct / ds);
        J.c2 = (T)(st / ds);
        J.hw = (T)(hh / ds);
        J.inv_hw = (T)(ds / hh);
        J.wgt = (T)(1.0 / hh);
        J.rows = rows ? 1 : 0;
    }
    dfree(h, h->jtab);
    h->jtab = dalloc(h, sizeof(JosephAngle<T>) * na);
    ck(cudaMemcpy(h->jtab, tab.data(), sizeof(JosephAngle<T>) * na, cudaMemcpyHostToDevice), "joseph table");
}

// Dispatch on the bulk type.
template <typename F>
void by_type(plsqr_ctx* h, F&& fn) {
    if (h->fp64) fn(double{});
    else fn(float{});
}

}  // namespace

// ---- separable blur without any device allocation ------------------------------------------
// Scratch of plsqr_blur_noalloc: the blur taps (first 2 KiB) and the intermediate volume of the
// 3D blur.  A file-scope array, so every GPU that loads this library holds it until exit; its
// device address is looked up once per device (the host-side name is only a stand-in).
constexpr size_t kNoallocTapsBytes = 2048;
constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;
constexpr int kNoallocMaxRadius = 32;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// The taps of plsqr_blur_noalloc travel as a kernel parameter (by value), so the call holds no
// pointer to host memory.  w[d][0 .. len[d]) are written at dst + off[d] as double (esz 8) or float.
struct NoallocTaps {
    double w[3][2 * kNoallocMaxRadius + 1];
    int32_t off[3], len[3];
    int32_t ndim, esz;
};

__global__ void k_noalloc_taps(const NoallocTaps t, unsigned char* dst) {
    for (int d = 0; d < t.ndim; ++d)
        for (int k = threadIdx.x; k < t.len[d]; k += blockDim.x) {
            if (t.esz == 8) reinterpret_cast<double*>(dst + t.off[d])[k] = t.w[d][k];
            else reinterpret_cast<float*>(dst + t.off[d])[k] = (float)t.w[d][k];
        }
}

namespace {

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[256] = {};

// Device address of the scratch on the current device (first call per device looks it up).
void* noalloc_scratch(int* err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        *err = PLSQR_E_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            *err = PLSQR_E_CUDA;
            return nullptr;
        }
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" {

int plsqr_create(const plsqr_config* cfg, void* stream, plsqr_handle* out) {
    if (!out) return PLSQR_E_INVALID;
    *out = nullptr;
    plsqr_ctx* h = new plsqr_ctx();
    int rc = guarded(h, [&]() -> int {
        Plan pl = make_plan(cfg, 0);
        h->cfg = *cfg;
        h->user_stream = (cudaStream_t)stream;
        h->fp64 = cfg->precision == PLSQR_FP64;
        h->esz = h->fp64 ? 8 : 4;
        h->d = pl.d;
        h->B = cfg->max_batch;
        h->L = pl.L;
        h->nu = cfg->mg_sweeps;
        h->cycles = cfg->mg_cycles;
        h->kfloor = cfg->kappa_floor;
        h->nc = pl.nc;
        h->bw = pl.bw;
        h->m = h->d.N;
        const char* eg = std::getenv("PLSQR_GRAPH");
        h->use_graph = !(eg && eg[0] == '0');
        const char* em = std::getenv("PLSQR_GENERIC_MG");
        h->generic_mg = em && em[0] == '1';
        const char* eu = std::getenv("PLSQR_FUSE_UPDATE");
        h->no_fuse_update = eu && eu[0] == '0';
        const char* egd = std::getenv("PLSQR_GUARD");
        h->guard = egd && egd[0] == '1';
        ck(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        ck(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming), "cudaEventCreate");
        const int64_t B = h->B, N = h->d.N;
        const size_t e = h->esz;
        h->f = dalloc(h, e * B * N);
        h->p = dalloc(h, e * B * N);
        h->v = dalloc(h, e * B * N);
        h->w = dalloc(h, e * B * N);
        h->kappa = dalloc(h, e * B * N);
        h->tmp = dalloc(h, e * B * N);
        if (h->cycles > 1) {
            h->r0 = dalloc(h, e * B * N);
            h->e0 = dalloc(h, e * B * N);
        }
        alloc_data_buffers(h);
        h->lv[0].d = h->d;
        for (int l = 1; l < h->L; ++l) {
            const Dims& pd = h->lv[l - 1].d;
            h->lv[l].d = make_dims(h->d.ndim, pd.nx / 2, pd.ny / 2, pd.nz / 2);
            const int64_t Nl = h->lv[l].d.N;
            h->lv[l].cond = dalloc(h, e * B * Nl * h->d.ndim);
            h->lv[l].b = dalloc(h, e * B * Nl);
            h->lv[l].x = dalloc(h, e * B * Nl);
            h->lv[l].x2 = dalloc(h, e * B * Nl);
        }
        if (h->d.ndim == 2)
            for (int l = 0; l + 1 < h->L; ++l) h->lv[l].rd = dalloc(h, e * B * h->lv[l].d.N);
        h->split3 = pl.split3;
        if (h->split3) {
            h->xs0 = dalloc(h, e * B * N);
            h->bs0 = dalloc(h, e * B * N);
        }
        h->coop_sync = (unsigned*)dalloc(h, 4 * sizeof(unsigned));
        {
            const char* ec = std::getenv("PLSQR_MG_COOP");
            // every level must be a TMA layout (rows of 16-byte multiples; the coarsest is staged
            // as the coarse-correction box of the level above it)
            bool rows16 = true;
            for (int l = 0; l < h->L; ++l) rows16 = rows16 && ((size_t)h->lv[l].d.nx * e) % 16 == 0;
            h->coop_ok = !h->generic_mg && h->d.ndim == 2 && h->L >= 2 && rows16 && tma_enabled() &&
                         mg2d_coop_supported(h->nu, h->esz, h->L, h->nc) && !(ec && ec[0] == '0');
            if (!h->coop_ok) h->coop = 0;
            else if (ec && ec[0] == '1') {
                h->coop = 1;
                const char* el = std::getenv("PLSQR_MG_COOP_LEVEL");
                h->coop_lc = el ? std::max(0, std::min(h->L - 2, std::atoi(el))) : 0;
            }
        }
        {
            Dims dl[16];
            for (int l = 0; l < h->L; ++l) dl[l] = h->lv[l].d;
            h->tail_lc = h->generic_mg ? h->L : mg2d_tail_level(dl, h->L, h->nu, h->esz, h->nc);
            h->tail.n = h->tail_lc < h->L ? h->L - h->tail_lc : 0;
            if (h->tail_lc < h->L) {  // the opt-in cluster tail and the cooperative V-cycle exclude each other
                h->coop_ok = false;
                h->coop = 0;
            }
            for (int q = 0; q < h->tail.n; ++q) {
                const Level& Lv = h->lv[h->tail_lc + q];
                h->tail.cond[q] = Lv.cond;
                h->tail.rd[q] = Lv.rd;
                h->tail.b[q] = Lv.b;
                h->tail.x[q] = Lv.x;
                h->tail.x2[q] = Lv.x2;
                h->tail.d[q] = Lv.d;
            }
        }
        h->gth = pl.gth;
        h->gthw = pl.gthw;
        if (h->gth || h->gthw) {  // tables in the handle's type (the wide route: float only)
            const size_t vsz = h->gth ? h->esz : sizeof(float);
            h->gcol = dalloc(h, vsz * B * (size_t)h->nc * gth_stride(h->bw));
            if (xblk_enabled(B)) h->xblk = dalloc(h, vsz * B * (size_t)xblk_scratch(h->nc, h->bw));
            h->grow = dalloc(h, vsz * B * (size_t)h->nc * gth_stride(h->bw));
            if (h->fp64) h->X = (double*)dalloc(h, sizeof(double) * B * (size_t)h->nc * h->nc);
        } else {
            h->band = (double*)dalloc(h, sizeof(double) * B * (size_t)h->nc * (h->bw + 1));
            h->rdiag = (double*)dalloc(h, sizeof(double) * B * (size_t)h->nc);
            h->X = (double*)dalloc(h, sizeof(double) * B * (size_t)h->nc * h->nc);
        }
        if (!h->fp64) h->Xf = (float*)dalloc(h, sizeof(float) * B * (size_t)h->nc * h->nc);
        h->st = (GkState*)dalloc(h, sizeof(GkState) * B);
        ck(cudaMemset(h->st, 0, sizeof(GkState) * B), "memset");
        h->prm_dev = (SolveParams*)dalloc(h, sizeof(SolveParams) * B);
        ck(cudaMallocHost((void**)&h->prm_host, sizeof(SolveParams) * B), "cudaMallocHost");
        std::memset(h->prm_host, 0, sizeof(SolveParams) * B);  // stopping rules off
        ck(cudaMallocHost((void**)&h->st_host, sizeof(GkState) * B), "cudaMallocHost");
        // per-block partials, and the 32 x 16 segments of the 2D V-cycle's alpha
        h->red.max_blocks =
            (int32_t)std::max<int64_t>(8192, (int64_t)((h->d.ny + 15) / 16) * ((h->d.nx + 31) / 32));
        h->red.partials = (double*)dalloc(h, sizeof(double) * B * h->red.max_blocks);
        h->red.counters = (unsigned*)dalloc(h, sizeof(unsigned) * B);
        ck(cudaMemset(h->red.counters, 0, sizeof(unsigned) * B), "memset");
        ck(cudaDeviceSynchronize(), "create");
        return PLSQR_OK;
    });
    if (rc != PLSQR_OK) {
        std::fprintf(stderr, "plsqr_create: %s\n", h->err.c_str());
        destroy_ctx(h);
        return rc;
    }
    *out = h;
    return PLSQR_OK;
}

int plsqr_set_operator(plsqr_handle h, const plsqr_operator* op) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (!op) throw InvalidArg("operator is NULL");
        if (h->serving) throw std::logic_error("set_operator on a handle in slot mode");
        const Dims& d = h->d;
        OpDev od{};
        od.d = d;
        od.kind = op->kind;
        const char* eg = std::getenv("PLSQR_GENERIC_BLUR");
        od.generic_blur = (eg && eg[0] == '1') ? 1 : 0;
        if (op->kind == PLSQR_OP_BLUR || op->kind == PLSQR_OP_BLUR_MASK) {
            for (int dd = 0; dd < d.ndim; ++dd) {
                if (!(op->sigma[dd] > 0.0) || op->radius[dd] < 0 || op->radius[dd] > 32)
                    throw InvalidArg("blur needs sigma > 0 and 0 <= radius <= 32 on every axis");
            }
            if (op->kind == PLSQR_OP_BLUR_MASK && !op->mask) throw InvalidArg("masked blur needs a mask");
        } else if (op->kind == PLSQR_OP_JOSEPH) {
            if (d.ndim != 2 || d.nx != d.ny) throw InvalidArg("Joseph projector needs a square 2D image");
            if (op->n_angles < 1 || op->n_angles > 100000 || op->n_bins < 1 || op->n_bins > (1 << 20))
                throw InvalidArg("bad Joseph geometry");
            if (!(op->bin_spacing > 0.0)) throw InvalidArg("bin_spacing must be > 0");
        } else if (op->kind != PLSQR_OP_IDENTITY) {
            throw InvalidArg("unknown operator kind");
        }
        clear_graphs(h);
        const int64_t m_new = op_data_len(op, d);
        if (m_new != h->m || !h->g) {
            h->m = m_new;
            alloc_data_buffers(h);
        }
        od.m = h->m;
        if (op->kind == PLSQR_OP_BLUR || op->kind == PLSQR_OP_BLUR_MASK) {
            by_type(h, [&](auto tv) {
                using T = decltype(tv);
                for (int dd = 0; dd < d.ndim; ++dd) upload_taps<T>(h, od, dd, op->sigma[dd], op->radius[dd]);
            });
            for (int dd = 0; dd < d.ndim; ++dd) {
                od.taps[dd] = h->taps[dd];
                od.R[dd] = op->radius[dd];
            }
            if (op->kind == PLSQR_OP_BLUR_MASK) {
                if (!h->mask) h->mask = (uint8_t*)dalloc(h, (size_t)d.N);
                ck(cudaMemcpy(h->mask, op->mask, (size_t)d.N, cudaMemcpyDefault), "mask");
                od.mask = h->mask;
            }
        } else if (op->kind == PLSQR_OP_JOSEPH) {
            by_type(h, [&](auto tv) {
                using T = decltype(tv);
                upload_joseph<T>(h, op->n_angles, op->bin_spacing);
            });
            od.jtab = h->jtab;
            od.na = op->n_angles;
            od.nb = op->n_bins;
            od.ds = op->bin_spacing;
            // the forward's two-part launches: instances with n_angles x B below 3 x 152
            dfree(h, h->jpart);
            dfree(h, h->jcnt);
            h->jpart = h->jcnt = nullptr;
            h->jcap = joseph_parts_cap(h->B, op->n_angles);
            if (h->jcap > 0) {
                h->jpart = dalloc(h, h->esz * 2 * h->jcap * (size_t)op->n_angles * op->n_bins);
                h->jcnt = dalloc(h, sizeof(unsigned) * h->jcap * (size_t)op->n_angles);
            }
            od.jpart = h->jpart;
            od.jcnt = static_cast<unsigned*>(h->jcnt);
            od.jcap = h->jcap;
        }
        h->od = od;
        h->op = *op;
        h->op_set = true;
        return PLSQR_OK;
    });
}

int plsqr_solve(plsqr_handle h, const void* g, int32_t reg, double T, double tau, int32_t n_outer, int32_t n_inner,
                void* f_out, plsqr_stats* stats) {
    if (!h) return PLSQR_E_INVALID;
    if (h->serving) return fail(h, PLSQR_E_STATE, "the handle is in slot mode");
    return guarded(h, [&]() -> int {
        int rc = 0;
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            rc = solve_impl<TT>(h, 1, &g, false, &reg, &T, &tau, n_outer, n_inner, &f_out, false, stats);
        });
        return rc;
    });
}

int plsqr_solve_host(plsqr_handle h, const void* g_host, int32_t reg, double T, double tau, int32_t n_outer,
                     int32_t n_inner, void* f_host_out, plsqr_stats* stats) {
    if (!h) return PLSQR_E_INVALID;
    if (h->serving) return fail(h, PLSQR_E_STATE, "the handle is in slot mode");
    return guarded(h, [&]() -> int {
        int rc = 0;
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            rc = solve_impl<TT>(h, 1, &g_host, true, &reg, &T, &tau, n_outer, n_inner, &f_host_out, true, stats);
        });
        return rc;
    });
}

int plsqr_solve_batch(plsqr_handle h, int32_t count, const void* const* g, const int32_t* reg, const double* T,
                      const double* tau, int32_t n_outer, int32_t n_inner, void* const* f_out, plsqr_stats* stats) {
    if (!h) return PLSQR_E_INVALID;
    if (h->serving) return fail(h, PLSQR_E_STATE, "the handle is in slot mode");
    return guarded(h, [&]() -> int {
        if (!g || !reg || !T || !tau || !f_out) throw InvalidArg("NULL array argument");
        int rc = 0;
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            rc = solve_impl<TT>(h, count, g, false, reg, T, tau, n_outer, n_inner, f_out, false, stats);
        });
        return rc;
    });
}

// ---- bfloat16 kappa -----------------------------------------------------------------------------

int plsqr_set_kappa_bf16(plsqr_handle h, int32_t on) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        // several V-cycles per application form b - M x with the float kappa, which bfloat16
        // storage does not keep
        if (on && (h->fp64 || h->d.ndim != 2 || !use_fused_mg(h) || h->cycles != 1))
            throw InvalidArg("bfloat16 kappa needs a 2D single-precision handle with the temporally blocked V-cycle "
                             "and one V-cycle per application");
        if (on && !h->kappa16) h->kappa16 = (__nv_bfloat16*)dalloc(h, sizeof(__nv_bfloat16) * h->B * h->d.N);
        if ((on != 0) != h->kbf16) {
            clear_graphs(h);
            if (!h->tiles_set) h->tuned = false;  // the finest level's timing depends on the kappa storage
            if (h->coop_ok && !coop_forced()) h->coop = -1;
        }
        h->kbf16 = on != 0;
        return PLSQR_OK;
    });
}

// ---- tile shapes of the 2D V-cycle --------------------------------------------------------------

int plsqr_autotune(plsqr_handle h, int32_t fresh) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (h->serving) throw std::logic_error("tile shapes cannot change while slots are in use");
        if (h->coop_ok && !coop_forced()) h->coop = -1;  // timed again
        by_type(h, [&](auto tv) {
            using T = decltype(tv);
            autotune<T>(h, fresh != 0);
        });
        h->tiles_set = false;
        clear_graphs(h);  // captured with the previous shapes
        return PLSQR_OK;
    });
}

// The process-wide choices of the autotuner as text, one entry per line:
// "nx ny batch element_size sweeps finest kappa_bf16 shape".
int64_t plsqr_tune_cache_export(char* buf, int64_t cap) {
    std::string text;
    {
        std::lock_guard<std::mutex> lk(tune_mutex());
        for (const auto& kv : tune_cache()) {
            const auto& k = kv.first;
            char line[160];
            std::snprintf(line, sizeof line, "%d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k),
                          std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), kv.second);
            text += line;
        }
    }
    if (buf && cap > 0) {
        const size_t n = std::min<size_t>(text.size(), (size_t)cap - 1);
        std::memcpy(buf, text.data(), n);
        buf[n] = '\0';
    }
    return (int64_t)text.size();
}

int32_t plsqr_tune_cache_import(const char* text) {
    if (!text) return -PLSQR_E_INVALID;
    std::vector<std::pair<std::tuple<int, int, int, int, int, int, int>, int>> entries;
    const char* p = text;
    while (*p) {
        const char* e = std::strchr(p, '\n');
        const std::string line(p, e ? (size_t)(e - p) : std::strlen(p));
        p = e ? e + 1 : p + line.size();
        if (line.find_first_not_of(" \t\r") == std::string::npos) continue;  // blank line
        int v[8];
        char extra = 0;
        if (std::sscanf(line.c_str(), "%d %d %d %d %d %d %d %d %c", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                        &v[7], &extra) != 8)
            return -PLSQR_E_INVALID;
        int tx, ty, nth;
        const bool sizes_ok = v[0] > 0 && v[1] > 0 && v[2] >= 1 && v[2] <= 4096 && (v[3] == 4 || v[3] == 8) &&
                              v[4] >= 1 && v[4] <= 3 && (v[5] == 0 || v[5] == 1) && (v[6] == 0 || v[6] == 1);
        if (!sizes_ok || v[7] < 0 || !mg2d_shape(v[5] == 1, v[7], &tx, &ty, &nth)) return -PLSQR_E_INVALID;
        entries.emplace_back(std::make_tuple(v[0], v[1], v[2], v[3], v[4], v[5], v[6]), v[7]);
    }
    std::lock_guard<std::mutex> lk(tune_mutex());
    for (const auto& kv : entries) tune_cache()[kv.first] = kv.second;
    return (int32_t)entries.size();
}

int plsqr_set_tile_shape(plsqr_handle h, int32_t level, int32_t shape) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (h->serving) throw std::logic_error("tile shapes cannot change while slots are in use");
        if (level < 0 || level >= h->L - 1) throw InvalidArg("level must be in 0..mg_levels-2");
        if (h->d.ndim == 3) {  // planes per thread of the 3D half sweeps
            if (shape != 1 && shape != 2 && shape != 4) throw InvalidArg("3D levels take 1, 2 or 4 planes per thread");
            h->zc3[level] = shape;
            h->tuned = true;
            h->tiles_set = true;
            clear_graphs(h);
            return PLSQR_OK;
        }
        int tx, ty, nth;
        if (shape < 0 || !mg2d_shape(level == 0, shape, &tx, &ty, &nth)) throw InvalidArg("no such tile shape");
        h->tile[level] = shape;
        h->tuned = true;
        h->tiles_set = true;
        clear_graphs(h);
        return PLSQR_OK;
    });
}

int plsqr_tile_shape(plsqr_handle h, int32_t level, int32_t* shape, int32_t* tx, int32_t* ty, int32_t* threads) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (level < 0 || level >= 16) throw InvalidArg("bad level");
        const bool fused = use_fused_mg(h) && level < h->L - 1;
        const bool planes = h->d.ndim == 3 && !h->generic_mg && !h->split3 && level < h->L - 1;
        int id = fused ? h->tile[level] : -1;
        int v[3] = {0, 0, 0};
        if (fused) mg2d_shape(level == 0, id, &v[0], &v[1], &v[2]);
        if (planes) {  // 3D: "shape" = planes per thread of the half sweeps (256 threads, one cell row each)
            id = h->zc3[level];
            v[0] = 1;
            v[1] = h->zc3[level];
            v[2] = 256;
        }
        if (shape) *shape = id;
        if (tx) *tx = v[0];
        if (ty) *ty = v[1];
        if (threads) *threads = v[2];
        return PLSQR_OK;
    });
}

int plsqr_mg_schedule(plsqr_handle h, int32_t* coop, int32_t* first_level, int32_t* max_blocks) {
    if (!h || !coop) return PLSQR_E_INVALID;
    *coop = h->coop_ok ? h->coop : 0;
    if (first_level) *first_level = *coop == 1 ? h->coop_lc : -1;
    if (max_blocks) *max_blocks = *coop == 1 ? h->coop_cap : 0;
    return PLSQR_OK;
}

// ---- stopping rules ----------------------------------------------------------------------------

int plsqr_set_stopping(plsqr_handle h, int32_t index, double eta, double delta, double r_rel) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (index < -1 || index >= h->B) throw InvalidArg("index must be -1 (all) or an instance in 0..max_batch-1");
        if (!(eta >= 0.0) || !std::isfinite(eta) || !(delta >= 0.0) || !std::isfinite(delta))
            throw InvalidArg("eta and delta must be finite and >= 0");
        if (!(r_rel >= 0.0) || !(r_rel < 1.0)) throw InvalidArg("r_rel must be in [0, 1)");
        for (int b = (index < 0 ? 0 : index); b < (index < 0 ? h->B : index + 1); ++b) {
            h->prm_host[b].eta_delta = eta * delta;
            h->prm_host[b].r_rel = r_rel;
        }
        return PLSQR_OK;
    });
}

// ---- slots: continuous batching -----------------------------------------------------------

namespace {

// Taps of one slot on the handle's radius R: exp(-k^2 / (2 sigma^2)) for |k| <= ceil(3 sigma),
// zero beyond, normalised to unit sum over the nonzero part.
void slot_taps(float* dst, double sigma, int R) {
    const int r = (int)std::ceil(3.0 * sigma);
    if (!(sigma > 0.0) || !std::isfinite(sigma) || r > R) throw InvalidArg("slot sigma: ceil(3 sigma) must be <= the handle's radius");
    double sum = 0.0;
    for (int k = -r; k <= r; ++k) sum += std::exp(-(double)(k * k) / (2.0 * sigma * sigma));
    for (int k = -R; k <= R; ++k)
        dst[k + R] = std::abs(k) <= r ? (float)(std::exp(-(double)(k * k) / (2.0 * sigma * sigma)) / sum) : 0.0f;
}

void enter_slot_mode(plsqr_ctx* h) {
    if (h->serving) return;
    h->serving = true;
    h->slot_active.assign(h->B, 0);
    h->slot_outer.assign(h->B, 0);
    h->slot_target.assign(h->B, 0);
    slots_state(h->st, h->prm_dev, h->B, -1, true, h->stream);  // every slot empty
}

}  // namespace

int plsqr_slot_start(plsqr_handle h, int32_t slot, const void* g, int32_t reg, double T, double tau, int32_t n_outer,
                     int32_t n_inner, const double* sigma) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (!h->op_set) throw std::logic_error("set_operator must be called before plsqr_slot_start");
        if (slot < 0 || slot >= h->B) throw InvalidArg("slot out of range");
        if (!g) throw InvalidArg("g is NULL");
        validate_solve(h, 1, &reg, &T, &tau, n_outer, n_inner);
        enter_slot_mode(h);
        if (h->slot_active[slot]) throw std::logic_error("slot is busy");
        bool any = false;
        for (int b = 0; b < h->B; ++b) any = any || h->slot_active[b];
        if (!any) ensure_hist(h, n_outer, n_inner);
        else if (n_inner != h->h_inner || n_outer > h->h_outer)
            throw InvalidArg("n_inner must equal, and n_outer not exceed, those of the running slots");
        const bool blur2d = h->op.kind == PLSQR_OP_BLUR && h->d.ndim == 2;
        if (sigma) {
            if (!blur2d || h->fp64 || h->od.R[0] != h->od.R[1] || h->od.generic_blur ||
                (h->od.R[0] != 6 && h->od.R[0] != 9 && h->od.R[0] != 12 && h->od.R[0] != 15))
                throw InvalidArg("per-slot sigma needs a 2D single-precision blur with radius 6, 9, 12 or 15 on both axes");
        }
        cudaStream_t s = h->stream;
        ck(cudaEventRecord(h->ev_in, h->user_stream), "cudaEventRecord");
        ck(cudaStreamWaitEvent(s, h->ev_in, 0), "cudaStreamWaitEvent");
        const int R = h->od.R[0], W = 2 * (2 * R + 1);
        if (sigma && !h->taps_inst) {  // from now on every slot reads its own taps
            h->taps_inst = (float*)dalloc(h, sizeof(float) * W * h->B);
            ck(cudaMallocHost((void**)&h->taps_inst_host, sizeof(float) * W * h->B), "cudaMallocHost");
            for (int b = 0; b < h->B; ++b)
                for (int k = 0; k < W; ++k) h->taps_inst_host[b * W + k] = (float)h->od.taps_host[k < W / 2 ? 0 : 1][k % (W / 2)];
            ck(cudaMemcpyAsync(h->taps_inst, h->taps_inst_host, sizeof(float) * W * h->B, cudaMemcpyHostToDevice, s),
               "taps");
            h->od.tapt = h->taps_inst;
            clear_graphs(h);
        }
        if (h->taps_inst) {
            float* row = h->taps_inst_host + (size_t)slot * W;
            if (sigma) {
                slot_taps(row, sigma[0], R);
                slot_taps(row + W / 2, sigma[1], R);
            } else {
                for (int k = 0; k < W; ++k) row[k] = (float)h->od.taps_host[k < W / 2 ? 0 : 1][k % (W / 2)];
            }
            ck(cudaMemcpyAsync(h->taps_inst + (size_t)slot * W, row, sizeof(float) * W, cudaMemcpyHostToDevice, s),
               "taps");
        }
        const size_t mb = h->esz * h->m, nb = h->esz * h->d.N;
        ck(cudaMemcpyAsync(h->g + slot * mb, g, mb, cudaMemcpyDeviceToDevice, s), "copy g");
        ck(cudaMemsetAsync(h->f + slot * nb, 0, nb, s), "f0");
        ck(cudaEventSynchronize(h->ev_out), "cudaEventSynchronize");  // no copy of the states in flight
        h->st_host[slot].status = ST_OK;
        h->prm_host[slot].reg = reg;
        h->prm_host[slot].T = T;
        h->prm_host[slot].tau = tau;
        ck(cudaMemcpyAsync(h->prm_dev + slot, h->prm_host + slot, sizeof(SolveParams), cudaMemcpyHostToDevice, s),
           "params");
        slots_state(h->st, h->prm_dev, h->B, slot, false, s);
        fill_nan(h->h_rbar + (int64_t)slot * h->h_outer * h->h_inner, (int64_t)h->h_outer * h->h_inner, s);
        fill_nan(h->h_R + (int64_t)slot * (h->h_outer + 1), h->h_outer + 1, s);
        fill_nan(h->h_resid + (int64_t)slot * h->h_outer, h->h_outer, s);
        h->slot_active[slot] = 1;
        h->slot_outer[slot] = 0;
        h->slot_target[slot] = n_outer;
        ck(cudaEventRecord(h->ev_out, s), "cudaEventRecord");
        ck(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0), "cudaStreamWaitEvent");
        return PLSQR_OK;
    });
}

int plsqr_step(plsqr_handle h) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (!h->serving) throw std::logic_error("no slot has been started");
        int n = 0;
        for (int b = 0; b < h->B; ++b)
            if (h->slot_active[b] && h->slot_outer[b] < h->slot_target[b]) ++n;
        if (n == 0) return PLSQR_OK;
        Range range("plsqr_step");
        cudaStream_t s = h->stream;
        const int64_t launches0 = h->prof.launches;
        // a slot that has reached its target is parked (skipped) until it is finished
        for (int b = 0; b < h->B; ++b)
            if (h->slot_active[b] && h->slot_outer[b] >= h->slot_target[b]) slots_state(h->st, h->prm_dev, h->B, b, true, s);
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            run_outer_steps<TT>(h, h->B, 1, h->h_inner);
        });
        for (int b = 0; b < h->B; ++b)
            if (h->slot_active[b] && h->slot_outer[b] < h->slot_target[b]) ++h->slot_outer[b];
        h->last_launches = h->prof.launches - launches0;
        // the instance states after the step, read by plsqr_slot_progress once the step is done
        ck(cudaMemcpyAsync(h->st_host, h->st, sizeof(GkState) * h->B, cudaMemcpyDeviceToHost, s), "state");
        h->st_after_step = true;
        ck(cudaEventRecord(h->ev_out, s), "cudaEventRecord");
        return PLSQR_OK;
    });
}

int plsqr_query(plsqr_handle h) {
    if (!h) return PLSQR_E_INVALID;
    const cudaError_t e = cudaEventQuery(h->ev_out);
    if (e == cudaErrorNotReady) return 1;
    if (e != cudaSuccess) {
        fail(h, PLSQR_E_CUDA, cudaGetErrorString(e));
        return -PLSQR_E_CUDA;
    }
    return 0;
}

int plsqr_slot_progress(plsqr_handle h, int32_t slot, int32_t* outer_done, int32_t* active) {
    if (!h) return PLSQR_E_INVALID;
    if (slot < 0 || slot >= h->B) return fail(h, PLSQR_E_INVALID, "slot out of range");
    const bool on = h->serving && h->slot_active[slot];
    int act = on ? 1 : 0;
    // stopped early by the outer rule (Algorithm 3 step 5): visible once the last step is done
    if (on && h->st_after_step) {
        const cudaError_t q = cudaEventQuery(h->ev_out);
        if (q == cudaSuccess && h->st_host[slot].status == ST_CONVERGED) act = 2;
        if (q == cudaErrorNotReady) cudaGetLastError();  // not ready is not an error
    }
    if (outer_done) *outer_done = on ? h->slot_outer[slot] : 0;
    if (active) *active = act;
    return PLSQR_OK;
}

// ---- checkpoint of a slot at an outer-step boundary ----------------------------------------------
// Between two outer steps of Algorithm 3 a request is f^k, its data g and its scalars (R(f^k) for
// the outer stop, the outer counter, the status, r, T, tau and the stopping rule), with the
// histories so far and, where set, its blur taps; every other vector is rebuilt by the next step.
// The blob: a header, then f (N values), g (m values), the histories (n_outer x n_inner, n_outer + 1
// and n_outer doubles of the handle that saved it) and the taps row.
namespace {
constexpr uint64_t kCkptMagic = 0x31544b43524c5350ull;  // "PLSRCKT1"
struct CkptHeader {
    uint64_t magic;
    int32_t esz, ndim, n[3], kind;
    int64_t m;
    int32_t h_outer, h_inner, outer_done, target, taps_w, kbf16;
    GkState st;
    SolveParams prm;
};

int64_t ckpt_bytes(const plsqr_ctx* h) {
    const int64_t no = h->h_outer, ni = h->h_inner;
    const int64_t W = h->taps_inst ? 2 * (2 * h->od.R[0] + 1) : 0;
    return (int64_t)sizeof(CkptHeader) + (int64_t)h->esz * (h->d.N + h->m) +
           (int64_t)sizeof(double) * (no * ni + (no + 1) + no) + (int64_t)sizeof(float) * W;
}
}  // namespace

int64_t plsqr_slot_state_bytes(plsqr_handle h) {
    if (!h || !h->serving || !h->h_rbar) return -1;
    return ckpt_bytes(h);
}

int plsqr_slot_save(plsqr_handle h, int32_t slot, void* buf, int64_t cap) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (slot < 0 || slot >= h->B) throw InvalidArg("slot out of range");
        if (!h->serving || !h->slot_active[slot]) throw std::logic_error("slot is not running");
        if (!buf) throw InvalidArg("buf is NULL");
        const int64_t need = ckpt_bytes(h);
        if (cap < need) throw InvalidArg("buffer smaller than plsqr_slot_state_bytes");
        cudaStream_t s = h->stream;
        ck(cudaStreamSynchronize(s), "cudaStreamSynchronize");  // the slot is between two outer steps
        CkptHeader hd{};
        hd.magic = kCkptMagic;
        hd.esz = (int32_t)h->esz;
        hd.ndim = h->d.ndim;
        hd.n[0] = h->d.nx;
        hd.n[1] = h->d.ny;
        hd.n[2] = h->d.nz;
        hd.kind = h->op.kind;
        hd.m = h->m;
        hd.h_outer = h->h_outer;
        hd.h_inner = h->h_inner;
        hd.outer_done = h->slot_outer[slot];
        hd.target = h->slot_target[slot];
        hd.taps_w = h->taps_inst ? 2 * (2 * h->od.R[0] + 1) : 0;
        hd.kbf16 = h->kbf16 ? 1 : 0;
        hd.prm = h->prm_host[slot];
        char* out = static_cast<char*>(buf);
        ck(cudaMemcpy(&hd.st, h->st + slot, sizeof(GkState), cudaMemcpyDeviceToHost), "state");
        std::memcpy(out, &hd, sizeof(hd));
        char* q = out + sizeof(hd);
        const size_t nb = h->esz * h->d.N, mb = h->esz * h->m;
        ck(cudaMemcpy(q, h->f + slot * nb, nb, cudaMemcpyDeviceToHost), "f");
        q += nb;
        ck(cudaMemcpy(q, h->g + slot * mb, mb, cudaMemcpyDeviceToHost), "g");
        q += mb;
        const int64_t nr = (int64_t)h->h_outer * h->h_inner, nR = h->h_outer + 1, ne = h->h_outer;
        ck(cudaMemcpy(q, h->h_rbar + slot * nr, sizeof(double) * nr, cudaMemcpyDeviceToHost), "hist");
        q += sizeof(double) * nr;
        ck(cudaMemcpy(q, h->h_R + slot * nR, sizeof(double) * nR, cudaMemcpyDeviceToHost), "hist");
        q += sizeof(double) * nR;
        ck(cudaMemcpy(q, h->h_resid + slot * ne, sizeof(double) * ne, cudaMemcpyDeviceToHost), "hist");
        q += sizeof(double) * ne;
        if (hd.taps_w) std::memcpy(q, h->taps_inst_host + (size_t)slot * hd.taps_w, sizeof(float) * hd.taps_w);
        return PLSQR_OK;
    });
}

int plsqr_slot_restore(plsqr_handle h, int32_t slot, const void* buf, int64_t len) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (!h->op_set) throw std::logic_error("set_operator must be called before plsqr_slot_restore");
        if (slot < 0 || slot >= h->B) throw InvalidArg("slot out of range");
        if (!buf || len < (int64_t)sizeof(CkptHeader)) throw InvalidArg("checkpoint too short");
        CkptHeader hd;
        std::memcpy(&hd, buf, sizeof(hd));
        if (hd.magic != kCkptMagic) throw InvalidArg("not a slot checkpoint");
        if (hd.esz != (int32_t)h->esz || hd.ndim != h->d.ndim || hd.n[0] != h->d.nx || hd.n[1] != h->d.ny ||
            hd.n[2] != h->d.nz || hd.kind != h->op.kind || hd.m != h->m)
            throw InvalidArg("checkpoint of another precision, grid or operator");
        if (hd.kbf16 != (h->kbf16 ? 1 : 0)) throw InvalidArg("checkpoint taken with another kappa storage");
        if (hd.h_outer < 1 || hd.h_inner < 1 || hd.outer_done < 0 || hd.outer_done > hd.target ||
            hd.target > hd.h_outer || hd.taps_w < 0 || hd.taps_w > 2 * (2 * 64 + 1))
            throw InvalidArg("corrupt checkpoint header");
        const int64_t nr = (int64_t)hd.h_outer * hd.h_inner, nR = hd.h_outer + 1, ne = hd.h_outer;
        const int64_t need = (int64_t)sizeof(CkptHeader) + (int64_t)h->esz * (h->d.N + h->m) +
                             (int64_t)sizeof(double) * (nr + nR + ne) + (int64_t)sizeof(float) * hd.taps_w;
        if (len < need) throw InvalidArg("checkpoint too short");
        const int W = 2 * (2 * h->od.R[0] + 1);
        if (hd.taps_w && hd.taps_w != W) throw InvalidArg("checkpoint taps of another blur radius");
        enter_slot_mode(h);
        if (h->slot_active[slot]) throw std::logic_error("slot is busy");
        bool any = false;
        for (int b = 0; b < h->B; ++b) any = any || h->slot_active[b];
        if (!any) ensure_hist(h, hd.h_outer, hd.h_inner);
        else if (hd.h_inner != h->h_inner || hd.target > h->h_outer)
            throw InvalidArg("n_inner must equal, and n_outer not exceed, those of the running slots");
        cudaStream_t s = h->stream;
        ck(cudaEventRecord(h->ev_in, h->user_stream), "cudaEventRecord");
        ck(cudaStreamWaitEvent(s, h->ev_in, 0), "cudaStreamWaitEvent");
        ck(cudaStreamSynchronize(s), "cudaStreamSynchronize");  // no step or copy of the states in flight
        const char* q = static_cast<const char*>(buf) + sizeof(hd);
        const size_t nb = h->esz * h->d.N, mb = h->esz * h->m;
        ck(cudaMemcpy(h->f + slot * nb, q, nb, cudaMemcpyHostToDevice), "f");
        q += nb;
        ck(cudaMemcpy(h->g + slot * mb, q, mb, cudaMemcpyHostToDevice), "g");
        q += mb;
        // histories: rows of the checkpoint's n_outer x n_inner layout into the handle's (NaN beyond)
        const int64_t hr = (int64_t)h->h_outer * h->h_inner, hR = h->h_outer + 1, he = h->h_outer;
        std::vector<double> tmp((size_t)std::max<int64_t>(hr, 1), std::nan(""));
        std::memcpy(tmp.data(), q, sizeof(double) * std::min(nr, hr));
        ck(cudaMemcpy(h->h_rbar + slot * hr, tmp.data(), sizeof(double) * hr, cudaMemcpyHostToDevice), "hist");
        q += sizeof(double) * nr;
        std::vector<double> tR((size_t)hR, std::nan(""));
        std::memcpy(tR.data(), q, sizeof(double) * std::min(nR, hR));
        ck(cudaMemcpy(h->h_R + slot * hR, tR.data(), sizeof(double) * hR, cudaMemcpyHostToDevice), "hist");
        q += sizeof(double) * nR;
        std::vector<double> te((size_t)std::max<int64_t>(he, 1), std::nan(""));
        std::memcpy(te.data(), q, sizeof(double) * std::min(ne, he));
        ck(cudaMemcpy(h->h_resid + slot * he, te.data(), sizeof(double) * he, cudaMemcpyHostToDevice), "hist");
        q += sizeof(double) * ne;
        if (hd.taps_w || h->taps_inst) {
            if (!h->taps_inst) {  // from now on every slot reads its own taps
                h->taps_inst = (float*)dalloc(h, sizeof(float) * W * h->B);
                ck(cudaMallocHost((void**)&h->taps_inst_host, sizeof(float) * W * h->B), "cudaMallocHost");
                for (int b = 0; b < h->B; ++b)
                    for (int k = 0; k < W; ++k)
                        h->taps_inst_host[b * W + k] = (float)h->od.taps_host[k < W / 2 ? 0 : 1][k % (W / 2)];
                ck(cudaMemcpy(h->taps_inst, h->taps_inst_host, sizeof(float) * W * h->B, cudaMemcpyHostToDevice),
                   "taps");
                h->od.tapt = h->taps_inst;
                clear_graphs(h);
            }
            float* row = h->taps_inst_host + (size_t)slot * W;
            if (hd.taps_w) std::memcpy(row, q, sizeof(float) * W);
            else
                for (int k = 0; k < W; ++k) row[k] = (float)h->od.taps_host[k < W / 2 ? 0 : 1][k % (W / 2)];
            ck(cudaMemcpy(h->taps_inst + (size_t)slot * W, row, sizeof(float) * W, cudaMemcpyHostToDevice), "taps");
        }
        h->prm_host[slot] = hd.prm;
        ck(cudaMemcpy(h->prm_dev + slot, &hd.prm, sizeof(SolveParams), cudaMemcpyHostToDevice), "params");
        GkState st = hd.st;
        st.frozen = 0;
        ck(cudaMemcpy(h->st + slot, &st, sizeof(GkState), cudaMemcpyHostToDevice), "state");
        h->st_host[slot] = st;
        h->slot_active[slot] = 1;
        h->slot_outer[slot] = hd.outer_done;
        h->slot_target[slot] = hd.target;
        ck(cudaEventRecord(h->ev_out, s), "cudaEventRecord");
        ck(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0), "cudaStreamWaitEvent");
        return PLSQR_OK;
    });
}

int plsqr_slot_finish(plsqr_handle h, int32_t slot, void* f_out, plsqr_stats* stats) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (slot < 0 || slot >= h->B) throw InvalidArg("slot out of range");
        if (!h->serving || !h->slot_active[slot]) throw std::logic_error("slot is not running");
        if (!f_out) throw InvalidArg("f_out is NULL");
        cudaStream_t s = h->stream;
        const size_t nb = h->esz * h->d.N;
        const int no = h->slot_outer[slot], ni = h->h_inner;
        // R(f^k) of this slot alone: the diffusivity pass on instance `slot` through shifted bases
        Hist hs = hist_of(h);
        hs.R = h->h_R + (int64_t)slot * (h->h_outer + 1);
        hs.rbar = nullptr;
        hs.resid = nullptr;
        slots_state(h->st, h->prm_dev, h->B, slot, false, s, /*keep_outer=*/true);
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            diffusivity<TT>(P<TT>(h->f) + (int64_t)slot * h->d.N, P<TT>(h->kappa) + (int64_t)slot * h->d.N, h->d, 1,
                            h->st + slot, hs, h->kfloor, h->red, s);
        });
        ck(cudaMemcpyAsync(f_out, h->f + slot * nb, nb, cudaMemcpyDeviceToDevice, s), "copy f");
        ck(cudaMemcpyAsync(h->st_host + slot, h->st + slot, sizeof(GkState), cudaMemcpyDeviceToHost, s), "state");
        const int64_t nr = (int64_t)h->h_outer * ni, nR = h->h_outer + 1, ne = h->h_outer;
        if (stats) {
            ck(cudaMemcpyAsync(h->h_stage, h->h_rbar + (int64_t)slot * nr, sizeof(double) * nr, cudaMemcpyDeviceToHost,
                               s), "hist");
            ck(cudaMemcpyAsync(h->h_stage + nr, h->h_R + (int64_t)slot * nR, sizeof(double) * nR,
                               cudaMemcpyDeviceToHost, s), "hist");
            ck(cudaMemcpyAsync(h->h_stage + nr + nR, h->h_resid + (int64_t)slot * ne, sizeof(double) * ne,
                               cudaMemcpyDeviceToHost, s), "hist");
        }
        slots_state(h->st, h->prm_dev, h->B, slot, true, s);  // empty again
        ck(cudaEventRecord(h->ev_out, s), "cudaEventRecord");
        ck(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0), "cudaStreamWaitEvent");
        ck(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        h->slot_active[slot] = 0;
        const int sb = h->st_host[slot].status_any;
        if (stats) {
            stats->status = sb;
            if (stats->rbar_hist) std::memcpy(stats->rbar_hist, h->h_stage, sizeof(double) * (size_t)no * ni);
            if (stats->R_hist) std::memcpy(stats->R_hist, h->h_stage + nr, sizeof(double) * (size_t)(no + 1));
            if (stats->resid_hist) std::memcpy(stats->resid_hist, h->h_stage + nr + nR, sizeof(double) * (size_t)no);
        }
        return sb != 0 ? PLSQR_E_BREAKDOWN : PLSQR_OK;
    });
}

void plsqr_destroy(plsqr_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    destroy_ctx(h);
}

const char* plsqr_last_error(plsqr_handle h) {
    if (!h) return "invalid handle";
    return h->err.c_str();
}

int64_t plsqr_workspace_bytes(const plsqr_config* cfg, const plsqr_operator* op) {
    try {
        Plan pl = make_plan(cfg, 0);
        int64_t m = op_data_len(op, pl.d);
        int64_t bytes = (int64_t)make_plan(cfg, m).bytes;
        if (op && op->kind == PLSQR_OP_JOSEPH) {
            const int64_t cap = joseph_parts_cap(cfg->max_batch, op->n_angles);
            const int64_t esz = cfg->precision == PLSQR_FP64 ? 8 : 4;
            bytes += cap * (2 * esz * m + (int64_t)sizeof(unsigned) * op->n_angles);
        }
        return bytes;
    } catch (...) {
        return -1;
    }
}

namespace {
// The single-operation entry points run on instance 0's state and the handle's scratch vectors,
// which the slots of continuous batching own.
void refuse_in_slot_mode(const plsqr_ctx* h) {
    if (h->serving) throw std::logic_error("the handle is in slot mode");
}
}  // namespace

int plsqr_apply_A(plsqr_handle h, const void* x, void* y) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        if (!h->op_set) throw std::logic_error("set_operator first");
        if (!x || !y) throw InvalidArg("NULL pointer");
        by_type(h, [&](auto tv) {
            using T = decltype(tv);
            op_apply<T>(h->od, false, EPI_PLAIN, (const T*)x, (T*)y, nullptr, P<T>(h->tmp), 1, h->st, h->red,
                        h->user_stream);
        });
        return PLSQR_OK;
    });
}

int plsqr_apply_At(plsqr_handle h, const void* y, void* x) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        if (!h->op_set) throw std::logic_error("set_operator first");
        if (!x || !y) throw InvalidArg("NULL pointer");
        by_type(h, [&](auto tv) {
            using T = decltype(tv);
            op_apply<T>(h->od, true, EPI_PLAIN, (const T*)y, (T*)x, nullptr, P<T>(h->tmp), 1, h->st, h->red,
                        h->user_stream);
        });
        return PLSQR_OK;
    });
}

int plsqr_diffusivity(plsqr_handle h, const void* f, int32_t reg, double T, void* kappa_out, double* R_out) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        if (!f || !kappa_out) throw InvalidArg("NULL pointer");
        if (reg < 0 || reg > 3) throw InvalidArg("bad regulariser");
        if (!(T > 0.0) || !std::isfinite(T)) throw InvalidArg("T must be positive and finite");
        cudaStream_t s = h->user_stream;
        h->prm_host[0].reg = reg;
        h->prm_host[0].T = T;
        h->prm_host[0].tau = 0.0;
        ck(cudaMemcpyAsync(h->prm_dev, h->prm_host, sizeof(SolveParams), cudaMemcpyHostToDevice, s), "params");
        set_params(h->st, h->prm_dev, 1, true, s);
        Hist hs{};
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            diffusivity<TT>((const TT*)f, (TT*)kappa_out, h->d, 1, h->st, hs, h->kfloor, h->red, s);
        });
        ck(cudaMemcpyAsync(h->st_host, h->st, sizeof(GkState), cudaMemcpyDeviceToHost, s), "state");
        ck(cudaStreamSynchronize(s), "sync");
        if (R_out) *R_out = h->st_host[0].R;
        return PLSQR_OK;
    });
}

int plsqr_prec_setup(plsqr_handle h, const void* kappa) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        if (!kappa) throw InvalidArg("NULL pointer");
        Range range("plsqr_prec_setup");
        cudaStream_t s = h->user_stream;
        ck(cudaMemcpyAsync(h->kappa, kappa, h->esz * h->d.N, cudaMemcpyDeviceToDevice, s), "kappa");
        if (h->kbf16) to_bf16(P<float>(h->kappa), h->kappa16, h->d.N, s);
        by_type(h, [&](auto tv) {
            using T = decltype(tv);
            prec_setup<T>(h, 1, s);
        });
        return PLSQR_OK;
    });
}

int plsqr_prec_apply(plsqr_handle h, const void* b, void* x) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        if (!b || !x) throw InvalidArg("NULL pointer");
        by_type(h, [&](auto tv) {
            using T = decltype(tv);
            prec_apply<T>(h, (const T*)b, (T*)x, 1, h->user_stream);
        });
        return PLSQR_OK;
    });
}

int plsqr_apply_M(plsqr_handle h, const void* x, void* y) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        if (!x || !y) throw InvalidArg("NULL pointer");
        by_type(h, [&](auto tv) {
            using T = decltype(tv);
            mg_apply_level<T>(P<T>(h->kappa), true, (const T*)x, nullptr, (T*)y, h->d, 1, h->user_stream);
        });
        return PLSQR_OK;
    });
}

int plsqr_mlsqr(plsqr_handle h, const void* g, double tau, int32_t n_inner, void* f_out, double* rbar_hist,
                int32_t* iters_done) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        refuse_in_slot_mode(h);
        Range range("plsqr_mlsqr");
        int32_t reg = 0;
        double T = 1.0;
        validate_solve(h, 1, &reg, &T, &tau, 1, n_inner);
        if (!g || !f_out) throw InvalidArg("NULL pointer");
        ensure_hist(h, 1, n_inner);
        cudaStream_t s = h->user_stream;
        ck(cudaMemcpyAsync(h->g, g, h->esz * h->m, cudaMemcpyDeviceToDevice, s), "g");
        h->prm_host[0].reg = reg;
        h->prm_host[0].T = T;
        h->prm_host[0].tau = tau;
        ck(cudaMemcpyAsync(h->prm_dev, h->prm_host, sizeof(SolveParams), cudaMemcpyHostToDevice, s), "params");
        set_params(h->st, h->prm_dev, 1, true, s);
        fill_nan(h->h_rbar, (int64_t)h->B * h->h_outer * h->h_inner, s);
        by_type(h, [&](auto tv) {
            using TT = decltype(tv);
            mlsqr_seq<TT>(h, 1, n_inner, s);
        });
        ck(cudaMemcpyAsync(f_out, h->f, h->esz * h->d.N, cudaMemcpyDeviceToDevice, s), "f");
        ck(cudaMemcpyAsync(h->st_host, h->st, sizeof(GkState), cudaMemcpyDeviceToHost, s), "state");
        if (rbar_hist)
            ck(cudaMemcpyAsync(h->h_stage, h->h_rbar, sizeof(double) * n_inner, cudaMemcpyDeviceToHost, s), "hist");
        ck(cudaStreamSynchronize(s), "sync");
        if (rbar_hist) std::memcpy(rbar_hist, h->h_stage, sizeof(double) * n_inner);
        if (iters_done) *iters_done = h->st_host[0].iter;
        return h->st_host[0].status != 0 ? PLSQR_E_BREAKDOWN : PLSQR_OK;
    });
}

int plsqr_selftest_wait(int32_t complete, int32_t* status_out) {
    if (!status_out) return PLSQR_E_INVALID;
    GkState* st = nullptr;
    if (cudaMalloc(&st, sizeof(GkState)) != cudaSuccess) {
        cudaGetLastError();
        return PLSQR_E_NOMEM;
    }
    int rc = PLSQR_OK;
    try {
        ck(cudaMemset(st, 0, sizeof(GkState)), "memset");
        selftest_wait(st, complete != 0, 1u << 16, nullptr);
        GkState h{};
        ck(cudaMemcpy(&h, st, sizeof(GkState), cudaMemcpyDeviceToHost), "state");
        *status_out = h.status;
    } catch (const std::exception&) {
        rc = PLSQR_E_CUDA;
    }
    cudaFree(st);
    return rc;
}

int plsqr_projected_solve(int32_t k, const double* alpha, const double* beta, double tau, double* y,
                          double* rbar) {
    if (k < 1 || !alpha || !beta || !y || !(tau >= 0.0)) return PLSQR_E_INVALID;
    // Algorithm 2 steps 8-20 on coefficient vectors in the basis V (x = sum_j y_j V_j, w likewise):
    // the damping rotation (eq. 3.6) and the plane rotation of each step, as in the device code.
    std::vector<double> w((size_t)k + 1, 0.0);
    for (int j = 0; j < k; ++j) y[j] = 0.0;
    w[0] = 1.0;  // w~_1 = v~_1
    double phibar = beta[0], rhobar = alpha[0], res2 = 0.0;
    const double sq = std::sqrt(tau);
    for (int i = 0; i < k; ++i) {
        double rhohat = rhobar, psi = 0.0;
        if (tau > 0.0) {
            rhohat = std::sqrt(rhobar * rhobar + tau);
            const double c1 = rhobar / rhohat, s1 = sq / rhohat;
            psi = s1 * phibar;
            phibar = c1 * phibar;
        }
        const double b = beta[i + 1], a = alpha[i + 1];
        const double rho = std::sqrt(rhohat * rhohat + b * b);
        if (!(rho > 0.0) || !std::isfinite(rho)) return PLSQR_E_BREAKDOWN;
        const double c = rhohat / rho, sn = b / rho;
        const double theta = sn * a;
        rhobar = -c * a;
        const double phi = c * phibar;
        phibar = sn * phibar;
        res2 += psi * psi;
        for (int j = 0; j <= i; ++j) y[j] += (phi / rho) * w[j];   // step 19
        for (int j = 0; j <= i; ++j) w[j] *= -(theta / rho);       // step 20
        w[i + 1] = 1.0;
        if (rbar) rbar[i] = std::sqrt(phibar * phibar + res2);
    }
    return PLSQR_OK;
}

int plsqr_mlsqr_multi_tau(plsqr_handle h, const void* g, int32_t n_inner, int32_t n_tau, const double* taus,
                          void* const* f_out, double* rbar_hist, int32_t* iters_done) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        if (!g || !f_out || !taus) throw InvalidArg("NULL pointer");
        if (n_tau < 1 || n_tau > MT_MAX) throw InvalidArg("n_tau must be in 1..32");
        for (int t = 0; t < n_tau; ++t) {
            if (!(taus[t] >= 0.0) || !std::isfinite(taus[t])) throw InvalidArg("tau must be finite and >= 0");
            if (!f_out[t]) throw InvalidArg("NULL pointer");
        }
        if (h->serving) throw std::logic_error("not while slots are in use");
        Range range("plsqr_mlsqr_multi_tau");
        int32_t reg = 0;
        double T = 1.0, tau0 = 0.0;
        validate_solve(h, 1, &reg, &T, &tau0, 1, n_inner);
        cudaStream_t s = h->user_stream;
        const int64_t N = h->d.N;
        char* V = nullptr;
        double *ab = nullptr, *coef = nullptr;
        int k = 0;
        auto release = [&]() {
            h->basis = nullptr;
            h->basis_ab = nullptr;
            h->basis_n = 0;
            if (V) cudaFree(V);
            if (ab) cudaFree(ab);
            if (coef) cudaFree(coef);
        };
        try {
            ck(cudaMalloc((void**)&V, h->esz * (size_t)n_inner * N), "cudaMalloc (stored Lanczos vectors)");
            ck(cudaMalloc((void**)&ab, sizeof(double) * 2 * (size_t)(n_inner + 1)), "cudaMalloc");
            ck(cudaMalloc((void**)&coef, sizeof(double) * (size_t)n_tau * n_inner), "cudaMalloc");
            ck(cudaMemsetAsync(ab, 0, sizeof(double) * 2 * (size_t)(n_inner + 1), s), "memset");
            h->basis = V;
            h->basis_ab = ab;
            h->basis_n = n_inner;
            // the bidiagonalisation does not depend on tau (Sec. 3.3): one run, undamped
            ensure_hist(h, 1, n_inner);
            ck(cudaMemcpyAsync(h->g, g, h->esz * h->m, cudaMemcpyDeviceToDevice, s), "g");
            h->prm_host[0].reg = reg;
            h->prm_host[0].T = T;
            h->prm_host[0].tau = 0.0;
            ck(cudaMemcpyAsync(h->prm_dev, h->prm_host, sizeof(SolveParams), cudaMemcpyHostToDevice, s), "params");
            set_params(h->st, h->prm_dev, 1, true, s);
            by_type(h, [&](auto tv) {
                using TT = decltype(tv);
                mlsqr_seq<TT>(h, 1, n_inner, s);
            });
            std::vector<double> abh(2 * (size_t)(n_inner + 1));
            ck(cudaMemcpyAsync(abh.data(), ab, sizeof(double) * abh.size(), cudaMemcpyDeviceToHost, s), "scalars");
            ck(cudaMemcpyAsync(h->st_host, h->st, sizeof(GkState), cudaMemcpyDeviceToHost, s), "state");
            ck(cudaStreamSynchronize(s), "sync");
            k = std::min<int>(n_inner, h->st_host[0].iter);
            if (iters_done) *iters_done = k;
            if (k < 1) {  // broke down before its first step: every f(tau) is the starting point 0
                for (int t = 0; t < n_tau; ++t) ck(cudaMemsetAsync(f_out[t], 0, h->esz * N, s), "memset");
                if (rbar_hist)
                    for (int i = 0; i < n_tau * n_inner; ++i) rbar_hist[i] = NAN;
                ck(cudaStreamSynchronize(s), "sync");
                release();
                return PLSQR_E_BREAKDOWN;
            }
            std::vector<double> alpha((size_t)k + 1), beta((size_t)k + 1);
            for (int j = 0; j <= k; ++j) {
                alpha[j] = abh[2 * j];
                beta[j] = abh[2 * j + 1];
            }
            std::vector<double> ch((size_t)n_tau * k), rb((size_t)k);
            for (int t = 0; t < n_tau; ++t) {
                if (plsqr_projected_solve(k, alpha.data(), beta.data(), taus[t], ch.data() + (size_t)t * k, rb.data()) !=
                    PLSQR_OK)
                    throw std::runtime_error("projected problem broke down");
                if (rbar_hist)
                    for (int i = 0; i < n_inner; ++i) rbar_hist[(size_t)t * n_inner + i] = i < k ? rb[i] : NAN;
            }
            ck(cudaMemcpyAsync(coef, ch.data(), sizeof(double) * ch.size(), cudaMemcpyHostToDevice, s), "coef");
            by_type(h, [&](auto tv) {
                using TT = decltype(tv);
                OutPtrs<TT> outs{};
                for (int t = 0; t < n_tau; ++t) outs.p[t] = (TT*)f_out[t];
                combine_basis<TT>(P<TT>(V), k, N, coef, n_tau, outs, s);
            });
            ck(cudaStreamSynchronize(s), "sync");
        } catch (...) {
            cudaStreamSynchronize(s);
            release();
            throw;
        }
        release();
        return k < n_inner ? PLSQR_E_BREAKDOWN : PLSQR_OK;
    });
}

int plsqr_profile(plsqr_handle h, int32_t enable) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        ck(cudaStreamSynchronize(h->stream), "sync");
        ck(cudaStreamSynchronize(h->user_stream), "sync");
        h->prof.collect();
        for (int c = 0; c < KC_COUNT; ++c) {
            h->prof.ms[c] = 0.0;
            h->prof.count[c] = 0;
        }
        h->prof.enabled = enable != 0;
        return PLSQR_OK;
    });
}

int plsqr_check_guards(plsqr_handle h, int64_t* n_checked, int64_t* n_bad) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        ck(cudaStreamSynchronize(h->stream), "sync");
        ck(cudaStreamSynchronize(h->user_stream), "sync");
        int64_t checked = 0, bad = 0;
        std::vector<unsigned char> band(2 * kGuard);
        for (const Alloc& a : h->allocs) {
            if (a.user == a.base) continue;
            ck(cudaMemcpy(band.data(), a.base, kGuard, cudaMemcpyDeviceToHost), "guard band");
            ck(cudaMemcpy(band.data() + kGuard, a.user + a.bytes, kGuard, cudaMemcpyDeviceToHost), "guard band");
            ++checked;
            for (unsigned char c : band)
                if (c != kGuardByte) {
                    ++bad;
                    break;
                }
        }
        if (n_checked) *n_checked = checked;
        if (n_bad) *n_bad = bad;
        return PLSQR_OK;
    });
}

int plsqr_profile_read(plsqr_handle h, double* ms, int64_t* counts, int32_t n) {
    if (!h) return PLSQR_E_INVALID;
    return guarded(h, [&]() -> int {
        h->prof.collect();
        for (int c = 0; c < n && c < KC_COUNT; ++c) {
            if (ms) ms[c] = h->prof.ms[c];
            if (counts) counts[c] = h->prof.count[c];
        }
        return PLSQR_OK;
    });
}

int64_t plsqr_last_launches(plsqr_handle h) { return h ? h->last_launches : -1; }

int plsqr_blur_noalloc(int32_t ndim, const int64_t* n, int32_t precision, const double* sigma, const int32_t* radius,
                       const void* x, void* y, void* stream) {
    if (!n || !sigma || !radius || !x || !y || (ndim != 2 && ndim != 3)) return PLSQR_E_INVALID;
    if (precision != PLSQR_FP32 && precision != PLSQR_FP64) return PLSQR_E_INVALID;
    const size_t esz = precision == PLSQR_FP64 ? 8 : 4;
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) {
        if (n[d] < 1 || n[d] > (1 << 20)) return PLSQR_E_INVALID;
        if (!(sigma[d] > 0.0) || radius[d] < 0 || radius[d] > kNoallocMaxRadius) return PLSQR_E_INVALID;
        N *= n[d];
    }
    if ((size_t)N * esz > kNoallocScratchBytes - kNoallocTapsBytes) return PLSQR_E_INVALID;  // beyond the maximum
    // the launch shapes of both passes (grid.y and grid.z are limited to 65535)
    if (ndim == 3 && (n[2] > 65535 || (n[1] + 7) / 8 > 65535)) return PLSQR_E_INVALID;
    // x and y must not overlap
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
    const uintptr_t bytes = (uintptr_t)N * esz;
    if (xa < ya + bytes && ya < xa + bytes) return PLSQR_E_INVALID;
    int err = PLSQR_OK;
    unsigned char* scratch = static_cast<unsigned char*>(noalloc_scratch(&err));
    if (!scratch) return err;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        OpDev od{};
        od.kind = OPK_BLUR;
        od.d = make_dims(ndim, n[0], n[1], ndim == 3 ? n[2] : 1);
        od.m = od.d.N;
        // taps of every axis: computed here, passed by value to a kernel that writes them, in the
        // element type, into the first 2 KiB of the scratch (no host-memory copy)
        NoallocTaps tp{};
        tp.ndim = ndim;
        tp.esz = (int32_t)esz;
        int32_t off = 0;
        for (int d = 0; d < ndim; ++d) {
            const int R = radius[d];
            double sum = 0.0;
            for (int k = -R; k <= R; ++k) sum += std::exp(-(double)(k * k) / (2.0 * sigma[d] * sigma[d]));
            od.R[d] = R;
            od.taps[d] = scratch + off;
            tp.off[d] = off;
            tp.len[d] = 2 * R + 1;
            for (int k = -R; k <= R; ++k) {
                const double w = std::exp(-(double)(k * k) / (2.0 * sigma[d] * sigma[d])) / sum;
                od.taps_host[d][k + R] = w;
                tp.w[d][k + R] = w;
            }
            off += (int32_t)(((2 * R + 1) * esz + 15) & ~(size_t)15);
        }
        k_noalloc_taps<<<1, 64, 0, s>>>(tp, scratch);
        klaunched("k_noalloc_taps");
        Red red{};
        if (esz == 8)
            op_apply<double>(od, false, EPI_PLAIN, (const double*)x, (double*)y, nullptr,
                             reinterpret_cast<double*>(scratch + kNoallocTapsBytes), 1, nullptr, red, s);
        else
            op_apply<float>(od, false, EPI_PLAIN, (const float*)x, (float*)y, nullptr,
                            reinterpret_cast<float*>(scratch + kNoallocTapsBytes), 1, nullptr, red, s);
        return PLSQR_OK;
    } catch (const std::exception& e) {
        std::fprintf(stderr, "plsqr_blur_noalloc: %s\n", e.what());
        return PLSQR_E_CUDA;
    }
}

}  // extern "C"
