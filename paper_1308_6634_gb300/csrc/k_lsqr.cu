// k_lsqr.cu -- Golub-Kahan scalar recurrences and vector updates of MLSQR (Algorithm 2).
//
// The norms beta = ||u|| and alpha = sqrt(v~ . p~) are reduced in double (per-thread partial
// in the bulk type over a handful of elements, double across threads and blocks, fixed
// order).  The last block of an instance runs the orthogonal transformation (Algorithm 1
// steps 10-16) on one thread in double, including the Paige-Saunders damping rotation
// that eliminates sqrt(tau) I (eq. 3.6), and records ||rbar_i||.
#include <cuda_runtime.h>

#include <algorithm>

#include <stdexcept>
#include <string>

#include <cudaTypedefs.h>

#include <cstdlib>

#include "kernels.cuh"
#include "tma.cuh"

namespace plsqr {


Profiler*& current_profiler() {
    static thread_local Profiler* p = nullptr;
    return p;
}

void Profiler::begin(int cls, cudaStream_t s) {
    if (!enabled || open) return;
    if (n_recs == cap) {
        const int nc = cap ? 2 * cap : 1024;
        Rec* nr = new Rec[nc];
        for (int i = 0; i < n_recs; ++i) nr[i] = recs[i];
        for (int i = n_recs; i < nc; ++i) {
            cudaEventCreate(&nr[i].a);
            cudaEventCreate(&nr[i].b);
        }
        delete[] recs;
        recs = nr;
        cap = nc;
    }
    recs[n_recs].cls = cls;
    cudaEventRecord(recs[n_recs].a, s);
    open = true;
}

void Profiler::finish(cudaStream_t s) {
    if (!enabled || !open) return;
    cudaEventRecord(recs[n_recs].b, s);
    ++n_recs;
    open = false;
}

void Profiler::collect() {
    for (int i = 0; i < n_recs; ++i) {
        float t = 0.f;
        cudaEventSynchronize(recs[i].b);
        if (cudaEventElapsedTime(&t, recs[i].a, recs[i].b) == cudaSuccess) {
            ms[recs[i].cls] += t;
            count[recs[i].cls] += 1;
        }
    }
    n_recs = 0;
}

void Profiler::release() {
    for (int i = 0; i < cap; ++i) {
        cudaEventDestroy(recs[i].a);
        cudaEventDestroy(recs[i].b);
    }
    delete[] recs;
    recs = nullptr;
    cap = n_recs = 0;
}

void kbegin(int cls, cudaStream_t s) {
    if (Profiler* p = current_profiler()) p->begin(cls, s);
}

void klaunched(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (Profiler* p = current_profiler()) p->launches += 1;
}

void kfinish(cudaStream_t s) {
    if (Profiler* p = current_profiler()) p->finish(s);
}

bool tma_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("PLSQR_TMA");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("PLSQR_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool tma_map_3d(CUtensorMap* map, const void* base, int esz, int64_t nx, int64_t ny, int64_t planes, int bx, int by,
                int bz) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode || !base) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (nx * esz) % 16 || ((int64_t)bx * esz) % 16) return false;
    if (bx < 1 || by < 1 || bz < 1 || bx > 256 || by > 256 || bz > 256 || nx < 1 || ny < 1 || planes < 1) return false;
    if (planes > (int64_t(1) << 31) - 1 || nx > (int64_t(1) << 31) - 1 || ny > (int64_t(1) << 31) - 1) return false;
    cuuint64_t gdim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    cuuint64_t gstride[2] = {(cuuint64_t)(nx * esz), (cuuint64_t)(nx * ny * esz)};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(map, esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                              const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int red_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 1024)); }

__global__ void k_set_params(GkState* st, const SolveParams* prm, int B, int reset_outer) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    GkState& s = st[b];
    s.reg = prm[b].reg;
    s.T = prm[b].T;
    s.tau = prm[b].tau;
    s.sqrt_tau = sqrt(prm[b].tau);
    s.eta_delta = prm[b].eta_delta;
    s.r_rel = prm[b].r_rel;
    s.frozen = 0;
    if (reset_outer) {
        s.outer = 0;
        s.status_any = ST_OK;
        s.status = ST_OK;
    }
}

// Slot states of a serving handle.  slot < 0: every slot empty.  idle: the slot is empty (or parked:
// kernels skip it).  Otherwise the slot takes its parameters from prm[slot] and starts afresh
// (outer counter 0, no breakdown), or, with keep_outer, a parked slot is only made runnable again.
__global__ void k_slots_state(GkState* st, const SolveParams* prm, int B, int slot, int idle, int keep_outer) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || (slot >= 0 && b != slot)) return;
    GkState& s = st[b];
    if (idle) {
        s.status = ST_IDLE;
        return;
    }
    if (keep_outer) {
        if (s.status == ST_IDLE) s.status = ST_OK;
        return;
    }
    s.reg = prm[b].reg;
    s.T = prm[b].T;
    s.tau = prm[b].tau;
    s.sqrt_tau = sqrt(prm[b].tau);
    s.eta_delta = prm[b].eta_delta;
    s.r_rel = prm[b].r_rel;
    s.frozen = 0;
    s.R = 0.0;
    s.outer = 0;
    s.status = ST_OK;
    s.status_any = ST_OK;
}

void slots_state(GkState* st, const SolveParams* prm, int B, int slot, bool idle, cudaStream_t s, bool keep_outer) {
    kbegin(KC_GK, s);
    k_slots_state<<<(B + 63) / 64, 64, 0, s>>>(st, prm, B, slot, idle ? 1 : 0, keep_outer ? 1 : 0);
    klaunched("k_slots_state");
    kfinish(s);
}

void set_params(GkState* st, const SolveParams* prm, int B, bool reset_outer, cudaStream_t s) {
    kbegin(KC_GK, s);
    k_set_params<<<(B + 63) / 64, 64, 0, s>>>(st, prm, B, reset_outer ? 1 : 0);
    klaunched("k_set_params");
    kfinish(s);
}

// beta_1 = ||g||, u_1 = g/beta_1 (kept raw), phibar_1 = beta_1 (Algorithm 2 steps 2, 7).
template <typename T>
__global__ void __launch_bounds__(256) k_init_norm(const T* __restrict__ g, int64_t m, GkState* st, Red red) {
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const T* gi = g + (int64_t)inst * m;
    T part = (T)0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < m; i += (int64_t)gridDim.x * 256)
        part = fma(gi[i], gi[i], part);
    double tot;
    if (reduce_last<256>((double)part, red, inst, blockIdx.x, gridDim.x, &tot)) {
        GkState& s = st[inst];
        const double b1 = sqrt(tot);
        s.beta1 = b1;
        s.beta = b1;
        s.beta_new = b1;
        s.phibar = b1;
        s.res2 = 0.0;
        s.iter = 0;
        s.frozen = 0;
        s.cf = 0.0;
        s.cw = 0.0;
        if (!(isfinite(b1) && b1 > 0.0)) {
            s.status = ST_BREAKDOWN;
            s.status_any = ST_BREAKDOWN;
        } else {
            s.status = ST_OK;
            s.c_adj_a = 1.0 / b1;
        }
    }
}

template <typename T>
void gk_init_norm(const T* g, int64_t m, int B, GkState* st, Red red, cudaStream_t s) {
    kbegin(KC_GK, s);
    int nblk = std::min(red_blocks(m), red.max_blocks);
    k_init_norm<T><<<dim3(nblk, B), 256, 0, s>>>(g, m, st, red);
    klaunched("k_init_norm");
    kfinish(s);
}

// alpha_{i+1} = sqrt(v~ . p~) (steps 5 / 13), then the rotations and the update coefficients.
template <typename T, bool INIT>
__global__ void __launch_bounds__(256) k_dot_rotate(const T* __restrict__ v, const T* __restrict__ p, int64_t N,
                                                    GkState* st, Hist hist, Red red) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    if (inner_off(st[inst])) return;
    const T* vi = v + (int64_t)inst * N;
    const T* pi = p + (int64_t)inst * N;
    T part = (T)0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
        part = fma(vi[i], pi[i], part);
    double tot;
    if (!reduce_last<256>((double)part, red, inst, blockIdx.x, gridDim.x, &tot)) return;
    finalize_alpha<INIT>(st[inst], tot, hist, inst);
}

template <typename T>
void gk_dot_rotate(const T* v, const T* p, int64_t N, int B, bool init, GkState* st, Hist hist, Red red,
                   cudaStream_t s) {
    kbegin(KC_GK, s);
    int nblk = std::min(red_blocks(N), red.max_blocks);
    if (init) launch_k(k_dot_rotate<T, true>, dim3(nblk, B), dim3(256), 0, s, v, p, N, st, hist, red);
    else launch_k(k_dot_rotate<T, false>, dim3(nblk, B), dim3(256), 0, s, v, p, N, st, hist, red);
    klaunched("k_dot_rotate");
    kfinish(s);
}

// Steps 19-20: f += (phi/rho) w~, w~ = v~ - (theta/rho) w~ with v~ = v_raw/alpha.
// INIT: f = 0, w~_1 = v~_1 (step 7).
template <typename T, bool INIT>
__global__ void __launch_bounds__(256) k_update(T* __restrict__ f, T* __restrict__ w, const T* __restrict__ v,
                                                int64_t N, const GkState* st) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const GkState& s = st[inst];
    if (parked(s) || (!INIT && inner_off(s))) return;
    const T cv = (T)s.c_upd_v, cf = (T)s.cf, cw = (T)s.cw;
    const int64_t off = (int64_t)inst * N;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
        if (INIT) {
            f[off + i] = (T)0;
            w[off + i] = v[off + i] * cv;
        } else {
            const T wi = w[off + i];
            f[off + i] = fma(cf, wi, f[off + i]);
            w[off + i] = v[off + i] * cv - cw * wi;
        }
    }
}

template <typename T>
void gk_update(T* f, T* w, const T* v, int64_t N, int B, bool init, const GkState* st, cudaStream_t s) {
    kbegin(KC_GK, s);
    int nblk = (int)std::min<int64_t>((N + 1023) / 1024, 2048);
    if (init) launch_k(k_update<T, true>, dim3(nblk, B), dim3(256), 0, s, f, w, v, N, st);
    else launch_k(k_update<T, false>, dim3(nblk, B), dim3(256), 0, s, f, w, v, N, st);
    klaunched("k_update");
    kfinish(s);
}

// ||g - A f^k|| for the outer history; advances the outer step counter.
template <typename T>
__global__ void __launch_bounds__(256) k_resid_norm(const T* __restrict__ g, const T* __restrict__ Af, int64_t m,
                                                    GkState* st, Hist hist, Red red) {
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const T* gi = g + (int64_t)inst * m;
    const T* ai = Af + (int64_t)inst * m;
    T part = (T)0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < m; i += (int64_t)gridDim.x * 256) {
        const T r = gi[i] - ai[i];
        part = fma(r, r, part);
    }
    double tot;
    if (reduce_last<256>((double)part, red, inst, blockIdx.x, gridDim.x, &tot)) {
        GkState& s = st[inst];
        if (hist.resid && s.outer < hist.n_outer) hist.resid[(int64_t)inst * hist.n_outer + s.outer] = sqrt(tot);
        s.outer += 1;
    }
}

template <typename T>
void resid_norm(const T* g, const T* Af, int64_t m, int B, GkState* st, Hist hist, Red red, cudaStream_t s) {
    kbegin(KC_GK, s);
    int nblk = std::min(red_blocks(m), red.max_blocks);
    k_resid_norm<T><<<dim3(nblk, B), 256, 0, s>>>(g, Af, m, st, hist, red);
    klaunched("k_resid_norm");
    kfinish(s);
}

__global__ void k_fill_nan(double* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) p[i] = nan("");
}

void fill_nan(double* p, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    kbegin(KC_GK, s);
    k_fill_nan<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(p, n);
    klaunched("k_fill_nan");
    kfinish(s);
}

// ---- self-test of the bounded wait ------------------------------------------------------------

// The wait of the TMA staging (tma_wait_tile) on an mbarrier that either completes (one plain
// arrival) or never does (an arrival that announces 16 bytes no copy will bring): the second case
// runs out after `limit` polls, twice, and records ST_TIMEOUT in the state.  No copy is ever issued.
__global__ void k_selftest_wait(GkState* st, int complete, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        if (complete) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        else mbar_expect_tx(&bar, 16);
    }
    __syncthreads();
    tma_wait_tile(&bar, st, 0, limit);
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&bar);
}

void selftest_wait(GkState* st, bool complete, uint32_t limit, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(st, complete ? 1 : 0, limit);
    klaunched("k_selftest_wait");
}

// ---- stored Lanczos vectors (reuse for several damping parameters, Sec. 3.3) -------------------

// V_j = v~ / alpha (the normalised basis vector the update of step 7 / 20 uses) and the current
// alpha, beta of the bidiagonalisation (one instance).
template <typename T>
__global__ void __launch_bounds__(256) k_store_basis(const T* __restrict__ v, T* __restrict__ Vj, int64_t N,
                                                     const GkState* st, double* ab, int store_v) {
    const GkState& s = st[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ab[0] = s.alpha;
        ab[1] = s.beta;
    }
    if (!store_v) return;
    const T c = (T)s.c_upd_v;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) Vj[i] = v[i] * c;
}

template <typename T>
void gk_store_basis(const T* v, T* Vj, int64_t N, const GkState* st, double* ab, bool store_v, cudaStream_t s) {
    kbegin(KC_GK, s);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 4096));
    k_store_basis<T><<<blocks, 256, 0, s>>>(v, Vj, N, st, ab, store_v ? 1 : 0);
    klaunched("k_store_basis");
    kfinish(s);
}

// outs[t] = sum_j coef[t][j] V_j for the n_tau <= MT_MAX coefficient rows, one pass over V.
template <typename T>
__global__ void __launch_bounds__(256) k_combine_basis(const T* __restrict__ V, int k, int64_t N,
                                                       const double* __restrict__ coef, int n_tau, OutPtrs<T> outs) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
        T acc[MT_MAX];
#pragma unroll
        for (int t = 0; t < MT_MAX; ++t) acc[t] = (T)0;
        for (int j = 0; j < k; ++j) {
            const T vj = V[(int64_t)j * N + i];
#pragma unroll
            for (int t = 0; t < MT_MAX; ++t)
                if (t < n_tau) acc[t] = fma((T)coef[t * k + j], vj, acc[t]);
        }
#pragma unroll
        for (int t = 0; t < MT_MAX; ++t)
            if (t < n_tau) outs.p[t][i] = acc[t];
    }
}

template <typename T>
void combine_basis(const T* V, int k, int64_t N, const double* coef, int n_tau, const OutPtrs<T>& outs,
                   cudaStream_t s) {
    kbegin(KC_GK, s);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 4096));
    k_combine_basis<T><<<blocks, 256, 0, s>>>(V, k, N, coef, n_tau, outs);
    klaunched("k_combine_basis");
    kfinish(s);
}

#define PLSQR_INST_LSQR(T)                                                                                   \
    template void gk_init_norm<T>(const T*, int64_t, int, GkState*, Red, cudaStream_t);                       \
    template void gk_dot_rotate<T>(const T*, const T*, int64_t, int, bool, GkState*, Hist, Red, cudaStream_t); \
    template void gk_update<T>(T*, T*, const T*, int64_t, int, bool, const GkState*, cudaStream_t);           \
    template void resid_norm<T>(const T*, const T*, int64_t, int, GkState*, Hist, Red, cudaStream_t);         \
    template void gk_store_basis<T>(const T*, T*, int64_t, const GkState*, double*, bool, cudaStream_t);     \
    template void combine_basis<T>(const T*, int, int64_t, const double*, int, const OutPtrs<T>&, cudaStream_t);

PLSQR_INST_LSQR(float)
PLSQR_INST_LSQR(double)

}  // namespace plsqr
