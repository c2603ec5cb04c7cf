// k_mg2d.cu -- the 2D V-cycle launches: the default tile shapes (with plain-load fallbacks), the
// dispatch over the shapes the autotuner picks (k_mg2d_alt.cu and k_mg2d_alt2.cu compile the
// others), and the opt-in one-launch coarse end.
#include "k_mg2d_impl.cuh"

#include <mutex>
#include <set>

namespace plsqr {

PLSQR_MG2D_SHAPE_DECL(, float, true, F0, true)
PLSQR_MG2D_SHAPE_DECL(, double, true, F0, true)
PLSQR_MG2D_SHAPE_DECL(, float, false, C0, true)
PLSQR_MG2D_SHAPE_DECL(, double, false, C0, true)
PLSQR_MG2D_ALT_FINE(extern)
PLSQR_MG2D_ALT_COARSE(extern)

struct TailMaps {
    Maps pre[TAIL_LEVELS - 1], post[TAIL_LEVELS - 1];
};

// Barrier between two phases of the coarse end: the generic-proxy writes of this phase are
// ordered before the TMA reads of the next, and the cluster barrier (release/acquire at cluster
// scope) makes them visible to every block of the cluster.
__device__ __forceinline__ void tail_phase_barrier() {
    fence_proxy_async();
    cluster_barrier();
    fence_proxy_async();
}

// The coarse end of the V-cycle in one launch: levels lc..L-2 (pre-smoothing going down, post-
// smoothing coming up) and the exact solve x = X b on the coarsest level, for one instance per
// cluster of CS blocks.  Each phase spreads the tiles (rows of X) of its level over the blocks of
// the cluster, separated by tail_phase_barrier.  The arithmetic per cell and the summation order
// are those of the per-level kernels and of the coarse symv kernel.
template <typename T, int NU, int CS, bool TMA>
__global__ void __launch_bounds__(TNT) k_mg_tail2d(const __grid_constant__ TailLevels tl,
                                                   const __grid_constant__ TailMaps tm, const T* X, int nc,
                                                   GkState* st) {
    extern __shared__ __align__(128) unsigned char smraw[];
    const int inst = blockIdx.y, rank = blockIdx.x;
    const int nl = tl.n;
    pdl_grid_sync();
    if (inner_off(st[inst])) return;  // the same answer in every block of the cluster
    for (int q = 0; q < nl - 1; ++q) {
        const Dims d = tl.d[q], dc = tl.d[q + 1];
        constexpr int MTX = TailShape::TX, MTY = TailShape::TY;
        const int tx = (d.nx + MTX - 1) / MTX, nt = tx * ((d.ny + MTY - 1) / MTY);
        for (int t = rank; t < nt; t += CS)
            pre_tile<T, false, NU, TMA, 0, TailShape>(smraw, tm.pre[q], (const T*)tl.cond[q], (const T*)tl.b[q],
                                                      (const T*)tl.rd[q], (T*)tl.x[q], (T*)tl.b[q + 1], d, dc, st,
                                                      inst, (t % tx) * MTX, (t / tx) * MTY);
        tail_phase_barrier();
    }
    {
        T* sbv = reinterpret_cast<T*>(smraw);
        const T* bL = (const T*)tl.b[nl - 1] + (int64_t)inst * nc;
        T* xL = (T*)tl.x2[nl - 1] + (int64_t)inst * nc;
        for (int i = threadIdx.x; i < nc; i += TNT) sbv[i] = bL[i];
        __syncthreads();
        const int per = (nc + CS - 1) / CS, r0 = rank * per, r1 = min(nc, r0 + per);
        const int lane = threadIdx.x & 31;
        for (int row = r0 + (threadIdx.x >> 5); row < r1; row += TNT / 32) {
            const T acc = coarse_row_dot<T>(X + (int64_t)inst * nc * nc + (int64_t)row * nc, sbv, nc, lane);
            if (lane == 0) xL[row] = acc;
        }
        __syncthreads();
        tail_phase_barrier();
    }
    for (int q = nl - 2; q >= 0; --q) {
        const Dims d = tl.d[q], dc = tl.d[q + 1];
        constexpr int MTX = TailShape::TX, MTY = TailShape::TY;
        const int tx = (d.nx + MTX - 1) / MTX, nt = tx * ((d.ny + MTY - 1) / MTY);
        for (int t = rank; t < nt; t += CS) {
            post_tile<T, false, NU, false, TMA, 0, TailShape>(smraw, tm.post[q], (const T*)tl.cond[q],
                                                              (const T*)tl.b[q], (const T*)tl.rd[q], (const T*)tl.x[q],
                                                              (T*)tl.x2[q], (const T*)tl.x2[q + 1], d, dc, st, inst,
                                                              (t % tx) * MTX, (t / tx) * MTY, nullptr, 0);
        }
        if (q > 0) tail_phase_barrier();
    }
}

bool mg2d_supported(int ndim, int nu) { return ndim == 2 && nu >= 1 && nu <= 3; }

void max_carveout_set(const void* kfn) {
    static std::mutex mu;
    static std::set<const void*> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(kfn)) return;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        cudaGetLastError();
    done.insert(kfn);
}

constexpr int TAIL_CS = 16;  // blocks per cluster (non-portable size; cudaOccupancyMaxActiveClusters is asked first)

// At least 120 KB per block, so that the blocks of a cluster land on different SMs (the tiles of
// a phase then run in parallel instead of sharing one SM's issue slots).
template <typename T, int NU>
static size_t tail_smem(int nc) {
    return std::max({Tile<T, false, 2 * NU + 1, TailShape>::bytes(), Tile<T, false, 2 * NU, TailShape, true>::bytes(),
                     sizeof(T) * (size_t)nc,
                     (size_t)120 * 1024});
}

template <typename T, int NU>
static cudaLaunchConfig_t tail_config(int B, size_t smem, cudaStream_t s, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(TAIL_CS, B, 1);
    cfg.blockDim = dim3(TNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = TAIL_CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    return cfg;
}

template <typename T, int NU, bool TMA>
static bool tail_prepare_one(int nc) {
    const size_t smem = tail_smem<T, NU>(nc);
    auto kfn = k_mg_tail2d<T, NU, TAIL_CS, TMA>;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = tail_config<T, NU>(1, smem, nullptr, at);
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kfn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

template <typename T, int NU>
static bool tail_prepare(int nc) {
    return tail_prepare_one<T, NU, true>(nc) && tail_prepare_one<T, NU, false>(nc);
}

int mg2d_tail_level(const Dims* d, int L, int nu, size_t elem, int nc) {
    // Opt-in (PLSQR_MG_TAIL=1): on the 1024^2 deblurring workload the cluster barriers and the
    // idle blocks of the small levels made the single launch slower than the per-level launches.
    const char* e = std::getenv("PLSQR_MG_TAIL");
    if (!(e && e[0] == '1') || !mg2d_supported(d[0].ndim, nu) || L < 3) return L;
    int lc = L;
    for (int l = std::max(1, L - TAIL_LEVELS); l < L - 1; ++l) {
        const int nt = ((d[l].nx + TailShape::TX - 1) / TailShape::TX) * ((d[l].ny + TailShape::TY - 1) / TailShape::TY);
        if (nt <= 2 * TAIL_CS) {
            lc = l;
            break;
        }
    }
    if (lc == L) return L;
    bool ok = false;
#define TAIL_PREP(NU_)                                                                  \
    case NU_:                                                                           \
        ok = elem == 8 ? tail_prepare<double, NU_>(nc) : tail_prepare<float, NU_>(nc); \
        break;
    switch (nu) {
        TAIL_PREP(1)
        TAIL_PREP(2)
        TAIL_PREP(3)
    }
#undef TAIL_PREP
    return ok ? lc : L;
}

template <typename T, int NU>
static void tail_launch(const TailLevels& tl, const T* X, int nc, int B, GkState* st, cudaStream_t s) {
    TailMaps tm;
    bool tma = tma_enabled();
    for (int q = 0; q + 1 < tl.n && tma; ++q) {
        const T* c = (const T*)tl.cond[q];
        const T* b = (const T*)tl.b[q];
        const T* rd = (const T*)tl.rd[q];
        tma = make_maps<T, false, 2 * NU + 1, TailShape, false>(tm.pre[q], c, b, rd, nullptr, nullptr, tl.d[q], tl.d[q + 1], B) &&
              make_maps<T, false, 2 * NU, TailShape, true>(tm.post[q], c, b, rd, (const T*)tl.x[q], (const T*)tl.x2[q + 1],
                                                tl.d[q], tl.d[q + 1], B);
    }
    cudaLaunchAttribute at[2];
    const cudaLaunchConfig_t cfg = tail_config<T, NU>(B, tail_smem<T, NU>(nc), s, at);
    const cudaError_t e = tma ? cudaLaunchKernelEx(&cfg, k_mg_tail2d<T, NU, TAIL_CS, true>, tl, tm, X, nc, st)
                              : cudaLaunchKernelEx(&cfg, k_mg_tail2d<T, NU, TAIL_CS, false>, tl, tm, X, nc, st);
    if (e != cudaSuccess) throw std::runtime_error(std::string("mg2d_tail: ") + cudaGetErrorString(e));
}

template <typename T>
void mg2d_tail(const TailLevels& tl, int nu, const T* X, int nc, int B, GkState* st, cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    switch (nu) {
        case 1: tail_launch<T, 1>(tl, X, nc, B, st, s); break;
        case 2: tail_launch<T, 2>(tl, X, nc, B, st, s); break;
        case 3: tail_launch<T, 3>(tl, X, nc, B, st, s); break;
        default: throw std::runtime_error("mg2d_tail: unsupported sweep count");
    }
    klaunched("k_mg_tail2d");
    kfinish(s);
}

template void mg2d_tail<float>(const TailLevels&, int, const float*, int, int, GkState*, cudaStream_t);
template void mg2d_tail<double>(const TailLevels&, int, const double*, int, int, GkState*, cudaStream_t);

bool mg2d_shape(bool fine, int id, int* tx, int* ty, int* nth) {
    int v[3];
    if (fine) {
        switch (id) {
            case 0: v[0] = F0::TX, v[1] = F0::TY, v[2] = F0::NTH; break;
            case 1: v[0] = F1::TX, v[1] = F1::TY, v[2] = F1::NTH; break;
            case 2: v[0] = F2::TX, v[1] = F2::TY, v[2] = F2::NTH; break;
            case 3: v[0] = F3::TX, v[1] = F3::TY, v[2] = F3::NTH; break;
            case 4: v[0] = F4::TX, v[1] = F4::TY, v[2] = F4::NTH; break;
            case 5: v[0] = F5::TX, v[1] = F5::TY, v[2] = F5::NTH; break;
            default: return false;
        }
    } else {
        switch (id) {
            case 0: v[0] = C0::TX, v[1] = C0::TY, v[2] = C0::NTH; break;
            case 1: v[0] = C1::TX, v[1] = C1::TY, v[2] = C1::NTH; break;
            case 2: v[0] = C2::TX, v[1] = C2::TY, v[2] = C2::NTH; break;
            case 3: v[0] = C3::TX, v[1] = C3::TY, v[2] = C3::NTH; break;
            case 4: v[0] = C4::TX, v[1] = C4::TY, v[2] = C4::NTH; break;
            case 5: v[0] = C5::TX, v[1] = C5::TY, v[2] = C5::NTH; break;
            default: return false;
        }
    }
    *tx = v[0], *ty = v[1], *nth = v[2];
    return true;
}

template <typename T>
void mg2d_pre(const T* cond, bool is_kappa, const T* b, const T* rd, T* x, T* bc, Dims d, Dims dc, int nu, int B,
              GkState* st, cudaStream_t s, const __nv_bfloat16* k16, int shape) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
    bool done = false;
    if (is_kappa) {
        if (shape == 1) done = pre_shape<T, true, F1, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, k16);
        if (shape == 2) done = pre_shape<T, true, F2, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, k16);
        if (shape == 3) done = pre_shape<T, true, F3, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, k16);
        if (shape == 4) done = pre_shape<T, true, F4, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, k16);
        if (shape == 5) done = pre_shape<T, true, F5, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, k16);
        if (!done) pre_shape<T, true, F0, true>(cond, b, rd, x, bc, d, dc, nu, B, st, s, k16);
    } else {
        switch (shape) {
            case 1: done = pre_shape<T, false, C1, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, nullptr); break;
            case 2: done = pre_shape<T, false, C2, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, nullptr); break;
            case 3: done = pre_shape<T, false, C3, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, nullptr); break;
            case 4: done = pre_shape<T, false, C4, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, nullptr); break;
            case 5: done = pre_shape<T, false, C5, false>(cond, b, rd, x, bc, d, dc, nu, B, st, s, nullptr); break;
            default: break;
        }
        if (!done) pre_shape<T, false, C0, true>(cond, b, rd, x, bc, d, dc, nu, B, st, s, nullptr);
    }
    klaunched("k_mg_pre2d");
    kfinish(s);
}

template <typename T>
void mg2d_post(const T* cond, bool is_kappa, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d,
               Dims dc, int nu, int B, int dot, GkState* st, Hist hist, Red red, cudaStream_t s,
               const __nv_bfloat16* k16, int shape) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
    bool done = false;
    if (is_kappa) {
        if (shape == 1)
            done = post_shape<T, true, F1, false>(cond, b, rd, xi, x, xc, d, dc, nu, B, dot, st, hist, red, s, k16);
        if (shape == 2)
            done = post_shape<T, true, F2, false>(cond, b, rd, xi, x, xc, d, dc, nu, B, dot, st, hist, red, s, k16);
        if (shape == 3)
            done = post_shape<T, true, F3, false>(cond, b, rd, xi, x, xc, d, dc, nu, B, dot, st, hist, red, s, k16);
        if (shape == 4)
            done = post_shape<T, true, F4, false>(cond, b, rd, xi, x, xc, d, dc, nu, B, dot, st, hist, red, s, k16);
        if (shape == 5)
            done = post_shape<T, true, F5, false>(cond, b, rd, xi, x, xc, d, dc, nu, B, dot, st, hist, red, s, k16);
        if (!done) post_shape<T, true, F0, true>(cond, b, rd, xi, x, xc, d, dc, nu, B, dot, st, hist, red, s, k16);
    } else {
        switch (shape) {
#define POST_ALT(ID, S_)                                                                                             \
    case ID:                                                                                                         \
        done = post_shape<T, false, S_, false>(cond, b, rd, xi, x, xc, d, dc, nu, B, 0, st, hist, red, s, nullptr); \
        break;
            POST_ALT(1, C1)
            POST_ALT(2, C2)
            POST_ALT(3, C3)
            POST_ALT(4, C4)
            POST_ALT(5, C5)
#undef POST_ALT
            default: break;
        }
        if (!done) post_shape<T, false, C0, true>(cond, b, rd, xi, x, xc, d, dc, nu, B, 0, st, hist, red, s, nullptr);
    }
    klaunched("k_mg_post2d");
    kfinish(s);
}

template void mg2d_pre<float>(const float*, bool, const float*, const float*, float*, float*, Dims, Dims, int, int,
                              GkState*, cudaStream_t, const __nv_bfloat16*, int);
template void mg2d_pre<double>(const double*, bool, const double*, const double*, double*, double*, Dims, Dims, int,
                               int, GkState*, cudaStream_t, const __nv_bfloat16*, int);
template void mg2d_post<float>(const float*, bool, const float*, const float*, const float*, float*, const float*,
                               Dims, Dims, int, int, int, GkState*, Hist, Red, cudaStream_t, const __nv_bfloat16*,
                               int);
template void mg2d_post<double>(const double*, bool, const double*, const double*, const double*, double*,
                                const double*, Dims, Dims, int, int, int, GkState*, Hist, Red, cudaStream_t,
                                const __nv_bfloat16*, int);

}  // namespace plsqr
