// k_mg2d_coop.cu -- the whole 2D V-cycle (Sec. 4.2 priorconditioner) in one cooperative launch.
//
// The per-level schedule launches two kernels per level (pre- and post-smoothing) and one for the
// coarse solve: 2 (L - 1) + 1 dependent launches per application, most of them on levels too
// small to fill the GPU, so at batch 1 every launch costs its own latency.  Here one persistent
// grid, all of whose blocks are resident at once (cooperative launch), walks the phases of the
// V-cycle -- pre-smoothing of levels 0 .. L-2, the exact solve on level L-1, post-smoothing of
// levels L-2 .. 0 -- and separates them by a grid-wide barrier.  A phase spreads the tiles of its
// level (of every instance of the batch) over the blocks.  Each tile runs the same device
// functions as the per-level kernels (pre_tile / post_tile with the same tile shapes), the coarse
// rows the same dot products as k_coarse_symv, and alpha (Algorithm 2 step 13) the same
// per-tile partial sums and reduction, so the result is the per-level schedule's bit for bit.
//
// The barrier is a counter in device memory: every block adds one when it arrives and waits until
// the counter reaches the number of blocks times the phase.  Every wait is bounded; a barrier that
// runs out records ST_TIMEOUT in every instance's state and the blocks return.  The last block to
// leave resets the counter for the next launch.
#include "k_mg2d_impl.cuh"

namespace plsqr {

constexpr uint32_t COOP_WAIT_LIMIT = 1u << 22;  // polls of one barrier wait (seconds at most)

// TMA maps of every smoothed level (pre- and post-smoothing boxes differ in their halo).
struct CoopMaps {
    Maps pre[COOP_LEVELS - 1], post[COOP_LEVELS - 1];
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `phase` (1, 2, ...).  The generic-proxy writes of the phase before it are
// ordered before the TMA (async-proxy) reads of the phase after it, in every block.  Returns false
// in every thread of a block whose wait ran out (or that found the abort flag set).
__device__ __forceinline__ bool coop_barrier(const CoopSync& sy, unsigned phase, GkState* st, int B) {
    __shared__ int ok;
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(sy.arrive, 1u);
        const unsigned target = phase * gridDim.x;
        bool good = true;
        uint32_t n = 0;
        while (ld_acquire_gpu(sy.arrive) < target) {
            if (++n > COOP_WAIT_LIMIT || *(volatile int*)sy.abort) {
                good = false;
                break;
            }
        }
        __threadfence();
        if (!good) {
            atomicExch(sy.abort, 1);
            for (int i = 0; i < B; ++i) {
                st[i].status = ST_TIMEOUT;
                st[i].status_any = ST_TIMEOUT;
            }
        }
        ok = good;
    }
    __syncthreads();
    fence_proxy_async();
    return ok != 0;
}

// Every block leaves through here: the last one resets the counters for the next launch.
__device__ __forceinline__ void coop_depart(const CoopSync& sy) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicAdd(sy.depart, 1u);
        if (old == gridDim.x - 1) {
            *sy.arrive = 0u;
            *sy.depart = 0u;
            *sy.abort = 0;
            __threadfence();
        }
    }
}

// DOTM: 0 no dot product, 1 alpha_1 (Algorithm 2 step 5), 2 alpha_{i+1} and the rotations
// (steps 13-17) fused into the finest post-smoothing tiles.  SF: tile shape of level 0, SC: of the
// coarser levels (both with NTH threads).
template <typename T, int NU, int DOTM, class SF, class SC>
__global__ void __launch_bounds__(SF::NTH) k_vcycle_coop(const __grid_constant__ CoopLevels cl,
                                                         const __grid_constant__ CoopMaps cm, const T* __restrict__ X,
                                                         int nc, int B, int lc, GkState* st, Hist hist, Red red,
                                                         CoopSync sy, const __nv_bfloat16* __restrict__ k16) {
    static_assert(SF::NTH == SC::NTH, "one block size for every phase");
    constexpr int NTH = SF::NTH;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int L = cl.L;
    unsigned phase = 0;
    // pre-smoothing, first level lc first; each tile also restricts its residual to the level below
    for (int l = lc; l < L - 1; ++l) {
        const Dims d = cl.d[l], dc = cl.d[l + 1];
        if (l == 0) {
            const int tx = (d.nx + SF::TX - 1) / SF::TX, nt = tx * ((d.ny + SF::TY - 1) / SF::TY);
            for (int u = blockIdx.x; u < nt * B; u += gridDim.x) {
                const int inst = u / nt, t = u - inst * nt;
                pre_tile<T, true, NU, true, 1, SF>(smraw, cm.pre[0], (const T*)cl.cond[0], (const T*)cl.b[0],
                                                   (const T*)cl.rd[0], (T*)cl.x[0], (T*)cl.b[1], d, dc, st, inst,
                                                   (t % tx) * SF::TX, (t / tx) * SF::TY, k16);
            }
        } else {
            const int tx = (d.nx + SC::TX - 1) / SC::TX, nt = tx * ((d.ny + SC::TY - 1) / SC::TY);
            for (int u = blockIdx.x; u < nt * B; u += gridDim.x) {
                const int inst = u / nt, t = u - inst * nt;
                pre_tile<T, false, NU, true, 1, SC>(smraw, cm.pre[l], (const T*)cl.cond[l], (const T*)cl.b[l],
                                                    (const T*)cl.rd[l], (T*)cl.x[l], (T*)cl.b[l + 1], d, dc, st,
                                                    inst, (t % tx) * SC::TX, (t / tx) * SC::TY);
            }
        }
        if (!coop_barrier(sy, ++phase, st, B)) {
            coop_depart(sy);
            return;
        }
    }
    {  // exact solve on the coarsest level: x = X b, eight rows per block (as k_coarse_symv)
        T* sbv = reinterpret_cast<T*>(smraw);
        const int groups = (nc + 7) / 8;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int u = blockIdx.x; u < groups * B; u += gridDim.x) {
            const int inst = u / groups, grp = u - inst * groups;
            if (parked(st[inst]) || st[inst].frozen >= 2) continue;  // the same answer in every thread
            const T* b = (const T*)cl.b[L - 1] + (int64_t)inst * nc;
            __syncthreads();  // the previous unit's reads of sbv are done
            for (int i = threadIdx.x; i < nc; i += NTH) sbv[i] = b[i];
            __syncthreads();
            for (int row = grp * 8 + w; row < min(nc, grp * 8 + 8); row += NTH / 32) {
                const T acc = coarse_row_dot<T>(X + (int64_t)inst * nc * nc + (int64_t)row * nc, sbv, nc, lane);
                if (lane == 0) ((T*)cl.x2[L - 1])[(int64_t)inst * nc + row] = acc;
            }
        }
        if (lc < L - 1 && !coop_barrier(sy, ++phase, st, B)) {
            coop_depart(sy);
            return;
        }
    }
    // post-smoothing, coarsest smoothed level first
    for (int l = L - 2; l >= max(lc, 1); --l) {
        const Dims d = cl.d[l], dc = cl.d[l + 1];
        const int tx = (d.nx + SC::TX - 1) / SC::TX, nt = tx * ((d.ny + SC::TY - 1) / SC::TY);
        for (int u = blockIdx.x; u < nt * B; u += gridDim.x) {
            const int inst = u / nt, t = u - inst * nt;
            post_tile<T, false, NU, false, true, 1, SC>(smraw, cm.post[l], (const T*)cl.cond[l], (const T*)cl.b[l],
                                                        (const T*)cl.rd[l], (const T*)cl.x[l], (T*)cl.x2[l],
                                                        (const T*)cl.x2[l + 1], d, dc, st, inst, (t % tx) * SC::TX,
                                                        (t / tx) * SC::TY, nullptr, 0);
        }
        if (l == lc) break;  // the last phase of a launch that starts below the finest level
        if (!coop_barrier(sy, ++phase, st, B)) {
            coop_depart(sy);
            return;
        }
    }
    if (lc == 0) {  // finest level, with alpha: per-tile partials reduced in tile order by the last tile
        const Dims d = cl.d[0], dc = cl.d[1];
        const int tx = (d.nx + SF::TX - 1) / SF::TX, nt = tx * ((d.ny + SF::TY - 1) / SF::TY);
        for (int u = blockIdx.x; u < nt * B; u += gridDim.x) {
            const int inst = u / nt, t = u - inst * nt;
            const int nseg = (d.nx + 31) / 32;
            if (!post_tile<T, true, NU, DOTM != 0, true, DOTM != 0 ? 2 : 1, SF>(
                    smraw, cm.post[0], (const T*)cl.cond[0], (const T*)cl.b[0], (const T*)cl.rd[0],
                    (const T*)cl.x[0], (T*)cl.x2[0], (const T*)cl.x2[1], d, dc, st, inst, (t % tx) * SF::TX,
                    (t / tx) * SF::TY, DOTM != 0 ? red.partials + (int64_t)inst * red.max_blocks : nullptr, nseg,
                    k16))
                continue;
            if (DOTM != 0) {
                double tot;
                if (sum_partials_last<NTH>(red, inst, nt, ((d.ny + 15) / 16) * nseg, &tot))
                    finalize_alpha<DOTM == 1>(st[inst], tot, hist, inst);
            }
        }
    }
    coop_depart(sy);
}

using CoopF = F1;  // 32 x 32 tiles, 256 threads
using CoopC = C3;  // 16 x 16 tiles, 256 threads

template <typename T, int NU>
static size_t coop_smem(int nc) {
    return std::max({Tile<T, true, 2 * NU + 1, CoopF>::bytes(), Tile<T, true, 2 * NU, CoopF, true>::bytes(),
                     Tile<T, false, 2 * NU + 1, CoopC>::bytes(), Tile<T, false, 2 * NU, CoopC, true>::bytes(),
                     sizeof(T) * (size_t)nc});
}

template <typename T, int NU, int DOTM>
static auto coop_kernel() {
    return k_vcycle_coop<T, NU, DOTM, CoopF, CoopC>;
}

// The coarse right-hand side is staged whole: only where it fits beside the tiles.
template <typename T, int NU>
static bool coop_fits(int nc) {
    return sizeof(T) * (size_t)nc <= std::max(Tile<T, true, 2 * NU, CoopF, true>::bytes(),
                                              Tile<T, false, 2 * NU, CoopC, true>::bytes());
}

// Blocks of one launch: every block resident at once (the occupancy of the kernel times the SMs),
// at most `cap` (0: no cap; fewer blocks make the barriers cheaper), and no more than the largest
// phase from level lc down has work units.
template <typename T, int NU, int DOTM>
static int coop_blocks(const CoopLevels& cl, int lc, int cap, int nc, int B) {
    if (!coop_fits<T, NU>(nc)) return 0;
    const size_t smem = coop_smem<T, NU>(nc);
    auto kfn = coop_kernel<T, NU, DOTM>();
    int dev = 0, sms = 0, ps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kfn, CoopF::NTH, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (ps <= 0) return 0;
    int64_t work = 0;
    for (int l = lc; l < cl.L - 1; ++l) {
        const int tw = l == 0 ? CoopF::TX : CoopC::TX, th = l == 0 ? CoopF::TY : CoopC::TY;
        work = std::max<int64_t>(work, (int64_t)B * ((cl.d[l].nx + tw - 1) / tw) * ((cl.d[l].ny + th - 1) / th));
    }
    work = std::max<int64_t>(work, (int64_t)B * ((nc + 7) / 8));
    int64_t n = std::min<int64_t>((int64_t)ps * sms, work);
    if (cap > 0) n = std::min<int64_t>(n, cap);
    return (int)n;
}

bool mg2d_coop_supported(int nu, size_t elem, int L, int nc) {
    if (nu != 2 || L < 2 || L > COOP_LEVELS) return false;
    CoopLevels cl{};
    cl.L = 1;
    return (elem == 8 ? coop_blocks<double, 2, 2>(cl, 0, 0, nc, 1) : coop_blocks<float, 2, 2>(cl, 0, 0, nc, 1)) > 0;
}

template <typename T, int NU, int DOTM>
static void coop_launch(const CoopLevels& cl, int lc, int cap, const T* X, int nc, int B, GkState* st, Hist hist,
                        Red red, CoopSync sy, const __nv_bfloat16* k16, cudaStream_t s) {
    CoopMaps cm;
    bool ok = true;
    for (int l = lc; l + 1 < cl.L && ok; ++l) {
        const T* c = (const T*)cl.cond[l];
        const T* b = (const T*)cl.b[l];
        const T* rd = (const T*)cl.rd[l];
        if (l == 0)
            ok = make_maps<T, true, 2 * NU + 1, CoopF, false>(cm.pre[0], c, b, rd, nullptr, nullptr, cl.d[0], cl.d[1],
                                                             B) &&
                 make_maps<T, true, 2 * NU, CoopF, true>(cm.post[0], c, b, rd, (const T*)cl.x[0],
                                                         (const T*)cl.x2[1], cl.d[0], cl.d[1], B);
        else
            ok = make_maps<T, false, 2 * NU + 1, CoopC, false>(cm.pre[l], c, b, rd, nullptr, nullptr, cl.d[l],
                                                              cl.d[l + 1], B) &&
                 make_maps<T, false, 2 * NU, CoopC, true>(cm.post[l], c, b, rd, (const T*)cl.x[l],
                                                          (const T*)cl.x2[l + 1], cl.d[l], cl.d[l + 1], B);
    }
    if (!ok) throw std::runtime_error("vcycle_coop: tensor maps unavailable for this layout");
    const int blocks = coop_blocks<T, NU, DOTM>(cl, lc, cap, nc, B);
    if (blocks <= 0) throw std::runtime_error("vcycle_coop: no resident blocks");
    if (DOTM != 0 && (int64_t)((cl.d[0].ny + 15) / 16) * ((cl.d[0].nx + 31) / 32) > red.max_blocks)
        throw std::runtime_error("vcycle_coop: too many segments for the reduction scratch");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(CoopF::NTH);
    cfg.dynamicSmemBytes = coop_smem<T, NU>(nc);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e =
        cudaLaunchKernelEx(&cfg, coop_kernel<T, NU, DOTM>(), cl, cm, X, nc, B, lc, st, hist, red, sy, k16);
    if (e != cudaSuccess) throw std::runtime_error(std::string("vcycle_coop: ") + cudaGetErrorString(e));
}

template <typename T>
void mg2d_vcycle_coop(const CoopLevels& cl, int lc, int cap, int nu, const T* X, int nc, int B, int dot,
                      GkState* st, Hist hist, Red red, CoopSync sy, const __nv_bfloat16* k16, cudaStream_t s) {
    if (nu != 2) throw std::runtime_error("vcycle_coop: unsupported sweep count");
    if (lc < 0 || lc > cl.L - 2) throw std::runtime_error("vcycle_coop: bad first level");
    if (lc > 0) dot = 0;  // alpha belongs to the finest level's launch
    kbegin(lc == 0 ? KC_GS_FINE : KC_MG_OTHER, s);
    switch (dot) {
        case 0: coop_launch<T, 2, 0>(cl, lc, cap, X, nc, B, st, hist, red, sy, k16, s); break;
        case 1: coop_launch<T, 2, 1>(cl, lc, cap, X, nc, B, st, hist, red, sy, k16, s); break;
        default: coop_launch<T, 2, 2>(cl, lc, cap, X, nc, B, st, hist, red, sy, k16, s); break;
    }
    klaunched("k_vcycle_coop");
    kfinish(s);
}

template void mg2d_vcycle_coop<float>(const CoopLevels&, int, int, int, const float*, int, int, int, GkState*, Hist,
                                      Red, CoopSync, const __nv_bfloat16*, cudaStream_t);
template void mg2d_vcycle_coop<double>(const CoopLevels&, int, int, int, const double*, int, int, int, GkState*,
                                       Hist, Red, CoopSync, const __nv_bfloat16*, cudaStream_t);

}  // namespace plsqr
