// k_mg2d.cu -- temporally blocked V-cycle kernels for 2D grids (Sec. 4.2 priorconditioner).
//
// A block owns a 64 x 32 tile of one level and stages the tile plus a halo of the right-hand
// side, the edge conductances and (post-smoothing) the iterate in shared memory, with TMA tile
// copies when the layout allows (zero fill outside the domain) and plain loads otherwise.
// Red-black Gauss-Seidel half sweeps then run entirely in shared memory: a cell updated in half
// sweep s needs neighbours from half sweep s-1, so after s half sweeps the values are exact on
// the region s cells inside the staged one.  With a halo H = 2 nu + 1 the pre-smoothing kernel
// also forms the residual on the tile and restricts it (sum of the 2 x 2 children); with
// H = 2 nu the post-smoothing kernel prolongs the coarse correction and smooths.  The arithmetic
// per cell is the same as in the one-half-sweep-per-launch kernels and the oracle: cells outside
// the domain are staged as zeros, which reproduces the zero ghost values beyond the high end,
// the missing edges at the low end and the summation order.  One launch replaces 2 nu + 1 (pre)
// or 2 nu + 1 (post) launches, and the iterate and coefficients are read from memory once per
// tile instead of once per half sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <stdexcept>
#include <string>

#include "kernels.cuh"
#include "tma.cuh"

namespace plsqr {

// Tile extent; threads per block on the finest level (many tiles), on the coarser levels (few
// tiles: more threads per tile) and in the one-launch coarse end.
constexpr int MTX = 64, MTY = 32, MNT = 256, CNT = 1024, TNT = 1024;

// Tile geometry: logical halo H on both axes; in storage the x halo is HX >= H (HX * sizeof(T)
// a multiple of 16 bytes, the TMA rule for the innermost coordinate), so logical column lx is
// stored at lx + OX.  Arrays: sb, scx, scy (scy == scx on the finest level), sx, sd (1 / diagonal)
// and, for post-smoothing (XC), the box of coarse-level cells that are parents of staged cells.
template <typename T, bool L0, int H, bool XC = false>
struct Tile {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int HX = ((H + VEC - 1) / VEC) * VEC, OX = HX - H;
    static constexpr int LX = MTX + 2 * H, LY = MTY + 2 * H;  // logical extents
    static constexpr int LXS = MTX + 2 * HX;                  // storage pitch
    static constexpr int NCS = LY * LXS;                      // one staged plane
    static constexpr int NCP = ((NCS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);  // 128-byte padded
    static constexpr int CPLANES = L0 ? 1 : 2;
    // Coarse box: it starts XB coarse columns and YB coarse rows before the parent (x0/2, y0/2)
    // of the tile's first cell (XB a multiple of VEC, so the copy's x stays 16-byte aligned).
    // The parent of staged cell (ly, lxs) is box cell ((ly + (H & 1)) >> 1, (lxs + 2 XB - HX) >> 1).
    static constexpr int XB = (((HX + 1) / 2 + VEC - 1) / VEC) * VEC;
    static constexpr int XW = ((((MTX + HX - 1) >> 1) + XB + 1 + VEC - 1) / VEC) * VEC;
    static constexpr int YB = (H + 1) / 2;
    static constexpr int YW = ((MTY + H - 1) >> 1) + YB + 1;
    static constexpr int NXC = XC ? ((XW * YW * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T) : 0;
    // layout: sb [NCP] | scx, scy [CPLANES * NCS, padded] | sx [NCP] | sd [NCP] | sxc [NXC] | mbarrier
    static constexpr int OFF_C = NCP;
    static constexpr int OFF_X = NCP + ((CPLANES * NCS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    static constexpr int OFF_D = OFF_X + NCP;
    static constexpr int OFF_XC = OFF_D + NCP;
    static constexpr int OFF_BAR = OFF_XC + NXC;
    static constexpr size_t bytes() { return sizeof(T) * (size_t)OFF_BAR + 16; }
};

struct Maps {
    CUtensorMap b, c, x, d, xc;
};

// Stage b, the conductances, the reciprocal diagonal rd and x_in when X_IN (x = 0 otherwise),
// and the coarse box of xc when XC.  k16 (finest level only, may be null): kappa stored in
// bfloat16, read with plain loads and widened in shared memory.  The copies are issued first;
// the instance state is read while they are in flight.  Returns whether the block skips the
// tile (SKIP 1: a parked or frozen instance, 2: an instance whose inner iteration is off, 0:
// never), the same answer in every thread.  Ends with a barrier.
template <typename T, bool L0, int H, bool TMA, bool X_IN, bool XC, int SKIP, int NTH>
__device__ __forceinline__ bool stage(T* sm, const Maps& maps, const T* __restrict__ cond, const T* __restrict__ b,
                                      const T* __restrict__ rd, const T* __restrict__ x_in,
                                      const T* __restrict__ xc, const Dims& d, const Dims& dc, int inst, int x0,
                                      int y0, GkState* st, const __nv_bfloat16* __restrict__ k16) {
    using TL = Tile<T, L0, H, XC>;
    T* sb = sm;
    T* sc = sm + TL::OFF_C;
    T* sx = sm + TL::OFF_X;
    T* sd = sm + TL::OFF_D;
    T* sxc = sm + TL::OFF_XC;
    auto skip_of = [&]() {
        if (SKIP == 1) return parked(st[inst]) || st[inst].frozen >= 2;
        if (SKIP == 2) return inner_off(st[inst]);
        return false;
    };
    if constexpr (TMA) {
        uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TL::OFF_BAR);
        const bool kb = L0 && k16;
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            const uint32_t plane = TL::NCS * sizeof(T);
            mbar_expect_tx(bar, plane * (2 + (kb ? 0 : TL::CPLANES) + (X_IN ? 1 : 0)) +
                                    (XC ? (uint32_t)(TL::XW * TL::YW * sizeof(T)) : 0u));
            const int gx = x0 - TL::HX, gy = y0 - H;
            tma_load_3d(sb, &maps.b, bar, gx, gy, inst);
            tma_load_3d(sd, &maps.d, bar, gx, gy, inst);
            if (!kb) tma_load_3d(sc, &maps.c, bar, gx, gy, L0 ? inst : 2 * inst);
            if (X_IN) tma_load_3d(sx, &maps.x, bar, gx, gy, inst);
            if (XC) tma_load_3d(sxc, &maps.xc, bar, (x0 >> 1) - TL::XB, (y0 >> 1) - TL::YB, inst);
        }
        const bool skip = skip_of();
        if (!X_IN)
            for (int i = threadIdx.x; i < TL::NCS; i += NTH) sx[i] = (T)0;
        if (kb) {  // meanwhile, kappa from bfloat16 (zero outside the domain, like the TMA fill)
            const __nv_bfloat16* k = k16 + (int64_t)inst * d.N;
            for (int i = threadIdx.x; i < TL::NCS; i += NTH) {
                const int ly = i / TL::LXS, lxs = i - ly * TL::LXS;
                const int gy = y0 - H + ly, gx = x0 - TL::HX + lxs;
                sc[i] = (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny && !skip)
                            ? (T)__bfloat162float(k[(int64_t)gy * d.nx + gx])
                            : (T)0;
            }
        }
        __syncthreads();  // the barrier's initialisation is visible to every thread
        tma_wait_tile(bar, st, inst);
        __syncthreads();
        if (threadIdx.x == 0) mbar_inval(bar);  // the next tile of this block initialises it again
        return skip;
    } else {
        if (skip_of()) return true;
        const int64_t off = (int64_t)inst * d.N;
        const T* c = cond + (L0 ? off : (int64_t)inst * 2 * d.N);
        for (int i = threadIdx.x; i < TL::NCS; i += NTH) {
            const int ly = i / TL::LXS, lxs = i - ly * TL::LXS;
            const int gy = y0 - H + ly, gx = x0 - TL::HX + lxs;
            T vb = (T)0, vx = (T)0, vy = (T)0, vv = (T)0, vd = (T)0;
            if (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny) {
                const int64_t g = (int64_t)gy * d.nx + gx;
                vb = b[off + g];
                vd = rd[off + g];
                vx = (L0 && k16) ? (T)__bfloat162float(k16[off + g]) : c[g];
                if (!L0) vy = c[d.N + g];
                if (X_IN) vv = x_in[off + g];
            }
            sb[i] = vb;
            sd[i] = vd;
            sc[i] = vx;
            if (!L0) sc[TL::NCS + i] = vy;
            sx[i] = vv;
        }
        if (XC) {
            const int64_t offc = (int64_t)inst * dc.N;
            for (int q = threadIdx.x; q < TL::XW * TL::YW; q += NTH) {
                const int cy = q / TL::XW, cx = q - cy * TL::XW;
                const int gy = (y0 >> 1) - TL::YB + cy, gx = (x0 >> 1) - TL::XB + cx;
                sxc[q] = (gx >= 0 && gx < dc.nx && gy >= 0 && gy < dc.ny) ? xc[offc + (int64_t)gy * dc.nx + gx]
                                                                          : (T)0;
            }
        }
        __syncthreads();
        return false;
    }
}

// One half sweep of `colour` over the logical cells at distance >= lo from the staged edge:
// x = (b + off) * sd.  Cells outside the domain have b = 0 and sd = 0 and stay 0.  Tiles start
// at even global coordinates (x0, y0 multiples of the tile extents) and the halo is the same on
// both axes, so the colour of logical cell (lx, ly), (gx + gy) mod 2, is (lx + ly) mod 2.
template <typename T, int LX, int LY, int LXS, int OX, int NTH>
__device__ __forceinline__ void half_sweep(const T* sb, const T* sd, const T* scx, const T* scy, T* sx, int lo,
                                          int colour) {
    const int hi = LX - 1 - lo, hiy = LY - 1 - lo;
    const int half = (hi - lo + 2) >> 1;
    const int rows = hiy - lo + 1;
    for (int k = threadIdx.x; k < rows * half; k += NTH) {
        const int ry = k / half, j = k - ry * half;
        const int ly = lo + ry;
        const int lx = lo + ((colour ^ ly ^ lo) & 1) + 2 * j;  // first lx >= lo of the colour, then every other
        if (lx > hi) continue;
        const int i = ly * LXS + lx + OX;
        T off = scx[i] * sx[i + 1];
        off += scx[i - 1] * sx[i - 1];
        off += scy[i] * sx[i + LXS];
        off += scy[i - LXS] * sx[i - LXS];
        sx[i] = (sb[i] + off) * sd[i];
    }
}

// Pre-smoothing of one tile from x = 0 (nu red->black sweeps), residual and restriction to bc.
// Returns false when the block skips the tile (see stage).  Ends with a barrier, so that a block
// can go on with another tile.
template <typename T, bool L0, int NU, bool TMA, int SKIP, int NTH>
__device__ __forceinline__ bool pre_tile(unsigned char* smraw, const Maps& maps, const T* cond, const T* b,
                                         const T* rd, T* x, T* bc, const Dims& d, const Dims& dc, GkState* st,
                                         int inst, int x0, int y0, const __nv_bfloat16* k16 = nullptr) {
    constexpr int H = 2 * NU + 1;
    using TL = Tile<T, L0, H>;
    constexpr int LXS = TL::LXS, OX = TL::OX;
    T* sm = reinterpret_cast<T*>(smraw);
    T* sb = sm;
    T* scx = sm + TL::OFF_C;
    T* scy = L0 ? scx : scx + TL::NCS;
    T* sx = sm + TL::OFF_X;
    const T* sd = sm + TL::OFF_D;
    if (stage<T, L0, H, TMA, false, false, SKIP, NTH>(sm, maps, cond, b, rd, nullptr, nullptr, d, dc, inst, x0, y0,
                                                      st, k16))
        return false;
#pragma unroll
    for (int s = 0; s < 2 * NU; ++s) {
        half_sweep<T, TL::LX, TL::LY, LXS, OX, NTH>(sb, sd, scx, scy, sx, s + 1, s & 1);
        __syncthreads();
    }
    // residual r = b - (diag x - off) on the tile, summed over the 2 x 2 children
    const int64_t offc = (int64_t)inst * dc.N;
    for (int k = threadIdx.x; k < (MTX / 2) * (MTY / 2); k += NTH) {
        const int cy = k / (MTX / 2), cx = k - cy * (MTX / 2);
        const int X = (x0 >> 1) + cx, Y = (y0 >> 1) + cy;
        if (X >= dc.nx || Y >= dc.ny) continue;
        T sum = (T)0;
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                const int i = (H + 2 * cy + oy) * LXS + (H + 2 * cx + ox) + OX;
                T diag = scx[i];
                diag += scx[i - 1];
                diag += scy[i];
                diag += scy[i - LXS];
                T off = scx[i] * sx[i + 1];
                off += scx[i - 1] * sx[i - 1];
                off += scy[i] * sx[i + LXS];
                off += scy[i - LXS] * sx[i - LXS];
                sum += sb[i] - (diag * sx[i] - off);
            }
        bc[offc + (int64_t)Y * dc.nx + X] = sum;
    }
    const int64_t off = (int64_t)inst * d.N;
    for (int k = threadIdx.x; k < MTX * MTY; k += NTH) {
        const int ty = k / MTX, tx = k - ty * MTX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < d.nx && gy < d.ny) x[off + (int64_t)gy * d.nx + gx] = sx[(H + ty) * LXS + H + tx + OX];
    }
    __syncthreads();
    return true;
}

template <typename T, bool L0, int NU, bool TMA, int NTH>
__global__ void __launch_bounds__(NTH) k_mg_pre2d(const __grid_constant__ Maps maps, const T* __restrict__ cond,
                                                  const T* __restrict__ b, const T* __restrict__ rd,
                                                  T* __restrict__ x, T* __restrict__ bc, Dims d, Dims dc, GkState* st,
                                                  const __nv_bfloat16* __restrict__ k16) {
    extern __shared__ __align__(128) unsigned char smraw[];
    pdl_grid_sync();
    pre_tile<T, L0, NU, TMA, 1, NTH>(smraw, maps, cond, b, rd, x, bc, d, dc, st, blockIdx.z, blockIdx.x * MTX,
                                     blockIdx.y * MTY, k16);
}

// One tile of x_out = smooth(x_in + P xc) with nu black->red sweeps (x_in and x_out must differ:
// blocks read neighbouring tiles of x_in as halo).  Returns false when the block skips the tile
// (see stage); *part is this thread's share of x_out . b over the tile when DOT.  Ends with a
// barrier.
template <typename T, bool L0, int NU, bool DOT, bool TMA, int SKIP, int NTH>
__device__ __forceinline__ bool post_tile(unsigned char* smraw, const Maps& maps, const T* cond, const T* b,
                                          const T* rd, const T* x_in, T* x_out, const T* xc, const Dims& d,
                                          const Dims& dc, GkState* st, int inst, int x0, int y0, T* part_out,
                                          const __nv_bfloat16* k16 = nullptr) {
    constexpr int H = 2 * NU;
    using TL = Tile<T, L0, H, true>;
    constexpr int LXS = TL::LXS, OX = TL::OX;
    T* sm = reinterpret_cast<T*>(smraw);
    T* sb = sm;
    T* scx = sm + TL::OFF_C;
    T* scy = L0 ? scx : scx + TL::NCS;
    T* sx = sm + TL::OFF_X;
    const T* sd = sm + TL::OFF_D;
    const T* sxc = sm + TL::OFF_XC;
    if (stage<T, L0, H, TMA, true, true, SKIP, NTH>(sm, maps, cond, b, rd, x_in, xc, d, dc, inst, x0, y0, st, k16))
        return false;
    // + P xc.  The extents are even (2^(levels-1) divides them), so a cell outside the domain has
    // its parent outside the coarse grid: it adds the zero fill and stays 0.
    for (int i = threadIdx.x; i < TL::NCS; i += NTH) {
        const int ly = i / LXS, lxs = i - ly * LXS;
        sx[i] = sx[i] + sxc[((ly + (H & 1)) >> 1) * TL::XW + ((lxs + 2 * TL::XB - TL::HX) >> 1)];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2 * NU; ++s) {
        half_sweep<T, TL::LX, TL::LY, LXS, OX, NTH>(sb, sd, scx, scy, sx, s + 1, 1 - (s & 1));
        __syncthreads();
    }
    const int64_t off = (int64_t)inst * d.N;
    T part = (T)0;
    for (int k = threadIdx.x; k < MTX * MTY; k += NTH) {
        const int ty = k / MTX, tx = k - ty * MTX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < d.nx && gy < d.ny) {
            const int i = (H + ty) * LXS + H + tx + OX;
            x_out[off + (int64_t)gy * d.nx + gx] = sx[i];
            if (DOT) part = fma(sx[i], sb[i], part);
        }
    }
    __syncthreads();
    *part_out = part;
    return true;
}

// DOT: also alpha = sqrt(x_out . b) and the rotations (finest level of the last V-cycle:
// x_out = v~, b = p~).
template <typename T, bool L0, int NU, bool DOT, bool INIT, bool TMA, int NTH>
__global__ void __launch_bounds__(NTH) k_mg_post2d(const __grid_constant__ Maps maps, const T* __restrict__ cond,
                                                   const T* __restrict__ b, const T* __restrict__ rd,
                                                   const T* __restrict__ x_in, T* __restrict__ x_out,
                                                   const T* __restrict__ xc, Dims d, Dims dc, GkState* st, Hist hist,
                                                   Red red, const __nv_bfloat16* __restrict__ k16) {
    extern __shared__ __align__(128) unsigned char smraw[];
    const int inst = blockIdx.z;
    pdl_grid_sync();
    T part;
    if (!post_tile<T, L0, NU, DOT, TMA, DOT ? 2 : 1, NTH>(smraw, maps, cond, b, rd, x_in, x_out, xc, d, dc, st, inst,
                                                          blockIdx.x * MTX, blockIdx.y * MTY, &part, k16))
        return;
    if (DOT) {
        const int nblk = gridDim.x * gridDim.y;
        double tot;
        if (reduce_last<NTH>((double)part, red, inst, blockIdx.x + gridDim.x * blockIdx.y, nblk, &tot))
            finalize_alpha<INIT>(st[inst], tot, hist, inst);
    }
}

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
        const int tx = (d.nx + MTX - 1) / MTX, nt = tx * ((d.ny + MTY - 1) / MTY);
        for (int t = rank; t < nt; t += CS)
            pre_tile<T, false, NU, TMA, 0, TNT>(smraw, tm.pre[q], (const T*)tl.cond[q], (const T*)tl.b[q],
                                             (const T*)tl.rd[q], (T*)tl.x[q], (T*)tl.b[q + 1], d, dc, st, inst,
                                             (t % tx) * MTX, (t / tx) * MTY);
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
            const T* Xr = X + (int64_t)inst * nc * nc + (int64_t)row * nc;
            T acc = (T)0;
            for (int c = lane; c < nc; c += 32) acc = fma(Xr[c], sbv[c], acc);
            acc = warp_sum_t<T>(acc);
            if (lane == 0) xL[row] = acc;
        }
        __syncthreads();
        tail_phase_barrier();
    }
    for (int q = nl - 2; q >= 0; --q) {
        const Dims d = tl.d[q], dc = tl.d[q + 1];
        const int tx = (d.nx + MTX - 1) / MTX, nt = tx * ((d.ny + MTY - 1) / MTY);
        for (int t = rank; t < nt; t += CS)
{
            T unused;
            post_tile<T, false, NU, false, TMA, 0, TNT>(smraw, tm.post[q], (const T*)tl.cond[q], (const T*)tl.b[q],
                                                        (const T*)tl.rd[q], (const T*)tl.x[q], (T*)tl.x2[q],
                                                        (const T*)tl.x2[q + 1], d, dc, st, inst, (t % tx) * MTX,
                                                        (t / tx) * MTY, &unused);
        }
        if (q > 0) tail_phase_barrier();
    }
}

// TMA maps for one launch; false when the layout rules are not met (plain loads instead).
// xc (post-smoothing): the coarse-level iterate, with the coarse dimensions dc.
template <typename T, bool L0, int H, bool XC>
static bool make_maps(Maps& m, const T* cond, const T* b, const T* rd, const T* x_in, const T* xc, const Dims& d,
                      const Dims& dc, int B) {
    using TL = Tile<T, L0, H, XC>;
    const int esz = (int)sizeof(T);
    bool ok = tma_map_3d(&m.b, b, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    ok = ok && tma_map_3d(&m.d, rd, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    ok = ok && tma_map_3d(&m.c, cond, esz, d.nx, d.ny, (int64_t)B * TL::CPLANES, TL::LXS, TL::LY, TL::CPLANES);
    if (x_in) ok = ok && tma_map_3d(&m.x, x_in, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    if (XC) ok = ok && tma_map_3d(&m.xc, xc, esz, dc.nx, dc.ny, B, TL::XW, TL::YW, 1);
    return ok;
}

template <typename T, bool L0, int NU>
static void pre_launch(const T* cond, const T* b, const T* rd, T* x, T* bc, Dims d, Dims dc, int B, GkState* st,
                       cudaStream_t s, const __nv_bfloat16* k16) {
    constexpr int H = 2 * NU + 1;
    const size_t smem = Tile<T, L0, H>::bytes();
    Maps maps;
    const bool tma = tma_enabled() && make_maps<T, L0, H, false>(maps, cond, b, rd, nullptr, nullptr, d, dc, B);
    constexpr int NTH = L0 ? MNT : CNT;
    auto kfn = tma ? k_mg_pre2d<T, L0, NU, true, NTH> : k_mg_pre2d<T, L0, NU, false, NTH>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((d.nx + MTX - 1) / MTX, (d.ny + MTY - 1) / MTY, B);
    launch_k(kfn, grid, dim3(NTH), smem, s, maps, cond, b, rd, x, bc, d, dc, st, k16);
}

template <typename T, bool L0, int NU, bool DOT, bool INIT>
static void post_launch(const T* cond, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d, Dims dc,
                        int B, GkState* st, Hist hist, Red red, cudaStream_t s, const __nv_bfloat16* k16) {
    constexpr int H = 2 * NU;
    const size_t smem = Tile<T, L0, H, true>::bytes();
    Maps maps;
    const bool tma = tma_enabled() && make_maps<T, L0, H, true>(maps, cond, b, rd, xi, xc, d, dc, B);
    constexpr int NTH = L0 ? MNT : CNT;
    auto kfn = tma ? k_mg_post2d<T, L0, NU, DOT, INIT, true, NTH> : k_mg_post2d<T, L0, NU, DOT, INIT, false, NTH>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((d.nx + MTX - 1) / MTX, (d.ny + MTY - 1) / MTY, B);
    if (DOT && (int64_t)grid.x * grid.y > red.max_blocks)
        throw std::runtime_error("mg_post2d: too many blocks for the reduction scratch");
    launch_k(kfn, grid, dim3(NTH), smem, s, maps, cond, b, rd, xi, x, xc, d, dc, st, hist, red, k16);
}

bool mg2d_supported(int ndim, int nu) { return ndim == 2 && nu >= 1 && nu <= 3; }

constexpr int TAIL_CS = 16;  // blocks per cluster (non-portable size; the driver is asked first)

// At least 120 KB per block, so that the blocks of a cluster land on different SMs (the tiles of
// a phase then run in parallel instead of sharing one SM's issue slots).
template <typename T, int NU>
static size_t tail_smem(int nc) {
    return std::max({Tile<T, false, 2 * NU + 1>::bytes(), Tile<T, false, 2 * NU, true>::bytes(), sizeof(T) * (size_t)nc,
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
        const int nt = ((d[l].nx + MTX - 1) / MTX) * ((d[l].ny + MTY - 1) / MTY);
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
        tma = make_maps<T, false, 2 * NU + 1, false>(tm.pre[q], c, b, rd, nullptr, nullptr, tl.d[q], tl.d[q + 1], B) &&
              make_maps<T, false, 2 * NU, true>(tm.post[q], c, b, rd, (const T*)tl.x[q], (const T*)tl.x2[q + 1],
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

template <typename T>
void mg2d_pre(const T* cond, bool is_kappa, const T* b, const T* rd, T* x, T* bc, Dims d, Dims dc, int nu, int B,
              GkState* st, cudaStream_t s, const __nv_bfloat16* k16) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
#define PRE_CASE(NU_)                                                                   \
    case NU_:                                                                           \
        if (is_kappa) pre_launch<T, true, NU_>(cond, b, rd, x, bc, d, dc, B, st, s, k16);  \
        else pre_launch<T, false, NU_>(cond, b, rd, x, bc, d, dc, B, st, s, nullptr);      \
        break;
    switch (nu) {
        PRE_CASE(1)
        PRE_CASE(2)
        PRE_CASE(3)
        default: throw std::runtime_error("mg2d_pre: unsupported sweep count");
    }
#undef PRE_CASE
    klaunched("k_mg_pre2d");
    kfinish(s);
}

template <typename T>
void mg2d_post(const T* cond, bool is_kappa, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d,
               Dims dc, int nu, int B, int dot, GkState* st, Hist hist, Red red, cudaStream_t s,
               const __nv_bfloat16* k16) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
#define POST_CASE(NU_)                                                                                           \
    case NU_:                                                                                                    \
        if (!is_kappa) post_launch<T, false, NU_, false, false>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s, nullptr); \
        else if (dot == 0) post_launch<T, true, NU_, false, false>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s, k16); \
        else if (dot == 1) post_launch<T, true, NU_, true, true>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s, k16); \
        else post_launch<T, true, NU_, true, false>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s, k16);             \
        break;
    switch (nu) {
        POST_CASE(1)
        POST_CASE(2)
        POST_CASE(3)
        default: throw std::runtime_error("mg2d_post: unsupported sweep count");
    }
#undef POST_CASE
    klaunched("k_mg_post2d");
    kfinish(s);
}

template void mg2d_pre<float>(const float*, bool, const float*, const float*, float*, float*, Dims, Dims, int, int,
                              GkState*, cudaStream_t, const __nv_bfloat16*);
template void mg2d_pre<double>(const double*, bool, const double*, const double*, double*, double*, Dims, Dims, int,
                               int, GkState*, cudaStream_t, const __nv_bfloat16*);
template void mg2d_post<float>(const float*, bool, const float*, const float*, const float*, float*, const float*,
                               Dims, Dims, int, int, int, GkState*, Hist, Red, cudaStream_t, const __nv_bfloat16*);
template void mg2d_post<double>(const double*, bool, const double*, const double*, const double*, double*,
                                const double*, Dims, Dims, int, int, int, GkState*, Hist, Red, cudaStream_t,
                                const __nv_bfloat16*);

}  // namespace plsqr
