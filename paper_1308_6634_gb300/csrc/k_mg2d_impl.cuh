// k_mg2d_impl.cuh -- temporally blocked V-cycle kernels for 2D grids (Sec. 4.2 priorconditioner),
// templated on the tile shape; k_mg2d.cu, k_mg2d_alt.cu and k_mg2d_alt2.cu instantiate them for
// the shapes the autotuner chooses from.
//
// A block owns a TX x TY tile of one level and stages the tile plus a halo of the right-hand
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
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <stdexcept>
#include <string>
#include <type_traits>

#include "kernels.cuh"
#include "tma.cuh"

namespace plsqr {

// Tile extents (TX, TY; even, TX a multiple of 8) and threads per block.  The finest level has
// many tiles; the coarser levels have few, so they take more threads per tile.
// MINB_: blocks per SM the finest-level float kernels are compiled for (register budget): the
// 32 x 32 post-smoothing tile then fits 8 blocks per SM (one wave for the 1024 tiles of a 1024^2
// level; 37 registers allowed only 6).
template <int TX_, int TY_, int NTH_, int MINB_ = 1>
struct Shape {
    static constexpr int TX = TX_, TY = TY_, NTH = NTH_, MINB = MINB_;
    static_assert(TX % 8 == 0 && TY % 2 == 0, "tiles start at even coordinates, x on 16-byte boundaries of xc");
};
// The shapes compiled in.  Level 0 (many tiles): F0 (default) .. F3.  Coarser levels (few tiles,
// so more threads per tile or smaller tiles spread over more SMs): C0 (default) .. C5.  The
// defaults also have plain-load variants; the others need TMA staging.  Every shape gives bit for
// bit the same V-cycle (the same arithmetic per cell in the same order), only the schedule differs.
using F0 = Shape<64, 32, 256>;
using F1 = Shape<32, 32, 256, 7>;
using F2 = Shape<32, 16, 256>;
using F3 = Shape<64, 32, 512>;
using F4 = Shape<16, 16, 256>;  // small tiles: more SMs on small grids (the fused alpha needs 32 x 16 segments)
using F5 = Shape<16, 8, 128>;
using C0 = Shape<64, 32, 1024>;
using C1 = Shape<32, 16, 512>;
using C2 = Shape<32, 16, 256>;
using C3 = Shape<16, 16, 256>;
using C4 = Shape<16, 16, 128>;
using C5 = Shape<16, 8, 128>;
using TailShape = Shape<64, 32, 1024>;  // the one-launch coarse end
constexpr int TNT = TailShape::NTH;

// Tile geometry: logical halo H on both axes; in storage the x halo is HX >= H (HX * sizeof(T)
// a multiple of 16 bytes, the TMA rule for the innermost coordinate), so logical column lx is
// stored at lx + OX.  Arrays: sb, scx, scy (scy == scx on the finest level), sx, sd (1 / diagonal)
// and, for post-smoothing (XC), the box of coarse-level cells that are parents of staged cells.
template <typename T, bool L0, int H, class S, bool XC = false>
struct Tile {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int HX = ((H + VEC - 1) / VEC) * VEC, OX = HX - H;
    static constexpr int LX = S::TX + 2 * H, LY = S::TY + 2 * H;  // logical extents
    static constexpr int LXS = S::TX + 2 * HX;                    // storage pitch
    static constexpr int NCS = LY * LXS;                      // one staged plane
    static constexpr int NCP = ((NCS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);  // 128-byte padded
    static constexpr int CPLANES = L0 ? 1 : 2;
    // Coarse box: it starts XB coarse columns and YB coarse rows before the parent (x0/2, y0/2)
    // of the tile's first cell (XB a multiple of VEC, so the copy's x stays 16-byte aligned).
    // The parent of staged cell (ly, lxs) is box cell ((ly + (H & 1)) >> 1, (lxs + 2 XB - HX) >> 1).
    static constexpr int XB = (((HX + 1) / 2 + VEC - 1) / VEC) * VEC;
    static constexpr int XW = ((((S::TX + HX - 1) >> 1) + XB + 1 + VEC - 1) / VEC) * VEC;
    static constexpr int YB = (H + 1) / 2;
    static constexpr int YW = ((S::TY + H - 1) >> 1) + YB + 1;
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
template <typename T, bool L0, int H, bool TMA, bool X_IN, bool XC, int SKIP, class S>
__device__ __forceinline__ bool stage(T* sm, const Maps& maps, const T* __restrict__ cond, const T* __restrict__ b,
                                      const T* __restrict__ rd, const T* __restrict__ x_in,
                                      const T* __restrict__ xc, const Dims& d, const Dims& dc, int inst, int x0,
                                      int y0, GkState* st, const __nv_bfloat16* __restrict__ k16) {
    using TL = Tile<T, L0, H, S, XC>;
    constexpr int NTH = S::NTH;
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

// The Gauss-Seidel update of one cell, x = (b + sum_nb c_nb x_nb) / diag with the reciprocal
// diagonal rd, in a fixed order of operations (every schedule and storage layout uses it, so they
// agree bit for bit): cE, cW are the conductances of the east / west edges (kappa of the cell and
// of its west neighbour on the finest level), cN, cS those of the north / south edges.
template <typename T>
__device__ __forceinline__ T gs_update(T b, T rd, T cE, T cW, T cN, T cS, T xE, T xW, T xN, T xS) {
    T off = cE * xE;
    off = fma(cW, xW, off);
    off = fma(cN, xN, off);
    off = fma(cS, xS, off);
    return (b + off) * rd;
}

// r = b - (diag x - off) of one cell, the residual the restriction sums (the same fixed order).
template <typename T>
__device__ __forceinline__ T gs_residual(T b, T x, T cE, T cW, T cN, T cS, T xE, T xW, T xN, T xS) {
    T diag = cE;
    diag += cW;
    diag += cN;
    diag += cS;
    T off = cE * xE;
    off = fma(cW, xW, off);
    off = fma(cN, xN, off);
    off = fma(cS, xS, off);
    return b - fma(diag, x, -off);
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
    // A thread keeps one column slot j of the colour and walks down the rows, rpp rows per step
    // (every row gets all of its cells: the first rpp * half threads cover rpp whole rows), so the
    // index advances by a constant instead of being divided out of a flat counter per cell.
    const int rpp = NTH / half;
    const int t = threadIdx.x;
    if (rpp == 0 || t >= rpp * half) {
        if (rpp == 0)  // rows longer than the block: the flat loop
            for (int k = t; k < rows * half; k += NTH) {
                const int ry = k / half, j = k - ry * half;
                const int ly = lo + ry;
                const int lx = lo + ((colour ^ ly ^ lo) & 1) + 2 * j;
                if (lx > hi) continue;
                const int i = ly * LXS + lx + OX;
                sx[i] = gs_update(sb[i], sd[i], scx[i], scx[i - 1], scy[i], scy[i - LXS], sx[i + 1], sx[i - 1],
                                  sx[i + LXS], sx[i - LXS]);
            }
        return;
    }
    const int j = t % half;
    for (int ry = t / half; ry < rows; ry += rpp) {
        const int ly = lo + ry;
        const int lx = lo + ((colour ^ ly ^ lo) & 1) + 2 * j;  // first lx >= lo of the colour, then every other
        if (lx > hi) continue;
        const int i = ly * LXS + lx + OX;
        sx[i] = gs_update(sb[i], sd[i], scx[i], scx[i - 1], scy[i], scy[i - LXS], sx[i + 1], sx[i - 1],
                          sx[i + LXS], sx[i - LXS]);
    }
}

// Pre-smoothing of one tile from x = 0 (nu red->black sweeps), residual and restriction to bc.
// Returns false when the block skips the tile (see stage).  Ends with a barrier, so that a block
// can go on with another tile.
template <typename T, bool L0, int NU, bool TMA, int SKIP, class S>
__device__ __forceinline__ bool pre_tile(unsigned char* smraw, const Maps& maps, const T* cond, const T* b,
                                         const T* rd, T* x, T* bc, const Dims& d, const Dims& dc, GkState* st,
                                         int inst, int x0, int y0, const __nv_bfloat16* k16 = nullptr) {
    constexpr int H = 2 * NU + 1;
    using TL = Tile<T, L0, H, S>;
    constexpr int LXS = TL::LXS, OX = TL::OX, NTH = S::NTH, MTX = S::TX, MTY = S::TY;
    T* sm = reinterpret_cast<T*>(smraw);
    T* sb = sm;
    T* scx = sm + TL::OFF_C;
    T* scy = L0 ? scx : scx + TL::NCS;
    T* sx = sm + TL::OFF_X;
    const T* sd = sm + TL::OFF_D;
    if (stage<T, L0, H, TMA, false, false, SKIP, S>(sm, maps, cond, b, rd, nullptr, nullptr, d, dc, inst, x0, y0,
                                                      st, k16))
        return false;
    const int64_t offc = (int64_t)inst * dc.N;
    const int64_t off = (int64_t)inst * d.N;
    {
#pragma unroll
        for (int s = 0; s < 2 * NU; ++s) {
            half_sweep<T, TL::LX, TL::LY, LXS, OX, NTH>(sb, sd, scx, scy, sx, s + 1, s & 1);
            __syncthreads();
        }
        // residual r = b - (diag x - off) on the tile, summed over the 2 x 2 children
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
                    sum += gs_residual(sb[i], sx[i], scx[i], scx[i - 1], scy[i], scy[i - LXS], sx[i + 1], sx[i - 1],
                                       sx[i + LXS], sx[i - LXS]);
                }
            bc[offc + (int64_t)Y * dc.nx + X] = sum;
        }
        for (int k = threadIdx.x; k < MTX * MTY; k += NTH) {
            const int ty = k / MTX, tx = k - ty * MTX;
            const int gx = x0 + tx, gy = y0 + ty;
            if (gx < d.nx && gy < d.ny) x[off + (int64_t)gy * d.nx + gx] = sx[(H + ty) * LXS + H + tx + OX];
        }
    }
    __syncthreads();
    return true;
}

template <typename T, bool L0, int NU, bool TMA, class S>
__global__ void __launch_bounds__(S::NTH, (sizeof(T) == 4 && L0) ? S::MINB : 1) k_mg_pre2d(const __grid_constant__ Maps maps, const T* __restrict__ cond,
                                                  const T* __restrict__ b, const T* __restrict__ rd,
                                                  T* __restrict__ x, T* __restrict__ bc, Dims d, Dims dc, GkState* st,
                                                  const __nv_bfloat16* __restrict__ k16) {
    extern __shared__ __align__(128) unsigned char smraw[];
    pdl_grid_sync();
    pre_tile<T, L0, NU, TMA, 1, S>(smraw, maps, cond, b, rd, x, bc, d, dc, st, blockIdx.z, blockIdx.x * S::TX,
                                   blockIdx.y * S::TY, k16);
}

// One tile of x_out = smooth(x_in + P xc) with nu black->red sweeps (x_in and x_out must differ:
// blocks read neighbouring tiles of x_in as halo).  Returns false when the block skips the tile
// (see stage).  DOT: also the partial sums of x_out . b over 32 x 16 segments of the grid (32
// columns, 16 rows, anchored at multiples of 32 and 16), written to segp[(y / 16) * nseg + x / 32]
// (nseg = ceil(nx / 32)): each row of a segment by one warp (the 32 products summed in T by a
// butterfly), then its 16 row sums in double in row order.  The segments do not depend on the
// tile shape, so alpha (their sum, see sum_partials_last) is the same whatever shape the
// autotuner picks.  Ends with a barrier.
template <typename T, bool L0, int NU, bool DOT, bool TMA, int SKIP, class S>
__device__ __forceinline__ bool post_tile(unsigned char* smraw, const Maps& maps, const T* cond, const T* b,
                                          const T* rd, const T* x_in, T* x_out, const T* xc, const Dims& d,
                                          const Dims& dc, GkState* st, int inst, int x0, int y0, double* segp,
                                          int nseg, const __nv_bfloat16* k16 = nullptr) {
    static_assert(!DOT || (S::TX % 32 == 0 && S::TY % 16 == 0), "tiles hold whole 32 x 16 segments");
    __shared__ double srow[DOT ? S::TY * (S::TX / 32) : 1];  // row sums of the tile's segments
    constexpr int H = 2 * NU;
    using TL = Tile<T, L0, H, S, true>;
    constexpr int LXS = TL::LXS, OX = TL::OX, NTH = S::NTH, MTX = S::TX, MTY = S::TY;
    T* sm = reinterpret_cast<T*>(smraw);
    T* sb = sm;
    T* scx = sm + TL::OFF_C;
    T* scy = L0 ? scx : scx + TL::NCS;
    T* sx = sm + TL::OFF_X;
    const T* sd = sm + TL::OFF_D;
    const T* sxc = sm + TL::OFF_XC;
    if (stage<T, L0, H, TMA, true, true, SKIP, S>(sm, maps, cond, b, rd, x_in, xc, d, dc, inst, x0, y0, st, k16))
        return false;
    const int64_t off = (int64_t)inst * d.N;
    {
        // + P xc.  The extents are even (2^(levels-1) divides them), so a cell outside the domain
        // has its parent outside the coarse grid: it adds the zero fill and stays 0.
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
        for (int k = threadIdx.x; k < MTX * MTY; k += NTH) {
            const int ty = k / MTX, tx = k - ty * MTX;
            const int gx = x0 + tx, gy = y0 + ty;
            T prod = (T)0;
            if (gx < d.nx && gy < d.ny) {
                const int i = (H + ty) * LXS + H + tx + OX;
                x_out[off + (int64_t)gy * d.nx + gx] = sx[i];
                if (DOT) prod = sx[i] * sb[i];
            }
            if (DOT) {  // the warp's 32 lanes are one 32-column row of a segment (TX is a multiple of 32)
                const T v = warp_sum_t<T>(prod);  // in T: a butterfly in double would load the FP64 pipe
                if ((threadIdx.x & 31) == 0) srow[ty * (MTX / 32) + (tx >> 5)] = (double)v;
            }
        }
        if (DOT) {
            __syncthreads();
            // one thread per segment of the tile: its 16 row sums in row order (rows beyond ny and
            // columns beyond nx added 0; segments wholly outside the grid do not exist)
            constexpr int NSX = MTX / 32, NSY = MTY / 16;
            if (threadIdx.x < NSX * NSY) {
                const int sy = threadIdx.x / NSX, sx_ = threadIdx.x - sy * NSX;
                const int gx0 = x0 + 32 * sx_, gy0 = y0 + 16 * sy;
                if (gx0 < d.nx && gy0 < d.ny) {
                    double v = 0.0;
#pragma unroll
                    for (int r = 0; r < 16; ++r) v += srow[(16 * sy + r) * NSX + sx_];
                    segp[(int64_t)(gy0 >> 4) * nseg + (gx0 >> 5)] = v;
                    __threadfence();
                }
            }
        }
    }
    __syncthreads();
    return true;
}

// DOT: also alpha = sqrt(x_out . b) and the rotations (finest level of the last V-cycle:
// x_out = v~, b = p~).
template <typename T, bool L0, int NU, bool DOT, bool INIT, bool TMA, class S>
__global__ void __launch_bounds__(S::NTH, (sizeof(T) == 4 && L0) ? S::MINB : 1) k_mg_post2d(const __grid_constant__ Maps maps, const T* __restrict__ cond,
                                                   const T* __restrict__ b, const T* __restrict__ rd,
                                                   const T* __restrict__ x_in, T* __restrict__ x_out,
                                                   const T* __restrict__ xc, Dims d, Dims dc, GkState* st, Hist hist,
                                                   Red red, const __nv_bfloat16* __restrict__ k16) {
    extern __shared__ __align__(128) unsigned char smraw[];
    const int inst = blockIdx.z;
    pdl_grid_sync();
    const int nseg = (d.nx + 31) / 32;
    if (!post_tile<T, L0, NU, DOT, TMA, DOT ? 2 : 1, S>(smraw, maps, cond, b, rd, x_in, x_out, xc, d, dc, st, inst,
                                                        blockIdx.x * S::TX, blockIdx.y * S::TY,
                                                        DOT ? red.partials + (int64_t)inst * red.max_blocks : nullptr,
                                                        nseg, k16))
        return;
    if (DOT) {
        double tot;
        if (sum_partials_last<S::NTH>(red, inst, gridDim.x * gridDim.y, ((d.ny + 15) / 16) * nseg, &tot))
            finalize_alpha<INIT>(st[inst], tot, hist, inst);
    }
}

// Ask for the largest shared-memory carveout (all of the unified L1 / shared storage an SM can give
// to shared memory), so that the occupancy is set by the blocks' needs and not by the driver's
// default split; once per kernel.
template <typename K>
void max_carveout(K kfn) {
    max_carveout_set(reinterpret_cast<const void*>(kfn));
}

// TMA maps for one launch; false when the layout rules are not met (plain loads instead).
// xc (post-smoothing): the coarse-level iterate, with the coarse dimensions dc.
template <typename T, bool L0, int H, class S, bool XC>
bool make_maps(Maps& m, const T* cond, const T* b, const T* rd, const T* x_in, const T* xc, const Dims& d,
                      const Dims& dc, int B) {
    using TL = Tile<T, L0, H, S, XC>;
    const int esz = (int)sizeof(T);
    bool ok = tma_map_3d(&m.b, b, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    ok = ok && tma_map_3d(&m.d, rd, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    ok = ok && tma_map_3d(&m.c, cond, esz, d.nx, d.ny, (int64_t)B * TL::CPLANES, TL::LXS, TL::LY, TL::CPLANES);
    if (x_in) ok = ok && tma_map_3d(&m.x, x_in, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    if (XC) ok = ok && tma_map_3d(&m.xc, xc, esz, dc.nx, dc.ny, B, TL::XW, TL::YW, 1);
    return ok;
}

// One launch with shape S.  Returns false (nothing launched) when the TMA layout rules are not
// met and S has no plain-load variant (PLAIN false).
template <typename T, bool L0, int NU, class S, bool PLAIN>
bool pre_launch(const T* cond, const T* b, const T* rd, T* x, T* bc, Dims d, Dims dc, int B, GkState* st,
                cudaStream_t s, const __nv_bfloat16* k16) {
    constexpr int H = 2 * NU + 1;
    const size_t smem = Tile<T, L0, H, S>::bytes();
    Maps maps;
    const bool tma = tma_enabled() && make_maps<T, L0, H, S, false>(maps, cond, b, rd, nullptr, nullptr, d, dc, B);
    if (!tma && !PLAIN) return false;
    auto kfn = k_mg_pre2d<T, L0, NU, true, S>;
    if constexpr (PLAIN)
        if (!tma) kfn = k_mg_pre2d<T, L0, NU, false, S>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    max_carveout(kfn);
    dim3 grid((d.nx + S::TX - 1) / S::TX, (d.ny + S::TY - 1) / S::TY, B);
    launch_k(kfn, grid, dim3(S::NTH), smem, s, maps, cond, b, rd, x, bc, d, dc, st, k16);
    return true;
}

template <typename T, bool L0, int NU, bool DOT, bool INIT, class S, bool PLAIN>
bool post_launch(const T* cond, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d, Dims dc, int B,
                 GkState* st, Hist hist, Red red, cudaStream_t s, const __nv_bfloat16* k16) {
    constexpr int H = 2 * NU;
    const size_t smem = Tile<T, L0, H, S, true>::bytes();
    Maps maps;
    const bool tma = tma_enabled() && make_maps<T, L0, H, S, true>(maps, cond, b, rd, xi, xc, d, dc, B);
    if (!tma && !PLAIN) return false;
    auto kfn = k_mg_post2d<T, L0, NU, DOT, INIT, true, S>;
    if constexpr (PLAIN)
        if (!tma) kfn = k_mg_post2d<T, L0, NU, DOT, INIT, false, S>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    max_carveout(kfn);
    dim3 grid((d.nx + S::TX - 1) / S::TX, (d.ny + S::TY - 1) / S::TY, B);
    if (DOT && (int64_t)((d.ny + 15) / 16) * ((d.nx + 31) / 32) > red.max_blocks)
        throw std::runtime_error("mg_post2d: too many segments for the reduction scratch");
    launch_k(kfn, grid, dim3(S::NTH), smem, s, maps, cond, b, rd, xi, x, xc, d, dc, st, hist, red, k16);
    return true;
}

// Pre- and post-smoothing of one level with shape S (L0: the finest level, conductances = kappa),
// nu = 1..3; dot as in mg2d_post.  False when S cannot stage this layout (see pre_launch).
template <typename T, bool L0, class S, bool PLAIN>
bool pre_shape(const T* cond, const T* b, const T* rd, T* x, T* bc, Dims d, Dims dc, int nu, int B, GkState* st,
               cudaStream_t s, const __nv_bfloat16* k16) {
    switch (nu) {
        case 1: return pre_launch<T, L0, 1, S, PLAIN>(cond, b, rd, x, bc, d, dc, B, st, s, k16);
        case 2: return pre_launch<T, L0, 2, S, PLAIN>(cond, b, rd, x, bc, d, dc, B, st, s, k16);
        case 3: return pre_launch<T, L0, 3, S, PLAIN>(cond, b, rd, x, bc, d, dc, B, st, s, k16);
        default: throw std::runtime_error("mg2d_pre: unsupported sweep count");
    }
}

template <typename T, bool L0, int NU, class S, bool PLAIN>
bool post_nu(const T* cond, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d, Dims dc, int B, int dot,
             GkState* st, Hist hist, Red red, cudaStream_t s, const __nv_bfloat16* k16) {
    if constexpr (!L0) {
        return post_launch<T, false, NU, false, false, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s,
                                                                 k16);
    } else if constexpr (S::TX % 32 != 0 || S::TY % 16 != 0) {  // no whole alpha segments: no fused alpha
        if (dot != 0) return false;
        return post_launch<T, true, NU, false, false, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s,
                                                                k16);
    } else {
        if (dot == 0)
            return post_launch<T, true, NU, false, false, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red,
                                                                    s, k16);
        if (dot == 1)
            return post_launch<T, true, NU, true, true, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s,
                                                                  k16);
        return post_launch<T, true, NU, true, false, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, st, hist, red, s,
                                                               k16);
    }
}

template <typename T, bool L0, class S, bool PLAIN>
bool post_shape(const T* cond, const T* b, const T* rd, const T* xi, T* x, const T* xc, Dims d, Dims dc, int nu,
                int B, int dot, GkState* st, Hist hist, Red red, cudaStream_t s, const __nv_bfloat16* k16) {
    switch (nu) {
        case 1: return post_nu<T, L0, 1, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, dot, st, hist, red, s, k16);
        case 2: return post_nu<T, L0, 2, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, dot, st, hist, red, s, k16);
        case 3: return post_nu<T, L0, 3, S, PLAIN>(cond, b, rd, xi, x, xc, d, dc, B, dot, st, hist, red, s, k16);
        default: throw std::runtime_error("mg2d_post: unsupported sweep count");
    }
}

#define PLSQR_MG2D_SHAPE_DECL(EXT, T, L0, S, PLAIN)                                                            \
    EXT template bool pre_shape<T, L0, S, PLAIN>(const T*, const T*, const T*, T*, T*, Dims, Dims, int, int,     \
                                                 GkState*, cudaStream_t, const __nv_bfloat16*);                  \
    EXT template bool post_shape<T, L0, S, PLAIN>(const T*, const T*, const T*, const T*, T*, const T*, Dims,    \
                                                  Dims, int, int, int, GkState*, Hist, Red, cudaStream_t,       \
                                                  const __nv_bfloat16*);

// the shapes of k_mg2d_alt.cu (level 0) and k_mg2d_alt2.cu (coarser levels), TMA staging only
#define PLSQR_MG2D_ALT_FINE(EXT)                            \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, true, F1, false)      \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, true, F1, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, true, F2, false)      \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, true, F2, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, true, F3, false)      \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, true, F3, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, true, F4, false)      \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, true, F4, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, true, F5, false)      \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, true, F5, false)
#define PLSQR_MG2D_ALT_COARSE(EXT)                          \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, false, C1, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, false, C1, false)    \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, false, C2, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, false, C2, false)    \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, false, C3, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, false, C3, false)    \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, false, C4, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, false, C4, false)    \
    PLSQR_MG2D_SHAPE_DECL(EXT, float, false, C5, false)     \
    PLSQR_MG2D_SHAPE_DECL(EXT, double, false, C5, false)

}  // namespace plsqr
