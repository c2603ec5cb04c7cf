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

#include <cstdlib>
#include <stdexcept>
#include <string>

#include "kernels.cuh"
#include "tma.cuh"

namespace plsqr {

constexpr int MTX = 64, MTY = 32, MNT = 256;

// Tile geometry: logical halo H on both axes; in storage the x halo is HX >= H (HX * sizeof(T)
// a multiple of 16 bytes, the TMA rule for the innermost coordinate), so logical column lx is
// stored at lx + OX.  Arrays: sb, scx, scy (scy == scx on the finest level), sx.
template <typename T, bool L0, int H>
struct Tile {
    static constexpr int VEC = 16 / (int)sizeof(T);
    static constexpr int HX = ((H + VEC - 1) / VEC) * VEC, OX = HX - H;
    static constexpr int LX = MTX + 2 * H, LY = MTY + 2 * H;  // logical extents
    static constexpr int LXS = MTX + 2 * HX;                  // storage pitch
    static constexpr int NCS = LY * LXS;                      // one staged plane
    static constexpr int NCP = ((NCS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);  // 128-byte padded
    static constexpr int CPLANES = L0 ? 1 : 2;
    // layout: sb [NCP] | scx, scy [CPLANES * NCS, padded] | sx [NCP] | mbarrier
    static constexpr int OFF_C = NCP;
    static constexpr int OFF_X = NCP + ((CPLANES * NCS * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    static constexpr size_t bytes() { return sizeof(T) * (size_t)(OFF_X + NCP) + 16; }
};

struct Maps {
    CUtensorMap b, c, x;
};

// Stage b and the conductances (and x_in when X_IN) of the tile.
template <typename T, bool L0, int H, bool TMA, bool X_IN>
__device__ __forceinline__ void stage(T* sm, const Maps& maps, const T* __restrict__ cond, const T* __restrict__ b,
                                      const T* __restrict__ x_in, const Dims& d, int inst, int x0, int y0,
                                      GkState* st) {
    using TL = Tile<T, L0, H>;
    T* sb = sm;
    T* sc = sm + TL::OFF_C;
    T* sx = sm + TL::OFF_X;
    if constexpr (TMA) {
        uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TL::OFF_X + TL::NCP);
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t plane = TL::NCS * sizeof(T);
            mbar_expect_tx(bar, plane * (1 + TL::CPLANES + (X_IN ? 1 : 0)));
            const int gx = x0 - TL::HX, gy = y0 - H;
            tma_load_3d(sb, &maps.b, bar, gx, gy, inst);
            tma_load_3d(sc, &maps.c, bar, gx, gy, L0 ? inst : 2 * inst);
            if (X_IN) tma_load_3d(sx, &maps.x, bar, gx, gy, inst);
        }
        tma_wait_tile(bar, st, inst);
    } else {
        const int64_t off = (int64_t)inst * d.N;
        const T* c = cond + (L0 ? off : (int64_t)inst * 2 * d.N);
        for (int i = threadIdx.x; i < TL::NCS; i += MNT) {
            const int ly = i / TL::LXS, lxs = i - ly * TL::LXS;
            const int gy = y0 - H + ly, gx = x0 - TL::HX + lxs;
            T vb = (T)0, vx = (T)0, vy = (T)0, vv = (T)0;
            if (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny) {
                const int64_t g = (int64_t)gy * d.nx + gx;
                vb = b[off + g];
                vx = c[g];
                if (!L0) vy = c[d.N + g];
                if (X_IN) vv = x_in[off + g];
            }
            sb[i] = vb;
            sc[i] = vx;
            if (!L0) sc[TL::NCS + i] = vy;
            if (X_IN) sx[i] = vv;
        }
        __syncthreads();
    }
}

// One half sweep of `colour` over the logical cells at distance >= lo from the staged edge.
template <typename T, int LX, int LY, int LXS, int OX, int H>
__device__ __forceinline__ void half_sweep(const T* sb, const T* scx, const T* scy, T* sx, int lo, int colour,
                                          const Dims& d, int x0, int y0) {
    const int hi = LX - 1 - lo, hiy = LY - 1 - lo;
    const int half = (hi - lo + 2) >> 1;
    const int rows = hiy - lo + 1;
    for (int k = threadIdx.x; k < rows * half; k += MNT) {
        const int ry = k / half, j = k - ry * half;
        const int ly = lo + ry;
        const int gy = y0 - H + ly;
        const int gx_lo = x0 - H + lo;
        const int p = (colour - gy - gx_lo) & 1;  // first lx in [lo, hi] with (gx + gy) % 2 == colour
        const int lx = lo + p + 2 * j;
        if (lx > hi) continue;
        const int gx = x0 - H + lx;
        if (gx < 0 || gx >= d.nx || gy < 0 || gy >= d.ny) continue;
        const int i = ly * LXS + lx + OX;
        T diag = scx[i];
        diag += scx[i - 1];
        diag += scy[i];
        diag += scy[i - LXS];
        T off = scx[i] * sx[i + 1];
        off += scx[i - 1] * sx[i - 1];
        off += scy[i] * sx[i + LXS];
        off += scy[i - LXS] * sx[i - LXS];
        sx[i] = (sb[i] + off) / diag;
    }
}

// Pre-smoothing from x = 0 (nu red->black sweeps), residual and restriction to bc.
template <typename T, bool L0, int NU, bool TMA>
__global__ void __launch_bounds__(MNT) k_mg_pre2d(const __grid_constant__ Maps maps, const T* __restrict__ cond,
                                                  const T* __restrict__ b, T* __restrict__ x, T* __restrict__ bc,
                                                  Dims d, Dims dc, GkState* st) {
    constexpr int H = 2 * NU + 1;
    using TL = Tile<T, L0, H>;
    constexpr int LXS = TL::LXS, OX = TL::OX;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    T* sb = sm;
    T* scx = sm + TL::OFF_C;
    T* scy = L0 ? scx : scx + TL::NCS;
    T* sx = sm + TL::OFF_X;
    const int inst = blockIdx.z, x0 = blockIdx.x * MTX, y0 = blockIdx.y * MTY;
    for (int i = threadIdx.x; i < TL::NCS; i += MNT) sx[i] = (T)0;
    stage<T, L0, H, TMA, false>(sm, maps, cond, b, nullptr, d, inst, x0, y0, st);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2 * NU; ++s) {
        half_sweep<T, TL::LX, TL::LY, LXS, OX, H>(sb, scx, scy, sx, s + 1, s & 1, d, x0, y0);
        __syncthreads();
    }
    // residual r = b - (diag x - off) on the tile, summed over the 2 x 2 children
    const int64_t offc = (int64_t)inst * dc.N;
    for (int k = threadIdx.x; k < (MTX / 2) * (MTY / 2); k += MNT) {
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
    for (int k = threadIdx.x; k < MTX * MTY; k += MNT) {
        const int ty = k / MTX, tx = k - ty * MTX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < d.nx && gy < d.ny) x[off + (int64_t)gy * d.nx + gx] = sx[(H + ty) * LXS + H + tx + OX];
    }
}

// x_out = smooth(x_in + P xc) with nu black->red sweeps (x_in and x_out must differ: blocks read
// neighbouring tiles of x_in as halo).  DOT: also alpha = sqrt(x_out . b) and the rotations
// (finest level of the last V-cycle: x_out = v~, b = p~).
template <typename T, bool L0, int NU, bool DOT, bool INIT, bool TMA>
__global__ void __launch_bounds__(MNT) k_mg_post2d(const __grid_constant__ Maps maps, const T* __restrict__ cond,
                                                   const T* __restrict__ b, const T* __restrict__ x_in,
                                                   T* __restrict__ x_out, const T* __restrict__ xc, Dims d, Dims dc,
                                                   GkState* st, Hist hist, Red red) {
    constexpr int H = 2 * NU;
    using TL = Tile<T, L0, H>;
    constexpr int LXS = TL::LXS, OX = TL::OX;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    T* sb = sm;
    T* scx = sm + TL::OFF_C;
    T* scy = L0 ? scx : scx + TL::NCS;
    T* sx = sm + TL::OFF_X;
    const int inst = blockIdx.z, x0 = blockIdx.x * MTX, y0 = blockIdx.y * MTY;
    if (DOT && st[inst].status != ST_OK) return;
    stage<T, L0, H, TMA, true>(sm, maps, cond, b, x_in, d, inst, x0, y0, st);
    const int64_t offc = (int64_t)inst * dc.N;
    for (int i = threadIdx.x; i < TL::NCS; i += MNT) {  // + P xc on the staged cells in the domain
        const int ly = i / LXS, lxs = i - ly * LXS;
        const int gy = y0 - H + ly, gx = x0 - TL::HX + lxs;
        if (gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny)
            sx[i] = sx[i] + xc[offc + (int64_t)(gy >> 1) * dc.nx + (gx >> 1)];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2 * NU; ++s) {
        half_sweep<T, TL::LX, TL::LY, LXS, OX, H>(sb, scx, scy, sx, s + 1, 1 - (s & 1), d, x0, y0);
        __syncthreads();
    }
    const int64_t off = (int64_t)inst * d.N;
    T part = (T)0;
    for (int k = threadIdx.x; k < MTX * MTY; k += MNT) {
        const int ty = k / MTX, tx = k - ty * MTX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < d.nx && gy < d.ny) {
            const int i = (H + ty) * LXS + H + tx + OX;
            x_out[off + (int64_t)gy * d.nx + gx] = sx[i];
            if (DOT) part = fma(sx[i], sb[i], part);
        }
    }
    if (DOT) {
        const int nblk = gridDim.x * gridDim.y;
        double tot;
        if (reduce_last<MNT>((double)part, red, inst, blockIdx.x + gridDim.x * blockIdx.y, nblk, &tot))
            finalize_alpha<INIT>(st[inst], tot, hist, inst);
    }
}

// TMA maps for one launch; false when the layout rules are not met (plain loads instead).
template <typename T, bool L0, int H>
static bool make_maps(Maps& m, const T* cond, const T* b, const T* x_in, const Dims& d, int B) {
    using TL = Tile<T, L0, H>;
    const int esz = (int)sizeof(T);
    bool ok = tma_map_3d(&m.b, b, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    ok = ok && tma_map_3d(&m.c, cond, esz, d.nx, d.ny, (int64_t)B * TL::CPLANES, TL::LXS, TL::LY, TL::CPLANES);
    if (x_in) ok = ok && tma_map_3d(&m.x, x_in, esz, d.nx, d.ny, B, TL::LXS, TL::LY, 1);
    return ok;
}

template <typename T, bool L0, int NU>
static void pre_launch(const T* cond, const T* b, T* x, T* bc, Dims d, Dims dc, int B, GkState* st, cudaStream_t s) {
    constexpr int H = 2 * NU + 1;
    const size_t smem = Tile<T, L0, H>::bytes();
    Maps maps;
    const bool tma = tma_enabled() && make_maps<T, L0, H>(maps, cond, b, nullptr, d, B);
    auto kfn = tma ? k_mg_pre2d<T, L0, NU, true> : k_mg_pre2d<T, L0, NU, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((d.nx + MTX - 1) / MTX, (d.ny + MTY - 1) / MTY, B);
    kfn<<<grid, MNT, smem, s>>>(maps, cond, b, x, bc, d, dc, st);
}

template <typename T, bool L0, int NU, bool DOT, bool INIT>
static void post_launch(const T* cond, const T* b, const T* xi, T* x, const T* xc, Dims d, Dims dc, int B,
                        GkState* st, Hist hist, Red red, cudaStream_t s) {
    constexpr int H = 2 * NU;
    const size_t smem = Tile<T, L0, H>::bytes();
    Maps maps;
    const bool tma = tma_enabled() && make_maps<T, L0, H>(maps, cond, b, xi, d, B);
    auto kfn = tma ? k_mg_post2d<T, L0, NU, DOT, INIT, true> : k_mg_post2d<T, L0, NU, DOT, INIT, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((d.nx + MTX - 1) / MTX, (d.ny + MTY - 1) / MTY, B);
    if (DOT && (int64_t)grid.x * grid.y > red.max_blocks)
        throw std::runtime_error("mg_post2d: too many blocks for the reduction scratch");
    kfn<<<grid, MNT, smem, s>>>(maps, cond, b, xi, x, xc, d, dc, st, hist, red);
}

bool mg2d_supported(int ndim, int nu) { return ndim == 2 && nu >= 1 && nu <= 3; }

template <typename T>
void mg2d_pre(const T* cond, bool is_kappa, const T* b, T* x, T* bc, Dims d, Dims dc, int nu, int B, GkState* st,
              cudaStream_t s) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
#define PRE_CASE(NU_)                                                                   \
    case NU_:                                                                           \
        if (is_kappa) pre_launch<T, true, NU_>(cond, b, x, bc, d, dc, B, st, s);       \
        else pre_launch<T, false, NU_>(cond, b, x, bc, d, dc, B, st, s);               \
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
void mg2d_post(const T* cond, bool is_kappa, const T* b, const T* xi, T* x, const T* xc, Dims d, Dims dc, int nu,
               int B, int dot, GkState* st, Hist hist, Red red, cudaStream_t s) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
#define POST_CASE(NU_)                                                                                           \
    case NU_:                                                                                                    \
        if (!is_kappa) post_launch<T, false, NU_, false, false>(cond, b, xi, x, xc, d, dc, B, st, hist, red, s); \
        else if (dot == 0) post_launch<T, true, NU_, false, false>(cond, b, xi, x, xc, d, dc, B, st, hist, red, s); \
        else if (dot == 1) post_launch<T, true, NU_, true, true>(cond, b, xi, x, xc, d, dc, B, st, hist, red, s); \
        else post_launch<T, true, NU_, true, false>(cond, b, xi, x, xc, d, dc, B, st, hist, red, s);             \
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

template void mg2d_pre<float>(const float*, bool, const float*, float*, float*, Dims, Dims, int, int, GkState*,
                              cudaStream_t);
template void mg2d_pre<double>(const double*, bool, const double*, double*, double*, Dims, Dims, int, int, GkState*,
                               cudaStream_t);
template void mg2d_post<float>(const float*, bool, const float*, const float*, float*, const float*, Dims, Dims, int,
                               int, int, GkState*, Hist, Red, cudaStream_t);
template void mg2d_post<double>(const double*, bool, const double*, const double*, double*, const double*, Dims, Dims,
                                int, int, int, GkState*, Hist, Red, cudaStream_t);

}  // namespace plsqr
