// k_mg.cu -- diffusivity and the geometric-multigrid priorconditioner (Sec. 4.2).
//
// M_f = sum_d D_d^T diag(kappa) D_d (eq. 1.13) on the tensor grid: forward differences,
// ghost value 0 beyond the high end of each axis.  In conductance form the edge from cell i
// to i+e_d carries c_d(i) (= kappa_i on the finest level), and
//     (M x)_i = sum_d c_d(i) (x_i - x_{i+e_d}) + c_d(i-e_d) (x_i - x_{i-e_d}).
// P approximates M^{-1} by V-cycles from a zero initial guess: red-black Gauss-Seidel
// (red = even index sum; nu sweeps red->black before, black->red after), restriction
// R = P^T (sum of the 2^d children), piecewise-constant prolongation, Galerkin coarse
// conductances (sum of the fine conductances crossing a coarse face), and an exact solve
// on the coarsest level through its explicit inverse (banded Cholesky factor in double,
// inverse columns by two triangular solves, stored symmetric).  Mirrored smoothing, R = P^T
// and the exact coarse solve keep P a fixed SPD operator.
#include <cuda_runtime.h>

#include <cstdlib>
#include <stdexcept>
#include <string>

#include "kernels.cuh"

namespace plsqr {

// ---- diffusivity (Algorithm 3 step 3) ----------------------------------------------------

template <typename T>
__device__ __forceinline__ T kappa_of(int reg, T Tp, T t) {
    const T q = t / Tp;
    switch (reg) {
        case REG_TIKHONOV: return (T)1;
        case REG_TV: return (T)1 / sqrt(Tp * Tp + t * t);
        case REG_PM_LOG: return (T)1 / ((T)1 + q * q);
        default: return exp(-q * q);
    }
}

template <typename T>
__device__ __forceinline__ T r_of(int reg, T Tp, T t) {
    const T q = t / Tp;
    switch (reg) {
        case REG_TIKHONOV: return (T)0.5 * t * t;
        case REG_TV: return Tp * sqrt((T)1 + q * q);
        case REG_PM_LOG: return (T)0.5 * Tp * Tp * log1p(q * q);
        default: return (T)-0.5 * Tp * Tp * expm1(-q * q);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_diffusivity(const T* __restrict__ f, T* __restrict__ kappa, Dims d,
                                                     GkState* st, Hist hist, double kfloor, Red red,
                                                     __nv_bfloat16* __restrict__ k16) {
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const int reg = st[inst].reg;
    const T Tp = (T)st[inst].T;
    const T kmin = (T)kfloor * kappa_of<T>(reg, Tp, (T)0);
    const T* fi = f + (int64_t)inst * d.N;
    T* ki = kappa + (int64_t)inst * d.N;
    __nv_bfloat16* k16i = k16 ? k16 + (int64_t)inst * d.N : nullptr;
    double part = 0.0;
    const int64_t plane = (int64_t)d.nx * d.ny;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * 256) {
        const uint32_t ri = fdiv((uint32_t)i, d.fx), zu = fdiv(ri, d.fy);
        const int x = (int)((uint32_t)i - ri * (uint32_t)d.nx);
        const int y = (int)(ri - zu * (uint32_t)d.ny);
        const int z = (int)zu;
        const T c = fi[i];
        T gx = (x + 1 < d.nx ? fi[i + 1] : (T)0) - c;
        T t2 = gx * gx;
        T gy = (y + 1 < d.ny ? fi[i + d.nx] : (T)0) - c;
        t2 += gy * gy;
        if (d.ndim == 3) {
            T gz = (z + 1 < d.nz ? fi[i + plane] : (T)0) - c;
            t2 += gz * gz;
        }
        const T t = sqrt(t2);
        const T k = kappa_of<T>(reg, Tp, t);
        const T kc = k > kmin ? k : kmin;
        if (k16i) k16i[i] = __float2bfloat16_rn((float)kc);  // bfloat16 storage: the only copy
        else ki[i] = kc;
        part += (double)r_of<T>(reg, Tp, t);
    }
    double tot;
    if (reduce_last<256>(part, red, inst, blockIdx.x, gridDim.x, &tot)) {
        GkState& s = st[inst];
        const double R_prev = s.R;
        s.R = tot;
        if (hist.R) hist.R[(int64_t)inst * (hist.n_outer + 1) + s.outer] = tot;
        // Algorithm 3 step 5: stop at f^k (k >= 2) when R(f^k) fell by less than r_rel R(f^{k-1})
        if (s.r_rel > 0.0 && s.outer >= 2 && R_prev > 0.0 && (tot - R_prev) / R_prev > -s.r_rel)
            s.status = ST_CONVERGED;
    }
}

template <typename T>
void diffusivity(const T* f, T* kappa, Dims d, int B, GkState* st, Hist hist, double kfloor, Red red,
                 cudaStream_t s, __nv_bfloat16* k16) {
    kbegin(KC_SETUP, s);
    int nblk = std::min(red_blocks(d.N), red.max_blocks);
    k_diffusivity<T><<<dim3(nblk, B), 256, 0, s>>>(f, kappa, d, st, hist, kfloor, red, k16);
    klaunched("k_diffusivity");
    kfinish(s);
}

// ---- level stencil -------------------------------------------------------------------------

// Conductance c_d(i) of the edge i -> i+e_d: kappa_i on the finest level, else cond[d][i].
template <typename T, bool KAPPA>
__device__ __forceinline__ T cond_at(const T* __restrict__ c, int dd, int64_t N, int64_t i) {
    return KAPPA ? c[i] : c[(int64_t)dd * N + i];
}

// diag = sum_d c_d(i) + c_d(i-e_d);  off = sum_d c_d(i) x_{i+e_d} + c_d(i-e_d) x_{i-e_d}
template <typename T, bool KAPPA, bool WITH_X>
__device__ __forceinline__ void stencil(const T* __restrict__ c, const T* x, const Dims& d, int64_t i, int cx,
                                        int cy, int cz, T& diag, T& off) {
    diag = (T)0;
    off = (T)0;
    const int co[3] = {cx, cy, cz};
    const int n[3] = {d.nx, d.ny, d.nz};
    const int64_t strd[3] = {1, (int64_t)d.nx, (int64_t)d.nx * d.ny};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        if (dd >= d.ndim) break;
        const T chi = cond_at<T, KAPPA>(c, dd, d.N, i);
        if (co[dd] > 0) {
            const T clo = cond_at<T, KAPPA>(c, dd, d.N, i - strd[dd]);
            diag += chi + clo;
            if (WITH_X) {
                if (co[dd] + 1 < n[dd]) off += chi * x[i + strd[dd]];
                off += clo * x[i - strd[dd]];
            }
        } else {
            diag += chi;
            if (WITH_X && co[dd] + 1 < n[dd]) off += chi * x[i + strd[dd]];
        }
    }
}

// One red-black Gauss-Seidel half sweep: cells of `colour` get x = (b + off) * (1 / diag) (the
// form of the temporally blocked kernels, which keep 1 / diag per cell).
// zero_init: x is implicitly 0 (first half sweep of a level); the other colour is written 0.
// ZC: each thread takes the cell (h, y) of ZC consecutive planes (3D; the loads of several planes in
// flight together); the arithmetic of a cell does not depend on ZC.
template <typename T, bool KAPPA, bool ZERO, int ZC>
__global__ void __launch_bounds__(256) k_gs_half(const T* __restrict__ cond, const T* __restrict__ b, T* x, Dims d,
                                                 int colour) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int hx = d.nx >> 1;
    const int nzc = (d.nz + ZC - 1) / ZC;
    const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (t >= (int64_t)hx * d.ny * nzc) return;
    const uint32_t rest = fdiv((uint32_t)t, d.fh), zc = fdiv(rest, d.fy);
    const int y = (int)(rest - zc * (uint32_t)d.ny);
    const int hh = (int)((uint32_t)t - rest * (uint32_t)hx);
    const T* c = cond + (KAPPA ? (int64_t)inst * d.N : (int64_t)inst * d.ndim * d.N);
    const T* bi = b + (int64_t)inst * d.N;
    T* xi = x + (int64_t)inst * d.N;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int z = (int)zc * ZC + k;
        if (z < d.nz) {
            const int par = (y + z + colour) & 1;
            const int xx = 2 * hh + par;
            const int64_t i = xx + (int64_t)d.nx * (y + (int64_t)d.ny * z);
            T diag, off;
            stencil<T, KAPPA, !ZERO>(c, xi, d, i, xx, y, z, diag, off);
            xi[i] = (bi[i] + off) * ((T)1 / diag);
            if (ZERO) xi[i + (par ? -1 : 1)] = (T)0;
        }
    }
}

template <typename T>
void mg_gs_half(const T* cond, bool is_kappa, const T* b, T* x, Dims d, int colour, bool zero_init, int B,
                cudaStream_t s, int zc) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
    if (zc != 2 && zc != 4) zc = 1;
    const int64_t threads = (int64_t)(d.nx / 2) * d.ny * ((d.nz + zc - 1) / zc);
    dim3 grid((unsigned)((threads + 255) / 256), B);
#define GS_HALF(K, Z, C) launch_k(k_gs_half<T, K, Z, C>, grid, dim3(256), 0, s, cond, b, x, d, colour)
#define GS_HALF_ZC(K, Z)                \
    switch (zc) {                       \
        case 2: GS_HALF(K, Z, 2); break; \
        case 4: GS_HALF(K, Z, 4); break; \
        default: GS_HALF(K, Z, 1); break; \
    }
    if (is_kappa) {
        if (zero_init) GS_HALF_ZC(true, true) else GS_HALF_ZC(true, false)
    } else {
        if (zero_init) GS_HALF_ZC(false, true) else GS_HALF_ZC(false, false)
    }
#undef GS_HALF_ZC
#undef GS_HALF
    klaunched("k_gs_half");
    kfinish(s);
}

// Coarse right-hand side: bc_I = sum over the 2^d children i of (b_i - (M x)_i).
template <typename T, bool KAPPA>
__global__ void __launch_bounds__(256) k_resid_restrict(const T* __restrict__ cond, const T* __restrict__ b,
                                                        const T* __restrict__ x, T* __restrict__ bc, Dims df,
                                                        Dims dc) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int64_t I = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (I >= dc.N) return;
    const uint32_t rI = fdiv((uint32_t)I, dc.fx), Zu = fdiv(rI, dc.fy);
    const int X = (int)((uint32_t)I - rI * (uint32_t)dc.nx), Y = (int)(rI - Zu * (uint32_t)dc.ny), Z = (int)Zu;
    const T* c = cond + (KAPPA ? (int64_t)inst * df.N : (int64_t)inst * df.ndim * df.N);
    const T* bi = b + (int64_t)inst * df.N;
    const T* xi = x + (int64_t)inst * df.N;
    T sum = (T)0;
    const int zc = df.ndim == 3 ? 2 : 1;
    for (int oz = 0; oz < zc; ++oz)
        for (int oy = 0; oy < 2; ++oy)
            for (int ox = 0; ox < 2; ++ox) {
                const int fx = 2 * X + ox, fy = 2 * Y + oy, fz = df.ndim == 3 ? 2 * Z + oz : 0;
                const int64_t i = fx + (int64_t)df.nx * (fy + (int64_t)df.ny * fz);
                T diag, off;
                stencil<T, KAPPA, true>(c, xi, df, i, fx, fy, fz, diag, off);
                sum += bi[i] - (diag * xi[i] - off);
            }
    bc[(int64_t)inst * dc.N + I] = sum;
}

template <typename T>
void mg_resid_restrict(const T* cond, bool is_kappa, const T* b, const T* x, T* bc, Dims df, Dims dc, int B,
                       cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    dim3 grid((unsigned)((dc.N + 255) / 256), B);
    if (is_kappa) launch_k(k_resid_restrict<T, true>, grid, dim3(256), 0, s, cond, b, x, bc, df, dc);
    else launch_k(k_resid_restrict<T, false>, grid, dim3(256), 0, s, cond, b, x, bc, df, dc);
    klaunched("k_resid_restrict");
    kfinish(s);
}

// x_i += xc_parent(i)
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(const T* __restrict__ xc, T* __restrict__ x, Dims df, Dims dc) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= df.N) return;
    const uint32_t ri = fdiv((uint32_t)i, df.fx), fzu = fdiv(ri, df.fy);
    const int fx = (int)((uint32_t)i - ri * (uint32_t)df.nx), fy = (int)(ri - fzu * (uint32_t)df.ny), fz = (int)fzu;
    const int64_t I = (fx >> 1) + (int64_t)dc.nx * ((fy >> 1) + (int64_t)dc.ny * (fz >> 1));
    x[(int64_t)inst * df.N + i] += xc[(int64_t)inst * dc.N + I];
}

template <typename T>
void mg_prolong_add(const T* xc, T* x, Dims df, Dims dc, int B, cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    launch_k(k_prolong_add<T>, dim3((unsigned)((df.N + 255) / 256), B), dim3(256), 0, s, xc, x, df, dc);
    klaunched("k_prolong_add");
    kfinish(s);
}

// ---- red-black split storage of a 3D level ---------------------------------------------------
//
// With x stored in natural order, a red-black half sweep reads the other colour's neighbours and
// its own right-hand side from sectors of which it uses half, and writes half of each sector of x.
// The split layout keeps the cells of colour c = (x + y + z) & 1 of row (y, z) contiguous:
// xs[c][z][y][h] holds cell x = 2h + p, p = (y + z + c) & 1 (nx even), [inst][2][N/2].  In it the
// other colour's neighbours of a cell (h, y, z) of colour c sit at h - 1 + p and h + p of its own
// row, and at h of the rows y +- 1 and z +- 1; the conductances stay in natural order (a half
// sweep reads all of them anyway).  The arithmetic of every cell is that of the natural-order
// kernels above, in the same order, so the V-cycle is bit for bit the same.

// stencil() for a cell of the split layout: xo = the other colour's array, hs = the cell's index in
// its own colour's array, p its parity in the row.
template <typename T, bool KAPPA, bool WITH_X>
__device__ __forceinline__ void stencil_split(const T* __restrict__ c, const T* xo, const Dims& d, int64_t i,
                                              int64_t hs, int nh, int p, int cx, int cy, int cz, T& diag, T& off) {
    diag = (T)0;
    off = (T)0;
    const int co[3] = {cx, cy, cz};
    const int n[3] = {d.nx, d.ny, d.nz};
    const int64_t strd[3] = {1, (int64_t)d.nx, (int64_t)d.nx * d.ny};
    const int64_t hi[3] = {hs + p, hs + nh, hs + (int64_t)nh * d.ny};
    const int64_t lo[3] = {hs - 1 + p, hs - nh, hs - (int64_t)nh * d.ny};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        const T chi = cond_at<T, KAPPA>(c, dd, d.N, i);
        if (co[dd] > 0) {
            const T clo = cond_at<T, KAPPA>(c, dd, d.N, i - strd[dd]);
            diag += chi + clo;
            if (WITH_X) {
                if (co[dd] + 1 < n[dd]) off += chi * xo[hi[dd]];
                off += clo * xo[lo[dd]];
            }
        } else {
            diag += chi;
            if (WITH_X && co[dd] + 1 < n[dd]) off += chi * xo[hi[dd]];
        }
    }
}

// One half sweep in the split layout.  MODE 0: first half sweep of the finest level (x = 0 before
// it): b is in natural order and is also written out split (bs) for the later sweeps; the other
// colour of x is written 0.  MODE 1: first half sweep of a coarser level (b split, x = 0 before).
// MODE 2: any other half sweep.  MODE 3: the last half sweep of the finest level, which also
// writes both colours of x in natural order to `out`.  Each thread takes the cells (h, y) of ZC
// consecutive planes, so that the loads of several planes are in flight together (xc and xo, this
// colour's and the other colour's halves of the split array, do not overlap).
template <typename T, bool KAPPA, int MODE, int ZC>
__global__ void __launch_bounds__(256) k_gs_half_split(const T* __restrict__ cond, const T* __restrict__ b,
                                                       T* __restrict__ bs, T* __restrict__ xc_all,
                                                       T* __restrict__ xo_all, T* __restrict__ out, Dims d,
                                                       int colour) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int nh = d.nx >> 1;
    const int64_t Nh = d.N >> 1;
    const int nzc = (d.nz + ZC - 1) / ZC;
    const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (t >= (int64_t)nh * d.ny * nzc) return;
    const uint32_t rest = fdiv((uint32_t)t, d.fh);
    const int zc = (int)fdiv(rest, d.fy), y = (int)(rest - (uint32_t)zc * (uint32_t)d.ny);
    const int h = (int)((uint32_t)t - rest * (uint32_t)nh);
    const T* c = cond + (KAPPA ? (int64_t)inst * d.N : (int64_t)inst * d.ndim * d.N);
    T* xc = xc_all + (int64_t)inst * d.N;  // colour-c half of instance inst (stride d.N between instances)
    T* xo = xo_all + (int64_t)inst * d.N;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int z = zc * ZC + k;
        if (z < d.nz) {
            const int p = (y + z + colour) & 1;
            const int xx = 2 * h + p;
            const int64_t hs = h + (int64_t)nh * (y + (int64_t)d.ny * z);
            const int64_t i = xx + (int64_t)d.nx * (y + (int64_t)d.ny * z);
            T diag, off;
            stencil_split<T, KAPPA, (MODE >= 2)>(c, xo, d, i, hs, nh, p, xx, y, z, diag, off);
            T bv;
            if (MODE == 0) {
                const T* bn = b + (int64_t)inst * d.N;
                bv = bn[i];
                const T bo = bn[i + (p ? -1 : 1)];  // the other colour's cell at the same h
                bs[(int64_t)inst * d.N + (int64_t)colour * Nh + hs] = bv;
                bs[(int64_t)inst * d.N + (int64_t)(1 - colour) * Nh + hs] = bo;
            } else {
                bv = b[(int64_t)inst * d.N + (int64_t)colour * Nh + hs];
            }
            const T xn = (bv + off) * ((T)1 / diag);
            xc[hs] = xn;
            if (MODE <= 1) xo[hs] = (T)0;
            if (MODE == 3) {
                T* o = out + (int64_t)inst * d.N;
                o[i] = xn;
                o[i + (p ? -1 : 1)] = xo[hs];
            }
        }
    }
}

// planes per thread of the split half sweep (PLSQR_MG3_ZC = 1, 2, 4 or 8; 2 measured best)
int split_planes() {
    static int zc = [] {
        const char* e = std::getenv("PLSQR_MG3_ZC");
        const int v = e ? std::atoi(e) : 2;
        return v == 1 || v == 4 || v == 8 ? v : 2;
    }();
    return zc;
}

template <typename T>
void mg_gs_half_split(const T* cond, bool is_kappa, const T* b, T* bs, T* xs, T* out, Dims d, int colour, int mode,
                      int B, cudaStream_t s) {
    kbegin(is_kappa ? KC_GS_FINE : KC_MG_OTHER, s);
    const int zcn = split_planes();
    const int64_t Nh = d.N / 2;
    T* xc = xs + (int64_t)colour * Nh;
    T* xo = xs + (int64_t)(1 - colour) * Nh;
    const int64_t threads = (int64_t)(d.nx / 2) * d.ny * ((d.nz + zcn - 1) / zcn);
    dim3 grid((unsigned)((threads + 255) / 256), B);
#define GS_SPLIT(K, M, Z) launch_k(k_gs_half_split<T, K, M, Z>, grid, dim3(256), 0, s, cond, b, bs, xc, xo, out, d, colour)
#define GS_SPLIT_Z(K, M)                 \
    switch (zcn) {                       \
        case 1: GS_SPLIT(K, M, 1); break; \
        default: GS_SPLIT(K, M, 2); break; \
        case 8: GS_SPLIT(K, M, 8); break; \
        case 4: GS_SPLIT(K, M, 4); break; \
    }
    if (is_kappa) {
        switch (mode) {
            case 0: GS_SPLIT_Z(true, 0); break;
            case 1: GS_SPLIT_Z(true, 1); break;
            case 2: GS_SPLIT_Z(true, 2); break;
            default: GS_SPLIT_Z(true, 3); break;
        }
    } else {
        switch (mode) {
            case 0: GS_SPLIT_Z(false, 0); break;
            case 1: GS_SPLIT_Z(false, 1); break;
            case 2: GS_SPLIT_Z(false, 2); break;
            default: GS_SPLIT_Z(false, 3); break;
        }
    }
#undef GS_SPLIT_Z
#undef GS_SPLIT
    klaunched("k_gs_half_split");
    kfinish(s);
}

// k_resid_restrict with b and x split; the coarse right-hand side is written split (OUT_SPLIT,
// for a coarse level that is smoothed) or in natural order (the coarsest level).
template <typename T, bool KAPPA, bool OUT_SPLIT>
__global__ void __launch_bounds__(256) k_resid_restrict_split(const T* __restrict__ cond, const T* __restrict__ bs,
                                                              const T* __restrict__ xs, T* __restrict__ bc, Dims df,
                                                              Dims dc) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int64_t I = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (I >= dc.N) return;
    const uint32_t rI = fdiv((uint32_t)I, dc.fx), Zu = fdiv(rI, dc.fy);
    const int X = (int)((uint32_t)I - rI * (uint32_t)dc.nx), Y = (int)(rI - Zu * (uint32_t)dc.ny), Z = (int)Zu;
    const T* c = cond + (KAPPA ? (int64_t)inst * df.N : (int64_t)inst * df.ndim * df.N);
    const int nh = df.nx >> 1;
    const int64_t Nh = df.N >> 1;
    const T* bi = bs + (int64_t)inst * df.N;
    const T* xi = xs + (int64_t)inst * df.N;
    T sum = (T)0;
    for (int oz = 0; oz < 2; ++oz)
        for (int oy = 0; oy < 2; ++oy)
            for (int ox = 0; ox < 2; ++ox) {
                const int fx = 2 * X + ox, fy = 2 * Y + oy, fz = 2 * Z + oz;
                const int64_t i = fx + (int64_t)df.nx * (fy + (int64_t)df.ny * fz);
                const int cc = (fx + fy + fz) & 1;
                const int64_t hs = (fx >> 1) + (int64_t)nh * (fy + (int64_t)df.ny * fz);
                T diag, off;
                stencil_split<T, KAPPA, true>(c, xi + (int64_t)(1 - cc) * Nh, df, i, hs, nh, fx & 1, fx, fy, fz, diag,
                                              off);
                sum += bi[(int64_t)cc * Nh + hs] - (diag * xi[(int64_t)cc * Nh + hs] - off);
            }
    if (OUT_SPLIT) {
        const int64_t Hs = (X >> 1) + (int64_t)(dc.nx >> 1) * (Y + (int64_t)dc.ny * Z);
        bc[(int64_t)inst * dc.N + (int64_t)((X + Y + Z) & 1) * (dc.N >> 1) + Hs] = sum;
    } else {
        bc[(int64_t)inst * dc.N + I] = sum;
    }
}

template <typename T>
void mg_resid_restrict_split(const T* cond, bool is_kappa, const T* bs, const T* xs, T* bc, bool out_split, Dims df,
                             Dims dc, int B, cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    dim3 grid((unsigned)((dc.N + 255) / 256), B);
#define RR_SPLIT(K, O) launch_k(k_resid_restrict_split<T, K, O>, grid, dim3(256), 0, s, cond, bs, xs, bc, df, dc)
    if (is_kappa) {
        if (out_split) RR_SPLIT(true, true);
        else RR_SPLIT(true, false);
    } else {
        if (out_split) RR_SPLIT(false, true);
        else RR_SPLIT(false, false);
    }
#undef RR_SPLIT
    klaunched("k_resid_restrict_split");
    kfinish(s);
}

// x_i += xc_parent(i) with x split; the coarse correction split (IN_SPLIT) or in natural order.
template <typename T, bool IN_SPLIT>
__global__ void __launch_bounds__(256) k_prolong_add_split(const T* __restrict__ xc, T* __restrict__ xs, Dims df,
                                                           Dims dc) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x;  // colour-major index of the split layout
    if (q >= df.N) return;
    const int nh = df.nx >> 1;
    const int64_t Nh = df.N >> 1;
    const int colour = q >= Nh ? 1 : 0;
    const int64_t hs = q - colour * Nh;
    const uint32_t rest = fdiv((uint32_t)hs, df.fh);
    const int fz = (int)fdiv(rest, df.fy), fy = (int)(rest - (uint32_t)fz * (uint32_t)df.ny);
    const int fx = 2 * (int)((uint32_t)hs - rest * (uint32_t)nh) + ((fy + fz + colour) & 1);
    const int X = fx >> 1, Y = fy >> 1, Z = fz >> 1;
    const int64_t I = IN_SPLIT ? (int64_t)((X + Y + Z) & 1) * (dc.N >> 1) + (X >> 1) +
                                     (int64_t)(dc.nx >> 1) * (Y + (int64_t)dc.ny * Z)
                               : X + (int64_t)dc.nx * (Y + (int64_t)dc.ny * Z);
    xs[(int64_t)inst * df.N + q] += xc[(int64_t)inst * dc.N + I];
}

template <typename T>
void mg_prolong_add_split(const T* xc, bool in_split, T* xs, Dims df, Dims dc, int B, cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    dim3 grid((unsigned)((df.N + 255) / 256), B);
    if (in_split) launch_k(k_prolong_add_split<T, true>, grid, dim3(256), 0, s, xc, xs, df, dc);
    else launch_k(k_prolong_add_split<T, false>, grid, dim3(256), 0, s, xc, xs, df, dc);
    klaunched("k_prolong_add_split");
    kfinish(s);
}

// y = M x, or y = b - M x when b is given.
template <typename T, bool KAPPA>
__global__ void __launch_bounds__(256) k_apply_level(const T* __restrict__ cond, const T* __restrict__ x,
                                                     const T* __restrict__ b, T* __restrict__ y, Dims d) {
    pdl_grid_sync();
    const int inst = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= d.N) return;
    const uint32_t ri = fdiv((uint32_t)i, d.fx), czu = fdiv(ri, d.fy);
    const int cx = (int)((uint32_t)i - ri * (uint32_t)d.nx), cy = (int)(ri - czu * (uint32_t)d.ny), cz = (int)czu;
    const T* c = cond + (KAPPA ? (int64_t)inst * d.N : (int64_t)inst * d.ndim * d.N);
    const T* xi = x + (int64_t)inst * d.N;
    T diag, off;
    stencil<T, KAPPA, true>(c, xi, d, i, cx, cy, cz, diag, off);
    const T mx = diag * xi[i] - off;
    y[(int64_t)inst * d.N + i] = b ? b[(int64_t)inst * d.N + i] - mx : mx;
}

template <typename T>
void mg_apply_level(const T* cond, bool is_kappa, const T* x, const T* b, T* y, Dims d, int B, cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    dim3 grid((unsigned)((d.N + 255) / 256), B);
    if (is_kappa) launch_k(k_apply_level<T, true>, grid, dim3(256), 0, s, cond, x, b, y, d);
    else launch_k(k_apply_level<T, false>, grid, dim3(256), 0, s, cond, x, b, y, d);
    klaunched("k_apply_level");
    kfinish(s);
}

template <typename T>
__global__ void k_axpy(T* y, const T* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) y[i] += x[i];
}

template <typename T>
void mg_axpy(T* y, const T* x, int64_t n, cudaStream_t s) {
    kbegin(KC_MG_OTHER, s);
    int nblk = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_axpy<T><<<nblk, 256, 0, s>>>(y, x, n);
    klaunched("k_axpy");
    kfinish(s);
}

// Galerkin coarsening: c_{l+1,d}(I) = sum of c_{l,d}(i) over the fine cells i of coarse
// cell I with i_d = 2 I_d + 1 (their edge i -> i+e_d crosses the high face of I).
template <typename T, bool KAPPA>
__global__ void __launch_bounds__(256) k_coarsen(const T* __restrict__ cf, T* __restrict__ cc, Dims df, Dims dc,
                                                 const __nv_bfloat16* __restrict__ k16) {
    const int inst = blockIdx.y;
    const int64_t I = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (I >= dc.N) return;
    const uint32_t rI = fdiv((uint32_t)I, dc.fx), Zu = fdiv(rI, dc.fy);
    const int X = (int)((uint32_t)I - rI * (uint32_t)dc.nx), Y = (int)(rI - Zu * (uint32_t)dc.ny), Z = (int)Zu;
    const T* c = cf + (KAPPA ? (int64_t)inst * df.N : (int64_t)inst * df.ndim * df.N);
    T* o = cc + (int64_t)inst * dc.ndim * dc.N;
    for (int dd = 0; dd < df.ndim; ++dd) {
        const int zlo = df.ndim == 3 ? (dd == 2 ? 2 * Z + 1 : 2 * Z) : 0;
        const int zhi = df.ndim == 3 ? 2 * Z + 1 : 0;
        const int ylo = dd == 1 ? 2 * Y + 1 : 2 * Y, yhi = 2 * Y + 1;
        const int xlo = dd == 0 ? 2 * X + 1 : 2 * X, xhi = 2 * X + 1;
        T s = (T)0;
        for (int fz = zlo; fz <= zhi; ++fz)
            for (int fy = ylo; fy <= yhi; ++fy)
                for (int fx = xlo; fx <= xhi; ++fx) {
                    const int64_t i = fx + (int64_t)df.nx * (fy + (int64_t)df.ny * fz);
                    s += (KAPPA && k16) ? (T)__bfloat162float(k16[(int64_t)inst * df.N + i])
                                        : cond_at<T, KAPPA>(c, dd, df.N, i);
                }
        o[(int64_t)dd * dc.N + I] = s;
    }
}

template <typename T>
void mg_coarsen(const T* cf, bool fine_is_kappa, T* cc, Dims df, Dims dc, int B, cudaStream_t s,
                const __nv_bfloat16* k16) {
    kbegin(KC_SETUP, s);
    dim3 grid((unsigned)((dc.N + 255) / 256), B);
    if (fine_is_kappa) k_coarsen<T, true><<<grid, 256, 0, s>>>(cf, cc, df, dc, k16);
    else k_coarsen<T, false><<<grid, 256, 0, s>>>(cf, cc, df, dc, nullptr);
    klaunched("k_coarsen");
    kfinish(s);
}

// 1 / diagonal of a 2D level: ((c_x(i) + c_x(i-1)) + c_y(i)) + c_y(i-nx), the edges missing at
// the low boundary counted as 0 -- the summation order of the red-black smoother, so the staged
// value is bit for bit the one a tile would form.  kappa may come from its bfloat16 copy.
template <typename T, bool KAPPA>
__global__ void __launch_bounds__(256) k_rdiag2d(const T* __restrict__ cond, T* __restrict__ rd, Dims d,
                                                 const __nv_bfloat16* __restrict__ k16) {
    const int inst = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= d.N) return;
    const int x = (int)(i % d.nx), y = (int)(i / d.nx);
    const T* c = cond + (KAPPA ? (int64_t)inst * d.N : (int64_t)inst * 2 * d.N);
    const __nv_bfloat16* k = k16 ? k16 + (int64_t)inst * d.N : nullptr;
    auto cx = [&](int64_t j) -> T { return (KAPPA && k) ? (T)__bfloat162float(k[j]) : c[j]; };
    auto cy = [&](int64_t j) -> T { return KAPPA ? cx(j) : c[d.N + j]; };
    T diag = cx(i);
    diag += x > 0 ? cx(i - 1) : (T)0;
    diag += cy(i);
    diag += y > 0 ? cy(i - d.nx) : (T)0;
    rd[(int64_t)inst * d.N + i] = (T)1 / diag;
}

template <typename T>
void mg_rdiag2d(const T* cond, bool is_kappa, T* rd, Dims d, int B, cudaStream_t s, const __nv_bfloat16* k16) {
    kbegin(KC_SETUP, s);
    dim3 grid((unsigned)((d.N + 255) / 256), B);
    if (is_kappa) k_rdiag2d<T, true><<<grid, 256, 0, s>>>(cond, rd, d, k16);
    else k_rdiag2d<T, false><<<grid, 256, 0, s>>>(cond, rd, d, nullptr);
    klaunched("k_rdiag2d");
    kfinish(s);
}

// ---- exact coarse solve ----------------------------------------------------------------------

// Lower band of the coarsest operator in double: band[i][k] = M(i, i-k), k = 0..bw.
template <typename T, bool KAPPA>
__global__ void __launch_bounds__(256) k_coarse_assemble(const T* __restrict__ cond, double* __restrict__ band,
                                                         Dims d, int bw) {
    const int inst = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= d.N) return;
    const int W = bw + 1;
    double* row = band + ((int64_t)inst * d.N + i) * W;
    for (int k = 0; k < W; ++k) row[k] = 0.0;
    const uint32_t ri = fdiv((uint32_t)i, d.fx), czu = fdiv(ri, d.fy);
    const int cx = (int)((uint32_t)i - ri * (uint32_t)d.nx), cy = (int)(ri - czu * (uint32_t)d.ny), cz = (int)czu;
    const T* c = cond + (KAPPA ? (int64_t)inst * d.N : (int64_t)inst * d.ndim * d.N);
    T diag, off;
    stencil<T, KAPPA, false>(c, (const T*)nullptr, d, i, cx, cy, cz, diag, off);
    row[0] = (double)diag;
    const int co[3] = {cx, cy, cz};
    const int64_t strd[3] = {1, (int64_t)d.nx, (int64_t)d.nx * d.ny};
    for (int dd = 0; dd < d.ndim; ++dd)
        if (co[dd] > 0) row[strd[dd]] = -(double)cond_at<T, KAPPA>(c, dd, d.N, i - strd[dd]);
}

template <typename T>
void coarse_assemble(const T* cond, bool is_kappa, double* band, Dims d, int bw, int B, cudaStream_t s) {
    kbegin(KC_SETUP, s);
    dim3 grid((unsigned)((d.N + 255) / 256), B);
    if (is_kappa) k_coarse_assemble<T, true><<<grid, 256, 0, s>>>(cond, band, d, bw);
    else k_coarse_assemble<T, false><<<grid, 256, 0, s>>>(cond, band, d, bw);
    klaunched("k_coarse_assemble");
    kfinish(s);
}

// In-place banded Cholesky M = L L^T, one block per instance.  The rows that column j touches
// live in a sliding window of bw+4 rows in shared memory.  Column j:
//  phase 1: the factors f_i = L(i,j)/a_j of the column (one per row), scaling of column j-1 by
//           1/sqrt(a_{j-1}) with L(j-1,j-1) = sqrt(a_{j-1}), write-back of the finished row j-2
//           and load of row j+bw+1 into the slot row j-3 left (all on disjoint entries);
//  phase 2: the trailing update L(i,k) -= f_i L(k,j), j < k <= i <= j+bw, with the
//           bw(bw+1)/2 pairs packed densely over the threads (the double-precision pipe is
//           narrow, so lanes that would sit predicated off cost as much as busy ones).
// The thread that updates the next pivot forms 1/a, sqrt(a) and 1/sqrt(a) once (triple-
// buffered in shared memory).  rdiag receives 1/L(j,j).
__global__ void __launch_bounds__(1024) k_chol_band(double* band_all, double* rdiag_all, int nc, int bw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int W = bw + 1, S = bw + 4;
    const int P = bw * (bw + 1) / 2;
    double* win = reinterpret_cast<double*>(smraw);
    double* sf = win + (size_t)S * W;                            // bw factors
    unsigned short* pii = reinterpret_cast<unsigned short*>(sf + bw);  // pair table
    unsigned short* pkk = pii + P;
    __shared__ double s_inv[3], s_sq[3], s_rsq[3];
    double* band = band_all + (int64_t)blockIdx.x * nc * W;
    double* rdiag = rdiag_all + (int64_t)blockIdx.x * nc;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int ii = tid; ii < bw; ii += nt) {  // pairs of row ii: (ii, 0..ii) at ii(ii+1)/2
        const int base = ii * (ii + 1) / 2;
        for (int kk = 0; kk <= ii; ++kk) {
            pii[base + kk] = (unsigned short)ii;
            pkk[base + kk] = (unsigned short)kk;
        }
    }
    const int nload = min(bw + 1, nc);
    for (int e = tid; e < nload * W; e += nt) {
        const int r = e / W, k = e - r * W;
        win[(r % S) * W + k] = band[(int64_t)r * W + k];
    }
    __syncthreads();
    if (tid == 0) {
        const double a = win[0], r = rsqrt_nr(a);
        s_inv[0] = r * r;
        s_sq[0] = a * r;
        s_rsq[0] = r;
    }
    __syncthreads();
    for (int j = 0; j <= nc; ++j) {
        // phase 1
        if (j < nc) {
            const double inv_a = s_inv[j % 3];
            const int base = (j + 1) % S;
            for (int ii = tid; ii < bw; ii += nt) {
                const int i = j + 1 + ii;
                int si = base + ii;
                if (si >= S) si -= S;
                sf[ii] = i < nc ? win[si * W + ii + 1] * inv_a : 0.0;  // L(i, j) / a_j
            }
        }
        if (j >= 1) {
            const int c = (j - 1) % 3;
            const double rs = s_rsq[c];
            for (int t = tid; t < W; t += nt) {
                const int i = j - 1 + t;
                if (i >= nc) break;
                double* Ri = win + (i % S) * W;
                if (t == 0) {
                    Ri[0] = s_sq[c];
                    rdiag[i] = rs;
                } else {
                    Ri[t] *= rs;
                }
            }
        }
        if (j >= 2) {
            const int r = j - 2;
            for (int k = tid; k < W; k += nt) band[(int64_t)r * W + k] = win[(r % S) * W + k];
        }
        {
            const int r = j + bw + 1;
            if (r < nc)
                for (int k = tid; k < W; k += nt) win[(r % S) * W + k] = band[(int64_t)r * W + k];
        }
        __syncthreads();
        // phase 2
        if (j < nc) {
            const int base = (j + 1) % S;
            for (int pidx = tid; pidx < P; pidx += nt) {
                const int ii = pii[pidx], kk = pkk[pidx];
                if (j + 1 + ii >= nc) continue;
                const double f = sf[ii];
                if (f == 0.0) continue;
                int si = base + ii, sk = base + kk;
                if (si >= S) si -= S;
                if (sk >= S) sk -= S;
                win[si * W + (ii - kk)] -= f * win[sk * W + kk + 1];  // L(i,k) -= f_i L(k,j)
            }
            if (tid == 0 && j + 1 < nc) {  // thread 0 owns the pair (0, 0): L(j+1, j+1)
                const double a = win[base * W], r = rsqrt_nr(a);
                const int c = (j + 1) % 3;
                s_inv[c] = r * r;
                s_sq[c] = a * r;
                s_rsq[c] = r;
            }
        }
        __syncthreads();
    }
    {
        const int r = nc - 1;
        for (int k = tid; k < W; k += nt) band[(int64_t)r * W + k] = win[(r % S) * W + k];
    }
}

void coarse_cholesky(double* band, double* rdiag, int nc, int bw, int B, cudaStream_t s) {
    kbegin(KC_SETUP, s);
    const int P = bw * (bw + 1) / 2;
    const size_t smem = sizeof(double) * ((size_t)(bw + 4) * (bw + 1) + bw) + sizeof(unsigned short) * 2 * P;
    if (smem > 227 * 1024) throw std::runtime_error("coarse_cholesky: band too wide for shared memory");
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_chol_band, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int nt = std::min(1024, std::max(64, ((P + 31) / 32) * 32));
    k_chol_band<<<B, nt, smem, s>>>(band, rdiag, nc, bw);
    klaunched("k_chol_band");
    kfinish(s);
}

// Inverse of the coarsest operator from its band factor, X = L^{-T} L^{-1}, stored full and
// exactly symmetric: for each column c,
//   forward  y_i = (delta_ic - sum_m L(i, i-m) y_{i-m}) / L(i,i),      i = c .. nc-1
//   backward x_i = (y_i      - sum_m L(i+m, i) x_{i+m}) / L(i,i),      i = nc-1 .. c
// y is parked in X(i, c); x overwrites it and is mirrored to X(c, i).  The rows are walked by a
// whole warp together, so the band row read is the same for all its lanes (broadcast).
// Narrow-band inverse with four lanes per column: lane q of the quad keeps window entries
// m = 8q .. 8q+7 and their partial sum; the quad adds the four partial sums (two butterfly
// shuffles) and passes the entry that leaves one lane's part of the window to the next lane
// (shuffle up within the quad).  Four times the parallelism of one lane per column, so the
// double-precision pipe stays busy even for one instance.
__device__ __forceinline__ double quad_sum(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2, 4);
    return v;
}

__global__ void __launch_bounds__(128) k_band_inverse_quad(const double* __restrict__ band_all,
                                                           const double* __restrict__ rdiag_all,
                                                           double* __restrict__ X_all, int nc, int bw) {
    const int inst = blockIdx.y;
    const int q = threadIdx.x & 3;
    const int c = blockIdx.x * 32 + (threadIdx.x >> 2);       // column of this quad
    const int c0 = blockIdx.x * 32 + ((threadIdx.x & ~31) >> 2);  // first column of this warp
    if (c0 >= nc) return;
    const int W = bw + 1;
    const double* band = band_all + (int64_t)inst * nc * W;
    const double* rdiag = rdiag_all + (int64_t)inst * nc;
    double* X = X_all + (int64_t)inst * nc * nc;
    const bool live = c < nc;
    const int mb = 8 * q;  // first window index of this lane
    double win[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) win[t] = 0.0;
    // forward: y_i = (delta_ic - sum_m L(i, i-1-m) y_{i-1-m}) / L(i,i); win[t] = y_{i-1-(mb+t)}
    for (int i = c0; i < nc; ++i) {
        const double* Li = band + (int64_t)i * W;
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            if (mb + t < bw) s0 = fma(Li[mb + t + 1], win[t], s0);
            if (mb + t + 1 < bw) s1 = fma(Li[mb + t + 2], win[t + 1], s1);
        }
        const double s = quad_sum(s0 + s1);
        double yi = ((i == c ? 1.0 : 0.0) - s) * rdiag[i];
        if (i < c || !live) yi = 0.0;
        const double carry = __shfl_up_sync(0xffffffffu, win[7], 1, 4);
#pragma unroll
        for (int t = 7; t > 0; --t) win[t] = win[t - 1];
        win[0] = q == 0 ? yi : carry;
        if (q == 0 && live && i >= c) X[(int64_t)i * nc + c] = yi;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) win[t] = 0.0;
    // backward: x_i = (y_i - sum_m L(i+1+m, i) x_{i+1+m}) / L(i,i); win[t] = x_{i+1+(mb+t)}
    for (int i = nc - 1; i >= c0; --i) {
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            const int m0 = mb + t, m1 = mb + t + 1;
            if (m0 < bw && i + 1 + m0 < nc) s0 = fma(band[(int64_t)(i + 1 + m0) * W + 1 + m0], win[t], s0);
            if (m1 < bw && i + 1 + m1 < nc) s1 = fma(band[(int64_t)(i + 1 + m1) * W + 1 + m1], win[t + 1], s1);
        }
        const double s = quad_sum(s0 + s1);
        double xi = 0.0;
        if (live && i >= c) xi = (X[(int64_t)i * nc + c] - s) * rdiag[i];
        const double carry = __shfl_up_sync(0xffffffffu, win[7], 1, 4);
#pragma unroll
        for (int t = 7; t > 0; --t) win[t] = win[t - 1];
        win[0] = q == 0 ? xi : carry;
        if (q == 0 && live && i >= c) {
            X[(int64_t)i * nc + c] = xi;
            X[(int64_t)c * nc + i] = xi;
        }
    }
}

__global__ void k_band_inverse(const double* __restrict__ band_all, const double* __restrict__ rdiag_all,
                               double* __restrict__ X_all, int nc, int bw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int inst = blockIdx.y;
    const int j = blockIdx.x * wpb + warp;
    if (j >= nc) return;
    const double* band = band_all + (int64_t)inst * nc * (bw + 1);
    const double* rdiag = rdiag_all + (int64_t)inst * nc;
    double* X = X_all + (int64_t)inst * nc * nc;
    double* y = reinterpret_cast<double*>(smraw) + (int64_t)warp * nc;
    const int W = bw + 1;
    for (int i = j; i < nc; ++i) {
        double s = 0.0;
        const int kmin = max(j, i - bw);
        for (int k = i - 1 - lane; k >= kmin; k -= 32) s += band[(int64_t)i * W + (i - k)] * y[k];
        s = warp_sum(s);
        const double yi = ((i == j ? 1.0 : 0.0) - s) * rdiag[i];
        if (lane == 0) y[i] = yi;
        __syncwarp();
    }
    for (int i = nc - 1; i >= j; --i) {
        double s = 0.0;
        const int kmax = min(i + bw, nc - 1);
        for (int k = i + 1 + lane; k <= kmax; k += 32) s += band[(int64_t)k * W + (k - i)] * y[k];
        s = warp_sum(s);
        const double xi = (y[i] - s) * rdiag[i];
        __syncwarp();
        if (lane == 0) y[i] = xi;
        __syncwarp();
    }
    for (int i = j + lane; i < nc; i += 32) {
        const double v = y[i];
        X[(int64_t)i * nc + j] = v;
        X[(int64_t)j * nc + i] = v;
    }
}

void coarse_inverse(const double* band, const double* rdiag, double* X, int nc, int bw, int B, cudaStream_t s) {
    if (bw <= 32) {
        kbegin(KC_SETUP, s);
        dim3 grid((nc + 31) / 32, B);  // 32 columns (8 warps of 4-lane quads) per block
        k_band_inverse_quad<<<grid, 128, 0, s>>>(band, rdiag, X, nc, bw);
        klaunched("k_band_inverse_quad");
        kfinish(s);
        return;
    }
    int wpb = 8;
    while (wpb > 1 && (size_t)wpb * nc * sizeof(double) > 200 * 1024) wpb >>= 1;
    size_t smem = (size_t)wpb * nc * sizeof(double);
    if (smem > 227 * 1024) throw std::runtime_error("coarse_inverse: coarsest level too large");
    kbegin(KC_SETUP, s);
    auto kfn = k_band_inverse;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((nc + wpb - 1) / wpb, B);
    kfn<<<grid, wpb * 32, smem, s>>>(band, rdiag, X, nc, bw);
    klaunched("k_band_inverse");
    kfinish(s);
}

// x = X b on the coarsest level, one warp per row.  Double-precision handles: X and the sums in
// double.  Single-precision handles: X rounded to float once per outer step (half the bytes per
// V-cycle), sums in float -- the coarse correction then carries an error of a few float ulps of
// |X||b|, below that of the single-precision smoothing around it.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_symv(const T* __restrict__ X_all, const T* __restrict__ b_all,
                                                     T* __restrict__ x_all, int nc, const GkState* st) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sb = reinterpret_cast<T*>(smraw);
    pdl_grid_sync();
    const int inst = blockIdx.y;
    if (st && (parked(st[inst]) || st[inst].frozen >= 2)) return;
    const T* b = b_all + (int64_t)inst * nc;
    for (int i = threadIdx.x; i < nc; i += 256) sb[i] = b[i];
    __syncthreads();
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= nc) return;
    const T acc = coarse_row_dot<T>(X_all + (int64_t)inst * nc * nc + (int64_t)row * nc, sb, nc, lane);
    if (lane == 0) x_all[(int64_t)inst * nc + row] = acc;
}

template <typename T>
void coarse_symv(const T* X, const T* b, T* x, int nc, int B, const GkState* st, cudaStream_t s) {
    kbegin(KC_COARSE, s);
    size_t smem = sizeof(T) * nc;
    auto kfn = k_coarse_symv<T>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_k(kfn, dim3((nc + 7) / 8, B), dim3(256), smem, s, X, b, x, nc, st);
    klaunched("k_coarse_symv");
    kfinish(s);
}

__global__ void k_round_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) b[i] = (float)a[i];
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
        b[i] = __float2bfloat16_rn(a[i]);
}

void to_bf16(const float* a, __nv_bfloat16* b, int64_t n, cudaStream_t s) {
    kbegin(KC_SETUP, s);
    k_to_bf16<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(a, b, n);
    klaunched("k_to_bf16");
    kfinish(s);
}

void round_to_float(const double* a, float* b, int64_t n, cudaStream_t s) {
    kbegin(KC_SETUP, s);
    k_round_to_float<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(a, b, n);
    klaunched("k_round_to_float");
    kfinish(s);
}

#define PLSQR_INST_MG(T)                                                                                  \
    template void diffusivity<T>(const T*, T*, Dims, int, GkState*, Hist, double, Red, cudaStream_t,         \
                                 __nv_bfloat16*);                                                         \
    template void mg_coarsen<T>(const T*, bool, T*, Dims, Dims, int, cudaStream_t, const __nv_bfloat16*);  \
    template void mg_rdiag2d<T>(const T*, bool, T*, Dims, int, cudaStream_t, const __nv_bfloat16*);        \
    template void mg_gs_half<T>(const T*, bool, const T*, T*, Dims, int, bool, int, cudaStream_t, int);    \
    template void mg_resid_restrict<T>(const T*, bool, const T*, const T*, T*, Dims, Dims, int,            \
                                       cudaStream_t);                                                     \
    template void mg_prolong_add<T>(const T*, T*, Dims, Dims, int, cudaStream_t);                          \
    template void mg_apply_level<T>(const T*, bool, const T*, const T*, T*, Dims, int, cudaStream_t);      \
    template void mg_axpy<T>(T*, const T*, int64_t, cudaStream_t);                                         \
    template void coarse_assemble<T>(const T*, bool, double*, Dims, int, int, cudaStream_t);               \
    template void coarse_symv<T>(const T*, const T*, T*, int, int, const GkState*, cudaStream_t);           \
    template void mg_gs_half_split<T>(const T*, bool, const T*, T*, T*, T*, Dims, int, int, int, cudaStream_t); \
    template void mg_resid_restrict_split<T>(const T*, bool, const T*, const T*, T*, bool, Dims, Dims, int,     \
                                             cudaStream_t);                                                    \
    template void mg_prolong_add_split<T>(const T*, bool, T*, Dims, Dims, int, cudaStream_t);

PLSQR_INST_MG(float)
PLSQR_INST_MG(double)

}  // namespace plsqr
