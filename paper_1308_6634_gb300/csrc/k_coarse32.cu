// k_coarse32.cu -- the exact coarse solve of the V-cycle in single precision (float handles).
//
// The coarsest operator M_c (Galerkin sums of the edge conductances, section 4.2) is a symmetric
// M-matrix: its off-diagonal entries are -c_e <= 0, and its row sums are the conductances of the
// edges to the zero ghost cells beyond the high boundary, s_i >= 0.  Gaussian elimination that
// carries the off-diagonal magnitudes and the row-sum excess s instead of the diagonal (the
// arrangement of Grassmann, Taksar and Heyman, 1985) forms each pivot as d_k = s_k + sum_i |a_ik|
// and each update as a sum of non-negative terms:
//
//     |a'_ij| = |a_ij| + |a_ik| |a_jk| / d_k,      s'_i = s_i + |a_ik| s_k / d_k.
//
// Nothing is ever subtracted, so every computed quantity carries a small componentwise relative
// error whatever the condition number of M_c, and single precision gives the inverse to a few
// float ulps per entry (M_c^{-1} is entrywise positive).  With M_c = L D L^T, L unit lower with
// entries -l_ik (l_ik >= 0), the inverse X = L^{-T} D^{-1} L^{-1} again needs only additions of
// non-negative terms.  This replaces the double-precision banded Cholesky and inverse, whose
// sequential column steps ran on the narrow double-precision pipe, for bandwidths <= 32 (2D
// coarsest grids up to 32 cells wide).
//
// Layout.  bw is the bandwidth (largest cell stride), BWP = round4(window + 1).  gcol[j][0] = s_j,
// gcol[j][t] = |a_{j+t,j}| (t = 1..bw, zero beyond); after the factorisation gcol[k][0] = 1/d_k and
// gcol[k][t] = l_{k+t,k}, and grow[i][t] = l_{i,i-t}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <stdexcept>

#include "kernels.cuh"
#include "tma.cuh"

namespace plsqr {

// Column j of the strictly lower triangle of M_c is the conductances of cell j's edges in the
// +x, +y (+z) directions; an edge to the ghost cell beyond the high boundary adds to s_j instead.
template <typename T, typename V, bool KAPPA>
__global__ void __launch_bounds__(256) k_gth_assemble(const T* __restrict__ cond, V* __restrict__ gcol, Dims d,
                                                      int BWP) {
    const int inst = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (j >= d.N) return;
    V* col = gcol + ((int64_t)inst * d.N + j) * BWP;
    for (int t = 0; t < BWP; ++t) col[t] = (V)0;
    const T* c = cond + (KAPPA ? (int64_t)inst * d.N : (int64_t)inst * d.ndim * d.N);
    const int co[3] = {(int)(j % d.nx), (int)((j / d.nx) % d.ny), (int)(j / ((int64_t)d.nx * d.ny))};
    const int n[3] = {d.nx, d.ny, d.nz};
    const int strd[3] = {1, d.nx, d.nx * d.ny};
    V s = (V)0;
    for (int dd = 0; dd < d.ndim; ++dd) {
        const V ce = (V)(KAPPA ? c[j] : c[(int64_t)dd * d.N + j]);
        if (co[dd] + 1 < n[dd]) col[strd[dd]] = ce;
        else s += ce;
    }
    col[0] = s;
}

template <int BWP>
__device__ __forceinline__ void load_row(float (&r)[BWP], const float* p) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int q = 0; q < BWP / 4; ++q) {
        const float4 v = p4[q];
        r[4 * q] = v.x;
        r[4 * q + 1] = v.y;
        r[4 * q + 2] = v.z;
        r[4 * q + 3] = v.w;
    }
}

template <int BWP>
__device__ __forceinline__ void load_row(double (&r)[BWP], const double* p) {
    const double2* p2 = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int q = 0; q < BWP / 2; ++q) {
        const double2 v = p2[q];
        r[2 * q] = v.x;
        r[2 * q + 1] = v.y;
    }
}

// correctly rounded reciprocal (the value of 1 / x)
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// d_k = s_k + sum_i |a_ik| of a staged column (excess first), in a fixed order: four partial sums
// over every fourth entry.
template <typename V, int BWP>
__device__ __forceinline__ V pivot_sum(const V (&c)[BWP]) {
    V a0 = (V)0, a1 = (V)0, a2 = (V)0, a3 = (V)0;
#pragma unroll
    for (int q = 0; q < BWP / 4; ++q) {
        a0 += c[4 * q];
        a1 += c[4 * q + 1];
        a2 += c[4 * q + 2];
        a3 += c[4 * q + 3];
    }
    return (a0 + a1) + (a2 + a3);
}

// L D L^T of one instance per warp.  The whole instance (nc * BWP floats) is staged in shared
// memory by one bulk copy, so the pivot loop makes no global loads.  Lane t-1 owns row offset t
// of every column: at step k it forms l_{k+t,k} = |a_{k+t,k}| / d_k and updates entry t of the
// columns k + tau (tau <= bw - t), lane t-1 also the excess of column k + t.  The loop is
// software-pipelined: step k first completes column k+1 (its update by pivot k and its excess),
// then issues the loads of column k+1 together with the rest of pivot k's update (columns k+2 ..),
// so the sum and reciprocal of pivot k+1 overlap that update.  l and 1/d_k go to global memory as
// they are formed; the staged copy of column k is left as is.  Measured on the 1024^2 workload's
// 32 x 32 coarse grid: 0.69 ms per factorisation, limited by one warp's dependent shared-memory
// and arithmetic chain.  k_ldl_gth_split below (four warps, the pivot chain on one of them) takes
// 0.29 ms and is the default; this kernel remains for comparisons (PLSQR_GTH_WARPS=1).
template <int BW>
__global__ void __launch_bounds__(32) k_ldl_gth_pipe(float* __restrict__ gcol_all, float* __restrict__ grow_all,
                                                     int nc, int bw, GkState* st) {
    constexpr int BWP = (BW + 1 + 3) & ~3;
    constexpr int SLW = BWP + BW;
    extern __shared__ __align__(128) float col[];
    __shared__ float sl[2][SLW];
    __shared__ __align__(8) uint64_t bar;
    const int inst = blockIdx.x, lane = threadIdx.x;
    if (parked(st[inst])) return;
    float* gc = gcol_all + (int64_t)inst * nc * BWP;
    float* gr = grow_all + (int64_t)inst * nc * BWP;
    if (lane == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, (uint32_t)(nc * BWP * sizeof(float)));
        bulk_load(col, gc, (uint32_t)(nc * BWP * sizeof(float)), &bar);
    }
    for (int e = lane; e < nc * BWP; e += 32)  // row layout: entries no pivot writes
        if (e % BWP == 0 || e % BWP > bw || e / BWP < e % BWP) gr[e] = 0.f;
    for (int e = lane; e < 2 * SLW; e += 32) (&sl[0][0])[e] = 0.f;  // l beyond the band stays 0
    for (int e = lane; e < BWP; e += 32) col[(int64_t)nc * BWP + e] = 0.f;
    __syncwarp();
    tma_wait_tile(&bar, st, inst);
    const int t = lane + 1;
    const bool mine = t <= bw;
    auto pivot = [&](const float (&c)[BWP]) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int q = 0; q < BWP / 4; ++q) {
            a0 += c[4 * q];
            a1 += c[4 * q + 1];
            a2 += c[4 * q + 2];
            a3 += c[4 * q + 3];
        }
        return 1.0f / ((a0 + a1) + (a2 + a3));
    };
    float cv[BWP];
    load_row<BWP>(cv, col);
    float rd = pivot(cv);
    float l = mine ? col[t] * rd : 0.f;
    for (int k = 0; k < nc; ++k) {
        float* slk = sl[k & 1];
        if (mine) {
            slk[t] = l;
            gc[(int64_t)k * BWP + t] = l;
            if (k + t < nc) gr[(int64_t)(k + t) * BWP + t] = l;
        }
        if (lane == 0) gc[(int64_t)k * BWP] = rd;
        __syncwarp();
        const int lim = min(bw - t, nc - 1 - k);  // the columns k + tau this lane updates: tau <= lim
        if (1 <= lim) {
            float* e = col + (int64_t)(k + 1) * BWP + t;
            *e = fmaf(slk[1 + t], cv[1], *e);
        }
        if (t == 1 && k + 1 < nc) {
            float* e = col + (int64_t)(k + 1) * BWP;
            *e = fmaf(l, cv[0], *e);
        }
        __syncwarp();
        // column k+1 is final: its loads go first (the staged table has one zero column beyond
        // the last, so the loads of the last step stay in bounds; that step's pivot is unused)
        float cn[BWP];
        load_row<BWP>(cn, col + (int64_t)(k + 1) * BWP);
        const float ln = mine ? col[(int64_t)(k + 1) * BWP + t] : 0.f;
        // the rest of pivot k's update: every entry this lane touches is read before any is
        // written (the entries are distinct, so this is the same arithmetic), which lets the
        // loads issue back to back instead of one load-use-store chain per column
        float ev[BW], sv[BW];
        float* ck1 = col + (int64_t)(k + 1) * BWP + t;
#pragma unroll
        for (int tau = 2; tau < BW; ++tau) {
            ev[tau] = tau <= lim ? ck1[(tau - 1) * BWP] : 0.f;
            sv[tau] = tau <= lim ? slk[tau + t] : 0.f;
        }
        const bool exc = t >= 2 && mine && k + t < nc;
        float* ex = col + (int64_t)(k + t) * BWP;
        const float exv = exc ? *ex : 0.f;
#pragma unroll
        for (int tau = 2; tau < BW; ++tau)
            if (tau <= lim) ck1[(tau - 1) * BWP] = fmaf(sv[tau], cv[tau], ev[tau]);
        if (exc) *ex = fmaf(l, cv[0], exv);
        rd = pivot(cn);
        l = ln * rd;
#pragma unroll
        for (int q = 0; q < BWP; ++q) cv[q] = cn[q];
        __syncwarp();
    }
}

// The same factorisation by four warps with look-ahead.  In step k warp 0 runs only the chain
// of pivots: it completes column k+1 (its update by pivot k and its excess), sums it and forms
// 1/d_{k+1} and l_{.,k+1}; meanwhile warps 1-3 apply pivot k to columns k+2 .. k+BW-1 (warp w
// the columns k + tau with tau = w + 1 (mod 3)) and warp 1 updates the excesses of columns
// k+2 .. k+bw.  A block barrier closes the step.  The l of consecutive pivots go to alternate
// shared buffers.  Every entry sees the operations of k_ldl_gth_pipe in the same order: the
// results are bit for bit the same.
constexpr int GTH_BULK = 3;  // warps applying the bulk of each pivot

template <typename V, int BW, int W>
__device__ __forceinline__ void gth_bulk(V* col, const V* slk, const V (&cv)[(BW + 1 + 3) & ~3],
                                         int k, int t, int lim) {
    constexpr int BWP = (BW + 1 + 3) & ~3;
    constexpr int NT = (BW - 1 - (W + 1) + GTH_BULK) / GTH_BULK;  // columns of this warp: tau = W+1, W+4, ..
    V ev[NT > 0 ? NT : 1], sv[NT > 0 ? NT : 1];
    V* ck = col + (int64_t)k * BWP + t;
#pragma unroll
    for (int q = 0; q < NT; ++q) {
        const int tau = W + 1 + GTH_BULK * q;
        ev[q] = tau <= lim ? ck[tau * BWP] : (V)0;
        sv[q] = tau <= lim ? slk[tau + t] : (V)0;
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) {
        const int tau = W + 1 + GTH_BULK * q;
        if (tau <= lim) ck[tau * BWP] = fma(sv[q], cv[tau], ev[q]);
    }
}

template <typename V, int BW>
__global__ void __launch_bounds__(32 * (1 + GTH_BULK)) k_ldl_gth_split(V* __restrict__ gcol_all,
                                                                        V* __restrict__ grow_all, int nc,
                                                                        int bw, GkState* st) {
    constexpr int BWP = (BW + 1 + 3) & ~3;
    constexpr int SLW = BWP + BW;
    constexpr int NTH = 32 * (1 + GTH_BULK);
    extern __shared__ __align__(128) unsigned char colraw[];
    V* col = reinterpret_cast<V*>(colraw);
    __shared__ V sl[2][SLW];
    __shared__ __align__(8) uint64_t bar;
    const int inst = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (parked(st[inst])) return;
    V* gc = gcol_all + (int64_t)inst * nc * BWP;
    V* gr = grow_all + (int64_t)inst * nc * BWP;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, (uint32_t)(nc * BWP * sizeof(V)));
        bulk_load(col, gc, (uint32_t)(nc * BWP * sizeof(V)), &bar);
    }
    for (int e = tid; e < nc * BWP; e += NTH)  // row layout: entries no pivot writes
        if (e % BWP == 0 || e % BWP > bw || e / BWP < e % BWP) gr[e] = (V)0;
    for (int e = tid; e < 2 * SLW; e += NTH) (&sl[0][0])[e] = (V)0;  // l beyond the band stays 0
    for (int e = tid; e < BWP; e += NTH) col[(int64_t)nc * BWP + e] = (V)0;
    __syncthreads();
    tma_wait_tile(&bar, st, inst);
    const int t = lane + 1;
    const bool mine = t <= bw;
    // warp 0 keeps the column of the current pivot in registers from the step that formed it
    V cw[BWP];
    if (warp == 0) {  // pivot 0
        load_row<BWP>(cw, col);
        const V rd = rcp_rn(pivot_sum<V, BWP>(cw));
        const V l = mine ? col[t] * rd : (V)0;
        if (mine) {
            sl[0][t] = l;
            gc[t] = l;
            if (t < nc) gr[(int64_t)t * BWP + t] = l;
        }
        if (lane == 0) gc[0] = rd;
    }
    __syncthreads();
    for (int k = 0; k < nc; ++k) {
        const V* slk = sl[k & 1];
        const int lim = min(bw - t, nc - 1 - k);  // the columns k + tau lane t-1 updates: tau <= lim
        if (warp == 0) {
            // pivot k's update of column k+1 and its excess; the lane's own entry stays in a register
            V* e1 = col + (int64_t)(k + 1) * BWP + t;
            V own = mine ? *e1 : (V)0;  // rows t > bw are outside the column (and the table)
            if (1 <= lim) {
                own = fma(slk[1 + t], cw[1], own);
                *e1 = own;
            }
            if (t == 1 && k + 1 < nc) {
                V* e = col + (int64_t)(k + 1) * BWP;
                *e = fma(slk[1], cw[0], *e);
            }
            __syncwarp();
            if (k + 1 < nc) {
                V* sln = sl[(k + 1) & 1];
                load_row<BWP>(cw, col + (int64_t)(k + 1) * BWP);
                const V rd = rcp_rn(pivot_sum<V, BWP>(cw));
                const V l = mine ? own * rd : (V)0;
                if (mine) {
                    sln[t] = l;
                    gc[(int64_t)(k + 1) * BWP + t] = l;
                    if (k + 1 + t < nc) gr[(int64_t)(k + 1 + t) * BWP + t] = l;
                }
                if (lane == 0) gc[(int64_t)(k + 1) * BWP] = rd;
            }
        } else {
            V cv[BWP];
            load_row<BWP>(cv, col + (int64_t)k * BWP);  // column k is final
            if (warp == 1) {
                gth_bulk<V, BW, 1>(col, slk, cv, k, t, lim);
                if (t >= 2 && mine && k + t < nc) {
                    V* e = col + (int64_t)(k + t) * BWP;
                    *e = fma(slk[t], cv[0], *e);
                }
            } else if (warp == 2) {
                gth_bulk<V, BW, 2>(col, slk, cv, k, t, lim);
            } else {
                gth_bulk<V, BW, 3>(col, slk, cv, k, t, lim);
            }
        }
        __syncthreads();
    }
}

// The inverse by one warp per column for double tables and batches up to 16; PLSQR_GTH_INV=thread
// or =warp forces one (comparisons).  Measured at batch 1 on the GB300: with double tables (16-wide
// band, 256 cells) the thread-per-column kernel runs its band of multiply-adds on the narrow
// double pipe and the warp kernel takes the setup of the 64^2 workload from 7.2 to 4.6 ms per
// solve; with float tables (32-wide band, 1024 cells) the warp kernel issues about ten
// instructions per row and column against under two for the thread kernel, and loses (272
// against 227 us).
bool gth_inverse_by_warp(int B, size_t esz) {
    const char* e = std::getenv("PLSQR_GTH_INV");
    if (e && e[0] == 't') return false;
    if (e && e[0] == 'w') return true;
    return esz == 8 && B <= 16;
}

// PLSQR_GTH_WARPS=1: the one-warp factorisation (comparisons)
bool gth_split_enabled() {
    const char* e = std::getenv("PLSQR_GTH_WARPS");
    return !(e && e[0] == '1');
}

// X = L^{-T} D^{-1} L^{-1}, one thread per column j (BW = window >= bw, a power of two).
// Forward: z = L^{-1} e_j column-oriented -- when z_k is final, z_{k+t} += l_{k+t,k} z_k -- with
// the BW pending sums in registers (rotating, the index fixed by unrolling), y_k = z_k / d_k kept
// in X[k][j].  Backward from the last row to row j: x_i = y_i + (pending), then the rows above
// receive l_{i,i-t} x_i.  x_i (i >= j) is stored at X[i][j] and X[j][i].  The factor tables are
// staged in shared memory for each pass.
template <typename V, int BW>
__global__ void __launch_bounds__(128) k_gth_inverse(const V* __restrict__ gcol_all,
                                                     const V* __restrict__ grow_all, V* __restrict__ X_all,
                                                     int nc, GkState* st) {
    constexpr int BWP = (BW + 1 + 3) & ~3;
    extern __shared__ __align__(128) unsigned char tabraw[];
    V* tab = reinterpret_cast<V*>(tabraw);
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const int jb = blockIdx.x * 128;
    const int j = jb + threadIdx.x;
    const int j0 = jb + (threadIdx.x & ~31);
    const V* gc = gcol_all + (int64_t)inst * nc * BWP;
    const V* gr = grow_all + (int64_t)inst * nc * BWP;
    V* X = X_all + (int64_t)inst * nc * nc;
    const bool live = j < nc;
    __shared__ __align__(8) uint64_t bar[2];
    const uint32_t bytes = (uint32_t)((nc - jb) * BWP * sizeof(V));
    // ---- forward ----
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_expect_tx(&bar[0], bytes);
        bulk_load(tab, gc + (int64_t)jb * BWP, bytes, &bar[0]);
    }
    __syncthreads();
    tma_wait_tile(&bar[0], st, inst);
    V pend[BW];
#pragma unroll
    for (int u = 0; u < BW; ++u) pend[u] = (V)0;
    if (j0 < nc) {
        for (int base = j0; base < nc; base += BW) {
#pragma unroll
            for (int u = 0; u < BW; ++u) {
                const int k = base + u;
                if (k < nc) {
                    V row[BWP];
                    load_row<BWP>(row, tab + (int64_t)(k - jb) * BWP);
                    const V z = pend[u] + (k == j ? (V)1 : (V)0);
                    pend[u] = (V)0;
                    if (live && k >= j) X[(int64_t)k * nc + j] = z * row[0];
#pragma unroll
                    for (int t = 1; t <= BW; ++t) pend[(u + t) & (BW - 1)] = fma(row[t], z, pend[(u + t) & (BW - 1)]);
                }
            }
        }
    }
    __syncthreads();
    // ---- backward ----
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar[1], bytes);
        bulk_load(tab, gr + (int64_t)jb * BWP, bytes, &bar[1]);
    }
    tma_wait_tile(&bar[1], st, inst);
#pragma unroll
    for (int u = 0; u < BW; ++u) pend[u] = (V)0;
    if (j0 >= nc) return;
    // y values of the next chunk are loaded one chunk ahead (they were written by this thread)
    V ynx[BW];
    const int top = nc - 1;
#pragma unroll
    for (int v = 0; v < BW; ++v) {
        const int i = top - v;
        ynx[v] = (live && i >= j) ? X[(int64_t)i * nc + j] : (V)0;
    }
    // the warp's chunk of x (BW rows x 32 columns) goes through shared memory so that the mirror
    // entries X[j][i] are written along rows
    V (*tile)[33] = reinterpret_cast<V (*)[33]>(tab + (size_t)nc * BWP) + (threadIdx.x >> 5) * BW;
    const int lane = threadIdx.x & 31;
    for (int base = top; base >= j0; base -= BW) {
        V ycur[BW];
#pragma unroll
        for (int v = 0; v < BW; ++v) ycur[v] = ynx[v];
#pragma unroll
        for (int v = 0; v < BW; ++v) {
            const int i = base - BW - v;
            ynx[v] = (live && i >= j && i >= j0) ? X[(int64_t)i * nc + j] : (V)0;
        }
#pragma unroll
        for (int v = 0; v < BW; ++v) {
            const int i = base - v;
            if (i >= j0) {
                V row[BWP];
                load_row<BWP>(row, tab + (int64_t)(i - jb) * BWP);
                const V x = ycur[v] + pend[v];
                pend[v] = (V)0;
                tile[v][lane] = x;
                if (live && i >= j) X[(int64_t)i * nc + j] = x;
#pragma unroll
                for (int t = 1; t <= BW; ++t) pend[(v + t) & (BW - 1)] = fma(row[t], x, pend[(v + t) & (BW - 1)]);
            }
        }
        __syncwarp();
        if (lane < BW) {
            const int i = base - lane;
            for (int r = 0; r < 32; ++r) {
                const int jr = j0 + r;
                if (jr < nc && i > jr) X[(int64_t)jr * nc + i] = tile[lane][r];
            }
        }
        __syncwarp();
    }
}

// The same inverse with one warp per column j, for small batches.  k_gth_inverse gives each
// column to one thread, whose chain of 2 nc rows (each a band of BW multiply-adds on one thread)
// sets the time of the whole launch at batch 1.  Here the BW pending sums of the column live one
// per lane: lane L keeps the pending sum of the row of residue L (mod 32), so that a row costs
// one shuffle of its finished entry from the lane that owns it and one multiply-add per lane, and
// a lane whose row is finished starts on the row 32 further on.  Forward: z_k = (pending of row k)
// (+1 at k = j), y_k = z_k / d_k stored at X[k][j], then z_{k+t} += l_{k+t,k} z_k.  Backward:
// x_i = y_i + (pending of row i), then x_{i-t} += l_{i,i-t} x_i.  Every entry of X sees the
// operations of k_gth_inverse in the same order (the +1 of row j is carried in the pending sum of
// its lane from the start, which adds only exact zeros to it), so the result is bit for bit the
// same.  The factor table (rows from the block's first column to the last) is staged in shared
// memory for each pass; the 32 band entries a lane needs in a run of 32 rows are read into
// registers before the run, off the shuffle-and-FMA chain.
template <typename V, int BW, int NWI>
__global__ void __launch_bounds__(32 * NWI) k_gth_inverse_warp(const V* __restrict__ gcol_all,
                                                               const V* __restrict__ grow_all,
                                                               V* __restrict__ X_all, int nc, GkState* st) {
    constexpr int BWP = (BW + 1 + 3) & ~3;
    extern __shared__ __align__(128) unsigned char tabraw[];
    V* tab = reinterpret_cast<V*>(tabraw);
    __shared__ __align__(8) uint64_t bar[2];
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = (blockIdx.x * NWI) & ~31;  // first staged row
    const int j = blockIdx.x * NWI + warp;
    const bool live = j < nc;
    const V* gc = gcol_all + (int64_t)inst * nc * BWP;
    const V* gr = grow_all + (int64_t)inst * nc * BWP;
    V* X = X_all + (int64_t)inst * nc * nc;
    const uint32_t bytes = (uint32_t)((nc - r0) * BWP * sizeof(V));
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_expect_tx(&bar[0], bytes);
        bulk_load(tab, gc + (int64_t)r0 * BWP, bytes, &bar[0]);
    }
    __syncthreads();
    tma_wait_tile(&bar[0], st, inst);
    // ---- forward over rows j, j+1, ... (runs of 32 rows aligned to multiples of 32) ----
    if (live) {
        V pend = lane == (j & 31) ? (V)1 : (V)0;
        for (int base = j & ~31; base < nc; base += 32) {
            V lt[32];
#pragma unroll
            for (int u = 0; u < 32; ++u) {  // lane's row at step k = base + u is k + t
                const int k = base + u, d = (lane - u) & 31, t = d ? d : 32;
                lt[u] = (k < nc && t <= BW) ? tab[(int64_t)(k - r0) * BWP + t] : (V)0;
            }
            const V rdv = base + lane < nc ? tab[(int64_t)(base + lane - r0) * BWP] : (V)0;
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int k = base + u;
                const V z = __shfl_sync(0xffffffffu, pend, u);
                if (lane == u) {
                    if (k >= j && k < nc) X[(int64_t)k * nc + j] = z * rdv;
                    pend = (V)0;
                }
                pend = fma(lt[u], z, pend);
            }
        }
    }
    __syncthreads();  // every warp is done with the forward table
    if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bar[1], bytes);
        bulk_load(tab, gr + (int64_t)r0 * BWP, bytes, &bar[1]);
    }
    tma_wait_tile(&bar[1], st, inst);
    if (!live) return;
    // ---- backward over rows nc-1, nc-2, ..., j ----
    const int top = nc - 1;
    V pend = (V)0;
    int cb = top & ~31;
    V yv = (cb + lane <= top && cb + lane >= j) ? X[(int64_t)(cb + lane) * nc + j] : (V)0;  // y of row cb + lane
    for (; cb >= (j & ~31); cb -= 32) {
        const int nb = cb - 32;  // y of the next run down, loaded one run ahead (this thread wrote them)
        const V ynx = (nb >= 0 && nb + lane >= j) ? X[(int64_t)(nb + lane) * nc + j] : (V)0;
        V lt[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {  // step i = cb + 31 - u; lane's row is i - t
            const int i = cb + 31 - u, d = (i - lane) & 31, t = d ? d : 32;
            lt[u] = (i <= top && t <= BW) ? tab[(int64_t)(i - r0) * BWP + t] : (V)0;
        }
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            const int i = cb + 31 - u, own = 31 - u;
            if (i <= top) {
                const V x = __shfl_sync(0xffffffffu, yv + pend, own);
                if (lane == own) {
                    if (i >= j) {
                        X[(int64_t)i * nc + j] = x;
                        if (i != j) X[(int64_t)j * nc + i] = x;
                    }
                    pend = (V)0;
                }
                pend = fma(lt[u], x, pend);
            }
        }
        yv = ynx;
    }
}

// ---- the inverse in 32 x 32 blocks ---------------------------------------------------------------
// With L = I - N (N >= 0: the l of the factor) cut into 32 x 32 blocks, L is block lower banded with
// K = ceil(bw / 32) blocks below the diagonal: N_ii strictly lower, N_{i,i-k} (k = 1..K).  Then
//   W = L^{-1}:  W_jj = G_j = (I - N_jj)^{-1},
//                W_ij = sum_{k=1..min(K, i-j)} P_{i,k} W_{i-k,j} with P_{i,k} = G_i N_{i,i-k} (i > j),
//   X = W^T D^{-1} W:  X_ab = sum_{i >= max(a,b)} W_ia^T D_i^{-1} W_ib.
// Every quantity is a sum of products of non-negative numbers, as in the row-by-row kernels, so the
// result keeps their componentwise accuracy; but the chains of dependent steps are 32 (G), nb (W)
// and nb (X) block steps spread over many blocks instead of 2 nc row steps on one thread.  Only X_ab
// with a <= b is formed (and the diagonal blocks' upper halves), and mirrored: X is exactly
// symmetric.  Rows beyond nc are padding (N = 0, 1/d = 0).  Scratch per instance: G and the P
// ((1 + K) nb blocks) and W (nb (nb + 1) / 2 blocks, packed by block rows).
constexpr int XB = 32;

template <typename V>
__device__ __forceinline__ V tab_l(const V* gc, int BWP, int bw, int nc, int r, int c) {  // l_{r,c}, r > c
    return (r < nc && c >= 0 && r > c && r - c <= bw) ? gc[(int64_t)c * BWP + (r - c)] : (V)0;
}

// G_i and P_{i,1..K} of block row i (one block of 32 x 32 threads per block row and instance)
template <typename V>
__global__ void __launch_bounds__(1024) k_xblk_diag(const V* __restrict__ gcol_all, V* __restrict__ gp_all, int nc,
                                                    int bw, int BWP, int nb, int K, GkState* st) {
    __shared__ V nd[XB][XB + 1], ns[XB][XB + 1], gs[XB][XB + 1];
    const int inst = blockIdx.y, i = blockIdx.x;
    if (parked(st[inst])) return;
    const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
    const V* gc = gcol_all + (int64_t)inst * nc * BWP;
    nd[r][c] = tab_l(gc, BWP, bw, nc, XB * i + r, XB * i + c);
    __syncthreads();
    // column c of G by warp c (= r here): lane l holds g_l; when g_s is final the rows below it
    // receive N_ls g_s
    {
        const int col = r, l = c;
        V g = l == col ? (V)1 : (V)0;
        for (int s2 = 0; s2 < XB; ++s2) {
            const V gsv = __shfl_sync(0xffffffffu, g, s2);
            if (l > s2) g = fma(nd[l][s2], gsv, g);
        }
        gs[l][col] = g;
    }
    __syncthreads();
    V* gp = gp_all + ((int64_t)inst * nb + i) * (1 + K) * XB * XB;
    gp[r * XB + c] = gs[r][c];
    for (int k = 1; k <= K; ++k) {
        ns[r][c] = i - k >= 0 ? tab_l(gc, BWP, bw, nc, XB * i + r, XB * (i - k) + c) : (V)0;
        __syncthreads();
        V acc = (V)0;
#pragma unroll 8
        for (int m = 0; m < XB; ++m) acc = fma(gs[r][m], ns[m][c], acc);
        gp[k * XB * XB + r * XB + c] = acc;
        __syncthreads();
    }
}

// 32 x 32 blocks in shared memory with a row stride of XS elements (pairs of a row 8- or 16-byte
// aligned for the vector loads of the 2 x 2 register tiles below)
constexpr int XS = XB + 2;

template <typename V> struct V2of;
template <> struct V2of<float> { using type = float2; };
template <> struct V2of<double> { using type = double2; };

// acc (2 x 2, rows r0, r0+1, columns c0, c0+1) += A^T B over m, A = sa[m][r], B = sb[m][c]
template <typename V>
__device__ __forceinline__ void tile_atb(const V (*sa)[XS], const V (*sb)[XS], int r0, int c0, V (&acc)[2][2]) {
    using V2 = typename V2of<V>::type;
#pragma unroll 8
    for (int m = 0; m < XB; ++m) {
        const V2 ar = *reinterpret_cast<const V2*>(&sa[m][r0]);
        const V2 bc = *reinterpret_cast<const V2*>(&sb[m][c0]);
        acc[0][0] = fma(ar.x, bc.x, acc[0][0]);
        acc[0][1] = fma(ar.x, bc.y, acc[0][1]);
        acc[1][0] = fma(ar.y, bc.x, acc[1][0]);
        acc[1][1] = fma(ar.y, bc.y, acc[1][1]);
    }
}

// W_jj .. W_{nb-1,j} of block column j: W_ij = sum_k P_{i,k} W_{i-k,j}.  256 threads, each a 2 x 2
// tile; the last K blocks of the column stay in a ring in shared memory (dynamic, K + 1 slots), and
// each P_{i,k} is staged transposed (pt[m][r] = P[r][m]) so that the product reads rows of both.
template <typename V>
__global__ void __launch_bounds__(256) k_xblk_wchain(const V* __restrict__ gp_all, V* __restrict__ w_all, int nb,
                                                     int K, GkState* st) {
    using V2 = typename V2of<V>::type;
    extern __shared__ __align__(16) unsigned char wraw[];
    V(*ws)[XB][XS] = reinterpret_cast<V(*)[XB][XS]>(wraw);  // K + 1 slots: W_{i,j} in slot (i - j) % (K + 1)
    __shared__ __align__(16) V pt[2][XB][XS];
    const int inst = blockIdx.y, j = blockIdx.x;
    if (parked(st[inst])) return;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const int r0 = 2 * ty, c0 = 2 * tx;
    const int64_t PS = (int64_t)(1 + K) * XB * XB;  // G and P blocks of one block row
    const V* gp = gp_all + (int64_t)inst * nb * PS;
    V* w = w_all + (int64_t)inst * (nb * (nb + 1) / 2) * XB * XB;
    auto ld2 = [&](const V* blk, int row) { return *reinterpret_cast<const V2*>(blk + row * XB + c0); };
    {
        const V* g = gp + (int64_t)j * PS;
        const V2 g0 = ld2(g, r0), g1 = ld2(g, r0 + 1);
        *reinterpret_cast<V2*>(&ws[0][r0][c0]) = g0;
        *reinterpret_cast<V2*>(&ws[0][r0 + 1][c0]) = g1;
        V* wj = w + ((int64_t)j * (j + 1) / 2 + j) * XB * XB;
        *reinterpret_cast<V2*>(wj + r0 * XB + c0) = g0;
        *reinterpret_cast<V2*>(wj + (r0 + 1) * XB + c0) = g1;
    }
    int use = 0;  // P blocks staged so far (alternating buffers)
    V2 p0{}, p1{};  // the next P block to stage, loaded one product ahead
    if (j + 1 < nb) {
        p0 = ld2(gp + (int64_t)(j + 1) * PS + XB * XB, r0);
        p1 = ld2(gp + (int64_t)(j + 1) * PS + XB * XB, r0 + 1);
    }
    for (int i = j + 1; i < nb; ++i) {
        const int kmax = min(K, i - j);
        V acc[2][2] = {{(V)0, (V)0}, {(V)0, (V)0}};
        for (int k = 1; k <= kmax; ++k) {
            const int cur = use++ & 1;
            pt[cur][c0][r0] = p0.x;  // transposed: pt[m][r] = P[r][m]
            pt[cur][c0 + 1][r0] = p0.y;
            pt[cur][c0][r0 + 1] = p1.x;
            pt[cur][c0 + 1][r0 + 1] = p1.y;
            if (k < kmax) {
                const V* pn = gp + (int64_t)i * PS + (int64_t)(k + 1) * XB * XB;
                p0 = ld2(pn, r0);
                p1 = ld2(pn, r0 + 1);
            } else if (i + 1 < nb) {  // P_{i+1,1}
                const V* pn = gp + (int64_t)(i + 1) * PS + XB * XB;
                p0 = ld2(pn, r0);
                p1 = ld2(pn, r0 + 1);
            }
            __syncthreads();
            tile_atb<V>(pt[cur], ws[(i - k - j) % (K + 1)], r0, c0, acc);
        }
        const V2 o0 = {acc[0][0], acc[0][1]}, o1 = {acc[1][0], acc[1][1]};
        __syncthreads();  // every thread is done with the slot W_{i-K-1,j} held
        *reinterpret_cast<V2*>(&ws[(i - j) % (K + 1)][r0][c0]) = o0;
        *reinterpret_cast<V2*>(&ws[(i - j) % (K + 1)][r0 + 1][c0]) = o1;
        V* wi = w + ((int64_t)i * (i + 1) / 2 + j) * XB * XB;
        *reinterpret_cast<V2*>(wi + r0 * XB + c0) = o0;
        *reinterpret_cast<V2*>(wi + (r0 + 1) * XB + c0) = o1;
        __syncthreads();
    }
}

// X_ab (a <= b) = sum_{i >= b} W_ia^T D_i^{-1} W_ib, written with its mirror.  256 threads, each a
// 2 x 2 tile; the next block row's two blocks are loaded into registers while this one is summed.
template <typename V>
__global__ void __launch_bounds__(256) k_xblk_syrk(const V* __restrict__ w_all, const V* __restrict__ gcol_all,
                                                   V* __restrict__ X_all, int nc, int BWP, int nb, GkState* st) {
    using V2 = typename V2of<V>::type;
    __shared__ __align__(16) V wa[2][XB][XS], wb[2][XB][XS];
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const int p = blockIdx.x;
    int b = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((b + 1) * (b + 2) / 2 <= p) ++b;
    while (b * (b + 1) / 2 > p) --b;
    const int a = p - b * (b + 1) / 2;  // a <= b
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const int r0 = 2 * ty, c0 = 2 * tx;
    const V* w = w_all + (int64_t)inst * (nb * (nb + 1) / 2) * XB * XB;
    const V* gc = gcol_all + (int64_t)inst * nc * BWP;
    // staging: this thread moves rows r0, r0+1, columns c0, c0+1 of W_ia and (scaled by 1/d) W_ib
    auto fetch = [&](int i, V2 (&fa)[2], V2 (&fb)[2]) {
        const V* A = w + ((int64_t)i * (i + 1) / 2 + a) * XB * XB;
        const V* Bm = w + ((int64_t)i * (i + 1) / 2 + b) * XB * XB;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int row = XB * i + r0 + q;
            const V dinv = row < nc ? gc[(int64_t)row * BWP] : (V)0;
            fa[q] = *reinterpret_cast<const V2*>(A + (r0 + q) * XB + c0);
            const V2 t = *reinterpret_cast<const V2*>(Bm + (r0 + q) * XB + c0);
            fb[q] = {dinv * t.x, dinv * t.y};
        }
    };
    V2 fa[2], fb[2];
    fetch(b, fa, fb);
    V acc[2][2] = {{(V)0, (V)0}, {(V)0, (V)0}};
    for (int i = b; i < nb; ++i) {
        const int cur = (i - b) & 1;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            *reinterpret_cast<V2*>(&wa[cur][r0 + q][c0]) = fa[q];
            *reinterpret_cast<V2*>(&wb[cur][r0 + q][c0]) = fb[q];
        }
        if (i + 1 < nb) fetch(i + 1, fa, fb);
        __syncthreads();
        tile_atb<V>(wa[cur], wb[cur], r0, c0, acc);  // sum over m of W_ia[m][r] (W_ib[m][c] / d_m)
        // the other buffer is written next; a barrier per block row keeps the reads of this one
        // ahead of that (two buffers, so one barrier suffices)
    }
    V* X = X_all + (int64_t)inst * nc * nc;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int r = r0 + q, c = c0 + e;
            const int gi = XB * a + r, gj = XB * b + c;
            if (gi < nc && gj < nc) {
                if (a < b || r <= c) X[(int64_t)gi * nc + gj] = acc[q][e];
                if (a < b || r < c) X[(int64_t)gj * nc + gi] = acc[q][e];
            }
        }
}

int xblk_blocks(int nc) { return (nc + XB - 1) / XB; }
int xblk_sub(int bw) { return std::max(1, (bw + XB - 1) / XB); }

// scratch elements per instance of the blocked inverse
int64_t xblk_scratch(int nc, int bw) {
    const int64_t nb = xblk_blocks(nc), K = xblk_sub(bw);
    return ((1 + K) * nb + nb * (nb + 1) / 2) * XB * XB;
}

template <typename V>
static void xblk_inverse(const V* gcol, V* X, V* scratch, int nc, int bw, int B, GkState* st, cudaStream_t s) {
    const int BWP = gth_stride(bw), nb = xblk_blocks(nc), K = xblk_sub(bw);
    V* gp = scratch;
    V* w = scratch + (int64_t)B * (1 + K) * nb * XB * XB;
    k_xblk_diag<V><<<dim3(nb, B), 1024, 0, s>>>(gcol, gp, nc, bw, BWP, nb, K, st);
    klaunched("k_xblk_diag");
    const size_t wsm = sizeof(V) * (size_t)(K + 1) * XB * XS;
    if (wsm > 48 * 1024) cudaFuncSetAttribute(k_xblk_wchain<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
    k_xblk_wchain<V><<<dim3(nb, B), 256, wsm, s>>>(gp, w, nb, K, st);
    klaunched("k_xblk_wchain");
    k_xblk_syrk<V><<<dim3(nb * (nb + 1) / 2, B), 256, 0, s>>>(w, gcol, X, nc, BWP, nb, st);
    klaunched("k_xblk_syrk");
}

// Wide bands (3D coarsest grids): the same elimination with a circular window of the bw + 1
// columns pivot k touches, in shared memory (column j in slot j mod (bw + 1), an odd slot stride
// so that consecutive rows of different slots fall in different banks).  The block has NQ groups
// of NT0 = round32(bw) threads (NQ * NT0 <= 1024).  Step k: d_k by a block reduction in a fixed
// order (warp partials to lane 0, then the warp totals in warp order, read by every thread; the
// warps of groups 1.. add zeros); l_{k+t,k} by thread t-1 of group 0; then thread t-1 of group g
// updates row offset t of the columns k + tau, tau = g+1, g+1+NQ, .. <= bw - t (its rows end
// there), GTH_WCH columns at a time with their loads issued before the stores; group 0 also
// updates the excess of column k + t.  Every entry receives one update per pivot, as in the
// narrow kernels.  Column k + bw + 1 is fetched into registers during the step and written to the
// freed slot at its end.  Output as the narrow kernels: gcol[k][0] = 1/d_k, gcol[k][t] = l_{k+t,k},
// grow[i][t] = l_{i,i-t}.
constexpr int GTH_WQ = 4;   // thread groups splitting each pivot's columns
constexpr int GTH_WCH = 4;  // columns per batch of loads

__global__ void __launch_bounds__(1024) k_ldl_gth_window(float* __restrict__ gcol_all, float* __restrict__ grow_all,
                                                         int nc, int bw, int BWP, GkState* st) {
    extern __shared__ __align__(16) float win[];
    __shared__ float sl[1024 + 2];
    __shared__ float wred[32];
    const int NT = blockDim.x, NW = NT >> 5;
    const int NT0 = max(32, ((bw + 31) / 32) * 32), NQ = NT / NT0;
    const int S = bw + 1, SW = S | 1;
    const int inst = blockIdx.x, tid = threadIdx.x, g = tid / NT0, t = tid - g * NT0 + 1;
    if (parked(st[inst])) return;
    float* gc = gcol_all + (int64_t)inst * nc * BWP;
    float* gr = grow_all + (int64_t)inst * nc * BWP;
    for (int e = tid; e < nc * BWP; e += NT)  // row layout: entries no pivot writes
        if (e % BWP == 0 || e % BWP > bw || e / BWP < e % BWP) gr[e] = 0.f;
    for (int e = tid; e < min(S, nc) * S; e += NT) {
        const int c = e / S, r = e - c * S;
        win[c * SW + r] = gc[(int64_t)c * BWP + r];
    }
    for (int e = tid; e < 1024 + 2; e += NT) sl[e] = 0.f;
    __syncthreads();
    for (int k = 0; k < nc; ++k) {
        const int sk = k % S;
        const float* ck = win + sk * SW;
        // the next column of the window, fetched while this step runs
        const bool nxt = k + S < nc;
        const float pre0 = (nxt && tid < S) ? gc[(int64_t)(k + S) * BWP + tid] : 0.f;
        const float pre1 = (nxt && tid + NT < S) ? gc[(int64_t)(k + S) * BWP + tid + NT] : 0.f;
        float part = (g == 0 && t <= bw ? ck[t] : 0.f) + (tid == 0 ? ck[0] : 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if ((tid & 31) == 0) wred[tid >> 5] = part;
        __syncthreads();
        float dk = 0.f;
        for (int w = 0; w < NW; ++w) dk += wred[w];
        const float rd = 1.0f / dk;
        const float s_k = ck[0];
        if (g == 0 && t <= bw) {
            const float l = ck[t] * rd;
            sl[t] = l;
            gc[(int64_t)k * BWP + t] = l;
            if (k + t < nc) gr[(int64_t)(k + t) * BWP + t] = l;
        }
        if (tid == 0) gc[(int64_t)k * BWP] = rd;
        __syncthreads();
        // row offset t of the columns k + tau, tau = g+1, g+1+NQ, .. <= min(bw - t, nc - 1 - k)
        const int last = min(bw - t, nc - 1 - k);
        int tau = g + 1;
        int slot = sk + tau;
        if (slot >= S) slot -= S;
        for (; tau + (GTH_WCH - 1) * NQ <= last; tau += GTH_WCH * NQ) {
            float* ep[GTH_WCH];
            float ev[GTH_WCH], lv[GTH_WCH], av[GTH_WCH];
#pragma unroll
            for (int c = 0; c < GTH_WCH; ++c) {
                ep[c] = win + slot * SW + t;
                ev[c] = *ep[c];
                lv[c] = sl[tau + c * NQ + t];
                av[c] = ck[tau + c * NQ];
                slot += NQ;
                if (slot >= S) slot -= S;
            }
#pragma unroll
            for (int c = 0; c < GTH_WCH; ++c) *ep[c] = fmaf(lv[c], av[c], ev[c]);
        }
        for (; tau <= last; tau += NQ) {
            float* e = win + slot * SW + t;
            *e = fmaf(sl[tau + t], ck[tau], *e);
            slot += NQ;
            if (slot >= S) slot -= S;
        }
        if (g == 0 && t <= bw && k + t < nc) {
            float* es = win + ((k + t) % S) * SW;
            *es = fmaf(sl[t], s_k, *es);
        }
        __syncthreads();
        if (nxt) {
            float* dst = win + sk * SW;
            if (tid < S) dst[tid] = pre0;
            if (tid + NT < S) dst[tid + NT] = pre1;
        }
    }
}

// The same elimination with look-ahead: in step k, warps 0 .. GP-1 (GP = ceil(bw / 32)) apply
// pivot k to column k+1 only, sum it and form 1/d_{k+1} and l_{.,k+1}, while the other warps apply
// pivot k to columns k+2 .. k+bw (thread t of group q: row offset t of the columns k + tau, tau =
// q + 2, q + 2 + NQ, ..; each thread takes the row offsets t and bw - t, so that every thread has
// about the same number of columns) and copy column k+bw+1 into the window.  One block barrier
// ends a step.
// The window holds bw + 2 slots (column c in slot c mod (bw + 2)), so the entering column never
// shares a slot with a column read in the same step.  The pivot sums use the warps, lanes and
// order of k_ldl_gth_window (thread i holds entry i + 1, thread 0 also the excess; shuffle-down
// within a warp, the warp totals in warp order), and every entry receives the same multiply-adds
// in the same order: bit for bit its factor.  In k_ldl_gth_window the pivot chain (sum, reciprocal,
// l) runs after each step's bulk update and both sit between block barriers: ~4400 cycles per
// pivot on the 192^3 workload's 12^3 coarse grid (band 144).
__global__ void __launch_bounds__(1024) k_ldl_gth_ahead(float* __restrict__ gcol_all, float* __restrict__ grow_all,
                                                        int nc, int bw, int BWP, GkState* st) {
    extern __shared__ __align__(16) float win[];
    __shared__ float sl[2][2 * 256 + 4];  // l of pivots k (k & 1) and k + 1, zero beyond bw
    __shared__ float pw[8];
    const int S = bw + 1, S2 = bw + 2, SW = S | 1;
    const int GP = (bw + 31) / 32;
    const int H = bw / 2 + 1;  // row pairs (r, bw - r) of the update group, r < H
    const int NU = blockDim.x - 32 * GP, NQ = NU / H;
    const int inst = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (parked(st[inst])) return;
    float* gc = gcol_all + (int64_t)inst * nc * BWP;
    float* gr = grow_all + (int64_t)inst * nc * BWP;
    for (int e = tid; e < nc * BWP; e += blockDim.x)  // row layout: entries no pivot writes
        if (e % BWP == 0 || e % BWP > bw || e / BWP < e % BWP) gr[e] = 0.f;
    for (int e = tid; e < min(S, nc) * S; e += blockDim.x) {
        const int c = e / S, r = e - c * S;
        win[c * SW + r] = gc[(int64_t)c * BWP + r];  // columns 0 .. bw in slots 0 .. bw
    }
    for (int e = tid; e < 2 * (2 * 256 + 4); e += blockDim.x) (&sl[0][0])[e] = 0.f;
    const bool pgrp = warp < GP;
    const int u = tid - 32 * GP;  // index in the update group
    const int q = pgrp ? 0 : u / H, tr = pgrp ? 0 : u - q * H;
    float pre = (!pgrp && u < S && S < nc) ? gc[(int64_t)S * BWP + u] : 0.f;  // column S, copied in step 0
    __syncthreads();
    // the pivot group's part of a step: column c (all previous pivots applied) -> 1/d_c and l_{.,c}
    auto pivot = [&](int c, float e, float e0) {
        const int t = tid + 1;
        float part = (t <= bw ? e : 0.f) + (tid == 0 ? e0 : 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) pw[warp] = part;
        asm volatile("bar.sync 1, %0;" ::"r"(32 * GP) : "memory");
        float dk = 0.f;
        for (int w = 0; w < GP; ++w) dk += pw[w];
        const float rd = 1.0f / dk;
        if (t <= bw) {
            const float l = e * rd;
            sl[c & 1][t] = l;
            gc[(int64_t)c * BWP + t] = l;
            if (c + t < nc) gr[(int64_t)(c + t) * BWP + t] = l;
        }
        if (tid == 0) gc[(int64_t)c * BWP] = rd;
    };
    if (pgrp) {  // pivot 0
        const int t = tid + 1;
        pivot(0, t <= bw ? win[t] : 0.f, win[0]);
    }
    __syncthreads();
    for (int k = 0; k < nc; ++k) {
        const float* ck = win + (k % S2) * SW;  // column k, the pivot
        const float* lk = sl[k & 1];
        if (pgrp) {
            if (k + 1 < nc) {
                float* c1 = win + ((k + 1) % S2) * SW;
                const int t = tid + 1;
                float e = t <= bw ? c1[t] : 0.f;
                if (t <= bw) {
                    e = fmaf(lk[1 + t], ck[1], e);
                    c1[t] = e;
                }
                float e0 = 0.f;
                if (tid == 0) {
                    e0 = fmaf(lk[1], ck[0], c1[0]);
                    c1[0] = e0;
                }
                pivot(k + 1, e, e0);
            }
        } else {
            if (q < NQ) {
                // row offsets tr and bw - tr (about bw / NQ columns together, whatever tr), columns
                // k + tau, tau = q + 2, q + 2 + NQ, ..; row 0 is the excess (l_{k+tau,k} s_k)
                for (int pass = 0; pass < 2; ++pass) {
                    const int r = pass == 0 ? tr : bw - tr;
                    if (pass == 1 && r == tr) break;
                    const int last = min(bw - r, nc - 1 - k);
                    int tau = q + 2;
                    if (tau > last) continue;
                    int slot = (k + tau) % S2;
                    const float* lp = lk + tau + r;
                    const float* ap = r == 0 ? ck : ck + tau;
                    const int as = r == 0 ? 0 : NQ;
                    for (; tau + 3 * NQ <= last; tau += 4 * NQ) {  // four columns: loads first
                        float* ep[4];
                        float ev[4], lv[4], av[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            ep[c] = win + slot * SW + r;
                            ev[c] = *ep[c];
                            lv[c] = lp[c * NQ];
                            av[c] = ap[c * as];
                            slot += NQ;
                            if (slot >= S2) slot -= S2;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) *ep[c] = fmaf(lv[c], av[c], ev[c]);
                        lp += 4 * NQ;
                        ap += 4 * as;
                    }
                    for (; tau <= last; tau += NQ) {
                        float* e = win + slot * SW + r;
                        *e = fmaf(*lp, *ap, *e);
                        slot += NQ;
                        if (slot >= S2) slot -= S2;
                        lp += NQ;
                        ap += as;
                    }
                }
            }
            if (u < S && k + S < nc) {  // column k + S enters its slot (read from step k + 1 on)
                win[((k + S) % S2) * SW + u] = pre;
                pre = k + S + 1 < nc ? gc[(int64_t)(k + S + 1) * BWP + u] : 0.f;
            }
        }
        __syncthreads();
    }
}

// The same elimination with the window in registers (bandwidths 33 .. 158, M = ceil(bw / 32)).
// Column c lives in slot c mod (bw + 2); slot sigma belongs to warp sigma mod 32 (its J =
// ceil((bw + 2) / 32) slots per warp as registers j = sigma / 32), lane i holding the row offsets r = 32 m + i + 1
// (m < M) and lane 0 also the excess (r = 0).  Step k: the warp holding column k + 1 applies
// pivot k to it, sums it (the lanes, shuffle-down trees and group order of the pivot group of
// k_ldl_gth_ahead, one group of 32 rows per warp there), forms 1/d_{k+1} and l_{.,k+1}, publishes
// l and the column (the multipliers of the next step) in shared memory and loads column
// k + 1 + bw + 2 for the freed slot (first updated two steps later); every warp applies
// pivot k to its other columns k + tau (2 <= tau <= bw), each entry with the multiply-add of the
// window kernels (those outside the band with l = 0: the entry is unchanged).  One block barrier
// per step and no shared-memory window.  Bit for bit k_ldl_gth_ahead.
template <int M>
__device__ __forceinline__ void gth_reg_pivot(const float (&e)[M], float e0, int c, int nc, int bw, int BWP,
                                              int lane, float* Ld, float* Ad, float* Sd, float* gc, float* gr) {
    float part[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int r = 32 * m + lane + 1;
        part[m] = (r <= bw ? e[m] : 0.f) + (m == 0 && lane == 0 ? e0 : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int m = 0; m < M; ++m) part[m] += __shfl_down_sync(0xffffffffu, part[m], o);
    }
    float dk = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) dk += part[m];  // the group totals, in group order (lane 0)
    dk = __shfl_sync(0xffffffffu, dk, 0);
    const float rd = 1.0f / dk;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int r = 32 * m + lane + 1;
        if (r <= bw) {
            const float l = e[m] * rd;
            Ld[r] = l;
            Ad[r] = e[m];
            gc[(int64_t)c * BWP + r] = l;
            if (c + r < nc) gr[(int64_t)(c + r) * BWP + r] = l;
        }
    }
    if (lane == 0) {
        *Sd = e0;
        gc[(int64_t)c * BWP] = rd;
    }
}

template <int M>
__device__ __forceinline__ void gth_reg_load(float (&e)[M], float& e0, const float* gc, int c, int nc, int bw,
                                             int BWP, int lane) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int r = 32 * m + lane + 1;
        e[m] = (c < nc && r <= bw) ? gc[(int64_t)c * BWP + r] : 0.f;
    }
    e0 = (c < nc && lane == 0) ? gc[(int64_t)c * BWP] : 0.f;
}

template <int M, int J>
__global__ void __launch_bounds__(1024, 1) k_ldl_gth_reg(float* __restrict__ gcol_all, float* __restrict__ grow_all,
                                                         int nc, int bw, int BWP, GkState* st) {
    // M = ceil(bw / 32) row groups, J = ceil((bw + 2) / 32) slots per warp
    constexpr int LW = 64 * M + 2;
    // l and the column of a pivot at t = 1 .. bw, zero beyond: a multiply-add of an entry outside
    // pivot k's band (tau + r > bw) reads l = 0 and leaves the entry as it is, exactly
    __shared__ float sL[2][LW], sA[2][LW];
    __shared__ float sS[2];
    const int S2 = bw + 2;
    const int inst = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (parked(st[inst])) return;
    float* gc = gcol_all + (int64_t)inst * nc * BWP;
    float* gr = grow_all + (int64_t)inst * nc * BWP;
    for (int e = tid; e < nc * BWP; e += blockDim.x)  // row layout: entries no pivot writes
        if (e % BWP == 0 || e % BWP > bw || e / BWP < e % BWP) gr[e] = 0.f;
    for (int e = tid; e < 2 * LW; e += blockDim.x) {
        (&sL[0][0])[e] = 0.f;
        (&sA[0][0])[e] = 0.f;
    }
    float ent[J][M], ex[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {  // columns 0 .. bw + 1 in slots 0 .. bw + 1
        const int sig = warp + 32 * j;
        gth_reg_load<M>(ent[j], ex[j], gc, sig < S2 ? sig : nc, nc, bw, BWP, lane);
    }
    __syncthreads();
    if (warp == 0) {  // pivot 0 (slot 0), then column bw + 2 enters the slot
        gth_reg_pivot<M>(ent[0], ex[0], 0, nc, bw, BWP, lane, sL[0], sA[0], &sS[0], gc, gr);
        gth_reg_load<M>(ent[0], ex[0], gc, S2, nc, bw, BWP, lane);
    }
    __syncthreads();
    // a column entering slot jpend: loaded into pf by the step that freed the slot and moved into
    // the slot's registers at the start of the next step (the load has landed by then, and no
    // instruction of the step that issued it waits for it)
    float pf[M], pf0 = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) pf[m] = 0.f;
    int jpend = -1;
    int kmod = 0;  // k mod S2
    for (int k = 0; k < nc; ++k) {
        const int b = k & 1;
        const float* Lk = sL[b];
        const float* Ak = sA[b];
        const float sk = sS[b];
        const int sn = kmod + 1 == S2 ? 0 : kmod + 1;  // slot of column k + 1
        if (jpend >= 0) {  // the same in every lane
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j == jpend) {
#pragma unroll
                    for (int m = 0; m < M; ++m) ent[j][m] = pf[m];
                    ex[j] = pf0;
                }
            }
            jpend = -1;
        }
        if (k + 1 < nc && (sn & 31) == warp) {
            const int jp = sn >> 5;
            float pe[M], pe0 = 0.f;
#pragma unroll
            for (int m = 0; m < M; ++m) pe[m] = 0.f;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j == jp) {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        ent[j][m] = fmaf(Lk[32 * m + lane + 2], Ak[1], ent[j][m]);
                        pe[m] = ent[j][m];
                    }
                    if (lane == 0) ex[j] = fmaf(Lk[1], sk, ex[j]);
                    pe0 = ex[j];
                }
            }
            gth_reg_pivot<M>(pe, pe0, k + 1, nc, bw, BWP, lane, sL[b ^ 1], sA[b ^ 1], &sS[b ^ 1], gc, gr);
            gth_reg_load<M>(pf, pf0, gc, k + 1 + S2, nc, bw, BWP, lane);  // slot jp, first read at step k + 3
            jpend = jp;
        }
        const int tmax = min(bw, nc - 1 - k);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int sig = warp + 32 * j;
            int tau = sig - kmod;
            if (tau < 0) tau += S2;
            if (sig < S2 && tau >= 2 && tau <= tmax) {  // the same in every lane
                const float a = Ak[tau];
                const float* lt = Lk + tau + lane + 1;  // row offset r = 32 m + lane + 1: l at tau + r
#pragma unroll
                for (int m = 0; m < M; ++m) ent[j][m] = fmaf(lt[32 * m], a, ent[j][m]);
                if (lane == 0) ex[j] = fmaf(Lk[tau], sk, ex[j]);
            }
        }
        kmod = sn;
        __syncthreads();
    }
}

// PLSQR_GTH_REG=0 keeps k_ldl_gth_ahead (comparisons)
bool gth_reg_supported(int bw, int nc) {
    const char* e = std::getenv("PLSQR_GTH_REG");
    return !(e && e[0] == '0') && bw > 32 && bw <= 158 && nc > 0;  // M <= 5, J <= 5 (64 registers)
}

// PLSQR_GTH_AHEAD=0 keeps k_ldl_gth_window (comparisons)
bool gth_ahead_supported(int bw, int nc) {
    const int S = bw + 1, SW = S | 1, GP = (bw + 31) / 32;
    const char* e = std::getenv("PLSQR_GTH_AHEAD");
    return !(e && e[0] == '0') && bw > 32 && bw <= 256 && GP <= 8 && (1024 - 32 * GP) / (bw / 2 + 1) >= 1 &&
           (size_t)(S + 1) * SW * sizeof(float) <= 200 * 1024 && nc > 0;
}

// X = L^{-T} D^{-1} L^{-1} for wide bands, one warp per column j: forward z_i = delta_ij +
// sum_t l_{i,i-t} z_{i-t} over the rows i >= j (row layout, consecutive lanes on consecutive t),
// y_i = z_i / d_i kept in X[i][j]; backward x_i = y_i + sum_t l_{i+t,i} x_{i+t} from the last row
// to row j (column layout), stored at X[i][j] and X[j][i].  The last bw values of z (x) sit in a
// ring in shared memory; the rows of the factor are loaded JW rows ahead into registers, the y
// values of a pass of 32 rows one per lane.  The warp sums go to lane 0 in a fixed order.  All
// terms are non-negative (l >= 0), as in the narrow kernel.  bw <= 32 * JT.
constexpr int JT = 8;  // factor entries per lane per row
constexpr int JW = 4;  // rows in flight

template <int NWARP>
__global__ void __launch_bounds__(32 * NWARP) k_gth_inverse_wide(const float* __restrict__ gcol_all,
                                                                 const float* __restrict__ grow_all,
                                                                 float* __restrict__ X_all, int nc, int bw, int BWP,
                                                                 GkState* st) {
    extern __shared__ float ring_all[];
    const int inst = blockIdx.y;
    if (parked(st[inst])) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * NWARP + warp;
    if (j >= nc) return;  // no block-wide barrier below
    const float* gc = gcol_all + (int64_t)inst * nc * BWP;
    const float* gr = grow_all + (int64_t)inst * nc * BWP;
    float* X = X_all + (int64_t)inst * nc * nc;
    const int R = bw + 1;
    float* ring = ring_all + warp * R;
    float fl[JW][JT];  // factor rows in flight (entry t = 1 + lane + 32 q)
    auto fetch = [&](const float* tab, int row, float (&dst)[JT]) {
#pragma unroll
        for (int q = 0; q < JT; ++q) {
            const int t = 1 + lane + 32 * q;
            dst[q] = (row >= 0 && row < nc && t <= bw) ? tab[(int64_t)row * BWP + t] : 0.f;
        }
    };
    // ---- forward over rows j, j+1, ... ----
    for (int e = lane; e < R; e += 32) ring[e] = 0.f;
#pragma unroll
    for (int w = 0; w < JW; ++w) fetch(gr, j + w, fl[w]);
    float dv = (j + lane < nc) ? gc[(int64_t)(j + lane) * BWP] : 0.f;  // 1/d of rows j + lane
    __syncwarp();
    int im = j % R;
    for (int i0 = j; i0 < nc; i0 += JW) {
#pragma unroll
        for (int w = 0; w < JW; ++w) {
            const int i = i0 + w;
            if (i < nc) {
                float part = 0.f;
#pragma unroll
                for (int q = 0; q < JT; ++q) {
                    const int t = 1 + lane + 32 * q;
                    if (t <= i - j && t <= bw) {
                        const int r = im - t;
                        part = fmaf(fl[w][q], ring[r < 0 ? r + R : r], part);
                    }
                }
                fetch(gr, i + JW, fl[w]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
                const float d = __shfl_sync(0xffffffffu, dv, (i - j) & 31);
                if (((i - j) & 31) == 31) dv = (i + 1 + lane < nc) ? gc[(int64_t)(i + 1 + lane) * BWP] : 0.f;
                __syncwarp();
                if (lane == 0) {
                    const float z = (i == j ? 1.f : 0.f) + part;
                    ring[im] = z;
                    X[(int64_t)i * nc + j] = z * d;
                }
                __syncwarp();
                im = im + 1 == R ? 0 : im + 1;
            }
        }
    }
    // ---- backward over rows nc-1, nc-2, ..., j ----
    for (int e = lane; e < R; e += 32) ring[e] = 0.f;
#pragma unroll
    for (int w = 0; w < JW; ++w) fetch(gc, nc - 1 - w, fl[w]);
    float yv = (nc - 1 - lane >= j) ? X[(int64_t)(nc - 1 - lane) * nc + j] : 0.f;  // y of rows nc-1-lane
    __syncwarp();
    im = (nc - 1) % R;
    for (int i0 = nc - 1; i0 >= j; i0 -= JW) {
#pragma unroll
        for (int w = 0; w < JW; ++w) {
            const int i = i0 - w;
            if (i >= j) {
                float part = 0.f;
#pragma unroll
                for (int q = 0; q < JT; ++q) {
                    const int t = 1 + lane + 32 * q;
                    if (t <= nc - 1 - i && t <= bw) {
                        const int r = im + t;
                        part = fmaf(fl[w][q], ring[r >= R ? r - R : r], part);
                    }
                }
                fetch(gc, i - JW, fl[w]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
                const float y = __shfl_sync(0xffffffffu, yv, (nc - 1 - i) & 31);
                if (((nc - 1 - i) & 31) == 31)
                    yv = (i - 1 - lane >= j) ? X[(int64_t)(i - 1 - lane) * nc + j] : 0.f;
                __syncwarp();
                if (lane == 0) {
                    const float x = y + part;
                    ring[im] = x;
                    X[(int64_t)i * nc + j] = x;
                    if (i != j) X[(int64_t)j * nc + i] = x;
                }
                __syncwarp();
                im = im == 0 ? R - 1 : im - 1;
            }
        }
    }
}

bool gth_wide_supported(int bw, int nc) {
    const int S = bw + 1, SW = S | 1;
    return bw > 0 && bw <= 32 * JT && (size_t)S * SW * sizeof(float) <= 200 * 1024 && nc > 0;
}

void gth_wide_factor_inverse(float* gcol, float* grow, float* X, float* xscr, int nc, int bw, int B, GkState* st,
                             cudaStream_t s) {
    if (!gth_wide_supported(bw, nc)) throw std::runtime_error("gth_wide_factor_inverse: bandwidth not supported");
    kbegin(KC_SETUP, s);
    const int BWP = gth_stride(bw);
    const int S = bw + 1, SW = S | 1;
    const size_t smem = sizeof(float) * (size_t)S * SW;
    const int nt0 = std::max(32, ((bw + 31) / 32) * 32);
    const int nt = nt0 * std::max(1, std::min(GTH_WQ, 1024 / nt0));
    if (gth_reg_supported(bw, nc)) {
        const int M = (bw + 31) / 32, J = (bw + 2 + 31) / 32;
        auto kfn = M == 2 ? (J == 2 ? k_ldl_gth_reg<2, 2> : k_ldl_gth_reg<2, 3>)
                 : M == 3 ? (J == 3 ? k_ldl_gth_reg<3, 3> : k_ldl_gth_reg<3, 4>)
                 : M == 4 ? (J == 4 ? k_ldl_gth_reg<4, 4> : k_ldl_gth_reg<4, 5>)
                          : k_ldl_gth_reg<5, 5>;
        kfn<<<B, 1024, 0, s>>>(gcol, grow, nc, bw, BWP, st);
        klaunched("k_ldl_gth_reg");
    } else if (gth_ahead_supported(bw, nc)) {
        const size_t smem2 = sizeof(float) * (size_t)(S + 1) * SW;
        if (smem2 > 48 * 1024)
            cudaFuncSetAttribute(k_ldl_gth_ahead, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        k_ldl_gth_ahead<<<B, 1024, smem2, s>>>(gcol, grow, nc, bw, BWP, st);
        klaunched("k_ldl_gth_ahead");
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_ldl_gth_window, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_ldl_gth_window<<<B, nt, smem, s>>>(gcol, grow, nc, bw, BWP, st);
        klaunched("k_ldl_gth_window");
    }
    if (xscr) {
        xblk_inverse<float>(gcol, X, xscr, nc, bw, B, st, s);
    } else {
        constexpr int NW = 4;
        dim3 grid((unsigned)((nc + NW - 1) / NW), B);
        k_gth_inverse_wide<NW><<<grid, 32 * NW, sizeof(float) * NW * (bw + 1), s>>>(gcol, grow, X, nc, bw, BWP, st);
        klaunched("k_gth_inverse_wide");
    }
    kfinish(s);
}

int gth_window(int bw) { return bw <= 8 ? 8 : bw <= 16 ? 16 : bw <= 32 ? 32 : 0; }

int gth_stride(int bw) {
    const int w = gth_window(bw);
    return ((w ? w : bw) + 1 + 3) & ~3;
}

bool gth_supported(int bw, int nc, size_t esz) {
    const int BWP = gth_stride(bw), W = gth_window(bw);
    if (W == 0 || (esz == 8 && W > 16)) return false;  // double: windows 8 and 16 (register budget)
    return (size_t)nc * BWP * esz + esz * 4 * W * 33 <= 220 * 1024;
}

template <typename T, typename V>
void gth_assemble(const T* cond, bool is_kappa, V* gcol, Dims d, int bw, int B, cudaStream_t s) {
    kbegin(KC_SETUP, s);
    const int BWP = gth_stride(bw);
    dim3 grid((unsigned)((d.N + 255) / 256), B);
    if (is_kappa) k_gth_assemble<T, V, true><<<grid, 256, 0, s>>>(cond, gcol, d, BWP);
    else k_gth_assemble<T, V, false><<<grid, 256, 0, s>>>(cond, gcol, d, BWP);
    klaunched("k_gth_assemble");
    kfinish(s);
}

template <typename V, int BW>
static void gth_launch(V* gcol, V* grow, V* X, V* xscr, int nc, int bw, int B, GkState* st, cudaStream_t s) {
    const int BWP = gth_stride(bw);
    const size_t stage = sizeof(V) * (size_t)nc * BWP;
    const size_t sp = stage + sizeof(V) * BWP;
    bool done = false;
    if constexpr (sizeof(V) == 4) {
        if (!gth_split_enabled()) {
            auto kp = k_ldl_gth_pipe<BW>;
            if (sp > 48 * 1024) cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
            kp<<<B, 32, sp, s>>>(gcol, grow, nc, bw, st);
            klaunched("k_ldl_gth_pipe");
            done = true;
        }
    }
    if (!done) {
        auto kq = k_ldl_gth_split<V, BW>;
        if (sp > 48 * 1024) cudaFuncSetAttribute(kq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
        kq<<<B, 32 * (1 + GTH_BULK), sp, s>>>(gcol, grow, nc, bw, st);
        klaunched("k_ldl_gth_split");
    }
    if (xscr) {  // the blocked inverse
        xblk_inverse<V>(gcol, X, xscr, nc, bw, B, st, s);
        return;
    }
    if (gth_inverse_by_warp(B, sizeof(V))) {
        constexpr int NWI = sizeof(V) == 8 ? 8 : 16;  // double: the registers of 32 band entries
        auto kw = k_gth_inverse_warp<V, BW, NWI>;
        if (stage > 48 * 1024) cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage);
        dim3 wgrid((unsigned)((nc + NWI - 1) / NWI), B);
        kw<<<wgrid, 32 * NWI, stage, s>>>(gcol, grow, X, nc, st);
        klaunched("k_gth_inverse_warp");
        return;
    }
    auto ki = k_gth_inverse<V, BW>;
    const size_t ism = stage + sizeof(V) * 4 * BW * 33;
    if (ism > 48 * 1024) cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
    dim3 igrid((unsigned)((nc + 127) / 128), B);
    ki<<<igrid, 128, ism, s>>>(gcol, grow, X, nc, st);
    klaunched("k_gth_inverse");
}

template <typename V>
void gth_factor_inverse(V* gcol, V* grow, V* X, V* xscr, int nc, int bw, int B, GkState* st, cudaStream_t s) {
    if (!gth_supported(bw, nc, sizeof(V)))
        throw std::runtime_error("gth_factor_inverse: bandwidth or size not supported");
    kbegin(KC_SETUP, s);
    switch (gth_window(bw)) {
        case 8: gth_launch<V, 8>(gcol, grow, X, xscr, nc, bw, B, st, s); break;
        case 16: gth_launch<V, 16>(gcol, grow, X, xscr, nc, bw, B, st, s); break;
        case 32:
            if constexpr (sizeof(V) == 4) gth_launch<V, 32>(gcol, grow, X, xscr, nc, bw, B, st, s);
            break;
    }
    kfinish(s);
}

template void gth_assemble<float, float>(const float*, bool, float*, Dims, int, int, cudaStream_t);
template void gth_assemble<double, float>(const double*, bool, float*, Dims, int, int, cudaStream_t);
template void gth_assemble<double, double>(const double*, bool, double*, Dims, int, int, cudaStream_t);
template void gth_factor_inverse<float>(float*, float*, float*, float*, int, int, int, GkState*, cudaStream_t);
template void gth_factor_inverse<double>(double*, double*, double*, double*, int, int, int, GkState*, cudaStream_t);

}  // namespace plsqr
