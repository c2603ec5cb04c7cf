// k_ops.cu -- forward maps A and adjoints A^T with the Golub-Kahan epilogues fused in.
//
// Gaussian blur (deblurring, Sec. 1): separable taps w_k = exp(-k^2/2s^2)/sum, |k| <= R,
// zero boundary, so B^T = B.  A 2D tile (64 x 32 outputs plus an R halo) is staged once in
// shared memory; the x pass writes an intermediate tile in shared memory and the y pass
// produces the output, so each input element is read from memory once per tile.  3D runs
// the same kernel per z-slice into a scratch volume, then a z pass with the epilogue.
// Masked blur (inpainting): A = D B (mask on the output), A^T = B D (mask on the input).
// Joseph projector (X-ray tomography, Sec. 1): one thread per ray steps along the dominant
// axis with linear interpolation; the adjoint is a gather per pixel over all angles of the
// (at most a few) rays whose interpolation touched the pixel, with the same weights: the
// exact transpose without atomics.
#include <cuda_runtime.h>

#include <stdexcept>
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "kernels.cuh"
#include "tma.cuh"

namespace plsqr {

template <typename T, int EPI>
__device__ __forceinline__ void epi_coefs(const GkState& s, T& ca, T& cp) {
    if (EPI == EPI_FWD) {
        ca = (T)s.c_fwd_a;
        cp = (T)s.c_fwd_p;
    } else if (EPI == EPI_ADJ) {
        ca = (T)s.c_adj_a;
        cp = (T)s.c_adj_p;
    } else if (EPI == EPI_ADJ_INIT) {
        ca = (T)s.c_adj_a;
        cp = (T)0;
    } else {
        ca = (T)1;
        cp = (T)0;
    }
}

// Apply the epilogue to one output element; returns the value written (for the norm).
template <typename T, int EPI>
__device__ __forceinline__ T epi_store(T acc, T ca, T cp, T* out, const T* prev, int64_t gi) {
    T v;
    if (EPI == EPI_PLAIN) {
        v = acc;
    } else if (EPI == EPI_FWD) {
        v = acc * ca - cp * prev[gi];
    } else if (EPI == EPI_ADJ) {
        v = acc * ca - cp * out[gi];
    } else {
        v = acc * ca;
    }
    out[gi] = v;
    return v;
}

// Finalise beta_{i+1} = ||u|| (Algorithm 2 step 10) in the last block.
// (1 / beta by the inverse square root of common.cuh; 1 / alpha is c_fwd_a.)
__device__ __forceinline__ void finalize_beta(GkState& s, double tot) {
    const double ib = tot > 0.0 ? rsqrt_nr(tot) : 0.0;
    const double bn = tot * ib;
    if (!good_pos(bn, s.beta1)) {
        s.status = ST_BREAKDOWN;
        s.status_any = ST_BREAKDOWN;
        return;
    }
    s.beta_new = bn;
    s.c_adj_a = ib;
    s.c_adj_p = bn * s.c_fwd_a;
}

constexpr int BTX = 64, BTY = 32, BNT = 256;

// TX x TY output tiles with NT threads; launch_blur2d picks smaller tiles when the grid would
// otherwise give few blocks (small double-precision images, where the blur is bound by the double
// pipe of the SMs it occupies).
template <typename T, int EPI, bool MASK_IN, bool MASK_OUT, int BTX = 64, int BTY = 32, int BNT = 256>
__global__ void __launch_bounds__(BNT) k_blur2d(const T* __restrict__ in, T* out, const T* prev,
                                                const uint8_t* __restrict__ mask, Dims d,
                                                const T* __restrict__ wx, int Rx, const T* __restrict__ wy,
                                                int Ry, GkState* st, Red red) {
    pdl_grid_sync();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int plane = blockIdx.z;  // z + nz * inst
    const int inst = plane / d.nz;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    const int tid = threadIdx.x;
    const int nwx = 2 * Rx + 1, nwy = 2 * Ry + 1;
    const int LX = BTX + 2 * Rx, LY = BTY + 2 * Ry;
    T* swx = reinterpret_cast<T*>(smraw);
    T* swy = swx + nwx;
    T* sin = swy + nwy;  // nwx + nwy is even: aligned for double
    T* smid = sin + LX * LY;
    for (int i = tid; i < nwx; i += BNT) swx[i] = wx[i];
    for (int i = tid; i < nwy; i += BNT) swy[i] = wy[i];
    const int x0 = blockIdx.x * BTX, y0 = blockIdx.y * BTY;
    const int64_t plane_off = (int64_t)plane * d.nx * d.ny;
    const int64_t mask_off = (int64_t)(plane - inst * d.nz) * d.nx * d.ny;
    for (int i = tid; i < LX * LY; i += BNT) {
        const int r = i / LX, c = i - r * LX;
        const int gy = y0 - Ry + r, gx = x0 - Rx + c;
        T v = (T)0;
        if (gy >= 0 && gy < d.ny && gx >= 0 && gx < d.nx) {
            const int64_t o = (int64_t)gy * d.nx + gx;
            v = in[plane_off + o];
            if (MASK_IN) v = mask[mask_off + o] ? v : (T)0;
        }
        sin[i] = v;
    }
    __syncthreads();
    for (int i = tid; i < LY * BTX; i += BNT) {
        const int r = i / BTX, c = i - r * BTX;
        const T* row = sin + r * LX + c;
        T acc = (T)0;
        for (int k = 0; k < nwx; ++k) acc = fma(swx[k], row[k], acc);
        smid[i] = acc;
    }
    __syncthreads();
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    T part = (T)0;
    for (int i = tid; i < BTY * BTX; i += BNT) {
        const int r = i / BTX, c = i - r * BTX;
        const int gy = y0 + r, gx = x0 + c;
        if (gy >= d.ny || gx >= d.nx) continue;
        const T* col = smid + r * BTX + c;
        T acc = (T)0;
        for (int k = 0; k < nwy; ++k) acc = fma(swy[k], col[k * BTX], acc);
        const int64_t o = (int64_t)gy * d.nx + gx;
        if (MASK_OUT) acc = mask[mask_off + o] ? acc : (T)0;
        T v = epi_store<T, EPI>(acc, ca, cp, out, prev, plane_off + o);
        if (EPI == EPI_FWD) part = fma(v, v, part);
    }
    if (EPI == EPI_FWD) {
        const int nblk = gridDim.x * gridDim.y * d.nz;
        const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * (plane - inst * d.nz));
        double tot;
        if (reduce_last<BNT>((double)part, red, inst, blk, nblk, &tot)) finalize_beta(st[inst], tot);
    }
}

// Register-blocked variant of k_blur2d for float with equal x / y radius R known at compile
// time.  The taps travel as kernel parameters (constant bank, FMA operands).  x pass: each
// thread produces 4 consecutive outputs of one row from a window of 4+2R inputs read as float4;
// y pass: each thread produces 8 consecutive outputs of one column from a window of 8+2R
// values held in registers.  Shared-memory loads per FMA drop from 2 to about 1/8.
template <int R>
struct TapsF {
    float w[2 * R + 1];
};

// TMA (R % 4 == 0): the whole halo tile arrives with one tensor copy (zero fill outside).
// UPD (with EPI_FWD): also the pending solution update of the previous iteration on the same
// cells, f += (phi/rho) w~, w~ = v~ - (theta/rho) w~ (Algorithm 2 steps 19-20), with v~ taken
// from the staged input tile.
// PI: the taps of each instance come from tapt[inst] ([2][2R+1], x then y) through shared memory
// instead of the kernel parameters.
template <int R, int EPI, bool MASK_IN, bool MASK_OUT, bool TMA, bool UPD, bool PI>
__global__ void __launch_bounds__(BNT) k_blur2d_rb(const __grid_constant__ CUtensorMap map_in,
                                                   const float* __restrict__ in, float* out, const float* prev,
                                                   const uint8_t* __restrict__ mask, Dims d, const TapsF<R> wx,
                                                   const TapsF<R> wy, GkState* st, Red red, float* __restrict__ fu,
                                                   float* __restrict__ wu, const float* __restrict__ tapt) {
    constexpr int LX = ((BTX + 2 * R) + 3) & ~3;  // row pitch (floats), multiple of 4
    constexpr int LY = BTY + 2 * R;
    constexpr int NW4 = (4 + 2 * R + 3) / 4;       // float4 loads per x-pass window
    static_assert(!TMA || (R % 4 == 0 && LX == BTX + 2 * R), "TMA tile needs a 16-byte aligned halo");
    __shared__ __align__(128) float sin[LY * LX];
    __shared__ __align__(16) float smid[LY * BTX];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float stap[PI ? 2 * (2 * R + 1) : 1];
    pdl_grid_sync();
    const int plane = blockIdx.z;
    const int inst = plane / d.nz;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * BTX, y0 = blockIdx.y * BTY;
    if constexpr (TMA) {  // the copy goes first; the instance state is read while it is in flight
        if (tid == 0) {
            mbar_init(&bar, 1);
            mbar_expect_tx(&bar, LX * LY * sizeof(float));
            tma_load_3d(sin, &map_in, &bar, x0 - R, y0 - R, plane);
        }
    }
    const bool skip = EPI != EPI_PLAIN && inner_off(st[inst]);  // the same in every thread
    if (!TMA && skip) return;
    if (PI)  // made visible by the barrier that follows the tile staging
        for (int k = tid; k < 2 * (2 * R + 1); k += BNT) stap[k] = tapt[(int64_t)inst * 2 * (2 * R + 1) + k];
    const int64_t plane_off = (int64_t)plane * d.nx * d.ny;
    const int64_t mask_off = (int64_t)(plane - inst * d.nz) * d.nx * d.ny;
    // this thread's outputs: column c, rows srow..srow+7 of the tile; their previous values
    // (and w~, f for UPD) are fetched now so the loads overlap the staging and the x pass
    const int oc = tid & (BTX - 1), srow = 8 * (tid / BTX);
    const int ogx = x0 + oc;
    float pv[8], wv[8], fv[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        pv[o] = wv[o] = fv[o] = 0.f;
        const int gy = y0 + srow + o;
        if (gy < d.ny && ogx < d.nx && !skip) {
            const int64_t gi = plane_off + (int64_t)gy * d.nx + ogx;
            if (EPI == EPI_FWD) pv[o] = prev[gi];
            if (EPI == EPI_ADJ) pv[o] = out[gi];
            if (UPD) {
                wv[o] = wu[gi];
                fv[o] = fu[gi];
            }
        }
    }
    if constexpr (TMA) {
        __syncthreads();  // the barrier's initialisation is visible to every thread
        tma_wait_tile(&bar, st, inst);
        if (skip) return;
    } else {
        for (int i = tid; i < LY * LX; i += BNT) {
            const int r = i / LX, c = i - r * LX;
            const int gy = y0 - R + r, gx = x0 - R + c;
            float v = 0.f;
            if (c < BTX + 2 * R && gy >= 0 && gy < d.ny && gx >= 0 && gx < d.nx) {
                const int64_t o = (int64_t)gy * d.nx + gx;
                v = in[plane_off + o];
                if (MASK_IN) v = mask[mask_off + o] ? v : 0.f;
            }
            sin[i] = v;
        }
        __syncthreads();
    }
    {  // x pass: rows r0, r0+16, ...; outputs 4q..4q+3
        const int q = tid & 15;
        for (int r = tid >> 4; r < LY; r += BNT / 16) {
            float win[4 * NW4];
            const float4* src = reinterpret_cast<const float4*>(sin + r * LX + 4 * q);
#pragma unroll
            for (int k = 0; k < NW4; ++k) {
                const float4 t = src[k];
                win[4 * k] = t.x;
                win[4 * k + 1] = t.y;
                win[4 * k + 2] = t.z;
                win[4 * k + 3] = t.w;
            }
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k)
#pragma unroll
                for (int o = 0; o < 4; ++o) acc[o] = fmaf(PI ? stap[k] : wx.w[k], win[o + k], acc[o]);
            *reinterpret_cast<float4*>(smid + r * BTX + 4 * q) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        }
    }
    __syncthreads();
    float ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<float, EPI>(st[inst], ca, cp);
    float part = 0.f;
    {  // y pass: column c, outputs rows 8s..8s+7
        const int c = oc;
        float win[8 + 2 * R];
#pragma unroll
        for (int k = 0; k < 8 + 2 * R; ++k) win[k] = smid[(srow + k) * BTX + c];
        float acc[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k)
#pragma unroll
            for (int o = 0; o < 8; ++o) acc[o] = fmaf(PI ? stap[2 * R + 1 + k] : wy.w[k], win[o + k], acc[o]);
        const int gx = ogx;
        float cv = 0.f, cf = 0.f, cw = 0.f;
        if (UPD) {
            cv = (float)st[inst].c_upd_v;
            cf = (float)st[inst].cf;
            cw = (float)st[inst].cw;
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int gy = y0 + srow + o;
            if (gy < d.ny && gx < d.nx) {
                const int64_t oo = (int64_t)gy * d.nx + gx;
                float a = acc[o];
                if (MASK_OUT) a = mask[mask_off + oo] ? a : 0.f;
                float v;
                if (EPI == EPI_PLAIN) v = a;
                else if (EPI == EPI_ADJ_INIT) v = a * ca;
                else v = a * ca - cp * pv[o];
                out[plane_off + oo] = v;
                if (EPI == EPI_FWD) part = fmaf(v, v, part);
                if (UPD) {
                    const float vin = sin[(srow + o + R) * LX + c + R];
                    fu[plane_off + oo] = fmaf(cf, wv[o], fv[o]);
                    wu[plane_off + oo] = vin * cv - cw * wv[o];
                }
            }
        }
    }
    if (EPI == EPI_FWD) {
        const int nblk = gridDim.x * gridDim.y * d.nz;
        const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * (plane - inst * d.nz));
        double tot;
        if (reduce_last<BNT>((double)part, red, inst, blk, nblk, &tot)) finalize_beta(st[inst], tot);
    }
}

constexpr int ZTZ = 16;  // z outputs per thread column; block = 32 (x) x 8 (y) threads

template <typename T, int EPI, bool MASK_OUT>
__global__ void __launch_bounds__(256) k_blur_z(const T* __restrict__ in, T* out, const T* prev,
                                                const uint8_t* __restrict__ mask, Dims d,
                                                const T* __restrict__ wz, int Rz, GkState* st, Red red) {
    pdl_grid_sync();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nzt = (d.nz + ZTZ - 1) / ZTZ;
    const int inst = blockIdx.z / nzt, zt = blockIdx.z - inst * nzt;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int nw = 2 * Rz + 1, LZ = ZTZ + 2 * Rz;
    T* sw = reinterpret_cast<T*>(smraw);
    T* s = sw + ((nw + 1) & ~1);
    for (int i = tid; i < nw; i += 256) sw[i] = wz[i];
    const int gx = blockIdx.x * 32 + tx, gy = blockIdx.y * 8 + ty, z0 = zt * ZTZ;
    const bool inxy = gx < d.nx && gy < d.ny;
    const int64_t plane = (int64_t)d.nx * d.ny;
    const int64_t base = (int64_t)inst * d.N + (int64_t)gy * d.nx + gx;
    for (int zz = 0; zz < LZ; ++zz) {
        const int gz = z0 - Rz + zz;
        T v = (T)0;
        if (inxy && gz >= 0 && gz < d.nz) v = in[base + gz * plane];
        s[zz * 256 + tid] = v;
    }
    __syncthreads();
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    T part = (T)0;
    if (inxy) {
        for (int zz = 0; zz < ZTZ; ++zz) {
            const int gz = z0 + zz;
            if (gz >= d.nz) break;
            T acc = (T)0;
            for (int k = 0; k < nw; ++k) acc = fma(sw[k], s[(zz + k) * 256 + tid], acc);
            const int64_t o = (int64_t)gz * plane + (int64_t)gy * d.nx + gx;
            if (MASK_OUT) acc = mask[o] ? acc : (T)0;
            T v = epi_store<T, EPI>(acc, ca, cp, out, prev, (int64_t)inst * d.N + o);
            if (EPI == EPI_FWD) part = fma(v, v, part);
        }
    }
    if (EPI == EPI_FWD) {
        const int nblk = gridDim.x * gridDim.y * nzt;
        const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zt);
        double tot;
        if (reduce_last<256>((double)part, red, inst, blk, nblk, &tot)) finalize_beta(st[inst], tot);
    }
}

// Register-blocked z pass for float with the z radius R known at compile time (the 3D workloads'
// 9, 12, 15): a thread owns one (x, y) column and ZR consecutive z outputs, loads the ZR + 2R
// input values of its column straight from memory into registers (coalesced across the 32 x
// lanes; all loads independent, so they are in flight together), and forms every output from
// them with the taps as FMA operands from the constant bank -- no shared memory and no reload of a
// value per tap.  The taps are summed in the order of k_blur_z, so the result is the same.
constexpr int ZR = 16;

template <int R>
struct TapsZ {
    float w[2 * R + 1];
};

template <int R, int EPI, bool MASK_OUT>
__global__ void __launch_bounds__(256) k_blur_z_rb(const float* __restrict__ in, float* out, const float* prev,
                                                   const uint8_t* __restrict__ mask, Dims d, const TapsZ<R> wz,
                                                   GkState* st, Red red) {
    pdl_grid_sync();
    const int nzt = (d.nz + ZR - 1) / ZR;
    const int inst = blockIdx.z / nzt, zt = blockIdx.z - inst * nzt;
    const bool skip = EPI != EPI_PLAIN && inner_off(st[inst]);  // the same in every thread of the block
    const int gx = blockIdx.x * 32 + (threadIdx.x & 31), gy = blockIdx.y * 8 + (threadIdx.x >> 5), z0 = zt * ZR;
    const bool inxy = gx < d.nx && gy < d.ny && !skip;
    const int64_t plane = (int64_t)d.nx * d.ny;
    const int64_t col = (int64_t)inst * d.N + (int64_t)gy * d.nx + gx;
    float win[ZR + 2 * R];
#pragma unroll
    for (int k = 0; k < ZR + 2 * R; ++k) {
        const int gz = z0 - R + k;
        win[k] = (inxy && gz >= 0 && gz < d.nz) ? __ldg(in + col + gz * plane) : 0.f;
    }
    float ca = 1.f, cp = 0.f;
    if (EPI != EPI_PLAIN && !skip) epi_coefs<float, EPI>(st[inst], ca, cp);
    float part = 0.f;
#pragma unroll
    for (int o = 0; o < ZR; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wz.w[k], win[o + k], acc);
        const int gz = z0 + o;
        if (inxy && gz < d.nz) {
            const int64_t oo = (int64_t)gz * plane + (int64_t)gy * d.nx + gx;
            if (MASK_OUT) acc = mask[oo] ? acc : 0.f;
            const float v = epi_store<float, EPI>(acc, ca, cp, out, prev, (int64_t)inst * d.N + oo);
            if (EPI == EPI_FWD) part = fmaf(v, v, part);
        }
    }
    if (EPI == EPI_FWD && !skip) {
        const int nblk = gridDim.x * gridDim.y * nzt;
        const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zt);
        double tot;
        if (reduce_last<256>((double)part, red, inst, blk, nblk, &tot)) finalize_beta(st[inst], tot);
    }
}

// A = I (denoising): the epilogue alone.
template <typename T, int EPI>
__global__ void __launch_bounds__(256) k_identity(const T* __restrict__ in, T* out, const T* prev, int64_t n,
                                                  GkState* st, Red red) {
    const int inst = blockIdx.y;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    T part = (T)0;
    const int64_t off = (int64_t)inst * n;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        T v = epi_store<T, EPI>(in[off + i], ca, cp, out, prev, off + i);
        if (EPI == EPI_FWD) part = fma(v, v, part);
    }
    if (EPI == EPI_FWD) {
        double tot;
        if (reduce_last<256>((double)part, red, inst, blockIdx.x, gridDim.x, &tot)) finalize_beta(st[inst], tot);
    }
}

// Joseph forward projection: one thread per ray (angle a, bin k).  Rows stepped: for each
// row i, x = (s - y_i sin)/cos, linear interpolation between the two bracketing columns,
// weight 1/|cos| (columns stepped: roles of x and y exchanged, weight 1/|sin|).
// Columns-stepped angles read the transposed image imgT (imgT[x][y] = img[y][x]), so that the
// lanes of a warp (neighbouring rays) gather from one row instead of 32 rows.
template <typename T, int EPI>
__global__ void __launch_bounds__(128) k_joseph_fwd(const T* __restrict__ img, const T* __restrict__ imgT, T* out,
                                                    const T* prev, const JosephAngle<T>* __restrict__ tab, int n,
                                                    int na, int nb, T ds, GkState* st, Red red) {
    const int inst = blockIdx.z, a = blockIdx.y, k = blockIdx.x * 128 + threadIdx.x;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    const JosephAngle<T> J = tab[a];
    const T cimg = (T)0.5 * (T)(n - 1), cdet = (T)0.5 * (T)(nb - 1);
    const T* im = (J.rows ? img : imgT) + (int64_t)inst * n * n;
    T acc = (T)0;
    if (k < nb) {
        const T s = ((T)k - cdet) * ds;
        const T u0 = s * J.a1 + cimg;
        // rows q with the sample inside (-1, n): u = u0 - (q - cimg) a2
        int qlo = 0, qhi = n - 1;
        if (fabs((double)J.a2) < 1e-7) {
            if (!(u0 > (T)-1 && u0 < (T)n)) qhi = -1;
        } else {
            const T q1 = (u0 - (T)n) / J.a2 + cimg, q2 = (u0 + (T)1) / J.a2 + cimg;
            const T lo = fmin(q1, q2), hi = fmax(q1, q2);
            qlo = max(0, (int)floor(lo) - 1);
            qhi = min(n - 1, (int)ceil(hi) + 1);
        }
        // samples outside the image add an exact 0
        for (int q = qlo; q <= qhi; ++q) {
            const T u = u0 - ((T)q - cimg) * J.a2;
            const T fl = floor(u);
            const int j0 = (int)fl;
            const T fr = u - fl;
            const T v0 = (j0 >= 0 && j0 < n) ? im[(int64_t)q * n + j0] : (T)0;
            const T v1 = (j0 + 1 >= 0 && j0 + 1 < n) ? im[(int64_t)q * n + j0 + 1] : (T)0;
            acc += ((T)1 - fr) * v0 + fr * v1;
        }
        acc *= J.wgt;
    }
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    T part = (T)0;
    if (k < nb) {
        T v = epi_store<T, EPI>(acc, ca, cp, out, prev, (int64_t)inst * na * nb + (int64_t)a * nb + k);
        if (EPI == EPI_FWD) part = v * v;
    }
    if (EPI == EPI_FWD) {
        double tot;
        if (reduce_last<128>((double)part, red, inst, blockIdx.x + gridDim.x * a, gridDim.x * gridDim.y, &tot))
            finalize_beta(st[inst], tot);
    }
}

// Joseph forward projection, band-staged: one block per (angle, instance), a thread per ray
// (bins tid, tid + 256, ...).  The image (img for rows-stepped angles, imgT for columns-stepped
// ones) is streamed through shared memory in bands of QB rows with cp.async double buffering, and
// every ray takes its samples of the band from shared memory, with the interpolation written
// x0 + fr (x1 - x0).  A ray's samples are summed in two parts, the rows below n/2 and the rest,
// each in increasing row order, and the parts are added.  One block takes both parts (H = 1), or,
// when the (angle, instance) pairs are too few to fill the GPU, two blocks take one part each
// (H = 2): the second to finish adds the two parts from the scratch `part` (its arrival counted in
// `cnt`, which it resets).  The sums do not depend on H or QB, so neither does the result.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int JF_RAYS = 4;  // rays per thread (nb <= 1024)
constexpr int JF_PAD = 4;   // zero elements on each side of a staged row

// acc += the samples of rows lo..hi (in order) of a ray; rowp = the staged row lo
template <typename T>
__device__ __forceinline__ void joseph_march(T& acc, int lo, int hi, T u0, T a2, T cimg, const T* rowp, int pitch) {
    T qc = (T)lo - cimg;  // q - cimg, exact
#pragma unroll 4
    for (int q = lo; q <= hi; ++q) {
        const T u = u0 - qc * a2;
        const T fl = floor(u);
        const int j0 = (int)fl;
        const T fr = u - fl;
        const T x0 = rowp[j0], x1 = rowp[j0 + 1];
        acc += x0 + fr * (x1 - x0);
        qc += (T)1;
        rowp += pitch;
    }
}

template <typename T, int EPI>
__global__ void __launch_bounds__(256, 5) k_joseph_fwd_band(const T* __restrict__ img, const T* __restrict__ imgT,
                                                         T* out, const T* prev,
                                                         const JosephAngle<T>* __restrict__ tab, int n, int na,
                                                         int nb, T ds, int QB, FDiv fvec, GkState* st, Red red,
                                                         T* part, unsigned* cnt) {
    // band rows are stored with JF_PAD zero elements on each side (pitch n + 2 JF_PAD), so that the
    // samples just outside the image (u in (-4, n + 3) for the conservative row ranges below, as
    // |a2| <= 1) read zeros without a bounds test
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned s_last;
    T* sbuf = reinterpret_cast<T*>(smraw);  // two bands of QB x pitch
    const int pitch = n + 2 * JF_PAD;
    const int inst = blockIdx.y, a = blockIdx.x, h = blockIdx.z, H = gridDim.z;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    const JosephAngle<T> J = tab[a];
    const T cimg = (T)0.5 * (T)(n - 1), cdet = (T)0.5 * (T)(nb - 1);
    const T* im = (J.rows ? img : imgT) + (int64_t)inst * n * n;
    for (int i = threadIdx.x; i < 2 * QB * 2 * JF_PAD; i += 256) {  // the pads of both buffers
        const int r = i / (2 * JF_PAD), c = i - r * (2 * JF_PAD);
        sbuf[(size_t)r * pitch + (c < JF_PAD ? c : n + c)] = (T)0;
    }
    T u0[JF_RAYS], acc[JF_RAYS], accA[JF_RAYS];
    int qlo[JF_RAYS], qhi[JF_RAYS];
#pragma unroll
    for (int r = 0; r < JF_RAYS; ++r) {
        const int k = threadIdx.x + 256 * r;
        acc[r] = (T)0;
        accA[r] = (T)0;
        qlo[r] = 0;
        qhi[r] = -1;
        u0[r] = (T)0;
        if (k < nb) {
            const T s = ((T)k - cdet) * ds;
            u0[r] = s * J.a1 + cimg;
            qhi[r] = n - 1;
            if (fabs((double)J.a2) < 1e-7) {
                if (!(u0[r] > (T)-1 && u0[r] < (T)n)) qhi[r] = -1;
            } else {
                const T q1 = (u0[r] - (T)n) / J.a2 + cimg, q2 = (u0[r] + (T)1) / J.a2 + cimg;
                const T lo = fmin(q1, q2), hi = fmax(q1, q2);
                qlo[r] = max(0, (int)floor(lo) - 1);
                qhi[r] = min(n - 1, (int)ceil(hi) + 1);
            }
        }
    }
    // bands: the rows [0, qs) of the first part in bands of QB from row 0, then the rows [qs, n)
    // of the second part in bands of QB from row qs
    const int qs = n / 2;
    const int nbA = (qs + QB - 1) / QB, nbB = (n - qs + QB - 1) / QB;
    const int b_lo = (H == 2 && h == 1) ? nbA : 0, b_hi = (H == 2 && h == 0) ? nbA : nbA + nbB;
    auto row0 = [&](int b) { return b < nbA ? b * QB : qs + (b - nbA) * QB; };
    auto row_end = [&](int b) { return b < nbA ? min(qs, (b + 1) * QB) : min(n, qs + (b - nbA + 1) * QB); };
    const int vec = n * (int)sizeof(T) / 16;  // 16-byte chunks per row
    auto stage = [&](int b) {
        T* dst = sbuf + (size_t)(b & 1) * QB * pitch + JF_PAD;
        const int q0 = row0(b), rows = row_end(b) - q0;
        const T* src = im + (int64_t)q0 * n;
        for (int c = threadIdx.x; c < rows * vec; c += 256) {
            const int r = (int)fdiv((uint32_t)c, fvec), v = c - r * vec;
            cp_async16(reinterpret_cast<char*>(dst + (size_t)r * pitch) + 16 * v,
                       reinterpret_cast<const char*>(src + (int64_t)r * n) + 16 * v);
        }
        cp_async_commit();
    };
    if (b_lo < b_hi) stage(b_lo);
    const T a2 = J.a2;
    for (int b = b_lo; b < b_hi; ++b) {
        if (b + 1 < b_hi) {
            stage(b + 1);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        if (b == nbA && b_lo == 0) {  // the first part is complete (one block takes both)
#pragma unroll
            for (int r = 0; r < JF_RAYS; ++r) {
                accA[r] = acc[r];
                acc[r] = (T)0;
            }
        }
        __syncthreads();
        const T* band = sbuf + (size_t)(b & 1) * QB * pitch + JF_PAD;
        const int q0 = row0(b), q1 = row_end(b) - 1;
#pragma unroll
        for (int r = 0; r < JF_RAYS; ++r) {
            const int lo = max(qlo[r], q0), hi = min(qhi[r], q1);
            joseph_march<T>(acc[r], lo, hi, u0[r], a2, cimg, band + (ptrdiff_t)(lo - q0) * pitch, pitch);
        }
        __syncthreads();  // the buffer of band b is refilled with band b + 2
    }
    if (H == 1) {
#pragma unroll
        for (int r = 0; r < JF_RAYS; ++r) acc[r] = accA[r] + acc[r];  // the loop passed band nbA (nbB >= 1)
    } else {
        T* pp = part + ((int64_t)h * gridDim.y + inst) * na * nb + (int64_t)a * nb;
#pragma unroll
        for (int r = 0; r < JF_RAYS; ++r) {
            const int k = threadIdx.x + 256 * r;
            if (k < nb) pp[k] = acc[r];
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned* c = cnt + (int64_t)inst * na + a;
            const unsigned old = atomicAdd(c, 1u);
            s_last = old == 1u;
            if (old == 1u) *c = 0u;  // for the next launch
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        const T* p0 = part + (int64_t)inst * na * nb + (int64_t)a * nb;
        const T* p1 = p0 + (int64_t)gridDim.y * na * nb;
#pragma unroll
        for (int r = 0; r < JF_RAYS; ++r) {
            const int k = threadIdx.x + 256 * r;
            acc[r] = k < nb ? __ldcg(p0 + k) + __ldcg(p1 + k) : (T)0;
        }
    }
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    T psum = (T)0;
#pragma unroll
    for (int r = 0; r < JF_RAYS; ++r) {
        const int k = threadIdx.x + 256 * r;
        if (k < nb) {
            const T v = epi_store<T, EPI>(acc[r] * J.wgt, ca, cp, out, prev, (int64_t)inst * na * nb + (int64_t)a * nb + k);
            if (EPI == EPI_FWD) psum = fma(v, v, psum);
        }
    }
    if (EPI == EPI_FWD) {
        double tot;
        if (reduce_last<256>((double)psum, red, inst, a, na, &tot)) finalize_beta(st[inst], tot);
    }
}

// imgT[x][y] = img[y][x] for each n x n instance, through 32 x 32 shared-memory tiles.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T* __restrict__ img, T* __restrict__ imgT, int n) {
    __shared__ T tile[32][33];
    const int inst = blockIdx.z;
    const T* a = img + (int64_t)inst * n * n;
    T* b = imgT + (int64_t)inst * n * n;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int r = threadIdx.x >> 5; r < 32; r += 8) {
        const int y = y0 + r, x = x0 + (threadIdx.x & 31);
        if (y < n && x < n) tile[r][threadIdx.x & 31] = a[(int64_t)y * n + x];
    }
    __syncthreads();
    for (int r = threadIdx.x >> 5; r < 32; r += 8) {
        const int x = x0 + r, y = y0 + (threadIdx.x & 31);
        if (y < n && x < n) b[(int64_t)x * n + y] = tile[threadIdx.x & 31][r];
    }
}

// Joseph adjoint, gather form: pixel (i, j) collects, for every angle, the rays k with
// |s_k - s_ij| < h (h = |cos| rows stepped, |sin| columns stepped), s_ij = x cos + y sin,
// with the forward weight (1 - |s_k - s_ij|/h)/h.  No atomics; exact transpose.
template <typename T, int EPI>
__global__ void __launch_bounds__(256) k_joseph_adj(const T* __restrict__ sino, T* out,
                                                    const JosephAngle<T>* __restrict__ tab, int n, int na, int nb,
                                                    int KB, GkState* st) {
    // A 16 x 16 pixel tile touches, per angle, at most KB consecutive bins: they are staged in
    // shared memory (zeros outside the detector) together with the angle table, so the loop over
    // angles reads only shared memory.
    extern __shared__ __align__(16) unsigned char smraw[];
    JosephAngle<T>* stab = reinterpret_cast<JosephAngle<T>*>(smraw);
    int* sk0 = reinterpret_cast<int*>(stab + na);
    T* sbin = reinterpret_cast<T*>(smraw + ((sizeof(JosephAngle<T>) * na + sizeof(int) * na + 15) & ~(size_t)15));
    const int inst = blockIdx.z;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    const T cimg = (T)0.5 * (T)(n - 1), cdet = (T)0.5 * (T)(nb - 1);
    const int tj = blockIdx.x * 16, ti = blockIdx.y * 16;
    const T xa = (T)tj - cimg, xb = (T)min(tj + 15, n - 1) - cimg;
    const T ya = (T)ti - cimg, yb = (T)min(ti + 15, n - 1) - cimg;
    for (int a = threadIdx.x; a < na; a += 256) {
        const JosephAngle<T> J = tab[a];
        stab[a] = J;
        const T tmin = fmin(xa * J.c1, xb * J.c1) + fmin(ya * J.c2, yb * J.c2) + cdet;
        sk0[a] = (int)floor(tmin - J.hw) - 1;
    }
    __syncthreads();
    const T* sg = sino + (int64_t)inst * na * nb;
    for (int e = threadIdx.x; e < na * KB; e += 256) {
        const int a = e / KB, kk = e - a * KB;
        const int k = sk0[a] + kk;
        sbin[e] = (k >= 0 && k < nb) ? sg[(int64_t)a * nb + k] : (T)0;
    }
    __syncthreads();
    const int j = tj + (threadIdx.x & 15), i = ti + (threadIdx.x >> 4);
    if (i >= n || j >= n) return;
    const T x = (T)j - cimg, y = (T)i - cimg;
    T acc = (T)0;
    for (int a = 0; a < na; ++a) {
        const JosephAngle<T>& J = stab[a];
        const T t = x * J.c1 + y * J.c2 + cdet;
        const int k0 = sk0[a];
        const int klo = (int)ceil(t - J.hw), khi = (int)floor(t + J.hw);
        const T* row = sbin + a * KB - k0;
        T acc_a = (T)0;
        for (int k = klo; k <= khi; ++k) {
            const T dist = fabs((T)k - t);
            if (dist < J.hw) acc_a += ((T)1 - dist * J.inv_hw) * row[k];
        }
        acc += acc_a * J.wgt;
    }
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    epi_store<T, EPI>(acc, ca, cp, out, out, (int64_t)inst * n * n + (int64_t)i * n + j);
}

// Gather adjoint when every half-width is at most one bin (ds >= max(|cos|, |sin|)): the rays that
// reach a pixel are the two bins around s_ij, floor(t) and floor(t) + 1, with weights
// max(0, 1 - |k - t| / h).  Tiles of 16 (x) x 32 (y) pixels, two pixels per thread (rows y and
// y + 16); per angle the tile's bin band (KB bins from k0) is staged in shared memory, and
// (c1, c2, cdet - k0, 1/h) and the weight 1/h are kept for every angle.
constexpr int JAX = 16, JAY = 32;

template <typename T>
struct __align__(4 * sizeof(T)) JosephAdjAngle {
    T c1, c2, off, ih;  // t - k0 = x c1 + y c2 + off; 1 / h
};

// The angles are taken in chunks of JA_CH (their bin bands staged one chunk at a time), so that
// the shared memory of a block stays small and every block of a launch is resident at once.  The
// per-pixel sums run over the angles in order, whatever the chunking.
constexpr int JA_CH = 128;

template <typename T, int EPI>
__global__ void __launch_bounds__(JAX * JAY / 2) k_joseph_adj2(const T* __restrict__ sino, T* out,
                                                               const JosephAngle<T>* __restrict__ tab, int n, int na,
                                                               int nb, int KB, GkState* st) {
    constexpr int NT = JAX * JAY / 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    using T4 = JosephAdjAngle<T>;
    T4* sp = reinterpret_cast<T4*>(smraw);                 // (c1, c2, cdet - k0, 1/h)
    T* sw = reinterpret_cast<T*>(sp + na);                 // 1/h (forward weight)
    int* sk0 = reinterpret_cast<int*>(sw + na);
    T* sbin = reinterpret_cast<T*>(smraw + ((sizeof(T4) * na + sizeof(T) * na + sizeof(int) * na + 15) & ~(size_t)15));
    const int inst = blockIdx.z;
    if (EPI != EPI_PLAIN && inner_off(st[inst])) return;
    const T cimg = (T)0.5 * (T)(n - 1), cdet = (T)0.5 * (T)(nb - 1);
    const int tj = blockIdx.x * JAX, ti = blockIdx.y * JAY;
    const T xa = (T)tj - cimg, xb = (T)min(tj + JAX - 1, n - 1) - cimg;
    const T ya = (T)ti - cimg, yb = (T)min(ti + JAY - 1, n - 1) - cimg;
    for (int a = threadIdx.x; a < na; a += NT) {
        const JosephAngle<T> J = tab[a];
        const T tmin = fmin(xa * J.c1, xb * J.c1) + fmin(ya * J.c2, yb * J.c2) + cdet;
        const int k0 = (int)floor(tmin - J.hw) - 1;
        sk0[a] = k0;
        T4 pv;
        pv.c1 = J.c1;
        pv.c2 = J.c2;
        pv.off = cdet - (T)k0;
        pv.ih = J.inv_hw;
        sp[a] = pv;
        sw[a] = J.wgt;
    }
    const T* sg = sino + (int64_t)inst * na * nb;
    const int j = tj + (threadIdx.x & (JAX - 1)), i0 = ti + (threadIdx.x / JAX), i1 = i0 + JAY / 2;
    // pixels beyond a ragged edge are evaluated at the edge (inside the staged band), not stored
    const T x = (T)min(j, n - 1) - cimg, y0 = (T)min(i0, n - 1) - cimg, y1 = (T)min(i1, n - 1) - cimg;
    T acc0 = (T)0, acc1 = (T)0;
    for (int a0 = 0; a0 < na; a0 += JA_CH) {
        const int a1 = min(na, a0 + JA_CH);
        __syncthreads();  // the table is written (first chunk) / the previous chunk's bins are read
#pragma unroll 4
        for (int e = threadIdx.x; e < (a1 - a0) * KB; e += NT) {
            const int a = a0 + e / KB, kk = e - (a - a0) * KB;
            const int k = sk0[a] + kk;
            sbin[e] = (k >= 0 && k < nb) ? sg[(int64_t)a * nb + k] : (T)0;
        }
        __syncthreads();
        for (int a = a0; a < a1; ++a) {
            const T4 pv = sp[a];
            const T wa = sw[a];
            const T* row = sbin + (a - a0) * KB;
            const T ux = fma(x, pv.c1, pv.off);
            {
                const T u = fma(y0, pv.c2, ux);  // t - k0
                const T fu = floor(u);
                const int q = (int)fu;
                const T fr = u - fu;
                const T w0 = fmax((T)0, (T)1 - fr * pv.ih), w1 = fmax((T)0, (T)1 - ((T)1 - fr) * pv.ih);
                acc0 += (w0 * row[q] + w1 * row[q + 1]) * wa;
            }
            {
                const T u = fma(y1, pv.c2, ux);
                const T fu = floor(u);
                const int q = (int)fu;
                const T fr = u - fu;
                const T w0 = fmax((T)0, (T)1 - fr * pv.ih), w1 = fmax((T)0, (T)1 - ((T)1 - fr) * pv.ih);
                acc1 += (w0 * row[q] + w1 * row[q + 1]) * wa;
            }
        }
    }
    T ca, cp;
    if (EPI != EPI_PLAIN) epi_coefs<T, EPI>(st[inst], ca, cp);
    if (j < n && i0 < n) epi_store<T, EPI>(acc0, ca, cp, out, out, (int64_t)inst * n * n + (int64_t)i0 * n + j);
    if (j < n && i1 < n) epi_store<T, EPI>(acc1, ca, cp, out, out, (int64_t)inst * n * n + (int64_t)i1 * n + j);
}

// Blocks per (angle, instance) of the band-staged forward projection: 2 when the launch has fewer
// than three (angle, instance) pairs per SM and the operator holds the scratch for B instances;
// PLSQR_JOSEPH_PARTS=1 or 2 forces one (2 only within the scratch).
static int joseph_fwd_parts(const OpDev& op, int B) {
    const bool room = op.jpart && op.jcnt && B <= op.jcap;
    if (const char* e = getenv("PLSQR_JOSEPH_PARTS")) {
        const int p = atoi(e);
        if (p == 1) return 1;
        if (p == 2) return room ? 2 : 1;
    }
    return room && (int64_t)op.na * B < 3 * 152 ? 2 : 1;
}

// Bins a JAX x JAY tile can touch for one angle (two-tap kernel), and whether every half-width
// is at most one bin.
static int joseph_tile_bins2(const OpDev& op, bool* two_tap) {
    const double ds = op.ds;
    double w = 0.0, hmax = 0.0;
    for (int a = 0; a < op.na; ++a) {
        const double th = 3.14159265358979323846 * (double)a / (double)op.na;
        const double c = std::fabs(std::cos(th)), sn = std::fabs(std::sin(th));
        const bool rows = (4 * a < op.na) || (4 * a > 3 * op.na);
        const double hw = (rows ? c : sn) / ds;
        hmax = std::max(hmax, hw);
        w = std::max(w, ((JAX - 1) * c + (JAY - 1) * sn) / ds + 2.0 * hw);
    }
    *two_tap = hmax <= 1.0;
    return (int)std::ceil(w) + 4;
}

// PLSQR_JOSEPH_GENERIC=1: the per-ray global-memory forward kernel (comparisons).
static bool op_generic_joseph() {
    static const bool on = [] {
        const char* e = std::getenv("PLSQR_JOSEPH_GENERIC");
        return e && e[0] == '1';
    }();
    return on;
}

// Bins a 16 x 16 tile can touch for one angle: 15 (|cos| + |sin|)/ds + 2 hw + 2 of slack, maximised
// over the angles.
template <typename T>
static int joseph_tile_bins(const OpDev& op) {
    const double ds = op.ds;
    double w = 0.0;
    for (int a = 0; a < op.na; ++a) {
        const double th = 3.14159265358979323846 * (double)a / (double)op.na;
        const double c = std::fabs(std::cos(th)), sn = std::fabs(std::sin(th));
        const bool rows = (4 * a < op.na) || (4 * a > 3 * op.na);
        const double hw = (rows ? c : sn) / ds;
        w = std::max(w, 15.0 * (c + sn) / ds + 2.0 * hw);
    }
    return (int)std::ceil(w) + 4;
}

// ---- launchers ---------------------------------------------------------------------------


template <int R, int EPI, bool MI, bool MO, bool UPD = false>
static void launch_blur2d_rb(const OpDev& op, const float* in, float* out, const float* prev, int B, GkState* st,
                             Red red, cudaStream_t s, float* fu = nullptr, float* wu = nullptr) {
    const Dims& d = op.d;
    TapsF<R> wx, wy;
    for (int k = 0; k <= 2 * R; ++k) {
        wx.w[k] = (float)op.taps_host[0][k];
        wy.w[k] = (float)op.taps_host[1][k];
    }
    dim3 grid((d.nx + BTX - 1) / BTX, (d.ny + BTY - 1) / BTY, d.nz * B);
    if (EPI == EPI_FWD && (int64_t)grid.x * grid.y * d.nz > red.max_blocks)
        throw std::runtime_error("blur2d: too many blocks for the reduction scratch");
    CUtensorMap map{};
    bool tma = false;
    if constexpr (R % 4 == 0 && !MI) {
        tma = tma_enabled() &&
              tma_map_3d(&map, in, 4, d.nx, d.ny, (int64_t)d.nz * B, BTX + 2 * R, BTY + 2 * R, 1);
        if (tma) {
            if constexpr (!MI && !MO) {
                if (op.tapt) {
                    max_carveout_set((const void*)k_blur2d_rb<R, EPI, MI, MO, true, UPD, true>);
                    launch_k(k_blur2d_rb<R, EPI, MI, MO, true, UPD, true>, grid, dim3(BNT), 0, s, map, in, out, prev,
                             (const uint8_t*)op.mask, d, wx, wy, st, red, fu, wu, op.tapt);
                    klaunched("k_blur2d_rb");
                    return;
                }
            }
            max_carveout_set((const void*)k_blur2d_rb<R, EPI, MI, MO, true, UPD, false>);
            launch_k(k_blur2d_rb<R, EPI, MI, MO, true, UPD, false>, grid, dim3(BNT), 0, s, map, in, out, prev,
                     (const uint8_t*)op.mask, d, wx, wy, st, red, fu, wu, (const float*)nullptr);
        }
    }
    if (!tma) {
        if constexpr (!MI && !MO) {
            if (op.tapt) {
                launch_k(k_blur2d_rb<R, EPI, MI, MO, false, UPD, true>, grid, dim3(BNT), 0, s, map, in, out, prev,
                         (const uint8_t*)op.mask, d, wx, wy, st, red, fu, wu, op.tapt);
                klaunched("k_blur2d_rb");
                return;
            }
        }
        launch_k(k_blur2d_rb<R, EPI, MI, MO, false, UPD, false>, grid, dim3(BNT), 0, s, map, in, out, prev,
                 (const uint8_t*)op.mask, d, wx, wy, st, red, fu, wu, (const float*)nullptr);
    }
    klaunched("k_blur2d_rb");
}

template <typename T, int EPI, bool MI, bool MO>
static void launch_blur2d(const OpDev& op, const T* in, T* out, const T* prev, int B, GkState* st, Red red,
                          cudaStream_t s) {
    const Dims& d = op.d;
    const int Rx = op.R[0], Ry = op.R[1];
    if constexpr (std::is_same<T, float>::value) {
        if (Rx == Ry && !op.generic_blur) {
            switch (Rx) {
                case 6: launch_blur2d_rb<6, EPI, MI, MO>(op, in, out, prev, B, st, red, s); return;
                case 9: launch_blur2d_rb<9, EPI, MI, MO>(op, in, out, prev, B, st, red, s); return;
                case 12: launch_blur2d_rb<12, EPI, MI, MO>(op, in, out, prev, B, st, red, s); return;
                case 15: launch_blur2d_rb<15, EPI, MI, MO>(op, in, out, prev, B, st, red, s); return;
                default: break;
            }
        }
    }
    // the largest of 64x32, 32x16, 16x16, 16x8 and 8x8 tiles that gives at least 152 blocks per
    // instance (else 8x8); the choice depends on the grid only, not on the batch
    auto blocks = [&](int tx, int ty) { return (int64_t)((d.nx + tx - 1) / tx) * ((d.ny + ty - 1) / ty) * d.nz; };
    int pick = 4;
    const int tiles[4][2] = {{64, 32}, {32, 16}, {16, 16}, {16, 8}};
    for (int q = 0; q < 4; ++q)
        if (blocks(tiles[q][0], tiles[q][1]) >= 152) {
            pick = q;
            break;
        }
    auto go = [&](auto kfn, int tx, int ty, int nt) {
        size_t smem = sizeof(T) * ((2 * Rx + 1) + (2 * Ry + 1) + (size_t)(tx + 2 * Rx) * (ty + 2 * Ry) +
                                   (size_t)(ty + 2 * Ry) * tx);
        if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        dim3 grid((d.nx + tx - 1) / tx, (d.ny + ty - 1) / ty, d.nz * B);
        if (EPI == EPI_FWD && (int64_t)grid.x * grid.y * d.nz > red.max_blocks)
            throw std::runtime_error("blur2d: too many blocks for the reduction scratch");
        launch_k(kfn, grid, dim3(nt), smem, s, in, out, prev, (const uint8_t*)op.mask, d, (const T*)op.taps[0], Rx,
                 (const T*)op.taps[1], Ry, st, red);
    };
    switch (pick) {
        case 0: go(k_blur2d<T, EPI, MI, MO, 64, 32, 256>, 64, 32, 256); break;
        case 1: go(k_blur2d<T, EPI, MI, MO, 32, 16, 256>, 32, 16, 256); break;
        case 2: go(k_blur2d<T, EPI, MI, MO, 16, 16, 256>, 16, 16, 256); break;
        case 3: go(k_blur2d<T, EPI, MI, MO, 16, 8, 128>, 16, 8, 128); break;
        default: go(k_blur2d<T, EPI, MI, MO, 8, 8, 64>, 8, 8, 64); break;
    }
    klaunched("k_blur2d");
}

template <int R, int EPI, bool MO>
static void launch_blur_z_rb(const OpDev& op, const float* in, float* out, const float* prev, int B, GkState* st,
                             Red red, cudaStream_t s) {
    const Dims& d = op.d;
    TapsZ<R> wz;
    for (int k = 0; k <= 2 * R; ++k) wz.w[k] = (float)op.taps_host[2][k];
    const int nzt = (d.nz + ZR - 1) / ZR;
    dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, nzt * B);
    if (EPI == EPI_FWD && (int64_t)grid.x * grid.y * nzt > red.max_blocks)
        throw std::runtime_error("blur_z: too many blocks for the reduction scratch");
    launch_k(k_blur_z_rb<R, EPI, MO>, grid, dim3(256), 0, s, in, out, prev, (const uint8_t*)op.mask, d, wz, st, red);
    klaunched("k_blur_z_rb");
}

template <typename T, int EPI, bool MO>
static void launch_blur_z(const OpDev& op, const T* in, T* out, const T* prev, int B, GkState* st, Red red,
                          cudaStream_t s) {
    const Dims& d = op.d;
    const int Rz = op.R[2];
    if constexpr (std::is_same<T, float>::value) {
        if (!op.generic_blur) {
            switch (Rz) {
                case 9: launch_blur_z_rb<9, EPI, MO>(op, in, out, prev, B, st, red, s); return;
                case 12: launch_blur_z_rb<12, EPI, MO>(op, in, out, prev, B, st, red, s); return;
                case 15: launch_blur_z_rb<15, EPI, MO>(op, in, out, prev, B, st, red, s); return;
                default: break;
            }
        }
    }
    const int nw = 2 * Rz + 1;
    size_t smem = sizeof(T) * ((size_t)((nw + 1) & ~1) + (size_t)(ZTZ + 2 * Rz) * 256);
    auto kfn = k_blur_z<T, EPI, MO>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int nzt = (d.nz + ZTZ - 1) / ZTZ;
    dim3 grid((d.nx + 31) / 32, (d.ny + 7) / 8, nzt * B);
    if (EPI == EPI_FWD && (int64_t)grid.x * grid.y * nzt > red.max_blocks)
        throw std::runtime_error("blur_z: too many blocks for the reduction scratch");
    launch_k(kfn, grid, dim3(256), smem, s, in, out, prev, (const uint8_t*)op.mask, d, (const T*)op.taps[2], Rz, st,
             red);
    klaunched("k_blur_z");
}

template <typename T, int EPI>
static void apply_epi(const OpDev& op, bool adjoint, const T* in, T* out, const T* prev, T* tmp, int B,
                      GkState* st, Red red, cudaStream_t s) {
    switch (op.kind) {
        case OPK_IDENTITY: {
            int nblk = (int)std::min<int64_t>((op.m + 255) / 256, 1024);
            nblk = std::min(nblk, red.max_blocks);
            k_identity<T, EPI><<<dim3(nblk, B), 256, 0, s>>>(in, out, prev, op.m, st, red);
            klaunched("k_identity");
            return;
        }
        case OPK_BLUR:
        case OPK_BLUR_MASK: {
            const bool mk = op.kind == OPK_BLUR_MASK;
            if (op.d.ndim == 2) {
                if (!mk) launch_blur2d<T, EPI, false, false>(op, in, out, prev, B, st, red, s);
                else if (adjoint) launch_blur2d<T, EPI, true, false>(op, in, out, prev, B, st, red, s);
                else launch_blur2d<T, EPI, false, true>(op, in, out, prev, B, st, red, s);
            } else {
                if (mk && adjoint) launch_blur2d<T, EPI_PLAIN, true, false>(op, in, tmp, nullptr, B, st, red, s);
                else launch_blur2d<T, EPI_PLAIN, false, false>(op, in, tmp, nullptr, B, st, red, s);
                if (mk && !adjoint) launch_blur_z<T, EPI, true>(op, tmp, out, prev, B, st, red, s);
                else launch_blur_z<T, EPI, false>(op, tmp, out, prev, B, st, red, s);
            }
            return;
        }
        case OPK_JOSEPH: {
            const int n = op.d.nx;
            const auto* tab = (const JosephAngle<T>*)op.jtab;
            if (!adjoint) {
                if (!tmp) throw std::runtime_error("joseph_fwd: scratch for the transposed image missing");
                dim3 tg((n + 31) / 32, (n + 31) / 32, B);
                k_transpose<T><<<tg, 256, 0, s>>>(in, tmp, n);
                klaunched("k_transpose");
                // band-staged form: rows of 16-byte multiples, at most JF_RAYS * 256 bins
                int QB = std::max(1, std::min(64, (int)(32768 / ((size_t)n * sizeof(T)))));
                if ((n * sizeof(T)) % 16 == 0 && op.nb <= JF_RAYS * 256 && !op_generic_joseph()) {
                    const int H = joseph_fwd_parts(op, B);
                    if (H == 2) {  // bands small enough that all 2 na B blocks are resident at once
                        const int64_t per_sm = ((int64_t)2 * op.na * B + 151) / 152;
                        const int64_t budget = 228 * 1024 / per_sm - 1024 - 128;
                        const int64_t qb = budget / (2 * (int64_t)sizeof(T) * (n + 2 * JF_PAD));
                        QB = (int)std::max<int64_t>(1, std::min<int64_t>(QB, qb));
                    }
                    const size_t smem = 2 * sizeof(T) * (size_t)QB * (n + 2 * JF_PAD);
                    auto kfn = k_joseph_fwd_band<T, EPI>;
                    if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (EPI == EPI_FWD && op.na > red.max_blocks)
                        throw std::runtime_error("joseph_fwd: too many blocks for the reduction scratch");
                    const FDiv fvec = make_fdiv((int64_t)n * sizeof(T) / 16);
                    kfn<<<dim3(op.na, B, H), 256, smem, s>>>(in, tmp, out, prev, tab, n, op.na, op.nb, (T)op.ds, QB,
                                                             fvec, st, red, (T*)op.jpart, op.jcnt);
                    klaunched("k_joseph_fwd_band");
                    return;
                }
                dim3 grid((op.nb + 127) / 128, op.na, B);
                if (EPI == EPI_FWD && (int64_t)grid.x * grid.y > red.max_blocks)
                    throw std::runtime_error("joseph_fwd: too many blocks for the reduction scratch");
                k_joseph_fwd<T, EPI><<<grid, 128, 0, s>>>(in, tmp, out, prev, tab, n, op.na, op.nb, (T)op.ds, st, red);
                klaunched("k_joseph_fwd");
            } else {
                bool two = false;
                const int KB2 = joseph_tile_bins2(op, &two);
                const size_t head2 =
                    (sizeof(T) * 4 * op.na + sizeof(T) * op.na + sizeof(int) * op.na + 15) & ~(size_t)15;
                const size_t smem2 = head2 + sizeof(T) * (size_t)std::min(op.na, JA_CH) * KB2;
                if (two && smem2 <= 227 * 1024) {
                    auto kfn = k_joseph_adj2<T, EPI>;
                    if (smem2 > 48 * 1024)
                        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
                    dim3 grid((n + JAX - 1) / JAX, (n + JAY - 1) / JAY, B);
                    kfn<<<grid, JAX * JAY / 2, smem2, s>>>(in, out, tab, n, op.na, op.nb, KB2, st);
                    klaunched("k_joseph_adj2");
                    return;
                }
                const int KB = joseph_tile_bins<T>(op);
                const size_t head = (sizeof(JosephAngle<T>) * op.na + sizeof(int) * op.na + 15) & ~(size_t)15;
                const size_t smem = head + sizeof(T) * (size_t)op.na * KB;
                if (smem > 227 * 1024) throw std::runtime_error("joseph_adj: too many angles for shared memory");
                auto kfn = k_joseph_adj<T, EPI>;
                if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                dim3 grid((n + 15) / 16, (n + 15) / 16, B);
                kfn<<<grid, 256, smem, s>>>(in, out, tab, n, op.na, op.nb, KB, st);
                klaunched("k_joseph_adj");
            }
            return;
        }
    }
    throw std::runtime_error("op_apply: unknown operator kind");
}

template <typename T>
void op_apply(const OpDev& op, bool adjoint, int epi, const T* in, T* out, const T* prev, T* tmp, int B,
              GkState* st, Red red, cudaStream_t s) {
    struct Scope {
        cudaStream_t s;
        ~Scope() { kfinish(s); }
    } scope{s};
    kbegin(epi == EPI_PLAIN ? KC_OP_PLAIN : (adjoint ? KC_ADJ : KC_FWD), s);
    switch (epi) {
        case EPI_PLAIN: apply_epi<T, EPI_PLAIN>(op, adjoint, in, out, prev, tmp, B, st, red, s); return;
        case EPI_FWD: apply_epi<T, EPI_FWD>(op, adjoint, in, out, prev, tmp, B, st, red, s); return;
        case EPI_ADJ: apply_epi<T, EPI_ADJ>(op, adjoint, in, out, prev, tmp, B, st, red, s); return;
        case EPI_ADJ_INIT: apply_epi<T, EPI_ADJ_INIT>(op, adjoint, in, out, prev, tmp, B, st, red, s); return;
    }
    throw std::runtime_error("op_apply: bad epilogue");
}

// Forward step fused with the previous iteration's solution update (2D float blur with a
// register-blocked radius); returns false when not applicable (caller runs them separately).
bool op_fwd_update(const OpDev& op, const float* v, float* u, float* f, float* w, int B, GkState* st, Red red,
                   cudaStream_t s) {
    if ((op.kind != OPK_BLUR && op.kind != OPK_BLUR_MASK) || op.d.ndim != 2 || op.R[0] != op.R[1] ||
        op.generic_blur)
        return false;
    const bool mo = op.kind == OPK_BLUR_MASK;
    struct Scope {
        cudaStream_t s;
        ~Scope() { kfinish(s); }
    } scope{s};
    kbegin(KC_FWD, s);
#define FU_CASE(R_)                                                                                      \
    case R_:                                                                                             \
        if (mo) launch_blur2d_rb<R_, EPI_FWD, false, true, true>(op, v, u, u, B, st, red, s, f, w);     \
        else launch_blur2d_rb<R_, EPI_FWD, false, false, true>(op, v, u, u, B, st, red, s, f, w);       \
        return true;
    switch (op.R[0]) {
        FU_CASE(6)
        FU_CASE(9)
        FU_CASE(12)
        FU_CASE(15)
        default: break;
    }
#undef FU_CASE
    kfinish(s);
    return false;
}

template void op_apply<float>(const OpDev&, bool, int, const float*, float*, const float*, float*, int, GkState*,
                              Red, cudaStream_t);
template void op_apply<double>(const OpDev&, bool, int, const double*, double*, const double*, double*, int,
                               GkState*, Red, cudaStream_t);

}  // namespace plsqr
