// common.cuh -- shared device types and helpers of libplsqr (sm_103a).
//
// Every kernel covers a batch of B independent instances of one grid size: bulk arrays
// are [B][N] (T = float or double), and each instance has its own double-precision Krylov
// state (GkState).  Norms and dot products are reduced deterministically: each block
// writes one double partial, the last block of the instance (atomic ticket) sums the
// partials in a fixed order and runs the scalar recurrence on one thread.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace plsqr {

constexpr int ST_IDLE = 7;       // an empty slot of a serving handle: kernels skip the instance
constexpr int ST_CONVERGED = 8;  // the fixed point stopped (Algorithm 3 step 5): kernels skip it


// Programmatic dependent launch.  A kernel launched with the programmatic-serialization attribute
// (launch_k) may be scheduled while its predecessor in the stream is finishing; it waits here,
// before its first access to global memory, until the predecessor has completed and its writes are
// visible.  Without the attribute this is a no-op.  (No kernel signals its dependents early:
// letting them become resident at the start of the predecessor measured slower on the V-cycle
// chain than letting them start at its completion.)
// Butterfly sum over the 32 lanes of a warp (every lane receives the total).
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Barrier over all threads of the thread-block cluster; the release/acquire pair at cluster scope
// makes the memory writes of every block before it visible to every block after it.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void pdl_grid_sync() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Status codes mirrored from plsqr.h (device side).
constexpr int ST_OK = 0;
constexpr int ST_BREAKDOWN = 4;

// Regulariser ids (plsqr_reg).
constexpr int REG_TIKHONOV = 0, REG_TV = 1, REG_PM_LOG = 2, REG_PM_EXP = 3;

// Per-instance scalar state of one MLSQR solve (Algorithm 2) and of the outer loop.
// alpha/beta hold alpha_i, beta_i of the current iteration; beta_new holds beta_{i+1}
// between the forward step and the rotation.  The c_* fields are the scale factors the
// bulk kernels apply to the raw (unnormalised) vectors; they are computed once by the
// thread that finalises a reduction so that no bulk thread divides in double:
//   c_fwd_a = 1/alpha_i, c_fwd_p = alpha_i/beta_i          (step 10)
//   c_adj_a = 1/beta_{i+1}, c_adj_p = beta_{i+1}/alpha_i    (step 11)
//   c_upd_v = 1/alpha_{i+1}, cf = phi_i/rho_i, cw = theta_{i+1}/rho_i  (steps 15, 19-20)
struct GkState {
    double alpha, beta, beta_new, beta1;
    double phibar, rhobar, res2;
    double cf, cw;
    double c_fwd_a, c_fwd_p, c_adj_a, c_adj_p, c_upd_v;
    double tau, sqrt_tau, T;
    double R;            // R(f) from the last diffusivity pass
    double eta_delta;    // S4: stop the inner solve once ||rbar_i|| <= eta delta (0: never)
    double r_rel;        // outer stop: R decreased by less than this fraction (0: never)
    int32_t reg;
    int32_t status;      // ST_OK, ST_BREAKDOWN (current inner solve), ST_IDLE, ST_CONVERGED
    int32_t status_any;  // sticky over the whole solve
    int32_t iter;        // completed inner iterations of the current inner solve
    int32_t outer;       // current outer step (0-based), history row
    int32_t frozen;      // S4: 0 running, 1 met at the last iteration, 2 inner solve finished
};

// The instance takes no part in the current outer step (empty slot, or converged).
__device__ __forceinline__ bool parked(const GkState& s) { return s.status == ST_IDLE || s.status == ST_CONVERGED; }
// The instance takes no part in the remaining inner iterations.
__device__ __forceinline__ bool inner_off(const GkState& s) { return s.status != ST_OK || s.frozen >= 2; }

// Per-instance solve parameters written by the host before a solve.
struct SolveParams {
    double T, tau;
    double eta_delta, r_rel;  // stopping rules (0: off)
    int32_t reg, pad_;
};

// Histories on the device: [B][n_outer][n_inner], [B][n_outer+1], [B][n_outer].
struct Hist {
    double* rbar;
    double* R;
    double* resid;
    int32_t n_outer, n_inner;
};

// Scratch of the two-level reductions: partials[B][max_blocks], counters[B].
struct Red {
    double* partials;
    unsigned* counters;
    int32_t max_blocks;
};

// Division of 0 <= n < 2^31 by a divisor d >= 1 fixed at launch, by one multiply-high, an add and
// a shift (the method of Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1 (< 2^32),
// floor(n / d) = (mulhi(m, n) + n) >> l, and mulhi(m, n) < n keeps the sum below 2^32.  The index
// arithmetic of the 3D kernels otherwise divides 64-bit integers, which the GPU does in software.
struct FDiv {
    uint32_t d, m;
    int32_t l;
};

inline FDiv make_fdiv(int64_t d) {
    FDiv f{};
    f.d = (uint32_t)(d < 1 ? 1 : d);
    while ((1ull << f.l) < f.d) ++f.l;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << f.l) - f.d)) / f.d) + 1);
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FDiv& f) { return (__umulhi(f.m, n) + n) >> f.l; }

// Grid extents of one level (nz = 1 for 2D), with the divisors of the index arithmetic (nx, ny and
// nx / 2), set by make_dims.
struct Dims {
    int32_t nx, ny, nz, ndim;
    int64_t N;  // nx*ny*nz
    FDiv fx, fy, fh;
};

// Per-level buffers of the coarse end of a 2D V-cycle (conductances, right-hand side, pre-smoothed
// iterate, post-smoothed result), indexed by level - lc for the levels lc..L-1 (at most
// TAIL_LEVELS - 1 smoothing levels and the coarsest).
constexpr int TAIL_LEVELS = 5;
struct TailLevels {
    const void* cond[TAIL_LEVELS];
    const void* rd[TAIL_LEVELS];
    void* b[TAIL_LEVELS];
    void* x[TAIL_LEVELS];
    void* x2[TAIL_LEVELS];
    Dims d[TAIL_LEVELS];
    int n;  // levels in use (the last one is the coarsest)
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One row of the coarsest level's exact solve, (X b)_row = sum_c X[row][c] b[c], by one warp: lane l
// takes the 16-byte groups l, l + 32, ... of the row (four floats or two doubles each; all of a
// row's loads are independent, so they are in flight together), multiplies them with the same
// group of b (16-byte aligned in shared memory) in column order within the group, and the warp
// sums the lanes (butterfly).  The rows of X are 16-byte aligned when nc is a multiple of 4;
// otherwise a plain strided loop.  Every schedule calls this function, so they agree bit for bit.
template <typename T>
__device__ __forceinline__ T coarse_row_dot(const T* __restrict__ Xr, const T* sb, int nc, int lane) {
    constexpr int V = 16 / (int)sizeof(T);
    T acc = (T)0;
    if (nc % 4 == 0) {
        using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        const V4* X4 = reinterpret_cast<const V4*>(Xr);
        const V4* B4 = reinterpret_cast<const V4*>(sb);
        const int ng = nc / V;
#pragma unroll 8
        for (int g = lane; g < ng; g += 32) {
            const V4 q = __ldg(X4 + g);
            const V4 bq = B4[g];
            if constexpr (sizeof(T) == 4) {
                acc = fma(q.x, bq.x, acc);
                acc = fma(q.y, bq.y, acc);
                acc = fma(q.z, bq.z, acc);
                acc = fma(q.w, bq.w, acc);
            } else {
                acc = fma(q.x, bq.x, acc);
                acc = fma(q.y, bq.y, acc);
            }
        }
    } else {
        for (int c = lane; c < nc; c += 32) acc = fma(Xr[c], sb[c], acc);
    }
    return warp_sum_t<T>(acc);
}

// Sum over the block; the result is valid in thread 0.  Fixed reduction tree.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh /* >= NT/32 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < NT / 32) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Two-level deterministic reduction.  Every block of instance `inst` calls this with its
// thread's contribution; returns true in thread 0 of the last block of the instance, with
// the instance total in *total.  nblk = blocks of this instance in this launch (<= rd.max_blocks).
// Threads must use a 1D thread index 0..NT-1 (threadIdx.x).
template <int NT>
__device__ __forceinline__ bool reduce_last(double v, const Red& rd, int inst, int blk, int nblk,
                                            double* total) {
    __shared__ double sh[NT / 32];
    __shared__ bool is_last;
    double bs = block_sum<NT>(v, sh);
    if (threadIdx.x == 0) {
        rd.partials[(int64_t)inst * rd.max_blocks + blk] = bs;
        __threadfence();
        unsigned prev = atomicAdd(&rd.counters[inst], 1u);
        is_last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += NT) s += __ldcg(&rd.partials[(int64_t)inst * rd.max_blocks + i]);
    double tot = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) {
        rd.counters[inst] = 0u;
        *total = tot;
        return true;
    }
    return false;
}

// Every block of instance `inst` calls this after its threads wrote (and fenced) their partial sums
// at fixed positions of rd.partials[inst][0 .. nparts); returns true in thread 0 of the last of the
// nblk blocks, with the sum of the nparts partials in *total: each thread sums the positions
// t, t + NT, ... in order, then a fixed tree.  The positions, not the blocks, fix the order, so the
// result does not depend on how the work was split into blocks.
template <int NT>
__device__ __forceinline__ bool sum_partials_last(const Red& rd, int inst, int nblk, int nparts, double* total) {
    __shared__ double sh[NT / 32];
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&rd.counters[inst], 1u);
        is_last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    const double* p = rd.partials + (int64_t)inst * rd.max_blocks;
    double s = 0.0;
#pragma unroll 8
    for (int i = threadIdx.x; i < nparts; i += NT) s += __ldcg(p + i);
    const double tot = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) {
        rd.counters[inst] = 0u;
        *total = tot;
        return true;
    }
    return false;
}

__device__ __forceinline__ bool good_pos(double x, double ref) {
    return isfinite(x) && x > 1e-30 * ref;
}

// 1 / sqrt(x) in double for x > 0, by the Newton-Raphson iteration for the inverse square root,
// y <- y (3/2 - (x/2) y^2), from the single-precision estimate rsqrtf (relative error ~1e-7; the
// iteration converges quadratically, so two steps reach double rounding).  GB300's double pipe is
// narrow and its square root and division run long dependent chains; this takes seven dependent
// double operations.  Outside the single-precision normal range it defers to rsqrt; a
// non-positive or non-finite x gives NaN, which callers turn into a breakdown.
__device__ __forceinline__ double rsqrt_nr(double x) {
    if (!(x > 0.0) || !isfinite(x)) return nan("");
    if (!(x > 1.2e-38 && x < 3.0e38)) return rsqrt(x);
    double y = (double)rsqrtf((float)x);
    const double h = 0.5 * x;
    y = y * fma(-h, y * y, 1.5);
    y = y * fma(-h, y * y, 1.5);
    return y;
}

// alpha_{i+1} = sqrt(v~ . p~) (Algorithm 2 steps 5 / 13) from the reduced dot product, then
// (INIT = false) the orthogonal transformation: the Paige-Saunders damping rotation that
// eliminates sqrt(tau) I (eq. 3.6) and Algorithm 1 steps 10-16, the coefficients of the
// pending update (steps 19-20) and ||rbar_i||.  Runs on one thread, on a copy of the state in
// registers; each rotation takes one inverse square root (c = a / r, s = b / r, r = (a^2 + b^2) / r
// with 1 / r = rsqrt_nr(a^2 + b^2)) instead of a square root and divisions.
template <bool INIT>
__device__ __forceinline__ void finalize_alpha(GkState& sg, double tot, const Hist& hist, int inst) {
    GkState s = sg;
    const double ian = tot > 0.0 ? rsqrt_nr(tot) : 0.0;  // 1 / alpha
    const double an = tot * ian;
    if (!good_pos(an, s.beta1)) {
        sg.status = ST_BREAKDOWN;
        sg.status_any = ST_BREAKDOWN;
        return;
    }
    if (INIT) {  // step 7: rhobar_1 = alpha_1, w~_1 = v~_1
        s.alpha = an;
        s.rhobar = an;
        s.c_upd_v = ian;
        s.c_fwd_a = ian;
        s.c_fwd_p = an / s.beta;
        sg = s;
        return;
    }
    double rhohat = s.rhobar, psi = 0.0;
    if (s.tau > 0.0) {
        const double q = s.rhobar * s.rhobar + s.tau;
        const double ir = rsqrt_nr(q);
        rhohat = q * ir;
        const double c1 = s.rhobar * ir, s1 = s.sqrt_tau * ir;
        psi = s1 * s.phibar;
        s.phibar = c1 * s.phibar;
    }
    const double beta = s.beta_new;
    const double q2 = rhohat * rhohat + beta * beta;
    const double irho = rsqrt_nr(q2);  // 1 / rho
    const double c = rhohat * irho, sn = beta * irho;
    const double theta = sn * an;
    s.rhobar = -c * an;
    const double phi = c * s.phibar;
    s.phibar = sn * s.phibar;
    s.res2 += psi * psi;
    s.cf = phi * irho;
    s.cw = theta * irho;
    if (s.frozen) {
        // S4 held after the previous iteration: its update was the last one; this iteration's
        // is void and the remaining iterations of the inner solve are skipped
        s.cf = 0.0;
        s.frozen = 2;
    } else {
        s.iter += 1;
        const double rq = s.phibar * s.phibar + s.res2;
        const double rb = rq > 0.0 ? rq * rsqrt_nr(rq) : 0.0;
        if (hist.rbar && s.outer < hist.n_outer && s.iter <= hist.n_inner)
            hist.rbar[((int64_t)inst * hist.n_outer + s.outer) * hist.n_inner + (s.iter - 1)] = rb;
        if (s.eta_delta > 0.0 && rb <= s.eta_delta) s.frozen = 1;  // S4 (Sec. 3.4)
    }
    s.alpha = an;
    s.beta = beta;
    s.c_upd_v = ian;
    s.c_fwd_a = ian;
    s.c_fwd_p = an * s.c_adj_a;  // alpha_{i+1} / beta_{i+1}; c_adj_a = 1 / beta_{i+1} (finalize_beta)
    sg = s;
}

}  // namespace plsqr
