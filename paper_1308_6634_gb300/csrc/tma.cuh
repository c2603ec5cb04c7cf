// tma.cuh -- tensor-memory-accelerator (TMA) tile loads for the stencil kernels.
//
// A block stages its halo tile with one cp.async.bulk.tensor copy issued by one thread and
// completed on an mbarrier (transaction bytes).  Elements of the box outside the tensor are
// filled with zeros by the hardware, which is exactly the zero boundary of the blur and of the
// diffusion stencil.  Every wait is bounded: after TMA_WAIT_LIMIT polls the block records a
// timeout in its instance state and waits once more (again bounded) for its own copy before
// going on with whatever is in shared memory.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace plsqr {

constexpr int ST_TIMEOUT = 5;
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 22;

// Host: a 3D tiled tensor map over a [planes][ny][nx] array of `esz`-byte floats with a box of
// (bx, by, bz).  Returns false when the layout does not satisfy the TMA rules (16-byte aligned
// base, row pitch a multiple of 16 bytes, box row a multiple of 16 bytes, boxes <= 256).
bool tma_map_3d(CUtensorMap* map, const void* base, int esz, int64_t nx, int64_t ny, int64_t planes, int bx, int by,
                int bz);
// TMA staging is used unless PLSQR_TMA=0 (plain loads, for comparisons).
bool tma_enabled();

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Untiled bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16), completed
// on an mbarrier like the tiled loads.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's generic-proxy memory accesses before later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = TMA_WAIT_LIMIT) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// All threads: wait for the tile; on timeout flag the instance and wait once more.
__device__ __forceinline__ void tma_wait_tile(uint64_t* bar, GkState* st, int inst, uint32_t limit = TMA_WAIT_LIMIT) {
    if (!mbar_wait_bounded(bar, 0, limit)) {
        if (threadIdx.x == 0 && st) {
            st[inst].status = ST_TIMEOUT;
            st[inst].status_any = ST_TIMEOUT;
        }
        mbar_wait_bounded(bar, 0, limit);
    }
}

}  // namespace plsqr
