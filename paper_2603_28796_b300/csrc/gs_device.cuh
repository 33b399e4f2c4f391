// Device helpers shared by the kernel translation units (gs_kernels.cu, gs_st.cu): mbarrier
// and 1-D bulk-copy PTX wrappers with bounded waits, the integer work queue, the debug-build row
// check, and the persistent-grid sizing of the tiled kernels. Internal linkage in each unit.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;   // bounded mbarrier wait: 2 s, then error status

// ------------------------------------------------------------------------------------------
// PTX helpers: mbarrier + 1-D bulk copy global -> shared.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for a phase of the mbarrier with a time limit (and an iteration limit, in case the
// timer does not advance). Returns false on timeout. The first probe is inline; the bounded
// polling loop is out of line.
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait_slow(bar, parity, limit_ns);
}

// Debug build (GS_DEBUG): a gathered row index must be below n_rows; otherwise the sticky status
// bit kStatusBounds is set and the caller skips the load. Release builds compile the check away.
__device__ __forceinline__ bool row_ok(uint64_t u, int64_t n_rows, int32_t* status) {
#ifdef GS_DEBUG
    if (u >= static_cast<uint64_t>(n_rows)) {
        atomicOr(status, kStatusBounds);
        return false;
    }
#else
    (void)u;
    (void)n_rows;
    (void)status;
#endif
    return true;
}

struct Span {
    uintptr_t src;
    uint32_t bytes;   // 16-byte multiple
};
// The 16-byte aligned superset [lo, hi) of [p, p + bytes); the device arrays carry 64 bytes of
// padding so that hi never leaves the allocation.
__device__ __forceinline__ Span span16(const void* p, uint32_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t lo = a & ~uintptr_t(15);
    const uintptr_t hi = (a + bytes + 15) & ~uintptr_t(15);
    Span s;
    s.src = lo;
    s.bytes = bytes ? static_cast<uint32_t>(hi - lo) : 0u;
    return s;
}

// Called once by every thread of every CTA of a work-queue kernel, after its loop: the last CTA
// to leave rewinds the queue (head and exit count back to 0), so the next launch needs no reset.
__device__ __forceinline__ void queue_exit(int32_t* head, int32_t* exit_cnt) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(exit_cnt, 1) == static_cast<int>(gridDim.x) - 1) {
            atomicExch(head, 0);
            atomicExch(exit_cnt, 0);
        }
    }
}

__device__ __forceinline__ int fetch_work(int32_t* head, int lane) {
    int w = 0;
    if (lane == 0) w = atomicAdd(head, 1);
    return __shfl_sync(0xffffffffu, w, 0);
}

// ------------------------------------------------------------------------------------------
// Host side: persistent grids (SMs x resident CTAs at the kernel's shared-memory footprint,
// static and dynamic). The occupancy is found with the whole unified L1/shared array offered as
// shared memory; the kernel's carve-out is then set to the smallest one that still holds those
// CTAs, so the rest of the array stays L1 cache for the gathers (a carve-out is a preference: if
// the smaller one would cost resident CTAs, the maximum is kept). A grid larger than the resident
// CTAs would leave the surplus waiting for a free slot, so both sides of this must agree.
int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

template <typename K>
int persistent_grid(K kernel, int smem_bytes, int threads = kThreads) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem_bytes) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int dev = 0, sm_smem = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa{};
    const int static_smem = cudaFuncGetAttributes(&fa, kernel) == cudaSuccess ? static_cast<int>(fa.sharedSizeBytes) : 0;
    if (sm_smem > 0) {
        const int64_t need = static_cast<int64_t>(per_sm) * (smem_bytes + static_smem + reserved);
        int pct = static_cast<int>((need * 100 + sm_smem - 1) / sm_smem);
        pct = pct < 0 ? 0 : (pct > 100 ? 100 : pct);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        int per_sm_l1 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_l1, kernel, threads, smem_bytes) != cudaSuccess ||
            per_sm_l1 < per_sm)
            cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    }
    return per_sm * sm_count();
}

}  // namespace
}  // namespace gs
