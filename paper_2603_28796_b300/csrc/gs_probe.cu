// Measurement kernels (roofline denominators; no counterpart in the paper): random row gathers
// with the access pattern of the variable-major pass, so that the pass's gather rate can be set
// against what the memory hierarchy delivers for the same row size and working set.
#include <cuda_runtime.h>

#include <cstdint>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kProbeBatch = 8;   // gathers in flight per lane group, as in the variable pass

// The load form of the variable pass's gathers: 16-byte non-coherent loads, no L2 policy.
__device__ __forceinline__ uint4 probe_ld16(const void* p) {
    uint4 r;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

// Each lane group of LPR lanes reads one row of LPR * 16 bytes per gather (16 bytes per lane);
// the G = 32 / LPR groups of a warp read different rows. Gathers are dealt to lane groups in
// order, kProbeBatch at a time, grid-stride; an index >= n_rows is skipped (no load). The loaded
// words are folded into one XOR per warp.
template <int LPR>
__global__ void __launch_bounds__(kThreads) k_gather_probe(const char* src, int64_t stride, uint32_t n_rows,
                                                           const uint32_t* idx, int64_t n, uint32_t* sink) {
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, li = lane % LPR;
    const int64_t groups_total = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32) * G;
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5)) * G + g;
    uint32_t acc = 0;
    for (int64_t base = gid * kProbeBatch; base < n; base += groups_total * kProbeBatch) {
        uint32_t r[kProbeBatch];
#pragma unroll
        for (int j = 0; j < kProbeBatch; ++j) r[j] = (base + j < n) ? __ldg(idx + base + j) : 0xffffffffu;
        uint4 v[kProbeBatch];
#pragma unroll
        for (int j = 0; j < kProbeBatch; ++j) {
            v[j] = make_uint4(0u, 0u, 0u, 0u);
            if (r[j] < n_rows) v[j] = probe_ld16(src + static_cast<int64_t>(r[j]) * stride + li * 16);
        }
#pragma unroll
        for (int j = 0; j < kProbeBatch; ++j) acc ^= v[j].x ^ v[j].y ^ v[j].z ^ v[j].w;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) atomicXor(sink, acc);
}

template <int LPR>
cudaError_t launch_probe(const char* src, int64_t stride, uint32_t n_rows, const uint32_t* idx, int64_t n,
                         uint32_t* sink, cudaStream_t s) {
    static int grid = 0;
    if (!grid) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gather_probe<LPR>, kThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        grid = per_sm * sm_count();
    }
    k_gather_probe<LPR><<<grid, kThreads, 0, s>>>(src, stride, n_rows, idx, n, sink);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather_probe(const void* src, int64_t stride, uint32_t n_rows, int32_t row_bytes, const uint32_t* idx,
                                int64_t n, uint32_t* sink, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const char* p = static_cast<const char*>(src);
    switch (row_bytes) {
        case 16: return launch_probe<1>(p, stride, n_rows, idx, n, sink, s);
        case 32: return launch_probe<2>(p, stride, n_rows, idx, n, sink, s);
        case 64: return launch_probe<4>(p, stride, n_rows, idx, n, sink, s);
        case 128: return launch_probe<8>(p, stride, n_rows, idx, n, sink, s);
        case 256: return launch_probe<16>(p, stride, n_rows, idx, n, sink, s);
        case 512: return launch_probe<32>(p, stride, n_rows, idx, n, sink, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gs
