// sm_103a kernels of the candidate pool and the branching-variable choice that follow training
// (Sec. "Partial Assignment Extraction for SAT Instances", the pool of Eq. 9, and Sec. "Guided
// Branching for UNSAT Instances").
//
// Pool: from one trained candidate's logits delta (the selected batch theta_sel), N samples
// x_hat^(k) = [delta + l^(k) > 0] with independent logistic noise (the two-logit form of adding
// Gumbel noise to each logit and taking the argmax, Eq. 3-4), and for each sample the S variables
// of highest confidence c^(k) = max_j y_j = sigma(|delta + l^(k)| / tau). sigma is increasing, so
// the order of c is the order of |delta + l|; it is used directly (float32 sigma saturates at 1 for
// |z| > 17 and would turn the top of the order into a tie). Ties go to the lower variable row.
// Branching: the d variables of lowest confidence sigma(|delta| / tau), i.e. smallest |delta|,
// ties to the lower row.
//
// Selection is exact: every (sample, row) gets a unique 64-bit key (32-bit |z| order, then the
// inverted row), and a 4-pass radix select with 16-bit digits finds each sample's S-th largest key
// T; the S rows with key >= T are appended (integer atomics), then sorted by row in one block per
// sample. Noise: the Philox4x32-10 stream of the straight-through step with step 0, candidate
// index k: counter (k / 4, row, 0, 0), key (seed mod 2^32, seed / 2^32), word k % 4.
#include <cuda.h>

#include <cstdint>

#include "gs_device.cuh"
#include "gs_internal.h"
#include "gs_noise.cuh"

namespace gs {
namespace {

constexpr int kDigits = 65536;

// Key of sample k at row v: larger = more confident (pool) or less confident (branch).
__device__ __forceinline__ uint64_t pool_key(float z, int64_t v, bool branch) {
    const uint32_t a = __float_as_uint(fabsf(z));   // non-negative float: bit order == value order
    const uint32_t hi = branch ? ~a : a;
    return (static_cast<uint64_t>(hi) << 32) | static_cast<uint32_t>(~static_cast<uint32_t>(v));
}

// The 32 samples 32 w .. 32 w + 31 (< N) of row v: z = delta + l (or delta alone when branching).
__device__ __forceinline__ void row_values(const PoolParams& P, int64_t v, int w, float (&z)[32]) {
    const float d = P.delta[v * P.stride];
    if (P.branch) {
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = d;
        return;
    }
    if (P.noise) {
        const float* row = P.noise + v * P.ldN;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int k = 32 * w + j;
            z[j] = d + ((k < P.N) ? row[k] : 0.0f);
        }
        return;
    }
    const uint32_t k0 = static_cast<uint32_t>(P.seed), k1 = static_cast<uint32_t>(P.seed >> 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint32_t x[4] = {static_cast<uint32_t>(8 * w + q), static_cast<uint32_t>(v), 0u, 0u};
        philox4x32_10(x, k0, k1);
#pragma unroll
        for (int j = 0; j < 4; ++j) z[4 * q + j] = d + logistic_from_word(x[j]);
    }
}

// One radix pass: histogram of the 16-bit digit at `shift` of the keys that match the prefix
// chosen so far; the first pass also writes the samples' bits.
__global__ void __launch_bounds__(256) k_pool_hist(const PoolParams P, int shift) {
    const int nw = P.nw32;
    const int64_t total = static_cast<int64_t>(P.n_rows) * nw;
    const uint64_t himask = (shift >= 48) ? 0ull : (~0ull << (shift + 16));
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = i / nw;
        const int w = static_cast<int>(i - v * nw);
        if (32 * w >= P.N) {
            if (P.bits32 && shift == 48) P.bits32[v * nw + w] = 0u;
            continue;
        }
        float z[32];
        row_values(P, v, w, z);
        uint32_t bits = 0u;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int k = 32 * w + j;
            if (k < P.N) {
                if (z[j] > 0.0f) bits |= 1u << j;
                const uint64_t key = pool_key(z[j], v, P.branch);
                if ((key & himask) == (P.prefix[k] & himask))
                    atomicAdd(&P.hist[static_cast<int64_t>(k) * kDigits + ((key >> shift) & 0xffffu)], 1u);
            }
        }
        if (P.bits32 && shift == 48) P.bits32[v * nw + w] = bits;
    }
}

// Per sample (one block of 1024 threads): the digit at which the count of keys above, taken from
// the largest digit down, reaches the remaining rank; extends the prefix and the remaining rank.
__global__ void __launch_bounds__(1024) k_pool_digit(const PoolParams P, int shift) {
    __shared__ uint32_t warp_sum[32];
    const int k = blockIdx.x;
    const uint32_t* h = P.hist + static_cast<int64_t>(k) * kDigits;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int top = kDigits - 1 - 64 * t;   // this thread's bins: top, top - 1, ..., top - 63
    uint32_t s = 0;
    for (int b = 0; b < 64; ++b) s += h[top - b];
    // exclusive scan over threads (thread 0 holds the largest digits)
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t ws = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        warp_sum[lane] = ws;
    }
    __syncthreads();
    const uint32_t before = x - s + (wid > 0 ? warp_sum[wid - 1] : 0u);
    const uint32_t rem = static_cast<uint32_t>(P.rem[k]);
    if (before < rem && before + s >= rem) {
        uint32_t cum = before;
        for (int b = 0; b < 64; ++b) {
            const uint32_t c = h[top - b];
            if (cum + c >= rem) {
                P.prefix[k] |= static_cast<uint64_t>(top - b) << shift;
                P.rem[k] = static_cast<int32_t>(rem - cum);
                break;
            }
            cum += c;
        }
    }
}

// Appends the rows whose key reaches the sample's threshold (exactly S per sample).
__global__ void __launch_bounds__(256) k_pool_collect(const PoolParams P) {
    const int nw = P.nw32;
    const int64_t total = static_cast<int64_t>(P.n_rows) * nw;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = i / nw;
        const int w = static_cast<int>(i - v * nw);
        if (32 * w >= P.N) continue;
        float z[32];
        row_values(P, v, w, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int k = 32 * w + j;
            if (k < P.N && pool_key(z[j], v, P.branch) >= P.prefix[k]) {
                const int pos = atomicAdd(&P.count[k], 1);
                if (pos < P.S)
                    P.sel[static_cast<int64_t>(k) * P.S + pos] = static_cast<int32_t>(v);
                else
                    atomicOr(P.status, kStatusSelect);
            }
        }
    }
}

// Sorts each sample's S rows ascending (bitonic sort in shared memory, S <= kPoolMaxS).
__global__ void __launch_bounds__(1024) k_pool_sort(const PoolParams P, int S2) {
    extern __shared__ int32_t buf[];
    const int k = blockIdx.x;
    int32_t* row = P.sel + static_cast<int64_t>(k) * P.S;
    for (int i = threadIdx.x; i < S2; i += blockDim.x) buf[i] = (i < P.S) ? row[i] : 0x7fffffff;
    __syncthreads();
    for (int size = 2; size <= S2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < S2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const int32_t a = buf[i], b = buf[j];
                    if ((a > b) == up) {
                        buf[i] = b;
                        buf[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < P.S; i += blockDim.x) row[i] = buf[i];
}

__global__ void k_pool_init(const PoolParams P) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.N; k += gridDim.x * blockDim.x) {
        P.prefix[k] = 0ull;
        P.rem[k] = P.S;
        P.count[k] = 0;
    }
}

int pool_blocks(int64_t total) {
    const int64_t blocks = (total + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    return static_cast<int>(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

cudaError_t launch_pool_select(const PoolParams& p, cudaStream_t s) {
    const int64_t total = static_cast<int64_t>(p.n_rows) * p.nw32;
    if (total <= 0 || p.N <= 0 || p.S <= 0) return cudaSuccess;
    cudaError_t e;
    k_pool_init<<<(p.N + 255) / 256, 256, 0, s>>>(p);
    for (int shift = 48; shift >= 0; shift -= 16) {
        e = cudaMemsetAsync(p.hist, 0, sizeof(uint32_t) * kDigits * static_cast<size_t>(p.N), s);
        if (e != cudaSuccess) return e;
        k_pool_hist<<<pool_blocks(total), 256, 0, s>>>(p, shift);
        k_pool_digit<<<p.N, 1024, 0, s>>>(p, shift);
    }
    k_pool_collect<<<pool_blocks(total), 256, 0, s>>>(p);
    int S2 = 1;
    while (S2 < p.S) S2 <<= 1;
    k_pool_sort<<<p.N, 1024, S2 * sizeof(int32_t), s>>>(p, S2);
    return cudaGetLastError();
}

}  // namespace gs
