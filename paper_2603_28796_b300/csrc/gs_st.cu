// sm_103a kernels of the straight-through Gumbel training step (Eq. 3 with noise, Eq. 4 in the
// forward pass).
//
// With two logits per variable the Gumbel-softmax of Eq. 3 puts y = sigma((delta + l) / tau) on
// state 1, delta = theta_1 - theta_0 and l = g_1 - g_0 ~ Logistic(0, 1). The forward pass uses
// the hard assignment x_hat = [delta + l > 0] (Eq. 4, ties to state 0); the backward pass takes
// the gradient of the loss at x_hat through the soft y: dL/d delta = dL/dx(x_hat) y (1 - y) / tau.
//
// At a Boolean point every leave-one-out product is 0 or 1, so dL/dx of variable v is an
// integer: (negated occurrences whose other literals are all false) - (positive ones). The pass
// therefore gathers 1 bit per (literal, candidate) instead of a float: a lane owns one 32-bit
// word of the bit-packed assignment (32 candidates), ORs the truth words of an occurrence's
// other literals, and adds the complement (all others false) into a signed bit-sliced counter,
// 10 bit planes of 32 candidates. The epilogue turns the planes into per-candidate integers,
// applies the soft chain and Adam, and writes the next step's hard assignment from the next
// step's noise. The loss at the hard point is the unsatisfied-clause count (gs_check_bits).
//
// Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key (seed mod 2^32, seed / 2^32),
// counter (b / 4, row, step mod 2^32, step / 2^32); candidate b takes output word b % 4;
// k = word >> 9, u = (k + 1/2) 2^-23 (exact in float32), l = log(u / (1 - u)).
#include <cuda.h>

#include <cstdint>

#include "gs_device.cuh"
#include "gs_internal.h"
#include "gs_noise.cuh"

namespace gs {
namespace {

// Logistic noise of candidates c0 .. c0 + 7 (c0 a multiple of 8) of batch row `row` at `step`.
__device__ __forceinline__ void logistic8(uint64_t seed, int64_t step, int64_t row, int c0, float (&l)[8]) {
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const uint32_t s0 = static_cast<uint32_t>(step), s1 = static_cast<uint32_t>(static_cast<uint64_t>(step) >> 32);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t x[4] = {static_cast<uint32_t>((c0 >> 2) + h), static_cast<uint32_t>(row), s0, s1};
        philox4x32_10(x, k0, k1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            l[4 * h + j] = logistic_from_word(x[j]);
        }
    }
}

// Eight consecutive floats from a row (16-byte aligned when c0 + 8 <= B), zero past B.
__device__ __forceinline__ void load8(const float* p, int c0, int B, float (&a)[8]) {
    if (c0 + 8 <= B) {
        const float4 x = __ldcs(reinterpret_cast<const float4*>(p));
        const float4 y = __ldcs(reinterpret_cast<const float4*>(p + 4));
        a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
        a[4] = y.x; a[5] = y.y; a[6] = y.z; a[7] = y.w;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = (c0 + j < B) ? p[j] : 0.0f;
    }
}
__device__ __forceinline__ void store8(float* p, int c0, int B, const float (&a)[8]) {
    if (c0 + 8 <= B) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(a[0], a[1], a[2], a[3]));
        __stcs(reinterpret_cast<float4*>(p + 4), make_float4(a[4], a[5], a[6], a[7]));
    } else {
        for (int j = 0; j < 8 && c0 + j < B; ++j) p[j] = a[j];
    }
}

__device__ __forceinline__ void noise8(const float* arr, uint64_t seed, int64_t step, int64_t row, int64_t ldB,
                                       int c0, int B, float (&l)[8]) {
    if (arr)
        load8(arr + row * ldB + c0, c0, B, l);
    else
        logistic8(seed, step, row, c0, l);
}

// Adam on delta with the straight-through chain: y = sigma(z), z = (delta + l) / tau,
// g = gx * y (1 - y) / tau, y (1 - y) = e / (1 + e)^2 with e = exp(-|z|) (no overflow).
__device__ __forceinline__ void st_adam1(float gx, float l, float& d, float& m, float& v, const AdamK& k) {
    const float z = (d + l) * k.inv_tau;
    const float e = expf(-fabsf(z));
    const float r = __frcp_rn(1.0f + e);
    const float q = e * r;
    const float g = gx * (r * q) * k.inv_tau;
    m = fmaf(k.beta1, m, k.one_minus_beta1 * g);
    v = fmaf(k.beta2, v, k.one_minus_beta2 * (g * g));
    const float den = sqrtf(v) * k.inv_sqrt_bc2 + k.eps;
    d = d - k.step_size * __fdividef(m, den);   // den >= eps > 0
}

// ------------------------------------------------------------------------------------------
// Signed bit-sliced counters: plane k holds bit k (two's complement) of 32 candidates' counts.
// P += x where s == 0, P -= x where s == ~0, for the candidates whose bit of x is set.
__device__ __forceinline__ void planes_step(uint32_t (&P)[kStPlanes], uint32_t x, uint32_t s) {
#pragma unroll
    for (int k = 0; k < kStPlanes; ++k) {
        const uint32_t c = (P[k] ^ s) & x;
        P[k] ^= x;
        x = c;
    }
}
// A += B (ripple-carry, modulo 2^kStPlanes).
__device__ __forceinline__ void planes_add(uint32_t (&A)[kStPlanes], const uint32_t (&Bp)[kStPlanes]) {
    uint32_t c = 0u;
#pragma unroll
    for (int k = 0; k < kStPlanes; ++k) {
        const uint32_t a = A[k], b = Bp[k], t = a ^ b;
        A[k] = t ^ c;
        c = (a & b) | (c & t);
    }
}
// Counts of the 8 candidates at bits j0 .. j0 + 7 as floats.
__device__ __forceinline__ void planes_get8(const uint32_t (&P)[kStPlanes], int j0, float (&gx)[8]) {
    int32_t val[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) val[j] = 0;
#pragma unroll
    for (int k = 0; k < kStPlanes; ++k) {
        const uint32_t byte = (P[k] >> j0) & 0xffu;
#pragma unroll
        for (int j = 0; j < 8; ++j) val[j] |= static_cast<int32_t>((byte >> j) & 1u) << k;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) gx[j] = static_cast<float>((val[j] << (32 - kStPlanes)) >> (32 - kStPlanes));
}

// Occurrence codes [cs, ce) of one lane group: for every occurrence, OR the truth words of its
// other literals; at its last code add (own literal negated) or subtract (positive) the
// candidates for which all of them are false. A unit clause's sentinel code has no literal.
template <int NB>
__device__ __forceinline__ void st_occ(const uint32_t* cd, int cs, int ce, const uint32_t* col, int nw32, bool wok,
                                       int64_t n_rows, int32_t* status, uint32_t (&Pl)[kStPlanes]) {
    uint32_t acc = 0u;
    for (int s = cs; s < ce; s += NB) {
        uint32_t cw[NB], wd[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) cw[j] = (s + j < ce) ? cd[s + j] : (kVSentinel << kVShift);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const uint32_t u = cw[j] >> kVShift;
            wd[j] = (wok && u != kVSentinel && row_ok(u, n_rows, status)) ? __ldg(col + static_cast<int64_t>(u) * nw32)
                                                                             : 0u;
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const uint32_t c = cw[j];
            acc |= wd[j] ^ (0u - (c & kVNeg));                  // literal true under x_hat
            const uint32_t end = 0u - ((c >> 1) & 1u);          // all ones at the occurrence's last code
            const uint32_t add = 0u - ((c >> 2) & 1u);          // own literal negated: +1
            planes_step(Pl, ~acc & end, ~add);
            acc &= ~end;
        }
    }
}

// Per variable: integer gradients, the soft chain and Adam, and the next hard assignment. The
// chunk's 32 * LW candidates are processed in runs of 256: lane L takes the 8 consecutive
// candidates 256 r + 8 L (coalesced 32-byte pieces of the state rows), whose counts sit in bits
// 8 (L % 4) .. + 7 of word 8 r + L / 4, i.e. in the planes of lane 8 r + L / 4 (every lane group
// holds the same reduced planes). get(src_lane, j0, base, gx) returns the 8 counts. The four
// lanes sharing a word merge their bytes and one of them stores the word.
template <int LW, typename F>
__device__ __forceinline__ void st_epilogue(const StParams& P, int v, int chunk, int lane, F&& get) {
    constexpr int CC = 32 * LW;                       // candidates per chunk
    constexpr int RUNS = (CC + 255) / 256;
    const int64_t off = static_cast<int64_t>(v) * P.ldB;
#pragma unroll 1
    for (int r = 0; r < RUNS; ++r) {
        const int base = 256 * r + 8 * lane;          // candidate offset within the chunk
        const int word_in_chunk = 8 * r + (lane >> 2);
        const int j0 = 8 * (lane & 3);
        const int c0 = chunk * CC + base;
        const bool act = base < CC && c0 < P.B;
        float gx[8];
        get(word_in_chunk < LW ? word_in_chunk : 0, j0, base, gx);
        uint32_t b8 = 0u;
        if (act) {
            float lt[8], ln[8], d[8], mm[8], vv[8];
            noise8(P.noise, P.seed, P.step, v, P.ldB, c0, P.B, lt);
            noise8(P.noise_next, P.seed, P.step + 1, v, P.ldB, c0, P.B, ln);
            if (P.noise_out) store8(P.noise_out + off + c0, c0, P.B, ln);
            load8(P.delta + off + c0, c0, P.B, d);
            load8(P.m + off + c0, c0, P.B, mm);
            load8(P.v + off + c0, c0, P.B, vv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                st_adam1(gx[j], lt[j], d[j], mm[j], vv[j], P.adam);
                if (c0 + j < P.B && d[j] + ln[j] > 0.0f) b8 |= 1u << j;
            }
            store8(P.delta + off + c0, c0, P.B, d);
            store8(P.m + off + c0, c0, P.B, mm);
            store8(P.v + off + c0, c0, P.B, vv);
        }
        uint32_t word = b8 << j0;
        word |= __shfl_xor_sync(0xffffffffu, word, 1);
        word |= __shfl_xor_sync(0xffffffffu, word, 2);
        const int gw = chunk * LW + word_in_chunk;
        if ((lane & 3) == 0 && word_in_chunk < LW && gw < P.nw32)
            P.bits_out[static_cast<int64_t>(v) * P.nw32 + gw] = word;
    }
}

// Counts of 8 candidates from the planes of another lane (all lanes take part in the shuffles).
__device__ __forceinline__ void planes_get8_from(const uint32_t (&Pl)[kStPlanes], int src, int j0, float (&gx)[8]) {
    uint32_t Q[kStPlanes];
#pragma unroll
    for (int k = 0; k < kStPlanes; ++k) Q[k] = __shfl_sync(0xffffffffu, Pl[k], src);
    planes_get8(Q, j0, gx);
}

template <int LW>
__device__ __forceinline__ void issue_st_item(const StParams& P, int item, unsigned char* buf, uint64_t* bar) {
    constexpr int G = 32 / LW;
    const VarItem it = P.items[item];
    const Span a = span16(P.vtab + it.vtab_base, static_cast<uint32_t>(it.nv + 1) * 4u);
    const Span b = (G > 1) ? span16(P.recs + it.rec_base, static_cast<uint32_t>(it.n_occ + 1) * 2u) : Span{0, 0};
    const Span c = span16(P.codes + it.code_base, static_cast<uint32_t>(it.n_codes) * 4u);
    mbar_expect_tx(bar, a.bytes + b.bytes + c.bytes);
    if (a.bytes) bulk_g2s(buf, reinterpret_cast<const void*>(a.src), a.bytes, bar);
    if (b.bytes) bulk_g2s(buf + kVarVtabBytes, reinterpret_cast<const void*>(b.src), b.bytes, bar);
    if (c.bytes) bulk_g2s(buf + kVarVtabBytes + kVarRecBytes, reinterpret_cast<const void*>(c.src), c.bytes, bar);
}

template <int LW>
__device__ __forceinline__ void reduce_groups(uint32_t (&Pl)[kStPlanes]) {
#pragma unroll
    for (int o = LW; o < 32; o <<= 1) {
        uint32_t Q[kStPlanes];
#pragma unroll
        for (int k = 0; k < kStPlanes; ++k) Q[k] = __shfl_xor_sync(0xffffffffu, Pl[k], o);
        planes_add(Pl, Q);
    }
}

template <int LW>
__device__ __forceinline__ void process_st_item(const StParams& P, int w, const unsigned char* buf, int g, int li,
                                                int lane) {
    constexpr int G = 32 / LW;
    constexpr int NB = 8;
    const int item = w % P.n_items;
    const int chunk = w / P.n_items;
    const VarItem it = P.items[item];
    const uint32_t* vt =
        reinterpret_cast<const uint32_t*>(buf + (reinterpret_cast<uintptr_t>(P.vtab + it.vtab_base) & 15));
    const uint16_t* rc = reinterpret_cast<const uint16_t*>(
        buf + kVarVtabBytes + (reinterpret_cast<uintptr_t>(P.recs + it.rec_base) & 15));
    const uint32_t* cd = reinterpret_cast<const uint32_t*>(
        buf + kVarVtabBytes + kVarRecBytes + (reinterpret_cast<uintptr_t>(P.codes + it.code_base) & 15));
    const int word = chunk * LW + li;
    const bool wok = word < P.nw32 && word * 32 < P.B;
    const uint32_t* col = P.bits_in + word;

    if (it.split < 0) {
        for (int vi = 0; vi < it.nv; ++vi) {
            const int v = it.v0 + vi;
            const uint32_t e0 = vt[vi], e1 = vt[vi + 1];
            int cs, ce;
            if constexpr (G == 1) {
                cs = static_cast<int>(e0 & 0xffffu);
                ce = static_cast<int>(e1 & 0xffffu);
            } else {
                const int oa = static_cast<int>(e0 >> 16);
                const int O = static_cast<int>(e1 >> 16) - oa;
                cs = rc[oa + (O * g) / G];
                ce = rc[oa + (O * (g + 1)) / G];
            }
            uint32_t Pl[kStPlanes];
#pragma unroll
            for (int k = 0; k < kStPlanes; ++k) Pl[k] = 0u;
            st_occ<NB>(cd, cs, ce, col, P.nw32, wok, P.n_rows, P.status, Pl);
            reduce_groups<LW>(Pl);
            st_epilogue<LW>(P, v, chunk, lane,
                            [&](int src, int j0, int, float (&gx)[8]) { planes_get8_from(Pl, src, j0, gx); });
        }
    } else {
        const int v = it.v0;
        int cs, ce;
        if constexpr (G == 1) {
            cs = 0;
            ce = it.n_codes;
        } else {
            const int O = it.n_occ;
            cs = rc[(O * g) / G];
            ce = rc[(O * (g + 1)) / G];
        }
        uint32_t Pl[kStPlanes];
#pragma unroll
        for (int k = 0; k < kStPlanes; ++k) Pl[k] = 0u;
        st_occ<NB>(cd, cs, ce, col, P.nw32, wok, P.n_rows, P.status, Pl);
        reduce_groups<LW>(Pl);
        // this part's integer counts of the lane's 32 candidates
        float* rowp = P.split_part + static_cast<int64_t>(it.split_row + it.part) * P.bpad + word * 32;
        if (g == 0 && word * 32 < P.bpad) {
#pragma unroll
            for (int j0 = 0; j0 < 32; j0 += 8) {
                float gx[8];
                planes_get8(Pl, j0, gx);
                __stcg(reinterpret_cast<float4*>(rowp + j0), make_float4(gx[0], gx[1], gx[2], gx[3]));
                __stcg(reinterpret_cast<float4*>(rowp + j0 + 4), make_float4(gx[4], gx[5], gx[6], gx[7]));
            }
        }
        __threadfence();
        __syncwarp();
        int prev = 0;
        if (lane == 0) prev = atomicAdd(&P.split_cnt[static_cast<int64_t>(it.split) * P.n_chunks + chunk], 1);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev == it.n_parts - 1) {
            if (lane == 0) P.split_cnt[static_cast<int64_t>(it.split) * P.n_chunks + chunk] = 0;   // rewind
            __threadfence();
            const float* rows = P.split_part + static_cast<int64_t>(it.split_row) * P.bpad + chunk * 32 * LW;
            st_epilogue<LW>(P, v, chunk, lane, [&](int, int, int base, float (&gx)[8]) {
#pragma unroll
                for (int j = 0; j < 8; ++j) gx[j] = 0.0f;
                if (base < 32 * LW) {
                    for (int q = 0; q < it.n_parts; ++q) {
                        const float* p = rows + static_cast<int64_t>(q) * P.bpad + base;
                        const float4 a = __ldcg(reinterpret_cast<const float4*>(p));
                        const float4 b = __ldcg(reinterpret_cast<const float4*>(p + 4));
                        gx[0] += a.x; gx[1] += a.y; gx[2] += a.z; gx[3] += a.w;
                        gx[4] += b.x; gx[5] += b.y; gx[6] += b.z; gx[7] += b.w;
                    }
                }
            });
        }
    }
}

template <int LW>
__global__ void __launch_bounds__(kThreads, 3) k_st_pass(const StParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LW, li = lane % LW;
    unsigned char* wbase = smem + warp * kVarWarpBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + 2 * kVarBufBytes);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int total = P.n_items * P.n_chunks;
    int w = fetch_work(P.head, lane);
    if (w < total && lane == 0) issue_st_item<LW>(P, w % P.n_items, wbase, &bars[0]);
    uint32_t phase[2] = {0u, 0u};
    int buf = 0;
    while (w < total) {
        const int wn = fetch_work(P.head, lane);
        if (wn < total && lane == 0) {
            fence_proxy_async();
            issue_st_item<LW>(P, wn % P.n_items, wbase + (buf ^ 1) * kVarBufBytes, &bars[buf ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bars[buf], phase[buf], kWaitNs);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicOr(P.status, kStatusTimeout);
                mbar_wait_bounded(&bars[buf], phase[buf], kWaitNs);
                if (wn < total) mbar_wait_bounded(&bars[buf ^ 1], phase[buf ^ 1], kWaitNs);
            }
            __syncwarp();
            break;
        }
        phase[buf] ^= 1u;
        process_st_item<LW>(P, w, wbase + buf * kVarBufBytes, g, li, lane);
        __syncwarp();
        w = wn;
        buf ^= 1;
    }
    queue_exit(P.head, P.exit_cnt);
}

// Logistic noise of one step, [n][ldB] float32: one thread per 8 candidates of a row.
__global__ void __launch_bounds__(256) k_st_noise(uint64_t seed, int64_t step, float* noise, int64_t n, int32_t B,
                                                  int64_t ldB) {
    const int runs = (B + 7) / 8;
    const int64_t total = n * runs;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t row = i / runs;
        const int c0 = static_cast<int>(i - row * runs) * 8;
        float l[8];
        logistic8(seed, step, row, c0, l);
        store8(noise + row * ldB + c0, c0, B, l);
    }
}

// Hard assignment [delta + l > 0] into bit words: one thread per 32-bit word of a row.
__global__ void __launch_bounds__(256) k_st_sample(const float* delta, const float* noise, uint64_t seed, int64_t step,
                                                   uint32_t* bits32, int64_t n, int32_t B, int64_t ldB, int32_t nw32) {
    const int64_t total = n * nw32;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t row = i / nw32;
        const int word = static_cast<int>(i - row * nw32);
        uint32_t bits = 0u;
        for (int r = 0; r < 4; ++r) {
            const int c0 = word * 32 + 8 * r;
            if (c0 >= B) break;
            float l[8], d[8];
            noise8(noise, seed, step, row, ldB, c0, B, l);
            load8(delta + row * ldB + c0, c0, B, d);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (c0 + j < B && d[j] + l[j] > 0.0f) bits |= 1u << (8 * r + j);
        }
        bits32[i] = bits;
    }
}

template <int LW>
int st_grid_t() {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_st_pass<LW>, kWarps * kVarWarpBytes);
    return grid;
}

int elementwise_blocks(int64_t total) {
    const int64_t blocks = (total + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    return static_cast<int>(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

int grid_st_pass(int lw) {
    switch (lw) {
        case 32: return st_grid_t<32>();
        case 16: return st_grid_t<16>();
        case 8: return st_grid_t<8>();
        case 4: return st_grid_t<4>();
        case 2: return st_grid_t<2>();
        default: return st_grid_t<1>();
    }
}

cudaError_t launch_st_pass(const StParams& p, int lw, int grid, cudaStream_t s) {
    const int smem = kWarps * kVarWarpBytes;
    grid_st_pass(lw);
    switch (lw) {
        case 32: k_st_pass<32><<<grid, kThreads, smem, s>>>(p); break;
        case 16: k_st_pass<16><<<grid, kThreads, smem, s>>>(p); break;
        case 8: k_st_pass<8><<<grid, kThreads, smem, s>>>(p); break;
        case 4: k_st_pass<4><<<grid, kThreads, smem, s>>>(p); break;
        case 2: k_st_pass<2><<<grid, kThreads, smem, s>>>(p); break;
        default: k_st_pass<1><<<grid, kThreads, smem, s>>>(p); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_st_noise(uint64_t seed, int64_t step, float* noise, int64_t n, int32_t B, int64_t ldB,
                            cudaStream_t s) {
    const int64_t total = n * ((B + 7) / 8);
    if (total <= 0) return cudaSuccess;
    k_st_noise<<<elementwise_blocks(total), 256, 0, s>>>(seed, step, noise, n, B, ldB);
    return cudaGetLastError();
}

cudaError_t launch_st_sample(const float* delta, const float* noise, uint64_t seed, int64_t step, uint32_t* bits32,
                             int64_t n, int32_t B, int64_t ldB, int32_t nw32, cudaStream_t s) {
    const int64_t total = n * nw32;
    if (total <= 0) return cudaSuccess;
    k_st_sample<<<elementwise_blocks(total), 256, 0, s>>>(delta, noise, seed, step, bits32, n, B, ldB, nw32);
    return cudaGetLastError();
}

}  // namespace gs
