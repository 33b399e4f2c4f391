// Device helpers of the variable-major pass (its tiled, owned-variable and TMA-ring forms in
// gs_kernels.cu): element types, gathers and streaming-operator loads/stores, literal factors,
// the leave-one-out occurrence loops, loss credits (in registers or shared memory), the Adam
// epilogue and the tile staging layout. Internal linkage.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

// ------------------------------------------------------------------------------------------
// Element types.
template <typename T>
struct Elem;
template <>
struct Elem<float> {
    static constexpr int VEC = 4;
};
template <>
struct Elem<__nv_bfloat16> {
    static constexpr int VEC = 8;
};
template <>
struct Elem<__half> {
    static constexpr int VEC = 8;
};

// One 16-byte piece of a relaxed-value row, through the non-coherent path. No L2 policy
// operand: each one costs the pass an instruction per gather (an explicit evict-last policy on
// the gathers measured 4-10 % slower across the workloads).
__device__ __forceinline__ uint4 ld_gather16(const void* p) {
    uint4 r;
    asm("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}
// Once-per-step state streams (delta, m, v read; delta, m, v, x_out written): the streaming cache
// operator (.cs, evict-first in L1 and L2) keeps them from displacing the gathered rows.
__device__ __forceinline__ float4 ld_first_f4(const float* p) {
    float4 r;
    asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ float2 ld_first_f2(const float* p) {
    float2 r;
    asm volatile("ld.global.cs.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ float ld_first_f1(const float* p) {
    float r;
    asm volatile("ld.global.cs.f32 %0, [%1];" : "=f"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ void st_first_u4(void* p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_first_u2(void* p, uint2 v) {
    asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void st_first_u1(void* p, uint32_t v) {
    asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ void unpack(const uint4& r, float* x);
template <>
__device__ __forceinline__ void unpack<float>(const uint4& r, float* x) {
    x[0] = __uint_as_float(r.x);
    x[1] = __uint_as_float(r.y);
    x[2] = __uint_as_float(r.z);
    x[3] = __uint_as_float(r.w);
}
template <>
__device__ __forceinline__ void unpack<__nv_bfloat16>(const uint4& r, float* x) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[2 * k] = __uint_as_float(w[k] << 16);
        x[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
template <>
__device__ __forceinline__ void unpack<__half>(const uint4& r, float* x) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h = *reinterpret_cast<const __half2*>(&w[k]);
        const float2 f = __half22float2(h);
        x[2 * k] = f.x;
        x[2 * k + 1] = f.y;
    }
}

template <typename T>
__device__ __forceinline__ T from_f32(float x);
template <>
__device__ __forceinline__ float from_f32<float>(float x) {
    return x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half from_f32<__half>(float x) {
    return __float2half_rn(x);
}

// N consecutive floats, streaming (read once / written once per step).
template <int N>
__device__ __forceinline__ void ld_stream(const float* p, float* x) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const float4 t = ld_first_f4(p + 4 * k);
            x[4 * k] = t.x;
            x[4 * k + 1] = t.y;
            x[4 * k + 2] = t.z;
            x[4 * k + 3] = t.w;
        }
    } else if constexpr (N == 2) {
        const float2 t = ld_first_f2(p);
        x[0] = t.x;
        x[1] = t.y;
    } else {
        x[0] = ld_first_f1(p);
    }
}
template <int N>
__device__ __forceinline__ void st_stream(float* p, const float* x) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k)
            st_first_u4(p + 4 * k, make_uint4(__float_as_uint(x[4 * k]), __float_as_uint(x[4 * k + 1]),
                                              __float_as_uint(x[4 * k + 2]), __float_as_uint(x[4 * k + 3])));
    } else if constexpr (N == 2) {
        st_first_u2(p, make_uint2(__float_as_uint(x[0]), __float_as_uint(x[1])));
    } else {
        st_first_u1(p, __float_as_uint(x[0]));
    }
}
// N consecutive values of T from floats (round to nearest even for 16-bit types).
template <typename T, int N>
__device__ __forceinline__ void st_vals(T* p, const float* x) {
    if constexpr (sizeof(T) == 4) {
        st_stream<N>(reinterpret_cast<float*>(p), x);
    } else {
        uint32_t w[(N + 1) / 2];
#pragma unroll
        for (int k = 0; k < (N + 1) / 2; ++k) {
            const T lo = from_f32<T>(x[2 * k]);
            const T hi = (2 * k + 1 < N) ? from_f32<T>(x[2 * k + 1]) : from_f32<T>(0.f);
            w[k] = static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(&lo)) |
                   (static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(&hi)) << 16);
        }
        if constexpr (N == 8) {
            st_first_u4(p, make_uint4(w[0], w[1], w[2], w[3]));
        } else if constexpr (N == 4) {
            st_first_u2(p, make_uint2(w[0], w[1]));
        } else if constexpr (N == 2) {
            st_first_u1(p, w[0]);
        } else {
            *p = from_f32<T>(x[0]);
        }
    }
}

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Literal factors f = a x + b of the VEC candidates in one 16-byte piece of a row, as pairs:
// a = -1, b = 1 for a positive literal (1 - x), a = 1, b = 0 for a negated one (x). For 16-bit
// values the product a x is formed by the mixed-precision FMA (16-bit a and x, float32 b and
// result), which equals converting x to float32 first: a x is exact and the sum rounds once.
template <typename T>
__device__ __forceinline__ void factors(const uint4& r, float a, float b, float2 (&f)[Elem<T>::VEC / 2]);
template <>
__device__ __forceinline__ void factors<float>(const uint4& r, float a, float b, float2 (&f)[2]) {
    f[0] = __ffma2_rn(dup2(a), make_float2(__uint_as_float(r.x), __uint_as_float(r.y)), dup2(b));
    f[1] = __ffma2_rn(dup2(a), make_float2(__uint_as_float(r.z), __uint_as_float(r.w)), dup2(b));
}
__device__ __forceinline__ float2 fma_bf16_pair(uint32_t w, uint16_t a, float b) {
    float lo, hi;
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "fma.rn.f32.bf16 %0, %3, l, %4;\n\tfma.rn.f32.bf16 %1, %3, h, %4;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(w), "h"(a), "f"(b));
    return make_float2(lo, hi);
}
__device__ __forceinline__ float2 fma_f16_pair(uint32_t w, uint16_t a, float b) {
    float lo, hi;
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "fma.rn.f32.f16 %0, %3, l, %4;\n\tfma.rn.f32.f16 %1, %3, h, %4;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(w), "h"(a), "f"(b));
    return make_float2(lo, hi);
}
template <>
__device__ __forceinline__ void factors<__nv_bfloat16>(const uint4& r, float a, float b, float2 (&f)[4]) {
    const uint16_t ab = a < 0.0f ? 0xBF80u : 0x3F80u;   // -1 / +1 in bfloat16
    f[0] = fma_bf16_pair(r.x, ab, b);
    f[1] = fma_bf16_pair(r.y, ab, b);
    f[2] = fma_bf16_pair(r.z, ab, b);
    f[3] = fma_bf16_pair(r.w, ab, b);
}
template <>
__device__ __forceinline__ void factors<__half>(const uint4& r, float a, float b, float2 (&f)[4]) {
    const uint16_t ab = a < 0.0f ? 0xBC00u : 0x3C00u;   // -1 / +1 in float16
    f[0] = fma_f16_pair(r.x, ab, b);
    f[1] = fma_f16_pair(r.y, ab, b);
    f[2] = fma_f16_pair(r.z, ab, b);
    f[3] = fma_f16_pair(r.w, ab, b);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Hardware approximations for the Adam epilogue: rcp.approx.f32 (at most 1 ulp from the
// reciprocal) and sqrt.approx.f32 (relative error at most 2^-23). The update's error bound in the
// tests allows a few float32 roundings per operation; the IEEE-rounded forms cost several
// instructions each and the pass is bound by instruction issue.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Logistic sigmoid, overflow-free: with e = exp(-|z|), sigma(|z|) = 1 / (1 + e) and
// sigma(-|z|) = e / (1 + e).
__device__ __forceinline__ float sigmoid(float z) {
    const float e = expf(-fabsf(z));
    const float r = rcp_fast(1.0f + e);
    return z >= 0.0f ? r : e * r;
}

// One Adam step on the logit difference delta given gx = dL/dx, x = sigma(delta / tau); the
// chain factor sigma(z) sigma(-z) is the product of the two halves above for either sign.
__device__ __forceinline__ void adam_update(float gx, float& d, float& m, float& v, float& x_new, const AdamK& k) {
    const float z = d * k.inv_tau;
    const float e = expf(-fabsf(z));
    const float r = rcp_fast(1.0f + e);
    const float q = e * r;
    const float g = gx * (r * q) * k.inv_tau;
    m = fmaf(k.beta1, m, k.one_minus_beta1 * g);
    v = fmaf(k.beta2, v, k.one_minus_beta2 * (g * g));
    const float den = sqrt_fast(v) * k.inv_sqrt_bc2 + k.eps;
    d = d - k.step_size * (m * rcp_fast(den));
    x_new = sigmoid(d * k.inv_tau);
}

template <int LC, int N>
__device__ __forceinline__ void group_sum(float (&a)[N]) {
#pragma unroll
    for (int off = LC; off < 32; off <<= 1) {
#pragma unroll
        for (int e = 0; e < N; ++e) a[e] += __shfl_xor_sync(0xffffffffu, a[e], off);
    }
}

// ------------------------------------------------------------------------------------------
// Variable-major pass: gradient (kModeGrad) or gradient + Adam + relaxed values + rounding
// (kModeAdam), optionally with the forward loss credited at each clause's position-0 literal.

// Literal factor f = a * x + b on two candidates at once (packed f32x2 arithmetic):
// (a, b) = (-1, 1) for a positive literal (f = 1 - x), (1, 0) for a negated one (f = x),
// (0, 1) for the unit-clause sentinel (f = 1, nothing loaded).

__device__ __forceinline__ void code_ab(uint32_t c, float& a, float& b) {
    const bool sent = (c >> kVShift) == kVSentinel;
    a = sent ? 0.0f : __uint_as_float(0xbf800000u ^ ((c & kVNeg) << 31));
    b = sent ? 1.0f : fmaf(-0.5f, a, 0.5f);
}
// Sign of d(own factor)/dx on the last code of an occurrence: +1 negated own literal, -1 positive.
__device__ __forceinline__ float occ_sign(uint32_t last) {
    return __uint_as_float(0xbf800000u ^ ((last & kVSelfNeg) << 29));
}

// Per-lane view of the relaxed values: row u of this lane's candidates is at base + u * row_bytes.
struct RowView {
    const char* base;
    uint32_t row_bytes;
    bool ok;   // the lane holds at least one candidate < B
#ifdef GS_DEBUG
    int64_t n_rows;
    int32_t* status;
#endif
};
__device__ __forceinline__ void set_row_bounds(RowView& rv, int64_t n_rows, int32_t* status) {
#ifdef GS_DEBUG
    rv.n_rows = n_rows;
    rv.status = status;
#else
    (void)rv;
    (void)n_rows;
    (void)status;
#endif
}
__device__ __forceinline__ uint4 load_row(const RowView& rv, uint32_t u) {
#ifdef GS_DEBUG
    if (!row_ok(u, rv.n_rows, rv.status)) return make_uint4(0u, 0u, 0u, 0u);
#endif
    return ld_gather16(rv.base + static_cast<uint64_t>(u) * rv.row_bytes);
}

// Cache-line prefetches (no data returned; the lines are asked into L1 resp. L2).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <bool GC>
__device__ __forceinline__ uint32_t ld_code(const uint32_t* cd, int i) {
    if constexpr (GC)
        return __ldg(cd + i);
    else
        return cd[i];
}

// Loss credits of one variable's occurrences: the clause value U_t = f_own * LOO is credited at
// the clause's position-0 literal. f_own is the variable's own factor, so the credits are summed
// separately for positive (Cp) and negated (Cn) own literals and multiplied by 1 - x resp. x once,
// when the variable is done.
template <int H>
struct Credits {
    float2 p[H], n[H];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int h = 0; h < H; ++h) p[h] = n[h] = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void add_p(const float2 (&r)[H]) {
#pragma unroll
        for (int h = 0; h < H; ++h) p[h] = __ffma2_rn(make_float2(1.0f, 1.0f), r[h], p[h]);
    }
    __device__ __forceinline__ void add_n(const float2 (&r)[H]) {
#pragma unroll
        for (int h = 0; h < H; ++h) n[h] = __ffma2_rn(make_float2(1.0f, 1.0f), r[h], n[h]);
    }
    // weighted form for several lane groups side by side (wp, wn in {0, 1})
    __device__ __forceinline__ void add_w(float wp, float wn, const float2 (&r)[H]) {
#pragma unroll
        for (int h = 0; h < H; ++h) {
            p[h] = __ffma2_rn(make_float2(wp, wp), r[h], p[h]);
            n[h] = __ffma2_rn(make_float2(wn, wn), r[h], n[h]);
        }
    }
    __device__ __forceinline__ void get(float2 (&pp)[H], float2 (&nn)[H]) const {
#pragma unroll
        for (int h = 0; h < H; ++h) {
            pp[h] = p[h];
            nn[h] = n[h];
        }
    }
};

// 16-byte shared-memory accesses the compiler keeps in place (a lane's own slots; volatile so
// that the sums are not hoisted back into registers).
__device__ __forceinline__ float4 ld_shared4(uint32_t x) {
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(x));
    return r;
}
__device__ __forceinline__ void st_shared4(uint32_t x, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(x), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// The same sums kept in shared memory (one warp, one lane group): a credit is a shared-memory
// read-add-write of the lane's slots, which leaves the 2 * VEC registers of Credits to the
// gathers. The additions are the same, in the same order, so the sums are bitwise those of
// Credits. Layout: 16-byte slots, slot q of lane l at q * 512 + l * 16 bytes (conflict-free
// 16-byte accesses), H / 2 slots of Cp then H / 2 of Cn.
template <int H>
struct CreditsSm {
    static_assert(H % 2 == 0, "16-byte slots hold two candidate pairs");
    uint32_t a;   // shared-memory address of the lane's first slot
    __device__ __forceinline__ static float4 lds(uint32_t x) { return ld_shared4(x); }
    __device__ __forceinline__ static void sts(uint32_t x, float4 v) { st_shared4(x, v); }
    __device__ __forceinline__ void zero() const {
#pragma unroll
        for (int q = 0; q < H; ++q) sts(a + q * 512, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    }
    __device__ __forceinline__ void add_at(uint32_t x, const float2 (&r)[H]) const {
#pragma unroll
        for (int q = 0; q < H / 2; ++q) {
            const float4 v = lds(x + q * 512);
            const float2 lo = __ffma2_rn(make_float2(1.0f, 1.0f), r[2 * q], make_float2(v.x, v.y));
            const float2 hi = __ffma2_rn(make_float2(1.0f, 1.0f), r[2 * q + 1], make_float2(v.z, v.w));
            sts(x + q * 512, make_float4(lo.x, lo.y, hi.x, hi.y));
        }
    }
    __device__ __forceinline__ void add_p(const float2 (&r)[H]) const { add_at(a, r); }
    __device__ __forceinline__ void add_n(const float2 (&r)[H]) const { add_at(a + (H / 2) * 512, r); }
    __device__ __forceinline__ void add_w(float, float, const float2 (&)[H]) const {}   // one lane group only
    __device__ __forceinline__ void get(float2 (&pp)[H], float2 (&nn)[H]) const {
#pragma unroll
        for (int q = 0; q < H / 2; ++q) {
            const float4 u = lds(a + q * 512), v = lds(a + (H / 2 + q) * 512);
            pp[2 * q] = make_float2(u.x, u.y);
            pp[2 * q + 1] = make_float2(u.z, u.w);
            nn[2 * q] = make_float2(v.x, v.y);
            nn[2 * q + 1] = make_float2(v.z, v.w);
        }
    }
};

// One batch of the general slot loop: NB occurrence codes from s (up to ce) of the group; an
// occurrence ends at a code carrying kVEnd. R is the running leave-one-out product (prefix then
// suffix of the occurrence's clause), restarted after each end.
// UNI: all 32 lanes of the warp process the same codes (one lane group), so branches on a code's
// flags are uniform and the loss credit is added only where a code carries it.
template <typename T, int VEC, int NB, bool LOSS, bool GC, bool UNI, typename CR>
__device__ __forceinline__ void slot_batch(const uint32_t* cd, int s, int ce, const RowView& rv, float2 (&R)[VEC / 2],
                                           float2 (&G2)[VEC / 2], CR& cr) {
    constexpr int H = VEC / 2;
    uint32_t cw[NB];
    uint4 raw[NB];
    if constexpr (GC) {
        if (s + 32 < ce) prefetch_l1(cd + s + 32);   // the codes four batches ahead
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) cw[j] = (s + j < ce) ? ld_code<GC>(cd, s + j) : (kVSentinel << kVShift);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const uint32_t u = cw[j] >> kVShift;
        raw[j] = make_uint4(0u, 0u, 0u, 0u);
        if (rv.ok && u != kVSentinel) raw[j] = load_row(rv, u);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const uint32_t c = cw[j];
        float a, b;
        code_ab(c, a, b);
        float2 f[H];
        factors<T>(raw[j], a, b, f);
        const bool end = (c & kVEnd) != 0u;
        float2 rn[H];
        if constexpr (UNI) {
            // one lane group: the end of an occurrence is a uniform branch
#pragma unroll
            for (int h = 0; h < H; ++h) rn[h] = __fmul2_rn(R[h], f[h]);
            if (end) {
                const float sg = occ_sign(c);
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    G2[h] = __ffma2_rn(dup2(sg), rn[h], G2[h]);
                    R[h] = dup2(1.0f);
                }
                // a credit sits on an occurrence's last code, so it is tested only there
                if (LOSS && (c & kVCredit)) {
                    if (c & kVSelfNeg)
                        cr.add_n(rn);
                    else
                        cr.add_p(rn);
                }
            } else {
#pragma unroll
                for (int h = 0; h < H; ++h) R[h] = rn[h];
            }
        } else {
            const float sg = end ? occ_sign(c) : 0.0f;
            const float e1 = end ? 1.0f : 0.0f;   // restart the running product after an end:
            const float keep = 1.0f - e1;         // R = rn * keep + e1 (rn is finite)
#pragma unroll
            for (int h = 0; h < H; ++h) {
                rn[h] = __fmul2_rn(R[h], f[h]);
                G2[h] = __ffma2_rn(dup2(sg), rn[h], G2[h]);
                R[h] = __ffma2_rn(rn[h], dup2(keep), dup2(e1));
            }
        }
        if (LOSS) {
            if constexpr (!UNI) {
                const uint32_t f = c & (kVEnd | kVCredit | kVSelfNeg);
                const float wp = (f == (kVEnd | kVCredit)) ? 1.0f : 0.0f;
                const float wn = (f == (kVEnd | kVCredit | kVSelfNeg)) ? 1.0f : 0.0f;
                cr.add_w(wp, wn, rn);
            }
        }
    }
}

// The general slot loop over the group's occurrence codes [cs, ce). With several lane groups
// the credits are predicated arithmetic on every code, so the loop is split: the credited
// occurrences come first in each variable's list, ending at cc, and batches run with the credit
// arithmetic only while some group of the warp is still before its cc.
template <typename T, int VEC, int NB, bool LOSS, bool GC, bool UNI, typename CR>
__device__ __forceinline__ void var_slots(const uint32_t* cd, int cs, int ce, int cc, const RowView& rv,
                                          float2 (&G2)[VEC / 2], CR& cr) {
    constexpr int H = VEC / 2;
    float2 R[H];
#pragma unroll
    for (int h = 0; h < H; ++h) R[h] = dup2(1.0f);
    int s = cs;
    if constexpr (LOSS && !UNI) {
        for (; s < ce && __any_sync(__activemask(), s < cc); s += NB)
            slot_batch<T, VEC, NB, true, GC, UNI>(cd, s, ce, rv, R, G2, cr);
        for (; s < ce; s += NB) slot_batch<T, VEC, NB, false, GC, UNI>(cd, s, ce, rv, R, G2, cr);
    } else {
        for (; s < ce; s += NB) slot_batch<T, VEC, NB, LOSS, GC, UNI>(cd, s, ce, rv, R, G2, cr);
    }
}

// Fixed-width occurrence loop: every occurrence in [cs, ce) has exactly K codes (all clauses
// of the tile have width K + 1, e.g. the paper's width-3 normal form with K = 2). OB whole
// occurrences per batch, their K * OB gathers issued together; full batches run without
// per-slot predicates, the last partial batch with them.
template <int K>
__device__ __forceinline__ void fixed_ab(uint32_t c, float& a, float& b) {
    if constexpr (K == 1) {
        code_ab(c, a, b);   // unit-clause sentinels only occur in K = 1 tiles
    } else {
        a = __uint_as_float(0xbf800000u ^ ((c & kVNeg) << 31));   // -1 positive, +1 negated
        b = fmaf(-0.5f, a, 0.5f);                                  //  1 positive,  0 negated
    }
}

template <typename T, int VEC, int K, int OB, bool LOSS, bool TAIL, bool GC, bool UNI, typename CR>
__device__ __forceinline__ void occ_batch(const uint32_t* cd, int s, int ce, const RowView& rv,
                                          float2 (&G2)[VEC / 2], CR& cr) {
    constexpr int H = VEC / 2;
    constexpr int NS = OB * K;
    uint32_t cw[NS];
    uint4 raw[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) cw[j] = (!TAIL || s + j < ce) ? ld_code<GC>(cd, s + j) : (kVSentinel << kVShift);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        raw[j] = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t u = cw[j] >> kVShift;
        const bool load = rv.ok && ((K > 1 && !TAIL) || u != kVSentinel);
        if (load) raw[j] = load_row(rv, u);
    }
#pragma unroll
    for (int o = 0; o < OB; ++o) {
        float2 prod[H];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float a, b;
            fixed_ab<(TAIL ? 1 : K)>(cw[o * K + j], a, b);
            float2 f[H];
            factors<T>(raw[o * K + j], a, b, f);
#pragma unroll
            for (int h = 0; h < H; ++h) prod[h] = (j == 0) ? f[h] : __fmul2_rn(prod[h], f[h]);
        }
        const uint32_t last = cw[o * K + K - 1];
        const bool valid = !TAIL || (s + o * K) < ce;
        if constexpr (UNI) {
            if (valid) {
                const float sg = (last & kVSelfNeg) ? 1.0f : -1.0f;
#pragma unroll
                for (int h = 0; h < H; ++h) G2[h] = __ffma2_rn(dup2(sg), prod[h], G2[h]);
                if (LOSS && (last & kVCredit)) {
                    if (last & kVSelfNeg)
                        cr.add_n(prod);
                    else
                        cr.add_p(prod);
                }
            }
            continue;
        }
        const float sg = valid ? occ_sign(last) : 0.0f;
#pragma unroll
        for (int h = 0; h < H; ++h) G2[h] = __ffma2_rn(dup2(sg), prod[h], G2[h]);
        if (LOSS) {
            const uint32_t f = valid ? (last & (kVCredit | kVSelfNeg)) : 0u;
            const float wp = (f == kVCredit) ? 1.0f : 0.0f;
            const float wn = (f == (kVCredit | kVSelfNeg)) ? 1.0f : 0.0f;
            cr.add_w(wp, wn, prod);
        }
    }
}

template <typename T, int VEC, int K, bool LOSS, bool GC, bool UNI, typename CR>
__device__ __forceinline__ void var_occ_fixed(const uint32_t* cd, int cs, int ce, int cc, const RowView& rv,
                                              float2 (&G2)[VEC / 2], CR& cr) {
    // occurrences per batch; width-4 clauses take 4 with float32 values (12 gathers in flight,
    // 6 % faster on 4-SAT) but keep 3 with 16-bit ones, whose 32-lane kernel would spill
    constexpr int OB = (K == 1) ? 8 : (K == 2 ? 4 : (VEC == 4 ? 4 : 3));
    constexpr int NS = OB * K;
    int s = cs;
    if constexpr (LOSS && !UNI && K >= 3) {
        // as in var_slots: the credit arithmetic only while some lane group is before its cc
        // (for width-3 clauses the credited third of the list is too short to pay for the vote)
        for (; s + NS <= ce && __any_sync(__activemask(), s < cc); s += NS)
            occ_batch<T, VEC, K, OB, true, false, GC, UNI>(cd, s, ce, rv, G2, cr);
        for (; s + NS <= ce; s += NS) occ_batch<T, VEC, K, OB, false, false, GC, UNI>(cd, s, ce, rv, G2, cr);
    } else {
        for (; s + NS <= ce; s += NS) occ_batch<T, VEC, K, OB, LOSS, false, GC, UNI>(cd, s, ce, rv, G2, cr);
    }
    if (s < ce) occ_batch<T, VEC, K, OB, LOSS, true, GC, UNI>(cd, s, ce, rv, G2, cr);
}

// Gradient and (with LOSS) loss credits of one variable's occurrence codes [cs, ce); the
// credited occurrences lie in [cs, cc) (cc = ce when that is not known: every code is then
// checked for a credit); GC: the codes are read from global memory instead of a shared-memory
// tile.
template <typename T, int VEC, int NB, bool LOSS, bool GC = false, bool UNI = false, typename CR = Credits<VEC / 2>>
__device__ __forceinline__ void var_gather(int kk, const uint32_t* cd, int cs, int ce, int cc, const RowView& rv,
                                           float (&gacc)[VEC], CR& cr) {
    constexpr int H = VEC / 2;
    float2 G2[H];
#pragma unroll
    for (int h = 0; h < H; ++h) G2[h] = dup2(0.0f);
    switch (kk) {
        case 1: var_occ_fixed<T, VEC, 1, LOSS, GC, UNI>(cd, cs, ce, cc, rv, G2, cr); break;
        case 2: var_occ_fixed<T, VEC, 2, LOSS, GC, UNI>(cd, cs, ce, cc, rv, G2, cr); break;
        case 3: var_occ_fixed<T, VEC, 3, LOSS, GC, UNI>(cd, cs, ce, cc, rv, G2, cr); break;
        default: var_slots<T, VEC, NB, LOSS, GC, UNI>(cd, cs, ce, cc, rv, G2, cr); break;
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        gacc[2 * h] = G2[h].x;
        gacc[2 * h + 1] = G2[h].y;
    }
}

template <typename T, int MODE, int LC>
struct VarCfg {
    static constexpr int VEC = Elem<T>::VEC;
    static constexpr int G = 32 / LC;
    static constexpr int BC = LC * VEC;
    static constexpr int NB = 8;                                // gathers in flight per slot batch
    static constexpr int VPG = (VEC / G) > 0 ? (VEC / G) : 1;   // epilogue candidates per lane
    static constexpr int GE = VEC / VPG;                        // groups active in the epilogue
    static constexpr int N32 = BC >= 32 ? BC / 32 : 1;          // 32-bit bit-words per chunk
    // Adam state loaded before the gathers when each lane keeps few epilogue candidates (16-bit
    // values in narrow chunks); with 32-lane chunks the registers go to the gathers instead
    static constexpr bool PREFETCH = (VEC == 8) && (LC < 32);
    // Per-warp staging buffer of one occurrence tile: the variable table, the occurrence offsets
    // (read only when several lane groups split a variable's occurrences) and the codes.
    static constexpr int REC_BYTES = (G > 1) ? kVarRecBytes : 0;
    static constexpr int CODE_OFF = kVarVtabBytes + REC_BYTES;
    static constexpr int BUF_BYTES = CODE_OFF + kVarCodeBytes;
    static constexpr int STAGE_BYTES = 2 * BUF_BYTES + 16;   // two buffers + two mbarriers
};

// Adam state (delta, m, v) of the epilogue candidates of one lane.
template <int VPG>
struct AdamState {
    float d[VPG], m[VPG], v[VPG];
};

template <typename T, int MODE, int LC>
__device__ __forceinline__ void adam_prefetch(const VarParams& P, int v, int chunk, int g, int li,
                                              AdamState<VarCfg<T, MODE, LC>::VPG>& st) {
    using C = VarCfg<T, MODE, LC>;
    constexpr int VPG = C::VPG;
    const int c0 = chunk * C::BC + li * C::VEC + g * VPG;
    const bool act = (g < C::GE) && (c0 < P.B);
    const int64_t off = static_cast<int64_t>(v) * P.ldB + c0;
    if (act && c0 + VPG <= P.B) {
        ld_stream<VPG>(P.delta + off, st.d);
        ld_stream<VPG>(P.m + off, st.m);
        ld_stream<VPG>(P.v + off, st.v);
    } else {
#pragma unroll
        for (int el = 0; el < VPG; ++el) {
            const bool ok = act && c0 + el < P.B;
            st.d[el] = ok ? P.delta[off + el] : 0.0f;
            st.m[el] = ok ? P.m[off + el] : 0.0f;
            st.v[el] = ok ? P.v[off + el] : 0.0f;
        }
    }
}

template <typename T, int MODE, int LC>
__device__ __forceinline__ void var_epilogue(const VarParams& P, int v, int inst, int chunk, int g, int li, int lane,
                                             const float (&ge)[VarCfg<T, MODE, LC>::VPG],
                                             const AdamState<VarCfg<T, MODE, LC>::VPG>& st) {
    using C = VarCfg<T, MODE, LC>;
    constexpr int VPG = C::VPG;
    const int r0 = li * C::VEC + g * VPG;
    const int c0 = chunk * C::BC + r0;
    const bool act = (g < C::GE) && (c0 < P.B);
    const bool full = act && (c0 + VPG <= P.B);
    const int64_t off = static_cast<int64_t>(v) * P.ldB + c0;
    if constexpr (MODE == kModeGrad) {
        if (act) {
            float out[VPG];
#pragma unroll
            for (int el = 0; el < VPG; ++el) {
                const float s = (P.dloss && c0 + el < P.B)
                                    ? static_cast<float>(P.dloss[static_cast<int64_t>(inst) * P.B + c0 + el])
                                    : 1.0f;
                out[el] = ge[el] * s;
            }
            if (full) {
                st_stream<VPG>(P.grad + off, out);
            } else {
                for (int el = 0; el < VPG && c0 + el < P.B; ++el) P.grad[off + el] = out[el];
            }
        }
    } else {
        uint32_t mybits = 0;
        if (act) {
            float d[VPG], mm[VPG], vv[VPG], xn[VPG];
#pragma unroll
            for (int el = 0; el < VPG; ++el) {
                d[el] = st.d[el];
                mm[el] = st.m[el];
                vv[el] = st.v[el];
            }
#pragma unroll
            for (int el = 0; el < VPG; ++el) {
                adam_update(ge[el], d[el], mm[el], vv[el], xn[el], P.adam);
                if (c0 + el < P.B && d[el] > 0.0f) mybits |= 1u << el;
            }
            T* xo = static_cast<T*>(P.x_out) + off;
            if (full) {
                st_stream<VPG>(P.delta + off, d);
                st_stream<VPG>(P.m + off, mm);
                st_stream<VPG>(P.v + off, vv);
                st_vals<T, VPG>(xo, xn);
            } else {
                for (int el = 0; el < VPG && c0 + el < P.B; ++el) {
                    P.delta[off + el] = d[el];
                    P.m[off + el] = mm[el];
                    P.v[off + el] = vv[el];
                    xo[el] = from_f32<T>(xn[el]);
                }
            }
        }
        if (P.bits32) {
            const int64_t row = static_cast<int64_t>(v) * 2 * P.nwd;
#pragma unroll
            for (int wi = 0; wi < C::N32; ++wi) {
                const uint32_t contrib = (act && (r0 >> 5) == wi) ? (mybits << (r0 & 31)) : 0u;
                const uint32_t word = __reduce_or_sync(0xffffffffu, contrib);
                const int hw = chunk * C::N32 + wi;
                if (lane == 0 && hw < 2 * P.nwd) P.bits32[row + hw] = word;
            }
            if (lane == 0 && chunk == P.n_chunks - 1) {
                for (int hw = P.n_chunks * C::N32; hw < 2 * P.nwd; ++hw) P.bits32[row + hw] = 0u;
            }
        }
    }
}

template <typename T, int MODE, int LC>
__device__ __forceinline__ void issue_var_item(const VarParams& P, int item, unsigned char* buf, uint64_t* bar) {
    using C = VarCfg<T, MODE, LC>;
    const VarItem it = P.items[item];
    const Span a = span16(P.vtab + it.vtab_base, static_cast<uint32_t>(it.nv + 1) * 4u);
    const Span b = (C::G > 1) ? span16(P.recs + it.rec_base, static_cast<uint32_t>(it.n_occ + 1) * 2u) : Span{0, 0};
    const Span c = span16(P.codes + it.code_base, static_cast<uint32_t>(it.n_codes) * 4u);
    mbar_expect_tx(bar, a.bytes + b.bytes + c.bytes);
    if (a.bytes) bulk_g2s(buf, reinterpret_cast<const void*>(a.src), a.bytes, bar);
    if (b.bytes) bulk_g2s(buf + kVarVtabBytes, reinterpret_cast<const void*>(b.src), b.bytes, bar);
    if (c.bytes) bulk_g2s(buf + C::CODE_OFF, reinterpret_cast<const void*>(c.src), c.bytes, bar);
}

}  // namespace
}  // namespace gs
