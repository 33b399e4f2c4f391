// sm_103a kernels of the GaloisSAT differentiable solving stage (arXiv 2603.28796).
//
// Layout: every candidate array is var-major, row v = variable v, columns = candidates, row
// stride ldB elements (16-byte rows). A lane owns VEC = 16 / sizeof(T) consecutive candidates
// and reads them with one 16-byte load; LC lanes cover a chunk of Bc = LC * VEC candidates;
// the G = 32 / LC lane groups of a warp work on different clauses / occurrences of one tile.
// Work items (tiles x candidate chunks) come from an integer work queue in chunk-major order,
// so that the rows of the current chunk stay resident in L2 while every tile gathers from it.
// Each warp stages its tile's index data into its own shared-memory buffer with 1-D bulk TMA
// (cp.async.bulk + mbarrier), double-buffered so the next tile loads while this one computes.
//
// No floating-point atomics: gradients are gathered per variable over the occurrence lists,
// split variables are combined in a fixed order by the last part to finish (integer counter),
// and loss partials are summed per tile in FP32 (Kahan) and across tiles in FP64 in tile order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "gs_device.cuh"
#include "gs_internal.h"
#include "gs_var.cuh"

namespace gs {
namespace {

// Where k_var_pass keeps a variable's loss credits. With one lane group per warp a credit is a
// warp-uniform branch taken on about one code in k, so the sums live in shared memory
// (CreditsSm) and their 2 * VEC registers go to the gathers: the 16-bit kernel keeps its third
// resident CTA that way, the float32 one its gathers in flight. Several lane groups credit by
// predicated arithmetic on every code and keep the sums in registers.
template <typename T, int LC>
__host__ __device__ constexpr bool credits_in_smem() {
    return LC == 32;
}

// Per-warp shared memory of k_var_pass: two staging buffers and their barriers (VarCfg), then the tile's
// compensated loss sums (sum and compensation, 32 lanes x VEC candidates each), which live in
// shared memory rather than registers to leave the registers to the gathers, then (see
// credits_in_smem) the variable's credit sums Cp and Cn (32 lanes x VEC candidates each).
template <typename T, int LC>
__host__ __device__ constexpr int var_warp_bytes() {
    return VarCfg<T, 1, LC>::STAGE_BYTES + 2 * 32 * Elem<T>::VEC * 4 +
           (credits_in_smem<T, LC>() ? 2 * 32 * Elem<T>::VEC * 4 : 0);
}

// The tile's compensated loss sums of one lane in shared memory: VEC / 4 16-byte slots of sums
// then VEC / 4 of compensations, slot q of lane l at q * 512 + l * 16 bytes (conflict-free).
template <int VEC>
struct LossSm {
    uint32_t a;   // shared-memory address of the lane's first slot
    __device__ __forceinline__ void zero() const {
#pragma unroll
        for (int q = 0; q < VEC / 2; ++q) st_shared4(a + q * 512, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    }
    __device__ __forceinline__ void load(float (&s)[VEC], float (&c)[VEC]) const {
#pragma unroll
        for (int q = 0; q < VEC / 4; ++q) {
            const float4 u = ld_shared4(a + q * 512), v = ld_shared4(a + (VEC / 4 + q) * 512);
            s[4 * q] = u.x, s[4 * q + 1] = u.y, s[4 * q + 2] = u.z, s[4 * q + 3] = u.w;
            c[4 * q] = v.x, c[4 * q + 1] = v.y, c[4 * q + 2] = v.z, c[4 * q + 3] = v.w;
        }
    }
    __device__ __forceinline__ void store(const float (&s)[VEC], const float (&c)[VEC]) const {
#pragma unroll
        for (int q = 0; q < VEC / 4; ++q) {
            st_shared4(a + q * 512, make_float4(s[4 * q], s[4 * q + 1], s[4 * q + 2], s[4 * q + 3]));
            st_shared4(a + (VEC / 4 + q) * 512, make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
        }
    }
};

// credit_flush on the loss sums in shared memory.
template <int VEC, typename CR>
__device__ __forceinline__ void credit_flush_v(const CR& cr, const float (&xs)[VEC], const LossSm<VEC>& L) {
    float s[VEC], c[VEC];
    float2 cp[VEC / 2], cn[VEC / 2];
    cr.get(cp, cn);
    L.load(s, c);
#pragma unroll
    for (int h = 0; h < VEC / 2; ++h) {
        kahan_add(s[2 * h], c[2 * h], fmaf(1.0f - xs[2 * h], cp[h].x, xs[2 * h] * cn[h].x));
        kahan_add(s[2 * h + 1], c[2 * h + 1], fmaf(1.0f - xs[2 * h + 1], cp[h].y, xs[2 * h + 1] * cn[h].y));
    }
    L.store(s, c);
}

template <typename T, int MODE, int LC>
__device__ __forceinline__ void process_var_item(const VarParams& P, int w, const unsigned char* buf, int g, int li,
                                                 int lane, float* lossbuf) {
    using C = VarCfg<T, MODE, LC>;
    constexpr int VEC = C::VEC, G = C::G, VPG = C::VPG, GE = C::GE;
    const int item = w % P.n_items;
    const int chunk = w / P.n_items;
    const VarItem it = P.items[item];
    const uint32_t* vt =
        reinterpret_cast<const uint32_t*>(buf + (reinterpret_cast<uintptr_t>(P.vtab + it.vtab_base) & 15));
    const uint16_t* rc = reinterpret_cast<const uint16_t*>(
        buf + kVarVtabBytes + (reinterpret_cast<uintptr_t>(P.recs + it.rec_base) & 15));
    const uint32_t* cd = reinterpret_cast<const uint32_t*>(
        buf + C::CODE_OFF + (reinterpret_cast<uintptr_t>(P.codes + it.code_base) & 15));
    const int cand0 = chunk * C::BC;
    const int lane_base = cand0 + li * VEC;
    const bool ld_ok = lane_base < P.B;
    RowView rv;
    rv.base = reinterpret_cast<const char*>(static_cast<const T*>(P.x_in) + lane_base);
    rv.row_bytes = static_cast<uint32_t>(P.ldB * sizeof(T));
    rv.ok = ld_ok;
    set_row_bounds(rv, P.n_rows, P.status);
    const bool loss = P.loss_part != nullptr;
    constexpr int H = VEC / 2;
    using CR = std::conditional_t<credits_in_smem<T, LC>(), CreditsSm<H>, Credits<H>>;
    CR cr0{};   // zero register sums, or the lane's shared-memory slots
    if constexpr (credits_in_smem<T, LC>())
        cr0.a = static_cast<uint32_t>(__cvta_generic_to_shared(lossbuf + 2 * 32 * VEC)) + lane * 16;

    LossSm<VEC> L;
    L.a = static_cast<uint32_t>(__cvta_generic_to_shared(lossbuf)) + lane * 16;
    if (loss) L.zero();

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
            AdamState<VPG> st;
            if constexpr (MODE == kModeAdam && C::PREFETCH) adam_prefetch<T, MODE, LC>(P, v, chunk, g, li, st);
            // otherwise ask the variable's Adam state into L2 now; it is loaded after the gathers
            if constexpr (MODE == kModeAdam && !C::PREFETCH) {
                const int c0p = chunk * C::BC + li * C::VEC + g * VPG;
                if (g < GE && c0p < P.B) {
                    const int64_t offp = static_cast<int64_t>(v) * P.ldB + c0p;
                    prefetch_l2(P.delta + offp);
                    prefetch_l2(P.m + offp);
                    prefetch_l2(P.v + offp);
                }
            }
            float gacc[VEC];
            CR cr = cr0;
            if (credits_in_smem<T, LC>() && loss) cr.zero();
            if (loss) {
                // the variable's own value (for its loss credits) is requested with the gathers
                uint4 own_raw = make_uint4(0u, 0u, 0u, 0u);
                if (ld_ok) own_raw = load_row(rv, static_cast<uint32_t>(v));
                var_gather<T, VEC, C::NB, true, false, (C::G == 1)>(it.kk, cd, cs, ce, ce, rv, gacc, cr);
                float xs[VEC];
                unpack<T>(own_raw, xs);
                credit_flush_v<VEC>(cr, xs, L);
            } else {
                var_gather<T, VEC, C::NB, false, false, (C::G == 1)>(it.kk, cd, cs, ce, ce, rv, gacc, cr);
            }
            group_sum<LC>(gacc);
            float ge[VPG];
#pragma unroll
            for (int el = 0; el < VPG; ++el) {
                float x = gacc[el];
#pragma unroll
                for (int q = 1; q < GE; ++q) x = (g == q) ? gacc[q * VPG + el] : x;
                ge[el] = x;
            }
            if constexpr (MODE == kModeAdam && !C::PREFETCH) adam_prefetch<T, MODE, LC>(P, v, chunk, g, li, st);
            var_epilogue<T, MODE, LC>(P, v, it.inst, chunk, g, li, lane, ge, st);
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
        float gacc[VEC];
        CR cr = cr0;
        if (credits_in_smem<T, LC>() && loss) cr.zero();
        if (loss) {
            var_gather<T, VEC, C::NB, true, false, (C::G == 1)>(it.kk, cd, cs, ce, ce, rv, gacc, cr);
            float xs[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) xs[e] = 0.0f;
            if (ld_ok) unpack<T>(load_row(rv, static_cast<uint32_t>(v)), xs);
            credit_flush_v<VEC>(cr, xs, L);
        } else {
            var_gather<T, VEC, C::NB, false, false, (C::G == 1)>(it.kk, cd, cs, ce, ce, rv, gacc, cr);
        }
        group_sum<LC>(gacc);
        float* rowp = P.split_part + static_cast<int64_t>(it.split_row + it.part) * P.bpad + lane_base;
        if (g == 0) {
#pragma unroll
            for (int e = 0; e < VEC; e += 4)
                __stcg(reinterpret_cast<float4*>(rowp + e), make_float4(gacc[e], gacc[e + 1], gacc[e + 2], gacc[e + 3]));
        }
        __threadfence();
        __syncwarp();
        int prev = 0;
        if (lane == 0) prev = atomicAdd(&P.split_cnt[static_cast<int64_t>(it.split) * P.n_chunks + chunk], 1);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev == it.n_parts - 1) {
            if (lane == 0) P.split_cnt[static_cast<int64_t>(it.split) * P.n_chunks + chunk] = 0;   // rewind
            __threadfence();
            float ge[VPG];
#pragma unroll
            for (int el = 0; el < VPG; ++el) ge[el] = 0.0f;
            if (g < GE) {
                const float* base = P.split_part + static_cast<int64_t>(it.split_row) * P.bpad + lane_base + g * VPG;
                for (int q = 0; q < it.n_parts; ++q) {
#pragma unroll
                    for (int el = 0; el < VPG; ++el) ge[el] += __ldcg(base + static_cast<int64_t>(q) * P.bpad + el);
                }
            }
            AdamState<VPG> st;
            if constexpr (MODE == kModeAdam) adam_prefetch<T, MODE, LC>(P, v, chunk, g, li, st);
            var_epilogue<T, MODE, LC>(P, v, it.inst, chunk, g, li, lane, ge, st);
        }
    }

    if (loss) {
        float lf[VEC], lc[VEC];
        L.load(lf, lc);
#pragma unroll
        for (int e = 0; e < VEC; ++e) lf[e] -= lc[e];
        group_sum<LC>(lf);
        if (g == 0) {
            float* dst = P.loss_part + static_cast<int64_t>(item) * P.bpad + lane_base;
#pragma unroll
            for (int e = 0; e < VEC; e += 4)
                __stcg(reinterpret_cast<float4*>(dst + e), make_float4(lf[e], lf[e + 1], lf[e + 2], lf[e + 3]));
        }
    }
}

// Register budget: float32 values run 3 CTAs (24 warps) per SM; 16-bit values hold twice the
// candidates per lane and run 3 CTAs per SM with one lane group per warp (credits in shared
// memory), 2 otherwise. Shared memory per warp: var_warp_bytes<T, LC>().
template <typename T, int MODE, int LC>
__global__ void __launch_bounds__(kThreads, (Elem<T>::VEC == 4 || credits_in_smem<T, LC>()) ? 3 : 2)
    k_var_pass(const VarParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LC, li = lane % LC;
    unsigned char* wbase = smem + warp * var_warp_bytes<T, LC>();
    using C = VarCfg<T, MODE, LC>;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + 2 * C::BUF_BYTES);
    float* lossbuf = reinterpret_cast<float*>(wbase + C::STAGE_BYTES);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int total = P.n_items * P.n_chunks;
    int w = fetch_work(P.head, lane);
    if (w < total && lane == 0) issue_var_item<T, MODE, LC>(P, w % P.n_items, wbase, &bars[0]);
    uint32_t phase[2] = {0u, 0u};
    int buf = 0;
    while (w < total) {
        const int wn = fetch_work(P.head, lane);
        if (wn < total && lane == 0) {
            fence_proxy_async();
            issue_var_item<T, MODE, LC>(P, wn % P.n_items, wbase + (buf ^ 1) * C::BUF_BYTES, &bars[buf ^ 1]);
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
        process_var_item<T, MODE, LC>(P, w, wbase + buf * C::BUF_BYTES, g, li, lane, lossbuf);
        __syncwarp();
        w = wn;
        buf ^= 1;
    }
    queue_exit(P.head, P.exit_cnt);
}

// ------------------------------------------------------------------------------------------
// Variable-major pass with variable-owning lane groups (chunks of LC < 32 lanes). The same
// arithmetic as k_var_pass, organised for small candidate rows: a work item is a run of whole
// variables of about a few thousand codes, listed largest first, and each of the G = 32 / LC
// lane groups of the warp takes every G-th of them and runs it start to end: occurrence loop,
// gradient, epilogue. The groups thus work on variables of similar size side by side; no group
// splits a variable, so nothing is reduced across groups per variable and a group's batches of
// gathers are only padded at the end of each of its variables. The codes are read straight from
// global memory (each group reads its variable's contiguous run; consecutive batches share
// cache lines).
template <typename T, int MODE, int LC>
__device__ __forceinline__ void own_epilogue(const VarParams& P, int v, int inst, int chunk, int li, uint32_t gmask,
                                             const float (&ge)[Elem<T>::VEC], const AdamState<Elem<T>::VEC>& st) {
    constexpr int VEC = Elem<T>::VEC;
    constexpr int BC = LC * VEC;
    const int c0 = chunk * BC + li * VEC;
    const bool act = c0 < P.B;
    const bool full = c0 + VEC <= P.B;
    const int64_t off = static_cast<int64_t>(v) * P.ldB + c0;
    if constexpr (MODE == kModeGrad) {
        if (act) {
            float out[VEC];
#pragma unroll
            for (int el = 0; el < VEC; ++el) {
                const float s = (P.dloss && c0 + el < P.B)
                                    ? static_cast<float>(P.dloss[static_cast<int64_t>(inst) * P.B + c0 + el])
                                    : 1.0f;
                out[el] = ge[el] * s;
            }
            if (full) {
                st_stream<VEC>(P.grad + off, out);
            } else {
                for (int el = 0; el < VEC && c0 + el < P.B; ++el) P.grad[off + el] = out[el];
            }
        }
    } else {
        uint32_t mybits = 0;
        if (act) {
            float d[VEC], mm[VEC], vv[VEC], xn[VEC];
#pragma unroll
            for (int el = 0; el < VEC; ++el) {
                d[el] = st.d[el];
                mm[el] = st.m[el];
                vv[el] = st.v[el];
            }
#pragma unroll
            for (int el = 0; el < VEC; ++el) {
                adam_update(ge[el], d[el], mm[el], vv[el], xn[el], P.adam);
                if (c0 + el < P.B && d[el] > 0.0f) mybits |= 1u << el;
            }
            T* xo = static_cast<T*>(P.x_out) + off;
            if (full) {
                st_stream<VEC>(P.delta + off, d);
                st_stream<VEC>(P.m + off, mm);
                st_stream<VEC>(P.v + off, vv);
                st_vals<T, VEC>(xo, xn);
            } else {
                for (int el = 0; el < VEC && c0 + el < P.B; ++el) {
                    P.delta[off + el] = d[el];
                    P.m[off + el] = mm[el];
                    P.v[off + el] = vv[el];
                    xo[el] = from_f32<T>(xn[el]);
                }
            }
        }
        if (P.bits32) {
            // lanes whose candidates share a 32-bit word OR their bits together (within the group)
            constexpr int LPW = (32 / VEC) < LC ? (32 / VEC) : LC;
            uint32_t word = mybits << (c0 & 31);
#pragma unroll
            for (int o = 1; o < LPW; o <<= 1) word |= __shfl_xor_sync(gmask, word, o);
            const int64_t row = static_cast<int64_t>(v) * 2 * P.nwd;
            const int hw = c0 >> 5;
            if (li % LPW == 0 && hw < 2 * P.nwd) P.bits32[row + hw] = word;
            if (li == 0 && chunk == P.n_chunks - 1) {
                for (int z = (P.n_chunks * BC + 31) >> 5; z < 2 * P.nwd; ++z) P.bits32[row + z] = 0u;
            }
        }
    }
}

template <typename T, int MODE, int LC>
__device__ __forceinline__ void process_own_item(const VarParams& P, int w, int g, int li, int lane, float* lossbuf) {
    constexpr int VEC = Elem<T>::VEC, G = 32 / LC, H = VEC / 2, BC = LC * VEC;
    // gathers in flight per batch: 8 per lane group; with the tile's loss sums in shared memory
    // the pass fits 80 registers and 3 CTAs (24 warps) per SM, which keeps more gathers in flight
    // per SM than 12-16 per batch at 2 CTAs (12.3 against 13.2 ms on the community workload)
    constexpr int NBL = 8, NBG = 8;
    const int item = w % P.n_items;
    const int chunk = w / P.n_items;
    const VarItem it = P.items[item];
    // the item's variables in the order the groups take them: group g takes entries g, g + G, ...
    const uint4* ent = reinterpret_cast<const uint4*>(P.vtab) + it.vtab_base;
    const uint32_t* cd = P.codes + it.code_base;
    const uint32_t gmask = (LC == 32) ? 0xffffffffu : (((1u << LC) - 1u) << (g * LC));
    const int lane_base = chunk * BC + li * VEC;
    const bool ld_ok = lane_base < P.B;
    RowView rv;
    rv.base = reinterpret_cast<const char*>(static_cast<const T*>(P.x_in) + lane_base);
    rv.row_bytes = static_cast<uint32_t>(P.ldB * sizeof(T));
    rv.ok = ld_ok;
    set_row_bounds(rv, P.n_rows, P.status);
    const bool loss = P.loss_part != nullptr;

    LossSm<VEC> L;
    L.a = static_cast<uint32_t>(__cvta_generic_to_shared(lossbuf)) + lane * 16;
    if (loss) L.zero();
    uint4 e = (g < it.nv) ? __ldg(ent + g) : make_uint4(0u, 0u, 0u, 0u);
    for (int j = g; j < it.nv; j += G) {
        const int v = it.v0 + static_cast<int>(e.x);
        const int cs = static_cast<int>(e.y), ce = static_cast<int>(e.z);
        // ahead of use: the group's next variable's entry and first codes (L1), this variable's
        // Adam state (L2; read after the gathers)
        const uint4 en = (j + G < it.nv) ? __ldg(ent + j + G) : e;
        if (j + G < it.nv) prefetch_l1(cd + en.y);
        if constexpr (MODE == kModeAdam) {
            if (ld_ok) {
                const int64_t off = static_cast<int64_t>(v) * P.ldB + lane_base;
                prefetch_l2(P.delta + off);
                prefetch_l2(P.m + off);
                prefetch_l2(P.v + off);
            }
        }
        float gacc[VEC];
        Credits<H> cr;
#pragma unroll
        for (int h = 0; h < H; ++h) cr.p[h] = cr.n[h] = dup2(0.0f);
        if (loss) {
            var_gather<T, VEC, NBL, true, true>(it.kk, cd, cs, ce, static_cast<int>(e.w), rv, gacc, cr);
            float xs[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) xs[e] = 0.0f;
            if (ld_ok) unpack<T>(load_row(rv, static_cast<uint32_t>(v)), xs);
            credit_flush_v<VEC>(cr, xs, L);
        } else {
            var_gather<T, VEC, NBG, false, true>(it.kk, cd, cs, ce, ce, rv, gacc, cr);
        }
        AdamState<VEC> st;
        if constexpr (MODE == kModeAdam) {
            const int64_t off = static_cast<int64_t>(v) * P.ldB + lane_base;
            if (ld_ok && lane_base + VEC <= P.B) {
                ld_stream<VEC>(P.delta + off, st.d);
                ld_stream<VEC>(P.m + off, st.m);
                ld_stream<VEC>(P.v + off, st.v);
            } else {
#pragma unroll
                for (int el = 0; el < VEC; ++el) {
                    const bool ok = lane_base + el < P.B;
                    st.d[el] = ok ? P.delta[off + el] : 0.0f;
                    st.m[el] = ok ? P.m[off + el] : 0.0f;
                    st.v[el] = ok ? P.v[off + el] : 0.0f;
                }
            }
        }
        own_epilogue<T, MODE, LC>(P, v, it.inst, chunk, li, gmask, gacc, st);
        e = en;
    }
    __syncwarp();
    if (loss) {
        float lf[VEC], lc[VEC];
        L.load(lf, lc);
#pragma unroll
        for (int e = 0; e < VEC; ++e) lf[e] -= lc[e];
        group_sum<LC>(lf);
        if (g == 0) {
            float* dst = P.loss_part + static_cast<int64_t>(item) * P.bpad + lane_base;
#pragma unroll
            for (int e = 0; e < VEC; e += 4)
                __stcg(reinterpret_cast<float4*>(dst + e), make_float4(lf[e], lf[e + 1], lf[e + 2], lf[e + 3]));
        }
    }
}

template <typename T, int MODE, int LC>
__global__ void __launch_bounds__(kThreads, 3) k_var_own(const VarParams P) {
    __shared__ __align__(16) float own_loss[kWarps][2 * 32 * Elem<T>::VEC];   // per warp: LossSm
    const int lane = threadIdx.x & 31;
    const int g = lane / LC, li = lane % LC;
    const int total = P.n_items * P.n_chunks;
    for (int w = fetch_work(P.head, lane); w < total; w = fetch_work(P.head, lane)) {
        process_own_item<T, MODE, LC>(P, w, g, li, lane, own_loss[threadIdx.x >> 5]);
        __syncwarp();
    }
    queue_exit(P.head, P.exit_cnt);
}

// ------------------------------------------------------------------------------------------
// Variable-major pass with TMA gathers (chunks of 32 lanes). The relaxed-value rows named by a
// tile's occurrence codes are fetched four at a time by cp.async.bulk.tensor ... tile::gather4
// into a per-warp ring of shared-memory slots, each completing on its own mbarrier, so many rows
// are in flight per warp without occupying registers; lanes read their 16-byte slice of each
// row from shared memory. A slot is refilled with the group kRingSlots ahead as soon as its four
// codes have been consumed.
__device__ __forceinline__ void gather4(void* dst, const CUtensorMap* tm, int col, int r0, int r1, int r2, int r3,
                                        uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

struct Ring {
    unsigned char* slots;
    uint64_t* bars;
    uint32_t phase;   // bit k: parity of slot k's next completion
    int pend_lo;      // after a failed wait: groups [pend_lo, pend_hi) still have copies in flight
    int pend_hi;
};

// Issues group g (codes 4g .. 4g+3 of the staged tile) into slot g % kRingSlots (lane 0 only).
__device__ __forceinline__ void ring_issue(Ring& r, const CUtensorMap* tm, const uint32_t* cd, int n_codes, int g,
                                           int col, uint32_t bytes) {
    int rows[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ci = 4 * g + i;
        const uint32_t u = (ci < n_codes) ? (cd[ci] >> kVShift) : kVSentinel;
        rows[i] = (u == kVSentinel) ? 0 : static_cast<int>(u);
    }
    const int slot = g % kRingSlots;
    fence_proxy_async();
    mbar_expect_tx(&r.bars[slot], bytes);
    gather4(r.slots + slot * kSlotBytes, tm, col, rows[0], rows[1], rows[2], rows[3], &r.bars[slot]);
}

template <typename T, int MODE>
__device__ __forceinline__ bool process_var_ring(const VarParams& P, const CUtensorMap* tm, int w,
                                                 const unsigned char* buf, Ring& ring, int lane) {
    using C = VarCfg<T, MODE, 32>;
    constexpr int VEC = C::VEC, H = VEC / 2, VPG = C::VPG;
    const int item = w % P.n_items;
    const int chunk = w / P.n_items;
    const VarItem it = P.items[item];
    const uint32_t* vt =
        reinterpret_cast<const uint32_t*>(buf + (reinterpret_cast<uintptr_t>(P.vtab + it.vtab_base) & 15));
    const uint32_t* cd = reinterpret_cast<const uint32_t*>(
        buf + C::CODE_OFF + (reinterpret_cast<uintptr_t>(P.codes + it.code_base) & 15));
    const int cand0 = chunk * C::BC;
    const int lane_base = cand0 + lane * VEC;
    const bool ld_ok = lane_base < P.B;
    const T* xcol = static_cast<const T*>(P.x_in) + lane_base;
    const bool loss = P.loss_part != nullptr;
    const int n_codes = it.n_codes;
    const int n_groups = (n_codes + 3) >> 2;
    const uint32_t bytes = 4u * kRowBytes;

    int issued = 0;
    if (lane == 0)
        for (int g = 0; g < n_groups && g < kRingSlots; ++g) ring_issue(ring, tm, cd, n_codes, g, cand0, bytes);
    issued = n_groups < kRingSlots ? n_groups : kRingSlots;

    float Ls[VEC], Lc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) Ls[e] = Lc[e] = 0.0f;
    int c = 0;
    const int nv = (it.split < 0) ? it.nv : 1;
    bool ok = true;
    for (int vi = 0; vi < nv; ++vi) {
        const int v = it.v0 + vi;
        const int ce = (it.split < 0) ? static_cast<int>(vt[vi + 1] & 0xffffu) : n_codes;
        float xs[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) xs[e] = 0.0f;
        if (loss && ld_ok && row_ok(v, P.n_rows, P.status)) unpack<T>(ld_gather16(xcol + static_cast<int64_t>(v) * P.ldB), xs);
        AdamState<VPG> st;
        if constexpr (MODE == kModeAdam)
            if (it.split < 0) adam_prefetch<T, MODE, 32>(P, v, chunk, 0, lane, st);
        float2 R[H], G2[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            R[h] = dup2(1.0f);
            G2[h] = dup2(0.0f);
        }
        for (; c < ce; ++c) {
            const int slot = (c >> 2) % kRingSlots;
            if ((c & 3) == 0) {
                const bool got = mbar_wait_bounded(&ring.bars[slot], (ring.phase >> slot) & 1u, kWaitNs);
                if (!__all_sync(0xffffffffu, got)) {
                    ring.pend_lo = c >> 2;
                    ring.pend_hi = issued;
                    ok = false;
                    break;
                }
                ring.phase ^= 1u << slot;
            }
            const uint4 raw = *reinterpret_cast<const uint4*>(ring.slots + slot * kSlotBytes + (c & 3) * kRowBytes +
                                                              lane * 16);
            float xv[VEC];
            unpack<T>(raw, xv);
            const uint32_t code = cd[c];
            float a, b;
            code_ab(code, a, b);
            const bool end = (code & kVEnd) != 0u;
            const float sg = end ? ((code & kVSelfNeg) ? 1.0f : -1.0f) : 0.0f;
            float2 rn[H];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                rn[h] = __fmul2_rn(R[h], __ffma2_rn(dup2(a), make_float2(xv[2 * h], xv[2 * h + 1]), dup2(b)));
                G2[h] = __ffma2_rn(dup2(sg), rn[h], G2[h]);
                R[h] = end ? dup2(1.0f) : rn[h];
            }
            if (loss && (code & kVCredit)) {
                const bool sneg = (code & kVSelfNeg) != 0u;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    kahan_add(Ls[2 * h], Lc[2 * h], (sneg ? xs[2 * h] : 1.0f - xs[2 * h]) * rn[h].x);
                    kahan_add(Ls[2 * h + 1], Lc[2 * h + 1], (sneg ? xs[2 * h + 1] : 1.0f - xs[2 * h + 1]) * rn[h].y);
                }
            }
            if ((c & 3) == 3) {   // group done: its slot takes the group kRingSlots ahead
                __syncwarp();
                if (lane == 0 && issued < n_groups) ring_issue(ring, tm, cd, n_codes, issued, cand0, bytes);
                if (issued < n_groups) ++issued;
            }
        }
        if (!ok) break;
        float gacc[VEC];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            gacc[2 * h] = G2[h].x;
            gacc[2 * h + 1] = G2[h].y;
        }
        if (it.split < 0) {
            var_epilogue<T, MODE, 32>(P, v, it.inst, chunk, 0, lane, lane, gacc, st);
        } else {
            float* rowp = P.split_part + static_cast<int64_t>(it.split_row + it.part) * P.bpad + lane_base;
#pragma unroll
            for (int e = 0; e < VEC; e += 4)
                __stcg(reinterpret_cast<float4*>(rowp + e), make_float4(gacc[e], gacc[e + 1], gacc[e + 2], gacc[e + 3]));
            __threadfence();
            __syncwarp();
            int prev = 0;
            if (lane == 0) prev = atomicAdd(&P.split_cnt[static_cast<int64_t>(it.split) * P.n_chunks + chunk], 1);
            prev = __shfl_sync(0xffffffffu, prev, 0);
            if (prev == it.n_parts - 1) {
                if (lane == 0) P.split_cnt[static_cast<int64_t>(it.split) * P.n_chunks + chunk] = 0;   // rewind
                __threadfence();
                float ge[VPG];
#pragma unroll
                for (int el = 0; el < VPG; ++el) ge[el] = 0.0f;
                const float* base = P.split_part + static_cast<int64_t>(it.split_row) * P.bpad + lane_base;
                for (int q = 0; q < it.n_parts; ++q) {
#pragma unroll
                    for (int el = 0; el < VPG; ++el) ge[el] += __ldcg(base + static_cast<int64_t>(q) * P.bpad + el);
                }
                if constexpr (MODE == kModeAdam) adam_prefetch<T, MODE, 32>(P, v, chunk, 0, lane, st);
                var_epilogue<T, MODE, 32>(P, v, it.inst, chunk, 0, lane, lane, ge, st);
            }
        }
    }
    if (!ok) return false;
    if (loss) {
        float* dst = P.loss_part + static_cast<int64_t>(item) * P.bpad + lane_base;
#pragma unroll
        for (int e = 0; e < VEC; e += 4)
            __stcg(reinterpret_cast<float4*>(dst + e), make_float4(Ls[e] - Lc[e], Ls[e + 1] - Lc[e + 1],
                                                                   Ls[e + 2] - Lc[e + 2], Ls[e + 3] - Lc[e + 3]));
    }
    return true;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kRingWarps * 32) k_var_ring(const VarParams P, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wbase = smem + warp * kRingWarpBytes;
    Ring ring;
    ring.slots = wbase;
    unsigned char* ibuf = wbase + kRingSlots * kSlotBytes;
    uint64_t* ibars = reinterpret_cast<uint64_t*>(ibuf + 2 * kVarBufBytes);
    ring.bars = ibars + 2;
    ring.phase = 0u;
    if (lane == 0) {
        mbar_init(&ibars[0], 1);
        mbar_init(&ibars[1], 1);
        for (int k = 0; k < kRingSlots; ++k) mbar_init(&ring.bars[k], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int total = P.n_items * P.n_chunks;
    int w = fetch_work(P.head, lane);
    if (w < total && lane == 0) issue_var_item<T, MODE, 32>(P, w % P.n_items, ibuf, &ibars[0]);
    uint32_t phase[2] = {0u, 0u};
    int buf = 0;
    while (w < total) {
        const int wn = fetch_work(P.head, lane);
        if (wn < total && lane == 0) {
            fence_proxy_async();
            issue_var_item<T, MODE, 32>(P, wn % P.n_items, ibuf + (buf ^ 1) * kVarBufBytes, &ibars[buf ^ 1]);
        }
        ring.pend_lo = ring.pend_hi = 0;
        bool idx_ok = mbar_wait_bounded(&ibars[buf], phase[buf], kWaitNs);
        idx_ok = __all_sync(0xffffffffu, idx_ok);
        bool ok = idx_ok;
        if (idx_ok) {
            phase[buf] ^= 1u;
            ok = process_var_ring<T, MODE>(P, &tm, w, ibuf + buf * kVarBufBytes, ring, lane);
        }
        if (!__all_sync(0xffffffffu, ok)) {
            // a bounded wait gave up: record it, let this warp's copies in flight land (each wait
            // bounded again), stop
            if (lane == 0) {
                atomicOr(P.status, kStatusTimeout);
                if (!idx_ok) mbar_wait_bounded(&ibars[buf], phase[buf], kWaitNs);
                if (wn < total) mbar_wait_bounded(&ibars[buf ^ 1], phase[buf ^ 1], kWaitNs);
                for (int g = ring.pend_lo; g < ring.pend_hi; ++g) {
                    const int k = g % kRingSlots;
                    mbar_wait_bounded(&ring.bars[k], (ring.phase >> k) & 1u, kWaitNs);
                    ring.phase ^= 1u << k;
                }
            }
            __syncwarp();
            break;
        }
        __syncwarp();
        w = wn;
        buf ^= 1;
    }
    queue_exit(P.head, P.exit_cnt);
}

// ------------------------------------------------------------------------------------------
// Forward (clause-major): per (clause, candidate) U_t = prod_i f_i, summed per tile.
template <typename T, int VEC, int NB>
__device__ __forceinline__ void fwd_slots(const uint32_t* cd, int cs, int ce, const T* xcol, int64_t ldB, bool ld_ok,
                                          int64_t n_rows, int32_t* status, float (&Ls)[VEC], float (&Lc)[VEC]) {
    constexpr uint32_t kPad = 0xffffffffu;
    float R[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) R[e] = 1.0f;
    for (int s = cs; s < ce; s += NB) {
        uint32_t cw[NB];
        uint4 raw[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) cw[j] = (s + j < ce) ? cd[s + j] : kPad;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            raw[j] = make_uint4(0u, 0u, 0u, 0u);
            if (ld_ok && cw[j] != kPad && row_ok(cw[j] >> kFShift, n_rows, status))
                raw[j] = ld_gather16(xcol + static_cast<int64_t>(cw[j] >> kFShift) * ldB);
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const uint32_t c = cw[j];
            const bool pad = (c == kPad);   // raw is zero: factor b = 1
            const float a = pad ? 0.0f : ((c & kFNeg) ? 1.0f : -1.0f);
            const float b = pad ? 1.0f : ((c & kFNeg) ? 0.0f : 1.0f);
            const bool end = !pad && (c & kFEnd);
            float2 f[VEC / 2];
            factors<T>(raw[j], a, b, f);
#pragma unroll
            for (int e = 0; e < VEC; e += 2) {
                R[e] *= f[e / 2].x;
                R[e + 1] *= f[e / 2].y;
            }
            if (end) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    kahan_add(Ls[e], Lc[e], R[e]);
                    R[e] = 1.0f;
                }
            }
        }
    }
}

__device__ __forceinline__ void issue_fwd_item(const FwdItem* items, const uint32_t* codes, const uint16_t* ctab,
                                               int item, unsigned char* buf, uint64_t* bar) {
    const FwdItem it = items[item];
    const Span a = span16(ctab + it.ctab_base, static_cast<uint32_t>(it.n_clauses + 1) * 2u);
    const Span c = span16(codes + it.code_base, static_cast<uint32_t>(it.n_codes) * 4u);
    mbar_expect_tx(bar, a.bytes + c.bytes);
    if (a.bytes) bulk_g2s(buf, reinterpret_cast<const void*>(a.src), a.bytes, bar);
    if (c.bytes) bulk_g2s(buf + kFwdCtabBytes, reinterpret_cast<const void*>(c.src), c.bytes, bar);
}

template <typename T, int LC>
__global__ void __launch_bounds__(kThreads) k_forward(const FwdParams P) {
    constexpr int VEC = Elem<T>::VEC, G = 32 / LC, BC = LC * VEC, NB = (VEC == 4) ? 8 : 4;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LC, li = lane % LC;
    unsigned char* wbase = smem + warp * kFwdWarpBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + 2 * kFwdBufBytes);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int total = P.n_items * P.n_chunks;
    int w = fetch_work(P.head, lane);
    if (w < total && lane == 0) issue_fwd_item(P.items, P.codes, P.ctab, w % P.n_items, wbase, &bars[0]);
    uint32_t phase[2] = {0u, 0u};
    int buf = 0;
    while (w < total) {
        const int wn = fetch_work(P.head, lane);
        if (wn < total && lane == 0) {
            fence_proxy_async();
            issue_fwd_item(P.items, P.codes, P.ctab, wn % P.n_items, wbase + (buf ^ 1) * kFwdBufBytes, &bars[buf ^ 1]);
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
        {
            const unsigned char* b = wbase + buf * kFwdBufBytes;
            const int item = w % P.n_items;
            const int chunk = w / P.n_items;
            const FwdItem it = P.items[item];
            const uint16_t* ct =
                reinterpret_cast<const uint16_t*>(b + (reinterpret_cast<uintptr_t>(P.ctab + it.ctab_base) & 15));
            const uint32_t* cd = reinterpret_cast<const uint32_t*>(
                b + kFwdCtabBytes + (reinterpret_cast<uintptr_t>(P.codes + it.code_base) & 15));
            const int nc = it.n_clauses;
            const int cs = ct[(nc * g) / G];
            const int ce = ct[(nc * (g + 1)) / G];
            const int lane_base = chunk * BC + li * VEC;
            const bool ld_ok = lane_base < P.B;
            const T* xcol = static_cast<const T*>(P.x) + lane_base;
            float Ls[VEC], Lc[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) Ls[e] = Lc[e] = 0.0f;
            fwd_slots<T, VEC, NB>(cd, cs, ce, xcol, P.ldB, ld_ok, P.n_rows, P.status, Ls, Lc);
            float lf[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) lf[e] = Ls[e] - Lc[e];
            group_sum<LC>(lf);
            if (g == 0) {
                float* dst = P.loss_part + static_cast<int64_t>(item) * P.bpad + lane_base;
#pragma unroll
                for (int e = 0; e < VEC; e += 4)
                    __stcg(reinterpret_cast<float4*>(dst + e), make_float4(lf[e], lf[e + 1], lf[e + 2], lf[e + 3]));
            }
        }
        __syncwarp();
        w = wn;
        buf ^= 1;
    }
    queue_exit(P.head, P.exit_cnt);
}

// ------------------------------------------------------------------------------------------
// Exact check on bit-packed rounded assignments: per clause, sat = OR_i (literal true) over 64
// candidates per word; the unsat words of a tile are added into 64 bit-sliced counters per lane
// (a tile has <= 256 clauses, so 9 planes), combined across lane groups, and written as one
// uint16 count per (tile, candidate). A fixed-order reduction over tiles follows; no atomics.
constexpr int kPlanes = 9;

template <int LW, typename W>
__global__ void __launch_bounds__(kThreads) k_check(const CheckParams P) {
    constexpr int G = 32 / LW, NB = 8;
    constexpr int WB = 8 * static_cast<int>(sizeof(W));   // candidates per word
    const W* bitsw = static_cast<const W*>(P.bits);
    constexpr uint32_t kPad = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LW, li = lane % LW;
    unsigned char* wbase = smem + warp * kFwdWarpBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + 2 * kFwdBufBytes);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int total = P.n_items * P.n_wchunks;
    // 32-bit words (B <= 32): each warp takes a fixed contiguous range of tiles instead of
    // pulling from the queue, so a CTA's warps work on neighbouring tiles (with tiles sorted by
    // median row, the same rows); the kernel runs 3 CTAs per SM and leaves the rest of the
    // SM's memory to L1, where those rows' compact words stay (community formula: 1.78 ->
    // 0.79 ms per check)
    constexpr bool STATIC = sizeof(W) == 4;
    const int gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    const int per = (total + nw - 1) / nw;
    const int w_end = min(total, (gw + 1) * per);
    auto next_w = [&](int cur) -> int {
        if constexpr (STATIC) return (cur + 1 < w_end) ? cur + 1 : total;
        else return fetch_work(P.head, lane);
    };
    int w = STATIC ? ((gw * per < total) ? gw * per : total) : fetch_work(P.head, lane);
    if (w < total && lane == 0) issue_fwd_item(P.items, P.codes, P.ctab, w % P.n_items, wbase, &bars[0]);
    uint32_t phase[2] = {0u, 0u};
    int buf = 0;
    while (w < total) {
        const int wn = next_w(w);
        if (wn < total && lane == 0) {
            fence_proxy_async();
            issue_fwd_item(P.items, P.codes, P.ctab, wn % P.n_items, wbase + (buf ^ 1) * kFwdBufBytes, &bars[buf ^ 1]);
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
        {
            const unsigned char* b = wbase + buf * kFwdBufBytes;
            const int item = w % P.n_items;
            const int wchunk = w / P.n_items;
            const FwdItem it = P.items[item];
            const int wd = wchunk * LW + li;
            const uint16_t* ct =
                reinterpret_cast<const uint16_t*>(b + (reinterpret_cast<uintptr_t>(P.ctab + it.ctab_base) & 15));
            const uint32_t* cd = reinterpret_cast<const uint32_t*>(
                b + kFwdCtabBytes + (reinterpret_cast<uintptr_t>(P.codes + it.code_base) & 15));
            const int nc = it.n_clauses;
            const int cs = ct[(nc * g) / G];
            const int ce = ct[(nc * (g + 1)) / G];
            const bool ok_w = wd < P.nwd;
            const int rem = P.B - wd * WB;
            const W vmask = (!ok_w || rem <= 0) ? W(0) : (rem >= WB ? ~W(0) : static_cast<W>((W(1) << rem) - W(1)));
            W planes[kPlanes];
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) planes[p] = W(0);
            W acc = W(0);
            if constexpr (G >= 8) {
                // narrow words (many lane groups): group g takes clauses g, g + G, ... so that the
                // groups' code reads fall on different shared-memory banks
                for (int c = g; c < nc; c += G) {
                    const int a = ct[c], e = ct[c + 1];
                    if (a == e) continue;   // empty clauses are counted per instance
                    acc = W(0);
                    for (int s = a; s < e; s += NB) {
                        uint32_t cw[NB];
                        W x[NB];
#pragma unroll
                        for (int j = 0; j < NB; ++j) cw[j] = (s + j < e) ? cd[s + j] : kPad;
#pragma unroll
                        for (int j = 0; j < NB; ++j)
                            x[j] = (ok_w && cw[j] != kPad && row_ok(cw[j] >> kFShift, P.n_rows, P.status))
                                       ? __ldg(bitsw + static_cast<int64_t>(cw[j] >> kFShift) * P.nwd + wd)
                                       : W(0);
#pragma unroll
                        for (int j = 0; j < NB; ++j)
                            if (cw[j] != kPad) acc |= (cw[j] & kFNeg) ? ~x[j] : x[j];
                    }
                    W carry = static_cast<W>(~acc & vmask);
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) {
                        const W t = planes[p] & carry;
                        planes[p] ^= carry;
                        carry = t;
                    }
                }
            }
            for (int s = (G >= 8) ? ce : cs; s < ce; s += NB) {
                uint32_t cw[NB];
                W x[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) cw[j] = (s + j < ce) ? cd[s + j] : kPad;
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    x[j] = (ok_w && cw[j] != kPad && row_ok(cw[j] >> kFShift, P.n_rows, P.status))
                               ? __ldg(bitsw + static_cast<int64_t>(cw[j] >> kFShift) * P.nwd + wd)
                               : W(0);
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const uint32_t c = cw[j];
                    if (c == kPad) continue;
                    acc |= (c & kFNeg) ? ~x[j] : x[j];
                    if (c & kFEnd) {
                        W carry = static_cast<W>(~acc & vmask);
                        acc = W(0);
#pragma unroll
                        for (int p = 0; p < kPlanes; ++p) {
                            const W t = planes[p] & carry;
                            planes[p] ^= carry;
                            carry = t;
                        }
                    }
                }
            }
#pragma unroll
            for (int off = LW; off < 32; off <<= 1) {
                W carry = W(0);
#pragma unroll
                for (int p = 0; p < kPlanes; ++p) {
                    const W a = planes[p];
                    const W o = __shfl_xor_sync(0xffffffffu, a, off);
                    const W sum = a ^ o ^ carry;
                    carry = (a & o) | (carry & (a ^ o));
                    planes[p] = sum;
                }
            }
            if (ok_w) {
                // every lane group now holds the word's totals: group g turns its WB / G of the
                // word's WB counts into uint16 (pairs packed in uint32) and stores them
                constexpr int PER = WB / G;
                const int c0 = g * PER;
                uint16_t* dst16 = P.part16 + static_cast<int64_t>(item) * P.bpad16 + wd * WB + c0;
                auto pair = [&](int b0) -> uint32_t {
                    uint32_t a = 0, b = 0;
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) {
                        a |= static_cast<uint32_t>((planes[p] >> b0) & W(1)) << p;
                        b |= static_cast<uint32_t>((planes[p] >> (b0 + 1)) & W(1)) << p;
                    }
                    return a | (b << 16);
                };
                if constexpr (PER >= 8) {
                    uint4* dst = reinterpret_cast<uint4*>(dst16);
#pragma unroll
                    for (int q = 0; q < PER / 8; ++q)
                        dst[q] = make_uint4(pair(c0 + 8 * q), pair(c0 + 8 * q + 2), pair(c0 + 8 * q + 4),
                                            pair(c0 + 8 * q + 6));
                } else if constexpr (PER >= 2) {
                    uint32_t* dst = reinterpret_cast<uint32_t*>(dst16);
#pragma unroll
                    for (int q = 0; q < PER / 2; ++q) dst[q] = pair(c0 + 2 * q);
                } else {
                    uint32_t a = 0;
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) a |= static_cast<uint32_t>((planes[p] >> c0) & W(1)) << p;
                    *dst16 = static_cast<uint16_t>(a);
                }
            }
        }
        __syncwarp();
        w = wn;
        buf ^= 1;
    }
    queue_exit(P.head, P.exit_cnt);
}

// Low 32-bit word of each row of a bit-packed assignment (the candidates 0..31), for the check
// of batches of at most 32 candidates: half the bytes a check gathers per literal.
__global__ void __launch_bounds__(256) k_compact_low32(const uint64_t* bits, int64_t n, int32_t nwd, uint32_t* out) {
    for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[v] = static_cast<uint32_t>(__ldcs(bits + v * nwd));
}

// ------------------------------------------------------------------------------------------
// Two-stage fixed-order reductions of per-tile partials over the tiles of each instance.
// Stage 1: block (candidate slice of 32, instance, segment s) sums the segment's tiles (its 8
// warps take tiles round-robin, then combine in warp order). Stage 2 sums the segments in order.
template <typename PT, typename AT>
__global__ void __launch_bounds__(256) k_reduce_tiles(const PT* part, int32_t stride, const int32_t* iptr,
                                                      const int32_t* items, int32_t B, int32_t n_seg, AT* stage) {
    __shared__ AT red[8][32];
    const int inst = blockIdx.y, seg = blockIdx.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    const int a = iptr[inst], e = iptr[inst + 1];
    const int len = e - a;
    const int per = (len + n_seg - 1) / n_seg;
    const int k0 = a + seg * per;
    const int k1 = min(e, k0 + per);
    AT s = AT(0);
    if (b < B) {
#pragma unroll 4
        for (int k = k0 + warp; k < k1; k += 8) s += static_cast<AT>(part[static_cast<int64_t>(items[k]) * stride + b]);
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && b < B) {
        AT t = AT(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[q][lane];
        stage[(static_cast<int64_t>(seg) * gridDim.y + inst) * B + b] = t;
    }
}

// Stage 2 of the loss: block (32-candidate slice, instance); its 32 warps sum the segments
// round-robin, then combine in warp order; empty clauses (product 1 each) are added.
__global__ void __launch_bounds__(1024) k_loss_final(const double* stage, int32_t n_seg, int32_t n_inst,
                                                     const int64_t* n_empty, int32_t B, double* loss) {
    __shared__ double red[32][32];
    const int inst = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    double t = 0.0;
    if (b < B) {
#pragma unroll 4
        for (int sgm = warp; sgm < n_seg; sgm += 32) t += stage[(static_cast<int64_t>(sgm) * n_inst + inst) * B + b];
    }
    red[warp][lane] = t;
    __syncthreads();
    if (warp == 0 && b < B) {
        double u = 0.0;
#pragma unroll
        for (int q = 0; q < 32; ++q) u += red[q][lane];
        loss[static_cast<int64_t>(inst) * B + b] = u + static_cast<double>(n_empty[inst]);
    }
}

// Per instance: unsat = sum of the segments + empty clauses (always unsatisfied); best = the
// lowest candidate with the fewest unsatisfied clauses.
__global__ void __launch_bounds__(1024) k_count_final(const int32_t* stage, int32_t n_seg, int32_t n_inst,
                                                      const int64_t* n_empty, int32_t B, int32_t* unsat,
                                                      int32_t* best) {
    __shared__ unsigned long long red[1024];
    const int inst = blockIdx.x;
    const int32_t add = static_cast<int32_t>(n_empty[inst]);
    unsigned long long key = ~0ull;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        int32_t c = add;
#pragma unroll 8
        for (int sgm = 0; sgm < n_seg; ++sgm) c += stage[(static_cast<int64_t>(sgm) * n_inst + inst) * B + b];
        unsat[static_cast<int64_t>(inst) * B + b] = c;
        const unsigned long long k = (static_cast<unsigned long long>(static_cast<uint32_t>(c)) << 32) |
                                     static_cast<uint32_t>(b);
        key = k < key ? k : key;
    }
    red[threadIdx.x] = key;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st && red[threadIdx.x + st] < red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0 && best) best[inst] = (B > 0) ? static_cast<int32_t>(red[0] & 0xffffffffull) : -1;
}

// ------------------------------------------------------------------------------------------
// Relaxed values x = sigma(delta / tau), written as T: one thread per 4 consecutive candidates of
// a row (16-byte loads; the row stride keeps every group aligned), scalar tail past B.
template <typename T>
__global__ void __launch_bounds__(256) k_relax(const float* delta, T* x, int64_t n, int32_t B, int64_t ldB,
                                               float inv_tau) {
    const int64_t groups = (B + 3) / 4;
    const int64_t total = n * groups;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = i / groups, b = (i - v * groups) * 4;
        const int64_t o = v * ldB + b;
        if (b + 4 <= B) {
            float d[4], y[4];
            ld_stream<4>(delta + o, d);
#pragma unroll
            for (int e = 0; e < 4; ++e) y[e] = sigmoid(d[e] * inv_tau);
            st_vals<T, 4>(x + o, y);
        } else {
            for (int64_t e = b; e < B; ++e) x[v * ldB + e] = from_f32<T>(sigmoid(delta[v * ldB + e] * inv_tau));
        }
    }
}

// Rounding (Eq. 4): bit b of row v = (delta[v][b] > 0), 32 candidates per warp ballot.
__global__ void __launch_bounds__(256) k_round(const float* delta, uint32_t* bits32, int64_t n, int32_t B, int64_t ldB,
                                               int32_t nwd) {
    const int lane = threadIdx.x & 31;
    const int64_t halves = 2LL * nwd;
    const int64_t total = n * halves;
    for (int64_t wi = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5; wi < total;
         wi += (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5) {
        const int64_t v = wi / halves, h = wi - v * halves;
        const int64_t b = h * 32 + lane;
        const bool bit = (b < B) && (delta[v * ldB + b] > 0.0f);
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) bits32[v * halves + h] = word;
    }
}

// Standalone Adam update from an external gradient dL/dx.
template <typename T>
__global__ void __launch_bounds__(256) k_adam(float* delta, float* m, float* v, const float* grad, T* x_out, int64_t n,
                                              int32_t B, int64_t ldB, const AdamK k) {
    const int64_t total = n * B;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / B, b = i - r * B;
        const int64_t o = r * ldB + b;
        float d = delta[o], mm = m[o], vv = v[o], xn;
        adam_update(grad[o], d, mm, vv, xn, k);
        delta[o] = d;
        m[o] = mm;
        v[o] = vv;
        if (x_out) x_out[o] = from_f32<T>(xn);
    }
}

// Self-test of the bounded-wait path: waits on an mbarrier phase that nothing completes (one
// expected arrival, none made, no copy issued), gives up after limit_ns and records the timeout
// in the status word. Nothing is in flight when it returns.
__global__ void k_wait_selftest(int32_t* status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

// ------------------------------------------------------------------------------------------
template <typename T, int MODE, int LC>
int var_grid_t() {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_var_pass<T, MODE, LC>, kWarps * var_warp_bytes<T, LC>());
    return grid;
}
template <typename T, int MODE>
int ring_grid_t() {
    static int grid = 0;
    if (!grid) {
        const int smem = kRingWarps * kRingWarpBytes;
        auto kernel = k_var_ring<T, MODE>;
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRingWarps * 32, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        grid = per_sm * sm_count();
    }
    return grid;
}
template <typename T, int LC>
int fwd_grid_t() {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_forward<T, LC>, kWarps * kFwdWarpBytes);
    return grid;
}
template <int LW, typename W>
int check_grid_t() {
    static int grid = 0;
    if (!grid) {
        if constexpr (sizeof(W) == 4) {
            // three CTAs per SM (126 KB of staging buffers) and a 57 % shared-memory carve-out
            // (the 132 KB configuration): the other 124 KB of the SM's memory is L1 for the
            // gathered words (community formula: 0.79 ms per check, against 0.84 with two CTAs
            // and 152 KB of L1, 0.97 with four and 60 KB)
            auto kernel = k_check<LW, W>;
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWarps * kFwdWarpBytes);
            cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 57);
            grid = 3 * sm_count();
        } else {
            grid = persistent_grid(k_check<LW, W>, kWarps * kFwdWarpBytes);
        }
    }
    return grid;
}

template <typename T, int MODE, int LC>
int own_grid_t() {
    static int grid = 0;
    if (!grid) grid = persistent_grid(k_var_own<T, MODE, LC>, 0);
    return grid;
}
template <typename T, int MODE>
int own_grid_lc(int lc) {
    switch (lc) {
        case 16: return own_grid_t<T, MODE, 16>();
        case 8: return own_grid_t<T, MODE, 8>();
        default: return own_grid_t<T, MODE, 4>();
    }
}
template <typename T, int MODE>
cudaError_t own_launch_lc(const VarParams& p, int lc, int grid, cudaStream_t s) {
    switch (lc) {
        case 16: own_grid_t<T, MODE, 16>(); k_var_own<T, MODE, 16><<<grid, kThreads, 0, s>>>(p); break;
        case 8: own_grid_t<T, MODE, 8>(); k_var_own<T, MODE, 8><<<grid, kThreads, 0, s>>>(p); break;
        default: own_grid_t<T, MODE, 4>(); k_var_own<T, MODE, 4><<<grid, kThreads, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

template <typename T, int MODE>
int var_grid_lc(int lc) {
    switch (lc) {
        case 32: return var_grid_t<T, MODE, 32>();
        case 16: return var_grid_t<T, MODE, 16>();
        case 8: return var_grid_t<T, MODE, 8>();
        default: return var_grid_t<T, MODE, 4>();
    }
}
template <typename T, int MODE>
cudaError_t var_launch_lc(const VarParams& p, int lc, int grid, cudaStream_t s) {
    constexpr int W = kWarps;
    switch (lc) {
        case 32:
            var_grid_t<T, MODE, 32>();
            k_var_pass<T, MODE, 32><<<grid, kThreads, W * var_warp_bytes<T, 32>(), s>>>(p);
            break;
        case 16:
            var_grid_t<T, MODE, 16>();
            k_var_pass<T, MODE, 16><<<grid, kThreads, W * var_warp_bytes<T, 16>(), s>>>(p);
            break;
        case 8:
            var_grid_t<T, MODE, 8>();
            k_var_pass<T, MODE, 8><<<grid, kThreads, W * var_warp_bytes<T, 8>(), s>>>(p);
            break;
        default:
            var_grid_t<T, MODE, 4>();
            k_var_pass<T, MODE, 4><<<grid, kThreads, W * var_warp_bytes<T, 4>(), s>>>(p);
            break;
    }
    return cudaGetLastError();
}
template <typename T>
cudaError_t fwd_launch_lc(const FwdParams& p, int lc, int grid, cudaStream_t s) {
    const int smem = kWarps * kFwdWarpBytes;
    switch (lc) {
        case 32: fwd_grid_t<T, 32>(); k_forward<T, 32><<<grid, kThreads, smem, s>>>(p); break;
        case 16: fwd_grid_t<T, 16>(); k_forward<T, 16><<<grid, kThreads, smem, s>>>(p); break;
        case 8: fwd_grid_t<T, 8>(); k_forward<T, 8><<<grid, kThreads, smem, s>>>(p); break;
        default: fwd_grid_t<T, 4>(); k_forward<T, 4><<<grid, kThreads, smem, s>>>(p); break;
    }
    return cudaGetLastError();
}
template <typename T>
int fwd_grid_lc(int lc) {
    switch (lc) {
        case 32: return fwd_grid_t<T, 32>();
        case 16: return fwd_grid_t<T, 16>();
        case 8: return fwd_grid_t<T, 8>();
        default: return fwd_grid_t<T, 4>();
    }
}

int elementwise_grid(int64_t total) {
    const int64_t blocks = (total + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    return static_cast<int>(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

// ------------------------------------------------------------------------------------------
int grid_var_pass(int dtype, int mode, int lc) {
    if (dtype == kF32) return mode == kModeAdam ? var_grid_lc<float, kModeAdam>(lc) : var_grid_lc<float, kModeGrad>(lc);
    if (dtype == kBF16)
        return mode == kModeAdam ? var_grid_lc<__nv_bfloat16, kModeAdam>(lc) : var_grid_lc<__nv_bfloat16, kModeGrad>(lc);
    return mode == kModeAdam ? var_grid_lc<__half, kModeAdam>(lc) : var_grid_lc<__half, kModeGrad>(lc);
}
int grid_forward(int dtype, int lc) {
    if (dtype == kF32) return fwd_grid_lc<float>(lc);
    if (dtype == kBF16) return fwd_grid_lc<__nv_bfloat16>(lc);
    return fwd_grid_lc<__half>(lc);
}
int grid_check(int lw, bool words32) {
    if (words32) return check_grid_t<1, uint32_t>();
    switch (lw) {
        case 32: return check_grid_t<32, uint64_t>();
        case 16: return check_grid_t<16, uint64_t>();
        case 8: return check_grid_t<8, uint64_t>();
        case 4: return check_grid_t<4, uint64_t>();
        case 2: return check_grid_t<2, uint64_t>();
        default: return check_grid_t<1, uint64_t>();
    }
}

cudaError_t launch_var_pass(const VarParams& p, int dtype, int mode, int lc, int grid, cudaStream_t s) {
    if (dtype == kF32)
        return mode == kModeAdam ? var_launch_lc<float, kModeAdam>(p, lc, grid, s)
                                 : var_launch_lc<float, kModeGrad>(p, lc, grid, s);
    if (dtype == kBF16)
        return mode == kModeAdam ? var_launch_lc<__nv_bfloat16, kModeAdam>(p, lc, grid, s)
                                 : var_launch_lc<__nv_bfloat16, kModeGrad>(p, lc, grid, s);
    return mode == kModeAdam ? var_launch_lc<__half, kModeAdam>(p, lc, grid, s)
                             : var_launch_lc<__half, kModeGrad>(p, lc, grid, s);
}

int grid_var_own(int dtype, int mode, int lc) {
    if (dtype == kF32) return mode == kModeAdam ? own_grid_lc<float, kModeAdam>(lc) : own_grid_lc<float, kModeGrad>(lc);
    if (dtype == kBF16)
        return mode == kModeAdam ? own_grid_lc<__nv_bfloat16, kModeAdam>(lc) : own_grid_lc<__nv_bfloat16, kModeGrad>(lc);
    return mode == kModeAdam ? own_grid_lc<__half, kModeAdam>(lc) : own_grid_lc<__half, kModeGrad>(lc);
}

cudaError_t launch_var_own(const VarParams& p, int dtype, int mode, int lc, int grid, cudaStream_t s) {
    if (dtype == kF32)
        return mode == kModeAdam ? own_launch_lc<float, kModeAdam>(p, lc, grid, s)
                                 : own_launch_lc<float, kModeGrad>(p, lc, grid, s);
    if (dtype == kBF16)
        return mode == kModeAdam ? own_launch_lc<__nv_bfloat16, kModeAdam>(p, lc, grid, s)
                                 : own_launch_lc<__nv_bfloat16, kModeGrad>(p, lc, grid, s);
    return mode == kModeAdam ? own_launch_lc<__half, kModeAdam>(p, lc, grid, s)
                             : own_launch_lc<__half, kModeGrad>(p, lc, grid, s);
}

int grid_var_ring(int dtype, int mode) {
    if (dtype == kF32) return mode == kModeAdam ? ring_grid_t<float, kModeAdam>() : ring_grid_t<float, kModeGrad>();
    if (dtype == kBF16)
        return mode == kModeAdam ? ring_grid_t<__nv_bfloat16, kModeAdam>() : ring_grid_t<__nv_bfloat16, kModeGrad>();
    return mode == kModeAdam ? ring_grid_t<__half, kModeAdam>() : ring_grid_t<__half, kModeGrad>();
}

cudaError_t launch_var_ring(const VarParams& p, const void* tmap, int dtype, int mode, int grid, cudaStream_t s) {
    const int smem = kRingWarps * kRingWarpBytes;
    const CUtensorMap& tm = *static_cast<const CUtensorMap*>(tmap);
    grid_var_ring(dtype, mode);
    if (dtype == kF32) {
        if (mode == kModeAdam)
            k_var_ring<float, kModeAdam><<<grid, kRingWarps * 32, smem, s>>>(p, tm);
        else
            k_var_ring<float, kModeGrad><<<grid, kRingWarps * 32, smem, s>>>(p, tm);
    } else if (dtype == kBF16) {
        if (mode == kModeAdam)
            k_var_ring<__nv_bfloat16, kModeAdam><<<grid, kRingWarps * 32, smem, s>>>(p, tm);
        else
            k_var_ring<__nv_bfloat16, kModeGrad><<<grid, kRingWarps * 32, smem, s>>>(p, tm);
    } else {
        if (mode == kModeAdam)
            k_var_ring<__half, kModeAdam><<<grid, kRingWarps * 32, smem, s>>>(p, tm);
        else
            k_var_ring<__half, kModeGrad><<<grid, kRingWarps * 32, smem, s>>>(p, tm);
    }
    return cudaGetLastError();
}

cudaError_t launch_forward(const FwdParams& p, int dtype, int lc, int grid, cudaStream_t s) {
    if (dtype == kF32) return fwd_launch_lc<float>(p, lc, grid, s);
    if (dtype == kBF16) return fwd_launch_lc<__nv_bfloat16>(p, lc, grid, s);
    return fwd_launch_lc<__half>(p, lc, grid, s);
}

cudaError_t launch_check(const CheckParams& p, int lw, bool words32, int grid, cudaStream_t s) {
    const int smem = kWarps * kFwdWarpBytes;
    if (words32) {
        check_grid_t<1, uint32_t>();
        k_check<1, uint32_t><<<grid, kThreads, smem, s>>>(p);
        return cudaGetLastError();
    }
    switch (lw) {
        case 32: check_grid_t<32, uint64_t>(); k_check<32, uint64_t><<<grid, kThreads, smem, s>>>(p); break;
        case 16: check_grid_t<16, uint64_t>(); k_check<16, uint64_t><<<grid, kThreads, smem, s>>>(p); break;
        case 8: check_grid_t<8, uint64_t>(); k_check<8, uint64_t><<<grid, kThreads, smem, s>>>(p); break;
        case 4: check_grid_t<4, uint64_t>(); k_check<4, uint64_t><<<grid, kThreads, smem, s>>>(p); break;
        case 2: check_grid_t<2, uint64_t>(); k_check<2, uint64_t><<<grid, kThreads, smem, s>>>(p); break;
        default: check_grid_t<1, uint64_t>(); k_check<1, uint64_t><<<grid, kThreads, smem, s>>>(p); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_compact_low32(const uint64_t* bits, int64_t n, int32_t nwd, uint32_t* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_compact_low32<<<elementwise_grid(n), 256, 0, s>>>(bits, n, nwd, out);
    return cudaGetLastError();
}

cudaError_t launch_loss_reduce2(const float* part, int32_t bpad, const int32_t* iptr, const int32_t* items,
                                const int64_t* n_empty, int32_t n_inst, int32_t B, int32_t n_seg, double* stage,
                                double* loss, cudaStream_t s) {
    if (B <= 0 || n_inst <= 0) return cudaSuccess;
    k_reduce_tiles<float, double><<<dim3((B + 31) / 32, n_inst, n_seg), 256, 0, s>>>(part, bpad, iptr, items, B,
                                                                                      n_seg, stage);
    k_loss_final<<<dim3((B + 31) / 32, n_inst), 1024, 0, s>>>(stage, n_seg, n_inst, n_empty, B, loss);
    return cudaGetLastError();
}

cudaError_t launch_count_reduce(const uint16_t* part16, int32_t bpad16, const int32_t* iptr, const int32_t* items,
                                const int64_t* n_empty, int32_t n_inst, int32_t B, int32_t n_seg, int32_t* stage,
                                int32_t* unsat, int32_t* best, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    if (B > 0)
        k_reduce_tiles<uint16_t, int32_t><<<dim3((B + 31) / 32, n_inst, n_seg), 256, 0, s>>>(part16, bpad16, iptr,
                                                                                            items, B, n_seg, stage);
    k_count_final<<<n_inst, 1024, 0, s>>>(stage, B > 0 ? n_seg : 0, n_inst, n_empty, B, unsat, best);
    return cudaGetLastError();
}

cudaError_t launch_relax(const float* delta, void* x, int dtype, int64_t n, int32_t B, int64_t ldB, float inv_tau,
                         cudaStream_t s) {
    if (n * B == 0) return cudaSuccess;
    const int grid = elementwise_grid(n * ((B + 3) / 4));
    if (dtype == kF32)
        k_relax<float><<<grid, 256, 0, s>>>(delta, static_cast<float*>(x), n, B, ldB, inv_tau);
    else if (dtype == kBF16)
        k_relax<__nv_bfloat16><<<grid, 256, 0, s>>>(delta, static_cast<__nv_bfloat16*>(x), n, B, ldB, inv_tau);
    else
        k_relax<__half><<<grid, 256, 0, s>>>(delta, static_cast<__half*>(x), n, B, ldB, inv_tau);
    return cudaGetLastError();
}

cudaError_t launch_round(const float* delta, uint32_t* bits32, int64_t n, int32_t B, int64_t ldB, int32_t nwd,
                         cudaStream_t s) {
    const int64_t warps = n * 2 * nwd;
    if (warps == 0) return cudaSuccess;
    k_round<<<elementwise_grid(warps * 32), 256, 0, s>>>(delta, bits32, n, B, ldB, nwd);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* delta, float* m, float* v, const float* grad, void* x_out, int dtype, int64_t n,
                        int32_t B, int64_t ldB, const AdamK& k, cudaStream_t s) {
    if (n * B == 0) return cudaSuccess;
    const int grid = elementwise_grid(n * B);
    if (dtype == kF32)
        k_adam<float><<<grid, 256, 0, s>>>(delta, m, v, grad, static_cast<float*>(x_out), n, B, ldB, k);
    else if (dtype == kBF16)
        k_adam<__nv_bfloat16><<<grid, 256, 0, s>>>(delta, m, v, grad, static_cast<__nv_bfloat16*>(x_out), n, B, ldB, k);
    else
        k_adam<__half><<<grid, 256, 0, s>>>(delta, m, v, grad, static_cast<__half*>(x_out), n, B, ldB, k);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int32_t* status, uint64_t limit_ns, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, limit_ns);
    return cudaGetLastError();
}

}  // namespace gs
