// Counter-based logistic noise shared by the straight-through step (gs_st.cu) and the candidate
// pool (gs_pool.cu): Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11) and the map from one 32-bit output word to one Logistic(0,1) draw.
#pragma once
#include <cstdint>

namespace gs {
namespace {

constexpr uint32_t kPhM0 = 0xD2511F53u;   // Philox4x32 round multipliers
constexpr uint32_t kPhM1 = 0xCD9E8D57u;
constexpr uint32_t kPhW0 = 0x9E3779B9u;   // Weyl increments of the key
constexpr uint32_t kPhW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox4x32_10(uint32_t (&x)[4], uint32_t k0, uint32_t k1) {
#pragma unroll 2   // smaller code: the straight-through kernel is otherwise instruction-fetch bound
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(kPhM0) * x[0];
        const uint64_t p1 = static_cast<uint64_t>(kPhM1) * x[2];
        const uint32_t y0 = static_cast<uint32_t>(p1 >> 32) ^ x[1] ^ k0;
        const uint32_t y2 = static_cast<uint32_t>(p0 >> 32) ^ x[3] ^ k1;
        x[1] = static_cast<uint32_t>(p1);
        x[3] = static_cast<uint32_t>(p0);
        x[0] = y0;
        x[2] = y2;
        k0 += kPhW0;
        k1 += kPhW1;
    }
}

// k = top 23 bits of the word, u = (k + 1/2) 2^-23 (exact in float32), l = log(u / (1 - u)).
__device__ __forceinline__ float logistic_from_word(uint32_t w) {
    const float u = (static_cast<float>(w >> 9) + 0.5f) * 0x1p-23f;
    // fast log: documented error 2^-21.41 absolute on [0.5, 2] and 3 ulp elsewhere, below the
    // spacing of the 23-bit draws (>= 4 * 2^-23 in l)
    return __logf(__fdiv_rn(u, 1.0f - u));
}

}  // namespace
}  // namespace gs
