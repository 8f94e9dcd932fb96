// Counter-based sampling of RANSAC minimal sets (the paper specifies no
// sampler; Sec. 2.2 only says that four correspondences are drawn).
//
// Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw ("Parallel
// random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32 ->
// 64-bit products by 0xD2511F53 / 0xCD9E8D57 with its Feistel-like word
// permutation; the key advances by 0x9E3779B9 / 0xBB67AE85 between rounds.
#pragma once
#include <stdint.h>

#include "fp32.cuh"

namespace aca {

struct U4 {
    uint32_t x, y, z, w;
};

ACA_HD uint32_t mulhi32(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

ACA_HD U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// rank j in [0, m): floor(u * m / 2^32)
ACA_HD uint32_t rank_of(uint32_t u, uint32_t m) { return mulhi32(u, m); }

// Four distinct indices in [0, N) (N >= 4) for hypothesis `hyp` of problem
// `prob`: ranks among the not-yet-drawn indices, mapped to indices by
// stepping over the earlier draws in ascending order.
ACA_HD void sample4(uint64_t seed, uint32_t prob, uint32_t hyp, uint32_t N, uint32_t idx[4])
{
    const U4 u = philox4x32_10(U4{hyp, prob, 0u, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t i0 = rank_of(u.x, N);
    uint32_t i1 = rank_of(u.y, N - 1u);
    i1 += (i1 >= i0);
    uint32_t a = i0 < i1 ? i0 : i1, b = i0 < i1 ? i1 : i0;       // sorted pair
    uint32_t i2 = rank_of(u.z, N - 2u);
    i2 += (i2 >= a);
    i2 += (i2 >= b);
    // sorted triple a <= b <= c
    uint32_t c = i2;
    if (c < b) { const uint32_t t = b; b = c; c = t; }
    if (b < a) { const uint32_t t = a; a = b; b = t; }
    uint32_t i3 = rank_of(u.w, N - 3u);
    i3 += (i3 >= a);
    i3 += (i3 >= b);
    i3 += (i3 >= c);
    idx[0] = i0;
    idx[1] = i1;
    idx[2] = i2;
    idx[3] = i3;
}

}  // namespace aca
