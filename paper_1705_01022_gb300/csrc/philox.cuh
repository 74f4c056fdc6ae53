// Philox-4x32-10 counter-based generator for device code.
//
// Written from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3" (SC'11): ten rounds, each multiplying counter words 0 and 2 by
// the round constants (32x32 -> 64 bit), swapping and xoring the high halves
// with the other counter words and the key; the key advances by a Weyl
// increment between rounds.
#pragma once
#include <cstdint>

namespace oct {

constexpr uint32_t kTagMcs = 1u;
constexpr uint32_t kTagSet = 2u;
constexpr uint32_t kTagSite = 3u;
constexpr uint32_t kTagAcc = 4u;
constexpr uint32_t kTagReplica = 6u;
constexpr uint32_t kTagTail = 7u;
constexpr uint32_t kTagSiteDb = 8u;
constexpr uint32_t kTagBorg = 9u;  // block-layer origin of DTrDTr

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int round = 0; round < 10; ++round) {
        // high and low halves of the two 32 x 32 -> 64-bit products
#ifdef __CUDA_ARCH__
        const uint32_t h0 = __umulhi(0xD2511F53u, c0), h1 = __umulhi(0xCD9E8D57u, c2);
#else
        const uint32_t h0 = static_cast<uint32_t>((static_cast<uint64_t>(0xD2511F53u) * c0) >> 32);
        const uint32_t h1 = static_cast<uint32_t>((static_cast<uint64_t>(0xCD9E8D57u) * c2) >> 32);
#endif
        const uint32_t l0 = 0xD2511F53u * c0, l1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = h1 ^ c1 ^ k0;
        const uint32_t n2 = h0 ^ c3 ^ k1;
        c1 = l1;
        c3 = l0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

}  // namespace oct
