// philox.cuh -- Philox4x32-10 counter-based generator on the device.
//
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): per round, two 32 x 32 -> 64-bit products of counter words 0 and 2
// with the multipliers 0xD2511F53 and 0xCD9E8D57; the high halves are xored
// with counter words 1 and 3 and the round key; the key advances by the Weyl
// constants 0x9E3779B9 and 0xBB67AE85 after every round; ten rounds.
#pragma once
#include <stdint.h>

namespace qmcdu {

struct u32x4 { uint32_t x0, x1, x2, x3; };

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x0, hi0 = __umulhi(0xD2511F53u, c.x0);
        const uint32_t lo1 = 0xCD9E8D57u * c.x2, hi1 = __umulhi(0xCD9E8D57u, c.x2);
        c = u32x4{hi1 ^ c.x1 ^ k0, lo1, hi0 ^ c.x3 ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// 53-bit uniform in [0, 1) from two words (exact in fp64).
__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo)
{
    const uint64_t bits = ((uint64_t)hi << 32) | lo;
    return (double)(bits >> 11) * 0x1.0p-53;
}

// Counter tags (word 2): 0 Metropolis uniform, 1 proposal Gaussians, 2 matrix.
enum : uint32_t { TAG_UNIFORM = 0, TAG_PROPOSAL = 1, TAG_MATRIX = 2 };

// Metropolis uniform of electron j in sweep s for a walker seed.
__device__ __forceinline__ double metropolis_uniform(unsigned long long seed, int j, int s)
{
    u32x4 o = philox4x32_10(u32x4{(uint32_t)j, (uint32_t)s, TAG_UNIFORM, 0u},
                            (uint32_t)seed, (uint32_t)(seed >> 32));
    return uniform53(o.x0, o.x1);
}

// Gaussian pair from the Philox output at counter (c0, c1, tag, blk) by the
// Box-Muller transform (Box and Muller, Ann. Math. Stat. 1958).
__device__ __forceinline__ double2 box_muller_pair(unsigned long long seed, uint32_t c0, uint32_t c1,
                                                   uint32_t tag, uint32_t blk)
{
    u32x4 o = philox4x32_10(u32x4{c0, c1, tag, blk}, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = uniform53(o.x0, o.x1);
    const double u2 = uniform53(o.x2, o.x3);
    const double rho = sqrt(-2.0 * log(1.0 - u1));
    const double ang = 2.0 * 3.141592653589793 * u2;
    double sn, cs;
    sincos(ang, &sn, &cs);
    return make_double2(rho * cs, rho * sn);
}

// Entries 2 blk and 2 blk + 1 of the proposal row of electron j, sweep s.
__device__ __forceinline__ double2 proposal_gaussian_pair(unsigned long long seed, int j, int s,
                                                          int blk)
{
    return box_muller_pair(seed, (uint32_t)j, (uint32_t)s, TAG_PROPOSAL, (uint32_t)blk);
}

// Entries 2 blk and 2 blk + 1 of row i of a walker's initial matrix, A_ij ~ N(0, 1).
__device__ __forceinline__ double2 matrix_gaussian_pair(unsigned long long seed, int i, int blk)
{
    return box_muller_pair(seed, (uint32_t)i, 0u, TAG_MATRIX, (uint32_t)blk);
}

}  // namespace qmcdu
