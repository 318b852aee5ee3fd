// forcing.cuh -- device pieces of the stirring force shared by the 2D and
// 3D lattices: the counter-based generator of the mode draws and the
// (cos, sin) pair of the phase tables.
#pragma once

namespace rlbk {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the
// published definition: per round two 32x32->64-bit products with the
// multipliers 0xD2511F53 and 0xCD9E8D57, words recombined as
// (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key bumped by the Weyl
// increments 0x9E3779B9 and 0xBB67AE85 after each round.
struct U4 {
    unsigned int w[4];
};

__device__ __forceinline__ U4 philox4x32_10(U4 ctr, unsigned int k0, unsigned int k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned int lo0 = 0xD2511F53u * ctr.w[0];
        const unsigned int hi0 = __umulhi(0xD2511F53u, ctr.w[0]);
        const unsigned int lo1 = 0xCD9E8D57u * ctr.w[2];
        const unsigned int hi1 = __umulhi(0xCD9E8D57u, ctr.w[2]);
        U4 n;
        n.w[0] = hi1 ^ ctr.w[1] ^ k0;
        n.w[1] = lo1;
        n.w[2] = hi0 ^ ctr.w[3] ^ k1;
        n.w[3] = lo0;
        ctr = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ctr;
}

__device__ __forceinline__ double u01_53(unsigned int a, unsigned int b) {
    const unsigned long long m = ((unsigned long long)a << 21) | (unsigned long long)(b >> 11);
    return (double)m * (1.0 / 9007199254740992.0);
}

template <typename TC>
struct C2 {
    TC c, s;
};

}  // namespace rlbk
