// Adaptive acceptance of one aligned pair (Section "Related works", BELLA
// paragraph: an adaptive threshold decides which X-drop alignments are
// kept; the paper gives no formula).  Reading: accepted iff the status is
// OK and the total score left + seed_len * match + right reaches
// (1 - delta) * L * (phi * match + (1 - phi) * mismatch), where L =
// min(seed_a, seed_b) + min(len_a - seed_a, len_b - seed_b) is the overlap
// the seed implies and phi = (1 - e)^2 the chance that a column pairs two
// correct bases.  e and delta come in units of 1e-4; the comparison is
// exact in 128-bit integers, scaled by 10^12.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define XA_HD __host__ __device__ __forceinline__
#else
#define XA_HD inline
#endif

namespace xa {

// Expected score of one overlap column, times 10^8.
XA_HD __int128 expected_e8(int32_t match, int32_t mismatch, uint32_t error_e4)
{
    const int64_t q = 10000;
    const int64_t phi = (q - (int64_t)error_e4) * (q - (int64_t)error_e4);
    return (__int128)phi * match + (__int128)(q * q - phi) * mismatch;
}

XA_HD uint8_t accept_one(int32_t status, int32_t left, int32_t right, uint32_t seed_a,
                         uint32_t seed_b, uint32_t seed_len, uint32_t len_a, uint32_t len_b,
                         int32_t match, __int128 expected, uint32_t delta_e4)
{
    if (status != 0) return 0;
    const int64_t q = 10000;
    const int64_t sa = seed_a, sb = seed_b, la = len_a, lb = len_b;
    const int64_t L = (sa < sb ? sa : sb) + (la - sa < lb - sb ? la - sa : lb - sb);
    const __int128 total = (__int128)left + (__int128)seed_len * match + right;
    return total * (q * q * q) >= (__int128)(q - (int64_t)delta_e4) * L * expected ? 1 : 0;
}

}  // namespace xa
