// CPU run of the per-pair acceptance arithmetic of
// paper_2309_07270_gb300/csrc/xd_accept.cuh (the function the kernel
// calls), for comparison with the oracle on the CPU (test infrastructure).
#include <stdint.h>

#include "../paper_2309_07270_gb300/csrc/xd_accept.cuh"

extern "C" void emulate_accept(const uint32_t *pairs, const int32_t *results, const uint32_t *read_len,
                               uint32_t n_reads, uint64_t n, int32_t match, int32_t mismatch,
                               uint32_t error_e4, uint32_t delta_e4, uint8_t *out)
{
    const __int128 expected = xa::expected_e8(match, mismatch, error_e4);
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t *p = pairs + 5 * i;  // a, b, seed_a, seed_b, seed_len
        const int32_t *r = results + 7 * i;
        const uint32_t a = p[0], b = p[1] & 0x7FFFFFFFu;
        out[i] = (a < n_reads && b < n_reads)
                     ? xa::accept_one(r[6], r[0], r[3], p[2], p[3], p[4], read_len[a], read_len[b],
                                      match, expected, delta_e4)
                     : 0;
    }
}
