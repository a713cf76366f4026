// CPU emulation of the seed-discovery pipeline (test infrastructure).
//
// Runs the per-element steps of paper_2309_07270_gb300/csrc/xd_seeds.cuh
// (the same functions the kernels call) in the pipeline's order, with
// std::stable_sort and plain loops where the device uses CUB's radix sort,
// run-length encoding, scan and reduce-by-key.  Comparing it with the
// oracle on the CPU checks the kernels' index arithmetic before any GPU
// run; it is neither the oracle nor the device path.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../paper_2309_07270_gb300/csrc/xd_seeds.cuh"

extern "C" int64_t emulate_candidates(const uint32_t *packed, const uint64_t *read_off,
                                      const uint32_t *read_len, uint32_t n_reads, uint32_t k,
                                      uint32_t stride, uint32_t lo, uint32_t hi, uint32_t *out,
                                      int64_t cap)
{
    std::vector<uint64_t> occ_off(n_reads + 1, 0);
    for (uint32_t r = 0; r < n_reads; ++r)
        occ_off[r + 1] = occ_off[r] + (read_len[r] >= k ? (read_len[r] - k) / stride + 1 : 0);
    const uint64_t n_occ = occ_off[n_reads];
    if (n_occ < 2) return 0;

    // kmer_kernel
    std::vector<uint64_t> keys(n_occ);
    std::vector<uint32_t> occ_rd(n_occ), fwd_bits((n_occ + 31) / 32, 0);
    for (uint64_t q = 0; q < n_occ; ++q) {
        uint32_t r;
        bool fwd;
        keys[q] = xs::occurrence(packed, read_off, occ_off.data(), n_reads, k, stride, q, &r, &fwd);
        occ_rd[q] = r;
        if (fwd) fwd_bits[q >> 5] |= 1u << (q & 31);
    }
    // stable sort of (code, occurrence id)
    std::vector<uint32_t> occ(n_occ);
    std::iota(occ.begin(), occ.end(), 0u);
    std::stable_sort(occ.begin(), occ.end(), [&](uint32_t x, uint32_t y) { return keys[x] < keys[y]; });
    std::vector<uint64_t> codes(n_occ);
    for (uint64_t i = 0; i < n_occ; ++i) codes[i] = keys[occ[i]];
    // runs of length >= 2
    std::vector<int> run_off, run_len;
    for (uint64_t i = 0; i < n_occ;) {
        uint64_t j = i;
        while (j < n_occ && codes[j] == codes[i]) ++j;
        if (j - i >= 2) {
            run_off.push_back((int)i);
            run_len.push_back((int)(j - i));
        }
        i = j;
    }
    const size_t n_runs = run_off.size();
    // count_kernel + inclusive scan
    std::vector<uint64_t> pair_end(n_runs);
    uint64_t acc = 0;
    for (size_t i = 0; i < n_runs; ++i) {
        acc += xs::run_pairs(occ.data(), occ_rd.data(), (uint64_t)run_off[i], (uint32_t)run_len[i],
                             lo, hi);
        pair_end[i] = acc;
    }
    const uint64_t n_ent = acc;
    if (n_ent == 0) return 0;
    // emit_kernel
    const uint32_t nb = xs::id_bits(n_reads);
    std::vector<uint64_t> ek(n_ent);
    std::vector<xs::Cand> ent(n_ent);
    std::vector<uint32_t> ei(n_ent);
    for (size_t i = 0; i < n_runs; ++i) {
        const uint64_t e0 = i ? pair_end[i - 1] : 0;
        if (pair_end[i] == e0) continue;
        const uint64_t s = (uint64_t)run_off[i];
        xs::run_emit(occ.data(), occ_rd.data(), fwd_bits.data(), occ_off.data(), read_len, codes[s],
                     s, (uint32_t)run_len[i], k, stride, nb, e0, ek.data(), ent.data(), ei.data());
    }
    // stable sort of the pair keys, gather, reduce by key
    std::vector<uint32_t> order(ei);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return ek[x] < ek[y]; });
    const xs::CandMerge merge;
    const uint64_t mask = nb >= 32 ? 0xFFFFFFFFull : (1ull << nb) - 1;
    int64_t n_cand = 0;
    for (uint64_t i = 0; i < n_ent;) {
        const uint64_t key = ek[order[i]];
        xs::Cand agg = ent[order[i]];
        uint64_t j = i + 1;
        for (; j < n_ent && ek[order[j]] == key; ++j) agg = merge(agg, ent[order[j]]);
        if (n_cand < cap) {
            uint32_t *o = out + 6 * n_cand;
            o[0] = (uint32_t)(key >> nb);
            o[1] = (uint32_t)(key & mask) | (agg.rc ? xs::kPairRC : 0u);
            o[2] = agg.pa;
            o[3] = agg.sb;
            o[4] = k;
            o[5] = agg.shared;
        }
        ++n_cand;
        i = j;
    }
    return n_cand;
}
