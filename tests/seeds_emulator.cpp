// CPU emulation of the seed-discovery pipeline (test infrastructure).
//
// Runs the per-element steps of paper_2309_07270_gb300/csrc/xd_seeds.cuh
// (the same functions the kernels call) in the pipeline's order, for both
// products (sort-based and row-wise), with std::stable_sort and plain loops
// where the device uses CUB's radix sort, run-length encoding, scan and
// reduce-by-key, and with one read's table at a time where the device
// fills many tables at once with shared-memory atomics.  Comparing it with the
// oracle on the CPU checks the kernels' index arithmetic before any GPU
// run; it is neither the oracle nor the device path.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../paper_2309_07270_gb300/csrc/xd_seeds.cuh"

namespace {

// The steps both products share: occurrences, their sort by code, the runs.
struct Front {
    std::vector<uint64_t> occ_off, codes;
    std::vector<uint32_t> occ, occ_rd, fwd_bits;
    std::vector<int> run_off, run_len;
};

bool front(const uint32_t *packed, const uint64_t *read_off, const uint32_t *read_len,
           uint32_t n_reads, uint32_t k, uint32_t stride, Front &f)
{
    f.occ_off.assign(n_reads + 1, 0);
    for (uint32_t r = 0; r < n_reads; ++r)
        f.occ_off[r + 1] = f.occ_off[r] + (read_len[r] >= k ? (read_len[r] - k) / stride + 1 : 0);
    const uint64_t n_occ = f.occ_off[n_reads];
    if (n_occ < 2) return false;
    std::vector<uint64_t> keys(n_occ);
    f.occ_rd.assign(n_occ, 0);
    f.fwd_bits.assign((n_occ + 31) / 32, 0);
    for (uint64_t q = 0; q < n_occ; ++q) {
        uint32_t r;
        bool fwd;
        keys[q] = xs::occurrence(packed, read_off, f.occ_off.data(), n_reads, k, stride, q, &r, &fwd);
        f.occ_rd[q] = r;
        if (fwd) f.fwd_bits[q >> 5] |= 1u << (q & 31);
    }
    f.occ.resize(n_occ);
    std::iota(f.occ.begin(), f.occ.end(), 0u);
    std::stable_sort(f.occ.begin(), f.occ.end(), [&](uint32_t x, uint32_t y) { return keys[x] < keys[y]; });
    f.codes.resize(n_occ);
    for (uint64_t i = 0; i < n_occ; ++i) f.codes[i] = keys[f.occ[i]];
    for (uint64_t i = 0; i < n_occ;) {
        uint64_t j = i;
        while (j < n_occ && f.codes[j] == f.codes[i]) ++j;
        if (j - i >= 2) {
            f.run_off.push_back((int)i);
            f.run_len.push_back((int)(j - i));
        }
        i = j;
    }
    return !f.run_off.empty();
}

struct RowCand {
    uint64_t key;   // (a << nb) | b
    uint64_t best;  // seed_key
    uint32_t shared;
};

}  // namespace

// The row-wise product with a table of 2^table_lg slots per read; returns
// -1 when some read has more partners than that (the library then takes
// the sort-based product), else the number of candidates.
extern "C" int64_t emulate_candidates_rowwise(const uint32_t *packed, const uint64_t *read_off,
                                              const uint32_t *read_len, uint32_t n_reads,
                                              uint32_t k, uint32_t stride, uint32_t lo,
                                              uint32_t hi, uint32_t table_lg, uint32_t *out,
                                              int64_t cap)
{
    Front f;
    if (!front(packed, read_off, read_len, n_reads, k, stride, f)) return 0;
    const size_t n_runs = f.run_off.size();
    // columns: distinct reads per reliable run, scanned
    std::vector<uint32_t> col_end(n_runs);
    uint64_t nnz = 0;
    for (size_t i = 0; i < n_runs; ++i) {
        nnz += xs::run_reads(f.occ.data(), f.occ_rd.data(), (uint64_t)f.run_off[i],
                             (uint32_t)f.run_len[i], lo, hi);
        col_end[i] = (uint32_t)nnz;
    }
    if (nnz == 0) return 0;
    std::vector<uint64_t> members(nnz);
    std::vector<uint32_t> col_of(nnz), row_cnt(n_reads, 0);
    for (size_t i = 0; i < n_runs; ++i) {
        const uint32_t c0 = i ? col_end[i - 1] : 0;
        if (col_end[i] == c0) continue;
        xs::run_members(f.occ.data(), f.occ_rd.data(), f.fwd_bits.data(), f.occ_off.data(),
                        (uint64_t)f.run_off[i], (uint32_t)f.run_len[i], stride, members.data() + c0);
        for (uint32_t j = c0; j < col_end[i]; ++j) {
            col_of[j] = (uint32_t)i;
            ++row_cnt[(uint32_t)(members[j] >> 32)];
        }
    }
    // rows: (column, position << 1 | forward) of each read's reliable k-mers
    std::vector<uint32_t> row_end(n_reads), fill(n_reads, 0);
    uint32_t acc = 0;
    for (uint32_t r = 0; r < n_reads; ++r) row_end[r] = acc += row_cnt[r];
    std::vector<uint32_t> row_col(nnz), row_pos(nnz);
    for (uint64_t j = 0; j < nnz; ++j) {
        const uint32_t r = (uint32_t)(members[j] >> 32);
        const uint32_t e = (r ? row_end[r - 1] : 0) + fill[r]++;
        row_col[e] = col_of[j];
        row_pos[e] = (uint32_t)(members[j] & 0xFFFFFFFFu);
    }
    // one table per read
    const uint32_t slots = 1u << table_lg;
    std::vector<uint32_t> tkey(slots), tcnt(slots);
    std::vector<unsigned long long> tbest(slots);
    const xs::RowTable t{tkey.data(), tcnt.data(), tbest.data(), table_lg};
    const uint32_t nb = xs::id_bits(n_reads);
    std::vector<RowCand> cands;
    for (uint32_t a = 0; a < n_reads; ++a) {
        const uint32_t e0 = a ? row_end[a - 1] : 0;
        if (row_end[a] == e0) continue;
        std::fill(tkey.begin(), tkey.end(), xs::kEmpty);
        std::fill(tcnt.begin(), tcnt.end(), 0u);
        std::fill(tbest.begin(), tbest.end(), ~0ull);
        for (uint32_t e = e0; e < row_end[a]; ++e) {
            const uint32_t col = row_col[e];
            const uint32_t pa = row_pos[e] >> 1;
            const bool fa = (row_pos[e] & 1u) != 0;
            for (uint32_t j = col ? col_end[col - 1] : 0; j < col_end[col]; ++j)
                if (!xs::row_term(t, a, pa, fa, members[j], read_len, k)) return -1;
        }
        for (uint32_t h = 0; h < slots; ++h)
            if (tkey[h] != xs::kEmpty)
                cands.push_back(RowCand{((uint64_t)a << nb) | tkey[h], tbest[h], tcnt[h]});
    }
    std::sort(cands.begin(), cands.end(),
              [](const RowCand &x, const RowCand &y) { return x.key < y.key; });
    const uint64_t mask = nb >= 32 ? 0xFFFFFFFFull : (1ull << nb) - 1;
    for (size_t i = 0; i < cands.size() && (int64_t)i < cap; ++i) {
        const RowCand &c = cands[i];
        uint32_t *o = out + 6 * i;
        o[0] = (uint32_t)(c.key >> nb);
        o[1] = (uint32_t)(c.key & mask) | ((c.best & 1u) ? xs::kPairRC : 0u);
        o[2] = (uint32_t)(c.best >> 32);
        o[3] = (uint32_t)(c.best & 0xFFFFFFFFu) >> 1;
        o[4] = k;
        o[5] = c.shared;
    }
    return (int64_t)cands.size();
}

extern "C" int64_t emulate_candidates(const uint32_t *packed, const uint64_t *read_off,
                                      const uint32_t *read_len, uint32_t n_reads, uint32_t k,
                                      uint32_t stride, uint32_t lo, uint32_t hi, uint32_t *out,
                                      int64_t cap)
{
    Front f;
    if (!front(packed, read_off, read_len, n_reads, k, stride, f)) return 0;
    const size_t n_runs = f.run_off.size();
    // count_kernel + inclusive scan
    std::vector<uint64_t> pair_end(n_runs);
    uint64_t acc = 0;
    for (size_t i = 0; i < n_runs; ++i) {
        acc += xs::run_pairs(f.occ.data(), f.occ_rd.data(), (uint64_t)f.run_off[i],
                             (uint32_t)f.run_len[i], lo, hi);
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
        const uint64_t s = (uint64_t)f.run_off[i];
        xs::run_emit(f.occ.data(), f.occ_rd.data(), f.fwd_bits.data(), f.occ_off.data(), read_len,
                     f.codes[s], s, (uint32_t)f.run_len[i], k, stride, nb, e0, ek.data(),
                     ent.data(), ei.data());
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
