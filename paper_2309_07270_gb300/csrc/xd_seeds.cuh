// Seed discovery: reliable k-mers and the candidate read pairs that share
// one (the nonzeros of A * A^T, A the read-by-reliable-k-mer matrix;
// Section "Related works", diBELLA 2D paragraph; Section "Experimental
// Setup": k = 31, stride 1, frequency window [20, 30] or [20, 50]).
//
// The per-element steps of the pipeline in xd_seeds.cu, as plain functions
// of indices and arrays so that each kernel is a thin loop around one of
// them.  Readings of what the paper leaves open:
//   * a k-mer's canonical code is the smaller of the 2k-bit codes (first
//     base most significant) of the k-mer and of its reverse complement;
//   * its count is its number of occurrences over all reads (several in one
//     read count separately); it is reliable iff lo <= count <= hi;
//   * read r's entry for a reliable k-mer is its first occurrence there;
//   * a candidate pair a < b shares at least one reliable k-mer; it counts
//     the shared k-mers and takes as seed the shared k-mer with the smallest
//     position in a (then in b, then the smallest code); if that k-mer was
//     read on opposite strands in a and b the pair names b's reverse
//     complement (flag 0x80000000 in b) with seed_b = len_b - k - pos_b.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define XS_HD __host__ __device__ __forceinline__
#else
#define XS_HD inline
#endif

namespace xs {

constexpr uint32_t kPairRC = 0x80000000u;
constexpr uint32_t kMaxK = 32;     // codes fit 64 bits
constexpr uint32_t kMaxHi = 1024;  // bounds the pairs one k-mer can make

// One shared reliable k-mer of a read pair, and after the reduction by
// pair the pair's chosen seed with the number of shared k-mers.
struct Cand {
    uint64_t code;    // canonical code of the k-mer
    uint32_t pa, pb;  // its first position in read a and in read b
    uint32_t sb;      // seed start in b, or in b's reverse complement
    uint32_t rc;      // 1: opposite strands
    uint32_t shared;  // number of shared reliable k-mers (1 before the reduction)
    uint32_t pad;
};

XS_HD uint64_t low_mask(uint32_t k)  // 2k low bits, 1 <= k <= 32
{
    return k >= 32 ? ~0ull : (1ull << (2 * k)) - 1;
}

// The 2-bit groups of x in reverse order.
XS_HD uint64_t rev2(uint64_t x)
{
    x = (x >> 32) | (x << 32);
    x = ((x >> 16) & 0x0000FFFF0000FFFFull) | ((x & 0x0000FFFF0000FFFFull) << 16);
    x = ((x >> 8) & 0x00FF00FF00FF00FFull) | ((x & 0x00FF00FF00FF00FFull) << 8);
    x = ((x >> 4) & 0x0F0F0F0F0F0F0F0Full) | ((x & 0x0F0F0F0F0F0F0F0Full) << 4);
    x = ((x >> 2) & 0x3333333333333333ull) | ((x & 0x3333333333333333ull) << 2);
    return x;
}

// Bases g .. g+k-1 of the packed buffer (16 per word, base g in bits
// 2(g mod 16) of word g/16), base g+i in bits 2i..2i+1.  Reads only the
// words that hold those bases.
XS_HD uint64_t window(const uint32_t *packed, uint64_t g, uint32_t k)
{
    const uint64_t w = g >> 4, wl = (g + k - 1) >> 4;
    const uint32_t o = 2u * (uint32_t)(g & 15);
    uint64_t lo = packed[w];
    if (wl > w) lo |= (uint64_t)packed[w + 1] << 32;
    uint64_t x = lo >> o;
    if (wl > w + 1) x |= (uint64_t)packed[w + 2] << (64 - o);  // here o >= 2
    return x & low_mask(k);
}

// Canonical code of the k-mer in window x; *fwd = the k-mer as read is
// the canonical one (ties count as forward).
XS_HD uint64_t canonical(uint64_t x, uint32_t k, bool *fwd)
{
    const uint64_t f = rev2(x) >> (64 - 2 * k);  // first base most significant
    const uint64_t r = ~x & low_mask(k);         // reverse complement, same order
    *fwd = f <= r;
    return f <= r ? f : r;
}

// The read of occurrence q: the largest r with occ_off[r] <= q, where
// occ_off[0] = 0 <= q < occ_off[n_reads] (reads without occurrences have
// occ_off[r] == occ_off[r+1] and are skipped).
XS_HD uint32_t occ_read(const uint64_t *occ_off, uint32_t n_reads, uint64_t q)
{
    uint32_t lo = 0, hi = n_reads;
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (occ_off[mid] <= q)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

XS_HD bool fwd_bit(const uint32_t *fwd_bits, uint64_t q)
{
    return (fwd_bits[q >> 5] >> (q & 31)) & 1u;
}

// Occurrence q: its canonical code, read and strand.  Occurrences are
// numbered read by read, positions 0, stride, 2*stride, ... <= len - k.
XS_HD uint64_t occurrence(const uint32_t *packed, const uint64_t *read_off,
                          const uint64_t *occ_off, uint32_t n_reads, uint32_t k,
                          uint32_t stride, uint64_t q, uint32_t *read, bool *fwd)
{
    const uint32_t r = occ_read(occ_off, n_reads, q);
    const uint64_t pos = (q - occ_off[r]) * stride;
    *read = r;
    return canonical(window(packed, read_off[r] + pos, k), k, fwd);
}

// A run is the occurrences [s, s + cnt) of one k-mer in the sorted order
// (ascending occurrence id, hence by read, then position).  Entry i is its
// read's first occurrence iff i == 0 or the previous entry is another read.
XS_HD bool first_in_read(const uint32_t *occ, const uint32_t *occ_rd, uint64_t s, uint32_t i)
{
    return i == 0 || occ_rd[occ[s + i]] != occ_rd[occ[s + i - 1]];
}

// Number of read pairs a reliable run makes: u(u-1)/2 over its u distinct
// reads; 0 for a run outside [lo, hi].
XS_HD uint64_t run_pairs(const uint32_t *occ, const uint32_t *occ_rd, uint64_t s,
                         uint32_t cnt, uint32_t lo, uint32_t hi)
{
    if (cnt < lo || cnt > hi) return 0;
    uint64_t u = 0;
    for (uint32_t i = 0; i < cnt; ++i) u += first_in_read(occ, occ_rd, s, i);
    return u * (u - 1) / 2;
}

// Writes the run's pairs to entries e0, e0+1, ...: key (a << nb) | b
// (a < b, nb bits per read id), the shared k-mer as a Cand, and the entry's
// own index (the payload of the key sort).  Same order as run_pairs counts.
XS_HD void run_emit(const uint32_t *occ, const uint32_t *occ_rd, const uint32_t *fwd_bits,
                    const uint64_t *occ_off, const uint32_t *read_len, uint64_t code,
                    uint64_t s, uint32_t cnt, uint32_t k, uint32_t stride, uint32_t nb,
                    uint64_t e0, uint64_t *keys, Cand *ent, uint32_t *idx)
{
    uint64_t e = e0;
    for (uint32_t x = 0; x < cnt; ++x) {
        if (!first_in_read(occ, occ_rd, s, x)) continue;
        const uint32_t qx = occ[s + x], ra = occ_rd[qx];
        const uint32_t pa = (uint32_t)((qx - occ_off[ra]) * stride);
        const bool fa = fwd_bit(fwd_bits, qx);
        for (uint32_t y = x + 1; y < cnt; ++y) {
            if (!first_in_read(occ, occ_rd, s, y)) continue;
            const uint32_t qy = occ[s + y], rb = occ_rd[qy];
            const uint32_t pb = (uint32_t)((qy - occ_off[rb]) * stride);
            const bool rc = fa != fwd_bit(fwd_bits, qy);
            Cand c;
            c.code = code;
            c.pa = pa;
            c.pb = pb;
            c.sb = rc ? read_len[rb] - k - pb : pb;
            c.rc = rc;
            c.shared = 1;
            c.pad = 0;
            keys[e] = ((uint64_t)ra << nb) | rb;
            ent[e] = c;
            idx[e] = (uint32_t)e;
            ++e;
        }
    }
}

// Reduction of the Cands of one read pair: the seed with the smallest
// (pa, pb, code), the shared counts summed.  Associative and commutative.
struct CandMerge {
    XS_HD Cand operator()(const Cand &x, const Cand &y) const
    {
        const bool xf = x.pa != y.pa ? x.pa < y.pa : x.pb != y.pb ? x.pb < y.pb : x.code <= y.code;
        Cand m = xf ? x : y;
        m.shared = x.shared + y.shared;
        return m;
    }
};

// Distinct reads of a run (the nonzeros of its column of A), 0 for a run
// outside [lo, hi].
XS_HD uint32_t run_reads(const uint32_t *occ, const uint32_t *occ_rd, uint64_t s, uint32_t cnt,
                         uint32_t lo, uint32_t hi)
{
    if (cnt < lo || cnt > hi) return 0;
    uint32_t u = 0;
    for (uint32_t i = 0; i < cnt; ++i) u += first_in_read(occ, occ_rd, s, i);
    return u;
}

// ---------------------------------------------------------------------------
// Row-wise product (Gustavson): read a's candidates are accumulated over its
// reliable k-mers (row a of A) and, for each, the other reads holding it
// (the k-mer's column).  Columns hold member words (read << 32) |
// (position << 1) | forward, in read order; rows hold (column, position << 1 |
// forward).  Per partner b > a the accumulator keeps the number of shared
// k-mers and the minimum of seed_key: the position in a decides alone (a
// position of a holds one k-mer, so the shared k-mers' positions in a are
// distinct), then seed_b and the strand ride along.

XS_HD uint64_t member_word(uint32_t read, uint32_t pos, bool fwd)
{
    return ((uint64_t)read << 32) | ((uint64_t)pos << 1) | (fwd ? 1u : 0u);
}

XS_HD uint64_t seed_key(uint32_t pa, uint32_t sb, bool rc)
{
    return ((uint64_t)pa << 32) | ((uint64_t)sb << 1) | (rc ? 1u : 0u);
}

// Column entries of a reliable run: its reads' first occurrences, in order.
XS_HD void run_members(const uint32_t *occ, const uint32_t *occ_rd, const uint32_t *fwd_bits,
                       const uint64_t *occ_off, uint64_t s, uint32_t cnt, uint32_t stride,
                       uint64_t *out)
{
    uint32_t j = 0;
    for (uint32_t i = 0; i < cnt; ++i) {
        if (!first_in_read(occ, occ_rd, s, i)) continue;
        const uint32_t q = occ[s + i], r = occ_rd[q];
        out[j++] = member_word(r, (uint32_t)((q - occ_off[r]) * stride), fwd_bit(fwd_bits, q));
    }
}

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kTableLg = 11;  // 2,048 partners per read in shared memory

struct RowTable {
    uint32_t *key;            // partner read id, kEmpty when free
    uint32_t *cnt;            // shared k-mers
    unsigned long long *best; // minimum seed_key
    uint32_t lg;              // 2^lg slots
};

XS_HD uint32_t table_slot(uint32_t b, uint32_t lg)
{
    return (b * 2654435761u) >> (32 - lg);  // multiplicative hash, top bits
}

// Adds one shared k-mer of partner b; false when the table is full.  On
// the device the slots are claimed and updated with shared-memory atomics
// (insertions from all threads of the block at once); on the host in order.
XS_HD bool table_add(const RowTable &t, uint32_t b, uint64_t key)
{
    const uint32_t mask = (1u << t.lg) - 1;
    uint32_t h = table_slot(b, t.lg);
    for (uint32_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
#if defined(__CUDA_ARCH__)
        const uint32_t prev = atomicCAS(&t.key[h], kEmpty, b);
#else
        const uint32_t prev = t.key[h];
        if (prev == kEmpty) t.key[h] = b;
#endif
        if (prev != kEmpty && prev != b) continue;
#if defined(__CUDA_ARCH__)
        atomicAdd(&t.cnt[h], 1u);
        atomicMin(&t.best[h], (unsigned long long)key);
#else
        t.cnt[h] += 1;
        if (key < t.best[h]) t.best[h] = key;
#endif
        return true;
    }
    return false;
}

// One (row entry, column member) product term of read a: a k-mer at
// position pa of a (forward fa) that read member>>32 also holds.
XS_HD bool row_term(const RowTable &t, uint32_t a, uint32_t pa, bool fa, uint64_t member,
                    const uint32_t *read_len, uint32_t k)
{
    const uint32_t b = (uint32_t)(member >> 32);
    if (b <= a) return true;
    const uint32_t pb = (uint32_t)(member & 0xFFFFFFFFu) >> 1;
    const bool rc = fa != ((member & 1u) != 0);
    return table_add(t, b, seed_key(pa, rc ? read_len[b] - k - pb : pb, rc));
}

// Bits per read id in a pair key: the smallest nb >= 1 with n_reads <= 2^nb.
inline uint32_t id_bits(uint32_t n_reads)
{
    uint32_t nb = 1;
    while (nb < 32 && ((uint64_t)1 << nb) < n_reads) ++nb;
    return nb;
}

}  // namespace xs
