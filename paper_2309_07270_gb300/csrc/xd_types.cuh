// Types and host/device helpers shared by the kernels and the host
// runtime (no kernels here).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace xd {

// Pruned cell.  Every threshold T - x is >= -x > -2^25 > NEG, and any
// live or pruned value times 16 plus 15 still fits in int32 (the packed
// best-cell key of the lockstep kernels).
constexpr int32_t NEG = -(1 << 26);
constexpr uint32_t FULL = 0xffffffffu;

struct Pair {
    uint32_t a, b, seed_a, seed_b, seed_len;
};

struct Scoring {
    int32_t match, mismatch, gap, x;
};

// Everything a kernel needs to decode and write one task.  Task t is the
// left (t even) or right (t odd) extension of pair t/2.
// Top bit of a pair's b: align against the reverse complement of read b
// (XDROP_PAIR_RC).  The library stores the reverse complement of every
// read after the reads themselves, rc_off bases further on, and an RC pair
// reads its b there; the band kernels never see the flag.
constexpr uint32_t kPairRC = 0x80000000u;

struct Job {
    const uint32_t *packed;  // the reads, then (rc_off > 0) their reverse complements
    int64_t n_words;         // words of the whole buffer
    int64_t rc_off;          // bases from a read to its reverse complement; 0 = none stored
    const uint64_t *read_off;
    const uint32_t *read_len;
    uint32_t n_reads;
    const Pair *pairs;
    uint64_t n_pairs;
    Scoring sc;
    int32_t *out;    // 7 int32 per pair (xdrop_result)
    int64_t *cells;  // per task cell count (counting launches only)
    // Serving requests only: finished / spilled task counters, the list of
    // spilled task ids, and the tag written to the host when all finished.
    uint32_t *ctr;
    uint32_t *spill_list;
    uint32_t tag;
};

// Overflow hand-off between tiers.
struct Spill {
    uint32_t *list;   // task ids
    uint32_t *count;  // number of ids in list
};

// One base stream c_k (k >= 1): c_k is base s0 + dir*(k-1) of the packed
// buffer.
struct Seq {
    const uint32_t *pk;
    int64_t nw;
    int64_t s0;
    int dir;
};

struct Ext {
    Seq A, B;
    int32_t m, n;
    uint32_t pair;
    int side;       // 0 left, 1 right
    uint32_t sa, sb, L;
    bool ok;
};

// ---------------------------------------------------------------------------
// Limits (also enforced on the host for host submits).
// ---------------------------------------------------------------------------
constexpr int64_t LEN_LIMIT = (int64_t)1 << 28;    // read length
constexpr int64_t SCORE_LIMIT = (int64_t)1 << 25;  // |score| * (len_a + len_b), and x

__host__ __device__ inline int32_t max_abs_score(const Scoring &s)
{
    int32_t a = s.match < 0 ? -s.match : s.match;
    int32_t b = s.mismatch < 0 ? -s.mismatch : s.mismatch;
    int32_t c = s.gap < 0 ? -s.gap : s.gap;
    int32_t m = a > b ? a : b;
    return m > c ? m : c;
}

// n_words: words of the reads themselves (without reverse complements);
// rc_ok: whether a pair may ask for the reverse strand of b.
__host__ __device__ inline bool pair_ok(const Pair &p, uint32_t n_reads,
                                        const uint32_t *read_len,
                                        const uint64_t *read_off,
                                        int64_t n_words, const Scoring &s, bool rc_ok)
{
    const uint32_t b = p.b & ~kPairRC;
    if ((p.b & kPairRC) && !rc_ok) return false;
    if (p.a >= n_reads || b >= n_reads) return false;
    uint64_t la = read_len[p.a], lb = read_len[b];
    if ((int64_t)la >= LEN_LIMIT || (int64_t)lb >= LEN_LIMIT) return false;
    if ((uint64_t)p.seed_a + p.seed_len > la) return false;
    if ((uint64_t)p.seed_b + p.seed_len > lb) return false;
    if ((int64_t)(la + lb) * max_abs_score(s) >= SCORE_LIMIT) return false;
    uint64_t oa = read_off[p.a], ob = read_off[b];
    if ((oa & 15) || (ob & 15)) return false;
    if ((int64_t)((oa + la + 15) / 16) > n_words) return false;
    if ((int64_t)((ob + lb + 15) / 16) > n_words) return false;
    return true;
}

__host__ __device__ inline bool job_pair_ok(const Job &J, const Pair &p)
{
    return pair_ok(p, J.n_reads, J.read_len, J.read_off, J.rc_off ? J.rc_off / 16 : J.n_words,
                   J.sc, J.rc_off > 0);
}

__device__ __forceinline__ Ext decode(const Job &J, uint32_t task)
{
    Ext e;
    e.pair = task >> 1;
    e.side = (int)(task & 1u);
    Pair p = J.pairs[e.pair];
    e.ok = job_pair_ok(J, p);
    e.sa = p.seed_a;
    e.sb = p.seed_b;
    e.L = p.seed_len;
    e.A.pk = e.B.pk = J.packed;
    e.A.nw = e.B.nw = J.n_words;
    e.m = e.n = 0;
    e.A.s0 = e.B.s0 = 0;
    e.A.dir = e.B.dir = 1;
    if (!e.ok) return e;
    const uint32_t b = p.b & ~kPairRC;
    int64_t oa = (int64_t)J.read_off[p.a];
    int64_t ob = (int64_t)J.read_off[b] + ((p.b & kPairRC) ? J.rc_off : 0);
    int64_t la = J.read_len[p.a], lb = J.read_len[b];
    if (e.side) {  // right: c_k = X[seed + L + k - 1]
        e.m = (int32_t)(la - p.seed_a - p.seed_len);
        e.n = (int32_t)(lb - p.seed_b - p.seed_len);
        e.A.s0 = oa + p.seed_a + p.seed_len;
        e.B.s0 = ob + p.seed_b + p.seed_len;
        e.A.dir = e.B.dir = 1;
    } else {       // left: c_k = X[seed - k]
        e.m = (int32_t)p.seed_a;
        e.n = (int32_t)p.seed_b;
        e.A.s0 = oa + (int64_t)p.seed_a - 1;
        e.B.s0 = ob + (int64_t)p.seed_b - 1;
        e.A.dir = e.B.dir = -1;
    }
    return e;
}

__device__ __forceinline__ void write_result(const Job &J, const Ext &e,
                                             int32_t score, int32_t bi,
                                             int32_t bj)
{
    int32_t *o = J.out + (size_t)e.pair * 7;
    if (e.side) {
        o[3] = score;
        o[4] = (int32_t)(e.sa + e.L) + bi;
        o[5] = (int32_t)(e.sb + e.L) + bj;
    } else {
        o[0] = score;
        o[1] = (int32_t)e.sa - bi;
        o[2] = (int32_t)e.sb - bj;
    }
}

}  // namespace xd
