"""Seeded synthetic inputs shaped like the paper's long-read workloads.

The paper measures on real E. coli long-read sets (29X: 8,605 reads, 100X:
91,394 reads; Section "Experimental Setup") that are not available here, so
these generators stand in for them.  They hold none of the alignment's
arithmetic: they only draw reads, plant seeds and pack bases.  Both the CUDA
path (through the C ABI) and the CPU oracle consume their output.

Error model (every workload): walk the template; per base draw u in [0, 1):
u < 0.04 substitute one of the three other bases uniformly, 0.04 <= u < 0.08
delete, 0.08 <= u < 0.12 insert one uniform random base and then emit the
template base, otherwise copy.  All randomness comes from
``numpy.random.Generator(PCG64(seed))``.

Packed layout: 2-bit codes A=0, C=1, G=2, T=3; 16 bases per little-endian
uint32, base k of the buffer in bits 2(k mod 16)..2(k mod 16)+1 of word
k / 16; every read starts at a multiple of 16 bases; the buffer ends with
at least ``PACK_TAIL_WORDS`` zero words.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PAIR_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("seed_a", "<u4"),
                       ("seed_b", "<u4"), ("seed_len", "<u4")])
SEED_LEN = 17
PACK_TAIL_WORDS = 64
PAIR_RC = 0x80000000  # in a pair's b: align against the reverse complement of read b
P_SUB, P_DEL, P_INS = 0.04, 0.04, 0.04
_CHUNK = 1 << 24


@dataclasses.dataclass
class Workload:
    """Packed reads, pair table and scoring of one synthetic workload."""
    name: str
    packed: np.ndarray      # uint32 words
    read_off: np.ndarray    # uint64, start of each read in bases
    read_len: np.ndarray    # uint32
    pairs: np.ndarray       # PAIR_DTYPE
    match: int = 1
    mismatch: int = -1
    gap: int = -1
    x: int = 50
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_pairs(self) -> int:
        return int(self.pairs.shape[0])

    @property
    def n_reads(self) -> int:
        return int(self.read_len.shape[0])

    def with_x(self, x: int) -> "Workload":
        return dataclasses.replace(self, x=int(x), name=f"{self.name}-x{x}")

    def subset(self, idx) -> "Workload":
        """The same reads with only the pairs at ``idx``."""
        return dataclasses.replace(self, pairs=np.ascontiguousarray(self.pairs[idx]))

    def codes(self, r: int) -> np.ndarray:
        """Unpacked codes of read r (slow; for tests and small cases)."""
        off, n = int(self.read_off[r]), int(self.read_len[r])
        w = self.packed[off // 16: (off + n + 15) // 16 + 1]
        sh = (2 * np.arange(16, dtype=np.uint32))
        c = ((w[:, None] >> sh[None, :]) & 3).astype(np.uint8).reshape(-1)
        return c[off % 16: off % 16 + n]


def pack_reads(reads) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Pack a list of code arrays (values 0..3) at 16-base-aligned offsets."""
    lens = np.array([len(r) for r in reads], dtype=np.uint64)
    padded = (lens + 15) // 16 * 16
    offs = np.zeros(len(reads), dtype=np.uint64)
    if len(reads) > 1:
        offs[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum()) if len(reads) else 0
    words = total // 16 + PACK_TAIL_WORDS
    packed = np.zeros(words, dtype=np.uint32)
    shifts = (2 * np.arange(16, dtype=np.uint32))[None, :]
    # Pack read by read, grouping small reads into one buffer pass.
    start_word = 0
    pending = []
    pending_len = 0

    def flush():
        nonlocal start_word, pending, pending_len
        if not pending:
            return
        cat = np.zeros(pending_len, dtype=np.uint8)
        pos = 0
        for r, pl in pending:
            cat[pos:pos + len(r)] = r
            pos += pl
        w = (cat.reshape(-1, 16).astype(np.uint32) << shifts)
        w = np.bitwise_or.reduce(w, axis=1)
        packed[start_word:start_word + w.shape[0]] = w
        start_word += w.shape[0]
        pending = []
        pending_len = 0

    for r, pl in zip(reads, padded):
        pending.append((np.asarray(r, dtype=np.uint8), int(pl)))
        pending_len += int(pl)
        if pending_len >= _CHUNK:
            flush()
    flush()
    return packed, offs, lens.astype(np.uint32)


def mutate(template: np.ndarray, rng: np.random.Generator,
           protect: np.ndarray | None = None, rates=None):
    """Apply the error model to ``template`` (codes); ``rates`` =
    (substitution, deletion, insertion) replaces the default 4% each.

    Returns (read, counts, sub, dele, ins): the erroneous copy, the number of
    read bases each template base emitted (0, 1 or 2), and the per-template
    base error flags.  ``protect`` (bool, template length) suppresses every
    error type on the flagged template bases.
    """
    L = template.shape[0]
    reads, counts_all, subs, dels, inss = [], [], [], [], []
    for c0 in range(0, max(L, 1), _CHUNK):
        t = template[c0:c0 + _CHUNK]
        n = t.shape[0]
        if n == 0:
            break
        p_sub, p_del, p_ins = rates if rates is not None else (P_SUB, P_DEL, P_INS)
        u = rng.random(n, dtype=np.float32)
        sub = u < p_sub
        dele = (u >= p_sub) & (u < p_sub + p_del)
        ins = (u >= p_sub + p_del) & (u < p_sub + p_del + p_ins)
        if protect is not None:
            keep = ~protect[c0:c0 + n]
            sub &= keep
            dele &= keep
            ins &= keep
        shift = rng.integers(1, 4, size=n, dtype=np.uint8)
        newbase = rng.integers(0, 4, size=n, dtype=np.uint8)
        base = np.where(sub, (t + shift) & 3, t).astype(np.uint8)
        counts = np.ones(n, dtype=np.uint8)
        counts[dele] = 0
        counts[ins] = 2
        ends = np.cumsum(counts, dtype=np.int64)
        out = np.empty(int(ends[-1]) if n else 0, dtype=np.uint8)
        emit = counts > 0
        out[ends[emit] - 1] = base[emit]
        out[ends[ins] - 2] = newbase[ins]
        reads.append(out)
        counts_all.append(counts)
        subs.append(sub)
        dels.append(dele)
        inss.append(ins)
    if not reads:
        z = np.zeros(0, dtype=np.uint8)
        zb = np.zeros(0, dtype=bool)
        return z, z, zb, zb, zb
    return (np.concatenate(reads), np.concatenate(counts_all),
            np.concatenate(subs), np.concatenate(dels), np.concatenate(inss))


def _template_to_read(counts: np.ndarray) -> np.ndarray:
    """Read position of each template base (meaningful where it was emitted)."""
    return (np.cumsum(counts, dtype=np.int64) - 1).astype(np.int64)


def _seed_ok(sub, dele, ins, k=SEED_LEN) -> np.ndarray:
    """ok[t]: template bases t..t+k-1 are each copied exactly (no
    substitution, no deletion) and no base was inserted between them, so
    they form k contiguous identical bases in the read."""
    n = sub.shape[0]
    if n < k:
        return np.zeros(0, dtype=bool)
    ce = np.concatenate([[0], np.cumsum((sub | dele).astype(np.int64))])
    ci = np.concatenate([[0], np.cumsum(ins.astype(np.int64))])
    t = np.arange(n - k + 1)
    inexact = ce[t + k] - ce[t]
    inserted = ci[t + k] - ci[t + 1]
    return (inexact == 0) & (inserted == 0)


# ----------------------------------------------------------------------------
# Workload 1: independent template pairs with one planted seed.
# ----------------------------------------------------------------------------

def template_pairs(n_pairs=200, len_lo=2000, len_hi=4000, seed=0, x=50,
                   name="template-pairs") -> Workload:
    """Two independent erroneous copies of a uniform random template per
    pair, with errors suppressed on one 17-base window (the planted seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reads = []
    pairs = np.zeros(n_pairs, dtype=PAIR_DTYPE)
    for p in range(n_pairs):
        L = int(rng.integers(len_lo, len_hi + 1))
        tpl = rng.integers(0, 4, size=L, dtype=np.uint8)
        t0 = int(rng.integers(0, L - SEED_LEN + 1))
        prot = np.zeros(L, dtype=bool)
        prot[t0:t0 + SEED_LEN] = True
        ra, ca, *_ = mutate(tpl, rng, prot)
        rb, cb, *_ = mutate(tpl, rng, prot)
        pairs[p] = (2 * p, 2 * p + 1, _template_to_read(ca)[t0],
                    _template_to_read(cb)[t0], SEED_LEN)
        reads += [ra, rb]
    packed, offs, lens = pack_reads(reads)
    return Workload(name, packed, offs, lens, pairs, 1, -1, -1, x,
                    dict(seed=seed, n_pairs=n_pairs, len=(len_lo, len_hi)))


# ----------------------------------------------------------------------------
# Workloads 2 and 4: reads sampled from one random genome, all true overlaps.
# ----------------------------------------------------------------------------

def _lognormal_lengths(rng, n, mean, sd, min_len, max_len):
    s2 = math.log(1.0 + (sd / mean) ** 2)
    mu = math.log(mean) - s2 / 2.0
    out = rng.lognormal(mu, math.sqrt(s2), size=n)
    bad = out < min_len
    while bad.any():
        out[bad] = rng.lognormal(mu, math.sqrt(s2), size=int(bad.sum()))
        bad = out < min_len
    return np.minimum(out.astype(np.int64), max_len)


def genome_overlaps(genome_len=4_600_000, coverage=29.0, mean_len=10_000,
                    sd_len=6_000, min_len=1_000, min_overlap=2_000, seed=1,
                    x=50, max_reads=None, name=None) -> Workload:
    """Forward-strand reads of one uniform random genome; every pair of reads
    whose template intervals overlap by >= min_overlap bases becomes a pair,
    seeded by the error-free 17-base window closest to the overlap centre
    (ties to the lower coordinate).  Pairs without such a window are
    dropped and counted in ``meta['dropped']``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    G = int(genome_len)
    genome = rng.integers(0, 4, size=G, dtype=np.uint8)
    n_reads = int(math.ceil(coverage * G / mean_len))
    if max_reads is not None:
        n_reads = min(n_reads, int(max_reads))
    lens = _lognormal_lengths(rng, n_reads, mean_len, sd_len, min_len, G)
    starts = rng.integers(0, G - lens + 1, dtype=np.int64)

    reads, tmaps, oks = [], [], []
    for r in range(n_reads):
        tpl = genome[starts[r]:starts[r] + lens[r]]
        rd, cnt, sub, dele, ins = mutate(tpl, rng)
        reads.append(rd)
        tmaps.append(_template_to_read(cnt).astype(np.int32))
        oks.append(_seed_ok(sub, dele, ins))
    ends = starts + lens

    # All pairs with template overlap >= min_overlap.
    order = np.argsort(starts, kind="stable")
    s_sorted = starts[order]
    pa, pb = [], []
    for rank, r in enumerate(order):
        hi = np.searchsorted(s_sorted, ends[r] - min_overlap, side="right")
        cand = order[rank + 1:hi]
        if cand.size == 0:
            continue
        ov = np.minimum(ends[r], ends[cand]) - np.maximum(starts[r], starts[cand])
        cand = cand[ov >= min_overlap]
        pa.append(np.full(cand.size, r, dtype=np.int64))
        pb.append(cand.astype(np.int64))
    pa = np.concatenate(pa) if pa else np.zeros(0, np.int64)
    pb = np.concatenate(pb) if pb else np.zeros(0, np.int64)

    seeds = _choose_seeds(pa, pb, starts, ends, oks)
    keep = seeds >= 0
    pa, pb, t = pa[keep], pb[keep], seeds[keep]
    pairs = np.zeros(pa.size, dtype=PAIR_DTYPE)
    pairs["a"] = pa
    pairs["b"] = pb
    sa = np.empty(pa.size, dtype=np.int64)
    sb = np.empty(pa.size, dtype=np.int64)
    for idx in range(pa.size):
        sa[idx] = tmaps[pa[idx]][t[idx] - starts[pa[idx]]]
        sb[idx] = tmaps[pb[idx]][t[idx] - starts[pb[idx]]]
    pairs["seed_a"] = sa
    pairs["seed_b"] = sb
    pairs["seed_len"] = SEED_LEN
    packed, offs, rl = pack_reads(reads)
    nm = name or f"genome-{coverage:g}x"
    return Workload(nm, packed, offs, rl, pairs, 1, -1, -1, x,
                    dict(seed=seed, genome_len=G, coverage=coverage,
                         n_reads=n_reads, dropped=int((~keep).sum()),
                         mean_len=mean_len, sd_len=sd_len))


def sequencing_reads(genome_len=200_000, coverage=29.0, mean_len=10_000, sd_len=6_000,
                     min_len=1_000, rc_frac=0.5, seed=11, error_rate=None):
    """Reads of one uniform random genome under the error model (or, with
    ``error_rate``, substitutions, deletions and insertions at a third of it
    each), each one stored as its reverse complement with probability
    ``rc_frac`` (reads come from both strands): the input of seed discovery.
    Lengths are lognormal as in genome_overlaps.  Returns (packed,
    read_off, read_len)."""
    rates = None if error_rate is None else (error_rate / 3,) * 3
    rng = np.random.Generator(np.random.PCG64(seed))
    G = int(genome_len)
    genome = rng.integers(0, 4, size=G, dtype=np.uint8)
    n_reads = max(int(math.ceil(coverage * G / mean_len)), 1)
    lens = _lognormal_lengths(rng, n_reads, mean_len, sd_len, min(min_len, G), G)
    starts = rng.integers(0, G - lens + 1, dtype=np.int64)
    flip = rng.random(n_reads) < rc_frac
    reads = []
    for r in range(n_reads):
        rd = mutate(genome[starts[r]:starts[r] + lens[r]], rng, rates=rates)[0]
        reads.append(revcomp(rd) if flip[r] else rd)
    return pack_reads(reads)


def _choose_seeds(pa, pb, starts, ends, oks, radius=1024):
    """Template coordinate of the chosen seed window per pair, -1 if none."""
    out = np.full(pa.size, -1, dtype=np.int64)
    lo = np.maximum(starts[pa], starts[pb])
    hi = np.minimum(ends[pa], ends[pb]) - SEED_LEN  # last window start
    c2 = lo + hi  # twice the centre of the window starts
    # Candidate order by (|2t - c2|, t): offsets from floor(c2/2).
    r = np.arange(radius)
    even = np.empty(2 * radius + 1, np.int64)
    even[0] = 0
    even[1::2] = -(r + 1)
    even[2::2] = r + 1
    odd = np.empty(2 * radius, np.int64)
    odd[0::2] = -r
    odd[1::2] = r + 1
    for idx in range(pa.size):
        if hi[idx] < lo[idx]:
            continue
        base = c2[idx] // 2
        offs = even if c2[idx] % 2 == 0 else odd
        t = base + offs
        t = t[(t >= lo[idx]) & (t <= hi[idx])]
        a_ok = oks[pa[idx]]
        b_ok = oks[pb[idx]]
        ok = a_ok[t - starts[pa[idx]]] & b_ok[t - starts[pb[idx]]]
        hit = np.flatnonzero(ok)
        if hit.size:
            out[idx] = t[hit[0]]
            continue
        # Rare: nothing near the centre; scan the whole overlap.
        tt = np.arange(lo[idx], hi[idx] + 1)
        ok = a_ok[tt - starts[pa[idx]]] & b_ok[tt - starts[pb[idx]]]
        hit = np.flatnonzero(ok)
        if hit.size:
            key = np.abs(2 * tt[hit] - c2[idx])  # argmin keeps the lower t
            out[idx] = tt[hit[np.argmin(key)]]
    return out


# ----------------------------------------------------------------------------
# Workload 3: heavy-tailed lengths, 80 % true overlaps, 20 % unrelated pairs.
# ----------------------------------------------------------------------------

def _pareto_lengths(rng, n, xm=100.0, alpha=1.5, cap=50_000):
    fmax = 1.0 - (xm / cap) ** alpha
    u = rng.random(n) * fmax
    return np.maximum((xm * (1.0 - u) ** (-1.0 / alpha)).astype(np.int64),
                      SEED_LEN)


def uneven_pairs(n_pairs=1_000_000, true_frac=0.8, seed=3, x=50,
                 name=None) -> Workload:
    """Pareto(x_m=100, alpha=1.5) lengths truncated at 50 kb.  A fraction
    ``true_frac`` of pairs are two erroneous copies of one template with a
    planted seed; the rest are two independent random reads of
    independently drawn lengths sharing one random 17-mer at random
    positions (X-drop dies early on them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_true = int(round(n_pairs * true_frac))
    n_rand = n_pairs - n_true
    kind = np.zeros(n_pairs, dtype=bool)
    kind[rng.permutation(n_pairs)[:n_true]] = True

    # True pairs: concatenate all templates and mutate them in one pass per
    # copy; split the copies at template boundaries.
    tl = _pareto_lengths(rng, n_true)
    tstart = np.concatenate([[0], np.cumsum(tl)])
    tpl = rng.integers(0, 4, size=int(tstart[-1]), dtype=np.uint8)
    t0 = (rng.random(n_true) * (tl - SEED_LEN + 1)).astype(np.int64)
    prot = np.zeros(tpl.size, dtype=bool)
    cov = np.zeros(tpl.size + 1, dtype=np.int32)
    np.add.at(cov, tstart[:-1] + t0, 1)
    np.add.at(cov, tstart[:-1] + t0 + SEED_LEN, -1)
    prot[:] = np.cumsum(cov[:-1]) > 0
    copies = []
    for _ in range(2):
        rd, cnt, *_ = mutate(tpl, rng, prot)
        ends = np.cumsum(cnt, dtype=np.int64)
        rstart = np.concatenate([[0], ends[tstart[1:] - 1]])
        seedpos = ends[tstart[:-1] + t0] - 1 - rstart[:-1]
        copies.append((rd, rstart, seedpos))

    # Random pairs: independent reads, one shared random 17-mer.
    la = _pareto_lengths(rng, n_rand)
    lb = _pareto_lengths(rng, n_rand)
    kmers = rng.integers(0, 4, size=(n_rand, SEED_LEN), dtype=np.uint8)
    pos_a = (rng.random(n_rand) * (la - SEED_LEN + 1)).astype(np.int64)
    pos_b = (rng.random(n_rand) * (lb - SEED_LEN + 1)).astype(np.int64)
    rand_a = rng.integers(0, 4, size=int(la.sum()), dtype=np.uint8)
    rand_b = rng.integers(0, 4, size=int(lb.sum()), dtype=np.uint8)
    sa_start = np.concatenate([[0], np.cumsum(la)])
    sb_start = np.concatenate([[0], np.cumsum(lb)])
    ia = (sa_start[:-1] + pos_a)[:, None] + np.arange(SEED_LEN)[None, :]
    ib = (sb_start[:-1] + pos_b)[:, None] + np.arange(SEED_LEN)[None, :]
    rand_a[ia.reshape(-1)] = kmers.reshape(-1)
    rand_b[ib.reshape(-1)] = kmers.reshape(-1)

    reads = []
    pairs = np.zeros(n_pairs, dtype=PAIR_DTYPE)
    it = ir = 0
    (ra, rsa, spa), (rb, rsb, spb) = copies
    for p in range(n_pairs):
        if kind[p]:
            reads.append(ra[rsa[it]:rsa[it + 1]])
            reads.append(rb[rsb[it]:rsb[it + 1]])
            pairs[p] = (2 * p, 2 * p + 1, spa[it], spb[it], SEED_LEN)
            it += 1
        else:
            reads.append(rand_a[sa_start[ir]:sa_start[ir + 1]])
            reads.append(rand_b[sb_start[ir]:sb_start[ir + 1]])
            pairs[p] = (2 * p, 2 * p + 1, pos_a[ir], pos_b[ir], SEED_LEN)
            ir += 1
    packed, offs, rl = pack_reads(reads)
    return Workload(name or f"uneven-{n_pairs}", packed, offs, rl, pairs,
                    1, -1, -1, x, dict(seed=seed, n_true=n_true,
                                       n_random=n_rand))


# ----------------------------------------------------------------------------
# Workload 5: arrival schedule of 25 producers drawing from a pair pool.
# ----------------------------------------------------------------------------

def serving_schedule(n_pool_pairs, n_producers=25, rate_pairs_per_s=1e6,
                     duration_s=60.0, batch_lo=1_000, batch_hi=20_000,
                     seed_base=100):
    """Per producer, a list of (arrival_time_s, pair_indices) with Poisson
    arrivals whose aggregate pair rate is ``rate_pairs_per_s``."""
    mean_batch = 0.5 * (batch_lo + batch_hi)
    per_prod_rate = rate_pairs_per_s / n_producers / mean_batch
    out = []
    for p in range(n_producers):
        rng = np.random.Generator(np.random.PCG64(seed_base + p))
        t = 0.0
        items = []
        while True:
            t += rng.exponential(1.0 / per_prod_rate)
            if t >= duration_s:
                break
            k = int(rng.integers(batch_lo, batch_hi + 1))
            idx = rng.integers(0, n_pool_pairs, size=k)
            items.append((t, idx))
        out.append(items)
    return out


def tiny_pairs(n_pairs=64, len_lo=0, len_hi=200, seed=7, x=20,
               name="tiny") -> Workload:
    """Small template pairs with lengths down to 0 (edge cases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reads = []
    pairs = np.zeros(n_pairs, dtype=PAIR_DTYPE)
    for p in range(n_pairs):
        L = int(rng.integers(len_lo, len_hi + 1)) + SEED_LEN
        tpl = rng.integers(0, 4, size=L, dtype=np.uint8)
        t0 = int(rng.integers(0, L - SEED_LEN + 1))
        prot = np.zeros(L, dtype=bool)
        prot[t0:t0 + SEED_LEN] = True
        ra, ca, *_ = mutate(tpl, rng, prot)
        rb, cb, *_ = mutate(tpl, rng, prot)
        pairs[p] = (2 * p, 2 * p + 1, _template_to_read(ca)[t0],
                    _template_to_read(cb)[t0], SEED_LEN)
        reads += [ra, rb]
    packed, offs, lens = pack_reads(reads)
    return Workload(name, packed, offs, lens, pairs, 1, -1, -1, x,
                    dict(seed=seed))


def from_sequences(seqs_a, seqs_b, seeds, match=1, mismatch=-1, gap=-1, x=50,
                   name="explicit") -> Workload:
    """Build a workload from explicit code arrays and (seed_a, seed_b,
    seed_len) triples, one pair per (a, b)."""
    reads = []
    pairs = np.zeros(len(seqs_a), dtype=PAIR_DTYPE)
    for p, (sa, sb, sd) in enumerate(zip(seqs_a, seqs_b, seeds)):
        reads += [np.asarray(sa, np.uint8), np.asarray(sb, np.uint8)]
        pairs[p] = (2 * p, 2 * p + 1, sd[0], sd[1], sd[2])
    packed, offs, lens = pack_reads(reads)
    return Workload(name, packed, offs, lens, pairs, match, mismatch, gap, x,
                    {})


ACGT = "ACGT"


def encode(s: str) -> np.ndarray:
    """Codes of an ACGT string."""
    return np.array([ACGT.index(ch) for ch in s], dtype=np.uint8)


def revcomp(codes: np.ndarray) -> np.ndarray:
    """Reverse complement of a code array (A=0, C=1, G=2, T=3)."""
    return (3 - np.asarray(codes, dtype=np.uint8)[::-1]).astype(np.uint8)


def reverse_strand(w: Workload, frac: float = 0.5, seed: int = 0) -> Workload:
    """The same alignments with a fraction of the pairs on the reverse
    strand: for each chosen pair the reverse complement of its read b is
    stored as a new read, and the pair points at that read with PAIR_RC
    set.  Aligning against the reverse complement of the stored read gives
    back read b, so every result must equal the original workload's."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = w.pairs.copy()
    pick = np.flatnonzero(rng.random(len(pairs)) < frac)
    reads = [w.codes(r) for r in range(len(w.read_len))]
    rc_of = {}
    for p in pick:
        b = int(pairs["b"][p])
        if b not in rc_of:
            rc_of[b] = len(reads)
            reads.append(revcomp(reads[b]))
        pairs["b"][p] = np.uint32(rc_of[b] | PAIR_RC)
    packed, off, lens = pack_reads(reads)
    return dataclasses.replace(w, packed=packed, read_off=off, read_len=lens.astype(np.uint32),
                               pairs=pairs, name=f"{w.name}-rc{frac:g}")
