"""Pins of the seed-discovery oracle (oracle/seeds.py) against closed forms,
exact-match invariants and a dense A * A^T built with numpy."""
import numpy as np

from oracle import seeds as S
from paper_2309_07270_gb300 import workloads as W


def pack(reads):
    return W.pack_reads([np.asarray(r, np.uint8) for r in reads])


def test_copies_and_reverse_copy_closed_form(orc):
    """Read 1 is read 0, read 2 its reverse complement: every k-mer of read 0
    occurs three times, so with the window [3, 3] all are reliable and the
    three pairs share all of them, with seeds at the start of each read."""
    rng = np.random.default_rng(1)
    while True:  # a read whose k-mers are all distinct, also across strands
        r0 = rng.integers(0, 4, 60).astype(np.uint8)
        codes = S.occurrences([r0.tolist()], 9)
        if len({c for c, *_ in codes}) == len(codes):
            break
    reads = [r0, r0.copy(), W.revcomp(r0)]
    packed, off, lens = pack(reads)
    n_k = 60 - 9 + 1
    got = S.candidate_pairs(packed, off, lens, k=9, lo=3, hi=3)
    assert got.tolist() == [(0, 1, 0, 0, 9, n_k), (0, 2 | S.PAIR_RC, 0, 0, 9, n_k),
                            (1, 2 | S.PAIR_RC, 0, 0, 9, n_k)]
    assert len(S.candidate_pairs(packed, off, lens, k=9, lo=4, hi=10)) == 0   # count 3 < lo
    assert len(S.candidate_pairs(packed, off, lens, k=9, lo=1, hi=2)) == 0    # count 3 > hi
    # the candidates align end to end: both extensions are exact
    res = orc.align_pairs(packed, off, lens, S.as_pairs(got), 1, -1, -1, 10)
    for r in res:
        assert (r["left_score"], r["left_begin_a"], r["left_begin_b"]) == (0, 0, 0)
        assert (r["right_score"], r["right_end_a"], r["right_end_b"]) == (51, 60, 60)


def overlap_set():
    """Overlapping noisy reads of a small genome, some stored reverse-complemented."""
    rng = np.random.default_rng(7)
    g = rng.integers(0, 4, 1500).astype(np.uint8)
    reads = []
    for s in range(0, 1200, 100):
        r, *_ = W.mutate(g[s:s + 300], rng)
        reads.append(W.revcomp(r) if rng.random() < 0.4 else r)
    return reads


def test_every_seed_is_an_exact_match_on_its_strand():
    reads = overlap_set()
    packed, off, lens = pack(reads)
    cands = S.candidate_pairs(packed, off, lens, k=15, lo=2, hi=6)
    assert len(cands) >= 8 and (cands["b"] >> 31).sum() >= 2
    for c in cands:
        a, b = reads[c["a"]], reads[c["b"] & 0x7FFFFFFF]
        if c["b"] >> 31:
            b = W.revcomp(b)
        sa, sb, k = int(c["seed_a"]), int(c["seed_b"]), int(c["seed_len"])
        assert np.array_equal(a[sa:sa + k], b[sb:sb + k])
        assert c["shared"] >= 1


def test_candidates_are_the_nonzeros_of_a_times_a_transpose():
    """A[r, m] = 1 when reliable k-mer m occurs in read r; the candidate set
    and its shared counts are the upper off-diagonal nonzeros of A @ A.T."""
    reads = overlap_set()
    packed, off, lens = pack(reads)
    codes = [r.tolist() for r in reads]
    keep = sorted(S.reliable_kmers(codes, 15, 2, 6))
    col = {c: i for i, c in enumerate(keep)}
    A = np.zeros((len(reads), len(keep)), np.int64)
    for code, r, _, _ in S.occurrences(codes, 15):
        if code in col:
            A[r, col[code]] = 1
    M = A @ A.T
    want = {(a, b): int(M[a, b]) for a in range(len(reads)) for b in range(a + 1, len(reads))
            if M[a, b]}
    cands = S.candidate_pairs(packed, off, lens, k=15, lo=2, hi=6)
    got = {(int(c["a"]), int(c["b"]) & 0x7FFFFFFF): int(c["shared"]) for c in cands}
    assert got == want


def test_seed_position_in_a_decides_alone():
    """A position of read a holds one k-mer, so the shared k-mers of a pair
    have distinct first positions in a: the smallest one picks the seed and
    the later tie-breaks (position in b, code) never decide.  Checked by
    brute force over every candidate pair."""
    reads = overlap_set()
    codes = [r.tolist() for r in reads]
    keep = S.reliable_kmers(codes, 15, 2, 6)
    first = {}
    for code, r, p, _ in S.occurrences(codes, 15):
        if code in keep:
            first.setdefault((r, code), p)
    by_read = {}
    for (r, code), p in first.items():
        by_read.setdefault(r, {})[code] = p
    packed, off, lens = pack(reads)
    cands = S.candidate_pairs(packed, off, lens, k=15, lo=2, hi=6)
    for c in cands:
        a, b = int(c["a"]), int(c["b"]) & 0x7FFFFFFF
        shared = set(by_read[a]) & set(by_read[b])
        pos_a = [by_read[a][m] for m in shared]
        assert len(pos_a) == len(set(pos_a)) == c["shared"]
        assert min(pos_a) == c["seed_a"]


def test_hand_case_golden():
    """The worked example of tests/golden/seeds_hand_case.md, derived by hand."""
    rc = S.PAIR_RC
    reads = [W.encode("ACGTA"), W.encode("CGTAC"), W.encode("GGGG")]
    packed, off, lens = pack(reads)
    for stride, lo, hi, want in ((1, 2, 3, [(0, 1 | rc, 0, 2, 3, 2)]),
                                 (1, 3, 3, [(0, 1 | rc, 0, 2, 3, 2)]),
                                 (1, 2, 2, []),
                                 (2, 2, 3, [(0, 1 | rc, 0, 2, 3, 2)])):
        got = S.candidate_pairs(packed, off, lens, k=3, lo=lo, hi=hi, stride=stride)
        assert got.tolist() == want, (stride, lo, hi)
    reads[1] = W.encode("GTACG")
    packed, off, lens = pack(reads)
    assert S.candidate_pairs(packed, off, lens, k=3, lo=2, hi=3).tolist() == [(0, 1, 0, 2, 3, 2)]
