"""Seed discovery oracle: TEST INFRASTRUCTURE ONLY.

The step upstream of seed-and-extend: reliable k-mers (a frequency window
over all k-mer occurrences) and the candidate read pairs that share one,
i.e. the nonzeros of the sparse product A * A^T of the read-by-k-mer matrix
A (Section "Related works", diBELLA 2D paragraph: overlap detection by
sparse matrix multiplication; Section "Experimental Setup": k = 31, stride
1, DNA alphabet, LOWER_KMER_FREQ = 20 and UPPER_KMER_FREQ = 30 or 50).
The paper does not spell the rest out; the readings fixed here:

  K1  A k-mer is k consecutive bases of a read (k <= 32), taken at every
      stride-th start.  Its canonical form is the smaller, as a 2k-bit
      integer with the first base most significant, of the k-mer and its
      reverse complement: reads come from both strands.
  K2  A canonical k-mer's count is its number of occurrences over all reads,
      several in one read counted separately.  It is reliable iff
      lo <= count <= hi (both inclusive).
  K3  A[r, kmer] is the first occurrence (smallest position) of a reliable
      k-mer in read r, with the strand it was read on.
  K4  A candidate pair is a pair of reads a < b sharing at least one
      reliable k-mer (a nonzero of A * A^T off the diagonal).  It carries
      the number of shared reliable k-mers and one seed: the shared k-mer
      whose position in a is smallest (then: smallest position in b, then:
      smallest canonical code).  If the k-mer was read on the same strand
      in both reads the pair is forward with seed (pos_a, pos_b); otherwise
      it is a reverse-strand pair (read b's reverse complement) with seed
      (pos_a, len_b - k - pos_b).  seed_len = k.

Everything is plain loops and dictionaries over the definitions; it is
meant for small read sets.  The CUDA library does not use it.
"""
from __future__ import annotations

import numpy as np

from .oracle import ORC_PAIR, unpack

PAIR_RC = 0x80000000
CANDIDATE = np.dtype([("a", "<u4"), ("b", "<u4"), ("seed_a", "<u4"), ("seed_b", "<u4"),
                      ("seed_len", "<u4"), ("shared", "<u4")])


def _code(bases) -> int:
    v = 0
    for c in bases:
        v = (v << 2) | int(c)
    return v


def _revcomp(bases) -> list:
    return [3 - int(c) for c in reversed(list(bases))]


def read_codes(packed, read_off, read_len) -> list:
    return [unpack(packed, int(o), int(n)).tolist() for o, n in zip(read_off, read_len)]


def occurrences(reads, k: int, stride: int = 1):
    """Every k-mer occurrence: (canonical code, read, position, forward?).
    forward is True when the canonical form is the k-mer as read (K1)."""
    out = []
    for r, seq in enumerate(reads):
        for p in range(0, len(seq) - k + 1, stride):
            fwd = _code(seq[p:p + k])
            rev = _code(_revcomp(seq[p:p + k]))
            out.append((min(fwd, rev), r, p, fwd <= rev))
    return out


def reliable_kmers(reads, k: int, lo: int, hi: int, stride: int = 1) -> set:
    """Canonical k-mers whose total count lies in [lo, hi] (K2)."""
    count = {}
    for code, _, _, _ in occurrences(reads, k, stride):
        count[code] = count.get(code, 0) + 1
    return {c for c, n in count.items() if lo <= n <= hi}


def candidate_pairs(packed, read_off, read_len, k: int = 31, lo: int = 20, hi: int = 30,
                    stride: int = 1) -> np.ndarray:
    """The candidate pairs of K4, sorted by (a, b), as CANDIDATE records."""
    reads = read_codes(packed, read_off, read_len)
    keep = reliable_kmers(reads, k, lo, hi, stride)
    first = {}  # (read, code) -> (position, forward)        (K3)
    for code, r, p, fwd in occurrences(reads, k, stride):
        if code in keep and (r, code) not in first:
            first[(r, code)] = (p, fwd)
    by_kmer = {}
    for (r, code), (p, fwd) in first.items():
        by_kmer.setdefault(code, []).append((r, p, fwd))
    best = {}  # (a, b) -> [shared, key, seed_a, seed_b, rc]
    for code, occ in by_kmer.items():
        for x in range(len(occ)):
            for y in range(len(occ)):
                ra, pa, fa = occ[x]
                rb, pb, fb = occ[y]
                if ra >= rb:
                    continue
                rc = fa != fb
                sb = (len(reads[rb]) - k - pb) if rc else pb
                key = (pa, pb, code)
                cur = best.get((ra, rb))
                if cur is None:
                    best[(ra, rb)] = [1, key, pa, sb, rc]
                else:
                    cur[0] += 1
                    if key < cur[1]:
                        cur[1:] = [key, pa, sb, rc]
    out = np.zeros(len(best), CANDIDATE)
    for i, ((a, b), (shared, _, sa, sb, rc)) in enumerate(sorted(best.items())):
        out[i] = (a, b | (PAIR_RC if rc else 0), sa, sb, k, shared)
    return out


def as_pairs(cands: np.ndarray) -> np.ndarray:
    """The candidates as pair records for the aligner (ORC_PAIR layout)."""
    p = np.zeros(len(cands), ORC_PAIR)
    for f in ("a", "b", "seed_a", "seed_b", "seed_len"):
        p[f] = cands[f]
    return p
