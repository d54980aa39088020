"""The method on Python strings, for tiny inputs -- TEST INFRASTRUCTURE ONLY.

Brute force: every function enumerates substrings and compares strings.  Since
'A' < 'C' < 'G' < 'T' in ASCII, Python's string order is the paper's
lexicographic order (Sect. 2.1).  Used to pin the C oracle (a different method:
2-bit numbers and a hash table) and for the paper's worked examples.
"""
from __future__ import annotations

from collections import Counter

BASES = "ACGT"
_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def revcomp(s: str) -> str:
    """Reverse complement (Sect. 2.1)."""
    return "".join(_COMP[c] for c in reversed(s))


def canonical(s: str) -> str:
    """Lexicographically smaller of a string and its reverse complement (Sect. 2.1)."""
    r = revcomp(s)
    return s if s <= r else r


def value(s: str) -> int:
    """2-bit number of a string, first symbol most significant (Suppl. S4 [map])."""
    v = 0
    for c in s:
        v = 4 * v + BASES.index(c)
    return v


def from_value(v: int, length: int) -> str:
    return "".join(BASES[(v >> (2 * (length - 1 - i))) & 3] for i in range(length))


def segments(read: str):
    """Maximal runs of A/C/G/T (any other byte breaks the read)."""
    seg = []
    cur = []
    for c in read:
        if c in _COMP:
            cur.append(c)
        else:
            if cur:
                seg.append("".join(cur))
            cur = []
    if cur:
        seg.append("".join(cur))
    return seg


def kmers(read: str, k: int):
    for s in segments(read):
        for i in range(len(s) - k + 1):
            yield s[i:i + k]


def count_brute(reads, k, cutoff_min=1, cutoff_max=2**32 - 1):
    """Plain definition: canonical k-mer -> count, kept if ci <= n <= cx."""
    c = Counter(canonical(s) for r in reads for s in kmers(r, k))
    return {s: n for s, n in c.items() if cutoff_min <= n <= cutoff_max}


def allowed(mm: str) -> bool:
    """Sect. 2.2: not starting with AAA, not starting with ACA, no AA except at the start."""
    if mm.startswith("AAA") or mm.startswith("ACA"):
        return False
    return "AA" not in mm[1:]


def signature(kmer: str, m: int):
    """Sect. 2.2 (reading A): smallest allowed canonical m-mer; None if none."""
    cands = [canonical(kmer[i:i + m]) for i in range(len(kmer) - m + 1)]
    cands = [c for c in cands if allowed(c)]
    return min(cands) if cands else None


def canonical_minimizer(kmer: str, m: int) -> str:
    """Sect. 2.1: minimum over the canonical m-mers (MSPKmerCounter's choice)."""
    return min(canonical(kmer[i:i + m]) for i in range(len(kmer) - m + 1))


def superkmers(read: str, k: int, m: int, use_minimizer: bool = False):
    """Fig. 1: maximal runs of consecutive k-mers with one signature -> [(substring, sig)]."""
    out = []
    f = canonical_minimizer if use_minimizer else signature
    for s in segments(read):
        i = 0
        n = len(s) - k + 1
        while i < n:
            sig = f(s[i:i + k], m)
            j = i + 1
            while j < n and f(s[j:j + k], m) == sig:
                j += 1
            out.append((s[i:j + k - 1], sig))
            i = j
    return out


def kxmers(superkmer: str, k: int, x: int):
    """Sect. 2.3 / Fig. 2: greedy split into (k,x)-mers -> [(x', stored string)]."""
    n = len(superkmer) - k + 1
    direct = [superkmer[i:i + k] <= revcomp(superkmer[i:i + k]) for i in range(n)]
    out = []
    i = 0
    while i < n:
        ln = 1
        while ln < x + 1 and i + ln < n and direct[i + ln] == direct[i]:
            ln += 1
        s = superkmer[i:i + k + ln - 1]
        out.append((ln - 1, s if direct[i] else revcomp(s)))
        i += ln
    return out


def sort_kxmers(kx):
    """Fig. 2 order: k-mers before (k+1)-mers, each group lexicographically."""
    return sorted(kx, key=lambda t: (t[0], t[1]))
