"""KMC 2 database files (.kmc_pre / .kmc_suf) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module.  It writes the two files of the
supplement's "Database format" section from a counting result (canonical
k-mers with their counts), reads them back with the procedure that section
gives, and answers single k-mer queries the way its worked example does
(signature -> map -> prefix array -> suffix range -> binary search).  Plain
Python on integers and bytes; the signature comes from the oracle's C
restatement of Sect. 2.2 (``oracle.signature_of``).

Layout (Suppl. "Database format"; all integers least significant byte first):

* ``.kmc_pre``: "KMCP", the prefix arrays (one array of 4^lut uint64 per bin,
  in bin order, then one uint64 guard), the map (4^m + 1 uint32: signature ->
  array), the header, the header's distance from the 8 last bytes (uint32),
  "KMCP".
* header: kmer_length, mode (0), counter_size, lut_prefix_length,
  signature_length, min_count, max_count (uint32 each), total_kmers (uint64),
  seven unused uint32, KMC_VER = 0x200 (uint32): 68 bytes, no padding.
* ``.kmc_suf``: "KMCS", the records, "KMCS".  A record is the k-mer's suffix
  (its last k - lut symbols, leftmost symbol first, four symbols per byte,
  first symbol in the top bits) then the count on counter_size bytes.
* Records are grouped by array (bin), then ordered by k-mer value; element x
  of a bin's prefix array is the index of the bin's first record whose top
  lut symbols have value x (so element x + 1 minus one is its last).

Readings where the section leaves a choice (listed with the other readings
of the paper in the design notes):

* lut_prefix_length: (k mod 4) + 4 when that is at most k and the prefix
  arrays of all bins hold at most 2^24 entries, else k mod 4 (the section
  requires only that 4 divides k - lut; its example uses 4).
* counter_size: the fewest bytes (1..4) that hold the largest stored count.
* min_count and max_count are the cutoffs applied: max(cutoff_min, 1) and
  cutoff_max clamped to 2^32 - 1.

Parity status: pinned by tests/test_oracle_db.py (the section's marker,
header-position and byte-packing rules, the worked example's signature and
prefix values, and lookups equal to brute-force string counts).
"""
from __future__ import annotations

import struct
from typing import Dict, List, Sequence

from . import signature_of

KMC_VER = 0x200
HEADER_BYTES = 68
CODE = {"A": 0, "C": 1, "G": 2, "T": 3}
SYM = "ACGT"


def lut_prefix_length(k: int, n_bins: int) -> int:
    base = k % 4
    wide = base + 4
    if wide <= k and n_bins * (4 ** wide) <= (1 << 24):
        return wide
    return base


def counter_size(max_count: int) -> int:
    for c in (1, 2, 3):
        if max_count < 256 ** c:
            return c
    return 4


def value(s: str) -> int:
    v = 0
    for ch in s:
        v = 4 * v + CODE[ch]
    return v


def string_of(v: int, k: int) -> str:
    return "".join(SYM[(v >> (2 * (k - 1 - i))) & 3] for i in range(k))


def canonical_str(s: str) -> str:
    rc = "".join({"A": "T", "C": "G", "G": "C", "T": "A"}[c] for c in reversed(s))
    return min(s, rc)


def suffix_bytes(kmer: str, lut: int) -> bytes:
    """The last k - lut symbols, four per byte, leftmost symbol in the top bits."""
    suf = kmer[lut:]
    assert len(suf) % 4 == 0
    out = bytearray()
    for i in range(0, len(suf), 4):
        b = 0
        for ch in suf[i:i + 4]:
            b = 4 * b + CODE[ch]
        out.append(b)
    return bytes(out)


def write(k: int, m: int, kmers: Sequence[int], counts: Sequence[int], bin_map: Sequence[int],
          n_bins: int, cutoff_min: int, cutoff_max: int):
    """Returns (kmc_pre bytes, kmc_suf bytes) for canonical k-mer values and counts."""
    lut = lut_prefix_length(k, n_bins)
    csize = counter_size(max(counts) if len(counts) else 0)
    rows: List[tuple] = []
    for v, c in zip(kmers, counts):
        s = string_of(int(v), k)
        b = int(bin_map[signature_of(s, m)])
        rows.append((b, int(v), s, int(c)))
    rows.sort(key=lambda r: (r[0], r[1]))
    # prefix arrays: per bin, the first record of each prefix value
    P = 4 ** lut
    firsts = [0] * (n_bins * P + 1)
    counts_bp = [0] * (n_bins * P)
    for b, v, s, c in rows:
        counts_bp[b * P + value(s[:lut])] += 1
    run = 0
    for i in range(n_bins * P):
        firsts[i] = run
        run += counts_bp[i]
    firsts[n_bins * P] = run
    pre = bytearray(b"KMCP")
    pre += struct.pack("<%dQ" % len(firsts), *firsts)
    pre += struct.pack("<%dI" % len(bin_map), *[int(x) for x in bin_map])
    header = struct.pack("<7IQ7II", k, 0, csize, lut, m, max(cutoff_min, 1), min(cutoff_max, 2 ** 32 - 1), len(rows),
                         0, 0, 0, 0, 0, 0, 0, KMC_VER)
    assert len(header) == HEADER_BYTES
    pre += header
    pre += struct.pack("<I", len(header))
    pre += b"KMCP"
    suf = bytearray(b"KMCS")
    for b, v, s, c in rows:
        suf += suffix_bytes(s, lut)
        suf += c.to_bytes(csize, "little")
    suf += b"KMCS"
    return bytes(pre), bytes(suf)


def read(pre: bytes, suf: bytes) -> Dict:
    """The section's opening procedure: markers, header position, header, data."""
    assert pre[:4] == b"KMCP" and pre[-4:] == b"KMCP", "kmc_pre markers"
    assert suf[:4] == b"KMCS" and suf[-4:] == b"KMCS", "kmc_suf markers"
    x = struct.unpack_from("<I", pre, len(pre) - 8)[0]
    h0 = len(pre) - (x + 8)
    f = struct.unpack_from("<7IQ7II", pre, h0)
    hd = dict(kmer_length=f[0], mode=f[1], counter_size=f[2], lut_prefix_length=f[3],
              signature_length=f[4], min_count=f[5], max_count=f[6], total_kmers=f[7], kmc_ver=f[15])
    n_map = 4 ** hd["signature_length"] + 1
    map_off = h0 - 4 * n_map
    mp = list(struct.unpack_from("<%dI" % n_map, pre, map_off))
    n_pref = (map_off - 4) // 8
    prefixes = list(struct.unpack_from("<%dQ" % n_pref, pre, 4))
    rec = (hd["kmer_length"] - hd["lut_prefix_length"]) // 4 + hd["counter_size"]
    data = suf[4:-4]
    assert len(data) == rec * hd["total_kmers"], "kmc_suf size"
    return dict(header=hd, map=mp, prefixes=prefixes, data=data, record_bytes=rec)


def lookup(db: Dict, kmer: str) -> int:
    """Count of a k-mer (either strand) in the database, 0 when absent."""
    hd = db["header"]
    k, lut, m = hd["kmer_length"], hd["lut_prefix_length"], hd["signature_length"]
    assert len(kmer) == k
    c = canonical_str(kmer)
    arr = db["map"][signature_of(c, m)]
    P = 4 ** lut
    x = value(c[:lut])
    lo = db["prefixes"][arr * P + x]
    hi = db["prefixes"][arr * P + x + 1]
    key = suffix_bytes(c, lut)
    rec, sb = db["record_bytes"], len(key)
    data = db["data"]
    while lo < hi:  # binary search over the suffixes of the range
        mid = (lo + hi) // 2
        s = data[mid * rec: mid * rec + sb]
        if s == key:
            return int.from_bytes(data[mid * rec + sb: (mid + 1) * rec], "little")
        if s < key:
            lo = mid + 1
        else:
            hi = mid
    return 0
