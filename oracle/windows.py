"""Exact counts of one prefix class of canonical k-mers over every window of
a large read set of one read length -- TEST INFRASTRUCTURE ONLY.

The plain definition (Sect. 2.1: every k-long window of a read that holds
only A/C/G/T is one occurrence of the canonical k-mer min(s, revcomp(s))),
evaluated with numpy over reads reshaped to a matrix, for the canonical
k-mers whose first q symbols are a given string Q.  A window can only be
such a k-mer when it starts with Q or ends with revcomp(Q), so the q-mer
value of every position is computed (from the values of shorter windows:
a window of length 2n is its first n symbols shifted left by 2n, or-ed with
its last n) and only the windows that pass this test are built in full.
This makes the full-size workloads checkable in seconds on a sample of
about 1/4^q of their k-mers.  k <= 64 (two 64-bit words above 32), q <= 16.

Parity status: pinned by tests/test_oracle_pins.py against the C oracle's
counts and valid-position total.
"""
from __future__ import annotations

import numpy as np

_CODE = np.full(256, 4, dtype=np.uint8)
for _i, _c in enumerate(b"ACGT"):
    _CODE[_c] = _i
_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def _value(s: str) -> int:
    v = 0
    for ch in s:
        v = 4 * v + "ACGT".index(ch)
    return v


def _qmer_values(c: np.ndarray, q: int) -> np.ndarray:
    """Values of the windows of length q (power-of-two doubling, then the
    remainder), shape (rows, L - q + 1); uint16 for q <= 8, else uint32."""
    t = np.uint16 if q <= 8 else np.uint32
    L = c.shape[1]
    f = {1: c.astype(t)}
    n = 1
    while 2 * n <= q:
        f[2 * n] = (f[n][:, :L - 2 * n + 1] << t(2 * n)) | f[n][:, n:L - n + 1]
        n *= 2
    W = L - q + 1
    v = np.zeros((c.shape[0], W), dtype=t)
    off = 0
    for size in sorted(f, reverse=True):
        while off + size <= q:
            v = (v << t(2 * size)) | f[size][:, off:off + W]
            off += size
    assert off == q
    return v


def _chunk_class(bases, offsets, r0, r1, L, k, q, qv, rv):
    """Canonical k-mers of the class among reads [r0, r1) (one array per
    call: uint64 values for k <= 32, else (hi, lo) rows) and the chunk's
    number of valid windows."""
    W = L - k + 1
    m = bases[int(offsets[r0]):int(offsets[r1])].reshape(r1 - r0, L)
    c = _CODE[m]
    bad = c == 4
    cs = np.zeros((r1 - r0, L + 1), dtype=np.int16 if L < 32767 else np.int32)
    np.cumsum(bad, axis=1, out=cs[:, 1:])
    valid = (cs[:, k:] - cs[:, :W]) == 0
    npos = int(np.count_nonzero(valid))
    c0 = c & np.uint8(3)  # the code 4 of a non-base becomes 0; its windows are not valid
    vq = _qmer_values(c0, q)
    sel = valid & ((vq[:, :W] == qv) | (vq[:, k - q:k - q + W] == rv))
    rows, cols = np.nonzero(sel)
    if rows.size == 0:
        return None, npos
    win = c0[rows[:, None], cols[:, None] + np.arange(k)].astype(np.uint64)  # (n_sel, k)
    if k <= 32:
        fw = np.bitwise_or.reduce(win << (2 * (k - 1 - np.arange(k))).astype(np.uint64), axis=1)
        rc = np.bitwise_or.reduce((np.uint64(3) - win) << (2 * np.arange(k)).astype(np.uint64), axis=1)
        canon = np.minimum(fw, rc)
        return canon[(canon >> np.uint64(2 * (k - q))) == np.uint64(qv)], npos
    # k > 32: value = hi (first k - 32 symbols) * 4^32 + lo (last 32 symbols)
    h = k - 32
    rwin = (np.uint64(3) - win)[:, ::-1]  # the reverse complement's symbols in order

    def words(x):
        hi = np.bitwise_or.reduce(x[:, :h] << (2 * (h - 1 - np.arange(h))).astype(np.uint64), axis=1)
        lo = np.bitwise_or.reduce(x[:, h:] << (2 * (31 - np.arange(32))).astype(np.uint64), axis=1)
        return hi, lo

    fh, fl = words(win)
    rh, rl = words(rwin)
    use_r = (rh < fh) | ((rh == fh) & (rl < fl))
    ch, cl = np.where(use_r, rh, fh), np.where(use_r, rl, fl)
    keep = (ch >> np.uint64(2 * (h - q))) == np.uint64(qv) if q <= h else \
        ((ch << np.uint64(2 * (q - h))) | (cl >> np.uint64(64 - 2 * (q - h)))) == np.uint64(qv)
    return np.stack([ch[keep], cl[keep]], axis=1), npos


def prefix_class_counts(bases, offsets, k: int, prefix: str, chunk_reads: int = 100_000, threads: int = 0):
    """(values, counts) of every canonical k-mer whose first len(prefix)
    symbols are `prefix`, over all valid windows, values ascending; and the
    number of valid windows of the whole read set.  All reads must have one
    length.  values: uint64[n] for k <= 32; for 32 < k <= 64 uint64[n, 2],
    the most significant word first (the first k - 32 symbols, then the last
    32).  Chunks of reads are processed by `threads` threads (0: all cores)."""
    import concurrent.futures as cf
    import os
    q = len(prefix)
    assert 1 <= q <= 16 and q <= k <= 64
    bases = np.asarray(bases, dtype=np.uint8)
    offsets = np.asarray(offsets, dtype=np.uint64)
    n = offsets.size - 1
    wide = k > 32
    empty = (np.zeros((0, 2) if wide else 0, np.uint64), np.zeros(0, np.int64))
    if n == 0:
        return empty + (0,)
    lengths = np.diff(offsets)
    L = int(lengths[0])
    assert np.all(lengths == L), "reads of one length only"
    if L < k:
        return empty + (0,)
    t = np.uint16 if q <= 8 else np.uint32
    qv = t(_value(prefix))
    rv = t(_value("".join(_COMP[ch] for ch in reversed(prefix))))
    spans = [(r0, min(n, r0 + chunk_reads)) for r0 in range(0, n, chunk_reads)]
    nt = threads or min(16, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        parts = list(ex.map(lambda sp: _chunk_class(bases, offsets, sp[0], sp[1], L, k, q, qv, rv), spans))
    npos = sum(p[1] for p in parts)
    found = [p[0] for p in parts if p[0] is not None and len(p[0])]
    if not found:
        return empty + (npos,)
    allv = np.concatenate(found)
    if not wide:
        vals, counts = np.unique(allv, return_counts=True)
        return vals, counts.astype(np.int64), npos
    vals, counts = np.unique(allv, axis=0, return_counts=True)  # rows in (hi, lo) order
    return vals, counts.astype(np.int64), npos
