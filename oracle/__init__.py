"""CPU oracle for KMC 2's k-mer counting -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path
(``paper_1407_1507_gb300``) and never imports it; the two meet only in the
seeded input generator ``paper_1407_1507_gb300.synth``, which holds none of the
method's arithmetic.

Two layers:

* ``kmc_oracle.c`` (plain C, built with gcc): the plain definition of the
  result (hash-map counting of canonical k-mers with cutoffs), the Sect. 2.2
  signature, the Fig. 1 super k-mer split, the Sect. 2.3 / Fig. 2 (k,x)-mer
  split and the Sect. 2.4 bin map.  Bound through ctypes below.
* ``strings.py``: the same definitions on Python strings for tiny inputs
  (brute force; the paper's worked examples).

Parity status of each function is listed in the module docstrings; every
function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkmc_oracle.so")
NO_KMER = 0xFFFFFFFF
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc; returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        intp = ctypes.POINTER(ctypes.c_int)
        lib.oracle_code.argtypes = [ctypes.c_uint8]
        lib.oracle_code.restype = ctypes.c_int
        lib.oracle_mmer_allowed.argtypes = [ctypes.c_uint32, ctypes.c_int]
        lib.oracle_mmer_allowed.restype = ctypes.c_int
        lib.oracle_signature.argtypes = [intp, ctypes.c_int, ctypes.c_int]
        lib.oracle_signature.restype = ctypes.c_uint32
        lib.oracle_position_sigs.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u32p]
        lib.oracle_position_sigs.restype = None
        lib.oracle_superkmers.argtypes = [u8p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint32, u64p, u32p, u32p, ctypes.c_uint64]
        lib.oracle_superkmers.restype = ctypes.c_uint64
        lib.oracle_kxmers.argtypes = [intp, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u64p, u32p,
                                      u32p, u64p, u64p, ctypes.c_uint64]
        lib.oracle_kxmers.restype = ctypes.c_uint64
        lib.oracle_bin_map.argtypes = [u64p, ctypes.c_uint32, ctypes.c_uint32, u32p]
        lib.oracle_bin_map.restype = None
        lib.oracle_count.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u64p, u32p,
                                     ctypes.c_uint64, u64p, u64p]
        lib.oracle_count.restype = ctypes.c_int
        lib.oracle_count_mode.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p,
                                          u32p, ctypes.c_uint64, u64p, u64p]
        lib.oracle_count_mode.restype = ctypes.c_int
        lib.oracle_count_sample.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, u64p, u32p, ctypes.c_uint64, u64p, u64p]
        lib.oracle_count_sample.restype = ctypes.c_int
        lib.oracle_hash_parts.argtypes = [u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64, u64p]
        lib.oracle_hash_parts.restype = None
        _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def as_reads(reads):
    """list[str|bytes] -> (bases uint8, offsets uint64)."""
    bs = [r.encode() if isinstance(r, str) else bytes(r) for r in reads]
    offsets = np.zeros(len(bs) + 1, dtype=np.uint64)
    np.cumsum([len(b) for b in bs], out=offsets[1:])
    bases = np.frombuffer(b"".join(bs), dtype=np.uint8).copy() if bs else np.zeros(0, np.uint8)
    return bases, offsets


def count(bases, offsets, k, cutoff_min=1, cutoff_max=2**32 - 1, threads=1, passes=1,
          return_npos=False, canonical=True, counter_max=0):
    """Plain-definition count (C).  Returns (kmers uint64[n, words], counts uint32[n]).

    canonical=False counts k-mers as read (Suppl. S1 -b).  counter_max > 0
    reports min(count, counter_max) for the k-mers the cutoffs keep (Suppl. S1
    -cs, "maximal value of a counter"; the cutoffs apply to the true count)."""
    lib = _load()
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    words = (k + 31) // 32
    n_out = ctypes.c_uint64(0)
    n_pos = ctypes.c_uint64(0)
    cap = 0
    kms = np.zeros((1, words), dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint32)
    for _ in range(2):
        rc = lib.oracle_count_mode(_p(bases, ctypes.c_uint8), _p(offsets, ctypes.c_uint64),
                                   offsets.size - 1, k, cutoff_min, cutoff_max, int(bool(canonical)),
                                   threads, passes, _p(kms, ctypes.c_uint64), _p(cnt, ctypes.c_uint32),
                                   cap, ctypes.byref(n_out), ctypes.byref(n_pos))
        if rc == -3:
            cap = n_out.value
            kms = np.zeros((max(cap, 1), words), dtype=np.uint64)
            cnt = np.zeros(max(cap, 1), dtype=np.uint32)
            continue
        if rc != 0:
            raise RuntimeError(f"oracle_count failed: {rc}")
        break
    n = n_out.value
    cnt = cnt[:n]
    if counter_max:
        cnt = np.minimum(cnt, np.uint32(min(counter_max, 2**32 - 1)))
    res = (kms[:n], cnt)
    return res + (n_pos.value,) if return_npos else res


def count_sample(bases, offsets, k, cutoff_min, cutoff_max, passes, which, threads=16):
    """Exact counts of one hash class of k-mers (about 1/passes of them) and
    the number of valid k-mer positions: (kmers, counts, n_pos).  The class
    is the k-mers c with in_sample(c) true for the same (passes, which,
    threads)."""
    lib = _load()
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    words = (k + 31) // 32
    n_out, n_pos = ctypes.c_uint64(0), ctypes.c_uint64(0)
    cap = 0
    kms = np.zeros((1, words), dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint32)
    for _ in range(2):
        rc = lib.oracle_count_sample(_p(bases, ctypes.c_uint8), _p(offsets, ctypes.c_uint64), offsets.size - 1,
                                     k, cutoff_min, cutoff_max, 1, threads, passes, which,
                                     _p(kms, ctypes.c_uint64), _p(cnt, ctypes.c_uint32), cap,
                                     ctypes.byref(n_out), ctypes.byref(n_pos))
        if rc == -3:
            cap = n_out.value
            kms = np.zeros((max(cap, 1), words), dtype=np.uint64)
            cnt = np.zeros(max(cap, 1), dtype=np.uint32)
            continue
        if rc != 0:
            raise RuntimeError(f"oracle_count_sample failed: {rc}")
        break
    n = n_out.value
    return kms[:n], cnt[:n], n_pos.value


def in_sample(kmers, k, passes, which, threads=16):
    """Boolean mask: which of the k-mers (uint64[n, words]) count_sample keeps."""
    kms = np.ascontiguousarray(kmers, dtype=np.uint64)
    h = np.empty(kms.shape[0], dtype=np.uint64)
    if kms.shape[0]:
        _load().oracle_hash_parts(_p(kms, ctypes.c_uint64), kms.shape[0], k, passes * threads,
                                  _p(h, ctypes.c_uint64))
    return (h // np.uint64(threads)) == np.uint64(which)


def position_sigs(bases, offsets, k, m):
    """Signature of every k-mer start position (NO_KMER where none)."""
    lib = _load()
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    out = np.empty(int(offsets[-1]), dtype=np.uint32)
    lib.oracle_position_sigs(_p(bases, ctypes.c_uint8), _p(offsets, ctypes.c_uint64),
                             offsets.size - 1, k, m, _p(out, ctypes.c_uint32))
    return out


def superkmers(read, k, m, use_minimizer=False, cut_every=0):
    """Fig. 1 split of one read: list of (start, n_kmers, signature).

    cut_every > 0 also cuts before read positions that are multiples of it."""
    lib = _load()
    b = np.frombuffer(read.encode() if isinstance(read, str) else bytes(read), dtype=np.uint8).copy()
    cap = max(1, b.size)
    st = np.zeros(cap, np.uint64)
    nk = np.zeros(cap, np.uint32)
    sg = np.zeros(cap, np.uint32)
    n = lib.oracle_superkmers(_p(b, ctypes.c_uint8), b.size, k, m, int(use_minimizer), cut_every,
                              _p(st, ctypes.c_uint64), _p(nk, ctypes.c_uint32),
                              _p(sg, ctypes.c_uint32), cap)
    return [(int(st[i]), int(nk[i]), int(sg[i])) for i in range(n)]


def kxmers(superkmer: str, k: int, x: int):
    """Sect. 2.3 split of one super k-mer: list of (first k-mer index, x', reversed, value)."""
    lib = _load()
    n_kmers = len(superkmer) - k + 1
    codes = (ctypes.c_int * max(1, len(superkmer)))(*[lib.oracle_code(ord(c)) for c in superkmer])
    cap = max(1, n_kmers)
    gs = np.zeros(cap, np.uint64)
    xp = np.zeros(cap, np.uint32)
    rv = np.zeros(cap, np.uint32)
    hi = np.zeros(cap, np.uint64)
    lo = np.zeros(cap, np.uint64)
    n = lib.oracle_kxmers(codes, n_kmers, k, x, _p(gs, ctypes.c_uint64), _p(xp, ctypes.c_uint32),
                          _p(rv, ctypes.c_uint32), _p(hi, ctypes.c_uint64), _p(lo, ctypes.c_uint64), cap)
    return [(int(gs[i]), int(xp[i]), int(rv[i]), (int(hi[i]) << 64) | int(lo[i])) for i in range(n)]


def signature_of(kmer: str, m: int) -> int:
    lib = _load()
    codes = (ctypes.c_int * len(kmer))(*[lib.oracle_code(ord(c)) for c in kmer])
    return int(lib.oracle_signature(codes, len(kmer), m))


def mmer_allowed(v: int, m: int) -> bool:
    return bool(_load().oracle_mmer_allowed(v, m))


def bin_map(weights, n_bins):
    """Sect. 2.4 bin map from per-signature sample weights (length 4^m + 1)."""
    w = np.ascontiguousarray(weights, dtype=np.uint64)
    out = np.empty(w.size, dtype=np.uint32)
    _load().oracle_bin_map(_p(w, ctypes.c_uint64), w.size, n_bins, _p(out, ctypes.c_uint32))
    return out


def kmers_to_int(kms: np.ndarray):
    """uint64[n, words] (most significant word first) -> list of Python ints."""
    out = []
    for row in kms:
        v = 0
        for w in row:
            v = (v << 64) | int(w)
        out.append(v)
    return out
