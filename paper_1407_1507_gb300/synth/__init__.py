"""Seeded synthetic genomes and reads (input generator shared by the CUDA path's
benchmarks and the oracle's tests; it holds none of the counting arithmetic).

The workloads are synthetic stand-ins for the paper's sequencing datasets
(short reads of 100-250 bp, high coverage, ~1 % substitution errors, human-like
GC content and interspersed repeats; paper Sect. 3, Table 1).  Every generator
is seeded; the C core draws from splitmix64 streams keyed by (seed, index) and
compares probabilities as integer thresholds, so a seed gives identical bytes on
every machine.

Workload presets (sizes as stated; ``scale`` shrinks read counts and genomes for
quick tests):

* ``tiny``:   1 Mbp iid genome, 200,000 reads x 100 bp, 1 % errors, no N;
              k=28, m=7, 64 bins, cutoffs [2, 1e9].
* ``mid``:    50 Mbp order-3 Markov genome (GC 0.41) + 50 repeat families x 40
              copies of 5 kbp at 10 % divergence; 20 M reads x 150 bp, 0.5 %
              errors, 0.1 % N; k=28, m=7, 512 bins, cutoffs [2, 1e9].
* ``large``:  300 Mbp Markov genome with the same repeats; 20 M x 150 bp, 1 %
              errors, 0.1 % N; k=28 or 55, m=9, 2048 bins.
* ``batch_set(i)``: set i of the batched workload (log-normal read count,
              median 200 k, clipped to [10 k, 5 M]; genome 1-20 Mbp; L in
              {100,150,250}; k in {21,28,31}; m=7; 1 % errors; no N).
              ``batch_sets(n)`` builds sets 0..n-1 on several threads.
* ``served_pools`` / ``served_request(i)``: the served workload.  Request i
              has the batched sizes (or, with probability 0.05, 10 M reads)
              and a k in {21,28,31}; its reads are a window of consecutive
              reads of one of 16 read pools, each pool drawn from its own
              genome (as a batched set's) at its own read length, so that
              5,000 requests (about 680 Gbases) need no per-request
              generation and no copy.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(os.path.dirname(_HERE), "_build")
_SO = os.path.join(_BUILD, "libkmc_synth.so")

BASE_SEED = 20140715
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator core with gcc (seconds); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.synth_genome_iid.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_genome_iid.restype = None
        lib.synth_markov3_table.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double, u32p]
        lib.synth_markov3_table.restype = ctypes.c_double
        lib.synth_genome_markov3.argtypes = [u8p, ctypes.c_uint64, u32p, ctypes.c_uint64]
        lib.synth_genome_markov3.restype = None
        lib.synth_insert_repeats.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64]
        lib.synth_insert_repeats.restype = ctypes.c_int
        lib.synth_reads.argtypes = [u8p, ctypes.c_uint64, u64p, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, u8p]
        lib.synth_reads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def genome_iid(n: int, seed: int) -> np.ndarray:
    g = np.empty(n, dtype=np.uint8)
    _load().synth_genome_iid(_ptr(g, ctypes.c_uint8), n, seed)
    return g


def markov3_table(seed: int, gc: float = 0.41, tol: float = 0.001):
    thr = np.empty(64 * 3, dtype=np.uint32)
    got = _load().synth_markov3_table(seed, gc, tol, _ptr(thr, ctypes.c_uint32))
    return thr, got


def genome_markov3(n: int, seed: int, gc: float = 0.41) -> np.ndarray:
    thr, _ = markov3_table(seed, gc)
    g = np.empty(n, dtype=np.uint8)
    _load().synth_genome_markov3(_ptr(g, ctypes.c_uint8), n, _ptr(thr, ctypes.c_uint32), seed)
    return g


def insert_repeats(g: np.ndarray, families: int, copies: int, elem_len: int,
                   divergence: float, seed: int) -> None:
    rc = _load().synth_insert_repeats(_ptr(g, ctypes.c_uint8), g.size, families, copies,
                                      elem_len, divergence, seed)
    if rc != 0:
        raise ValueError(f"repeat insertion failed ({rc}): genome too short for the copies")


def reads(g: np.ndarray, lengths, sub_rate: float, n_rate: float, seed: int):
    """Sample reads; ``lengths`` is an int (all reads) plus a count, or an array.

    Returns (bases uint8[total], offsets uint64[n_reads+1])."""
    lengths = np.asarray(lengths, dtype=np.uint64)
    offsets = np.zeros(lengths.size + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    out = np.empty(int(offsets[-1]), dtype=np.uint8)
    rc = _load().synth_reads(_ptr(g, ctypes.c_uint8), g.size, _ptr(offsets, ctypes.c_uint64),
                             lengths.size, sub_rate, n_rate, seed, _ptr(out, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("a read is longer than the genome")
    return out, offsets


@dataclass
class Workload:
    name: str
    bases: np.ndarray      # uint8 ASCII, reads concatenated
    offsets: np.ndarray    # uint64[n_reads+1]
    k: int
    m: int
    n_bins: int
    cutoff_min: int = 2
    cutoff_max: int = 1_000_000_000

    @property
    def n_reads(self) -> int:
        return self.offsets.size - 1


def _scaled(n: int, scale: float, lo: int = 1) -> int:
    return max(lo, int(round(n * scale)))


def tiny(scale: float = 1.0) -> Workload:
    c = 1
    g = genome_iid(_scaled(1_000_000, scale, 1000), BASE_SEED + c)
    b, o = reads(g, np.full(_scaled(200_000, scale), 100), 0.01, 0.0, BASE_SEED + 100 + c)
    return Workload("tiny", b, o, k=28, m=7, n_bins=64)


def _markov_with_repeats(n: int, seed: int, scale: float) -> np.ndarray:
    g = genome_markov3(n, seed)
    fam = max(1, _scaled(50, math.sqrt(scale)))
    cop = max(1, _scaled(40, math.sqrt(scale)))
    elem = 5000 if n >= fam * cop * 5000 else max(50, n // (fam * cop))
    insert_repeats(g, fam, cop, elem, 0.10, seed + 7)
    return g


def mid(scale: float = 1.0) -> Workload:
    c = 2
    g = _markov_with_repeats(_scaled(50_000_000, scale, 20_000), BASE_SEED + c, scale)
    b, o = reads(g, np.full(_scaled(20_000_000, scale), 150), 0.005, 0.001, BASE_SEED + 100 + c)
    return Workload("mid", b, o, k=28, m=7, n_bins=512)


def large(k: int = 28, scale: float = 1.0) -> Workload:
    c = 3
    g = _markov_with_repeats(_scaled(300_000_000, scale, 20_000), BASE_SEED + c, scale)
    b, o = reads(g, np.full(_scaled(20_000_000, scale), 150), 0.01, 0.001, BASE_SEED + 100 + c)
    return Workload(f"large_k{k}", b, o, k=k, m=9, n_bins=2048)


def batch_set_params(i: int):
    """Parameters of set i of the batched workload (deterministic in i)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 10_000 + i))
    n_reads = int(np.clip(round(math.exp(math.log(200_000) + 1.0 * rng.standard_normal())),
                          10_000, 5_000_000))
    genome = int(rng.integers(1_000_000, 20_000_001))
    L = int(rng.choice([100, 150, 250]))
    k = int(rng.choice([21, 28, 31]))
    return n_reads, genome, L, k


def batch_set(i: int, scale: float = 1.0) -> Workload:
    n_reads, genome, L, k = batch_set_params(i)
    seed = BASE_SEED + 10_000 + i
    g = genome_markov3(max(_scaled(genome, scale, 1000), L), seed)
    b, o = reads(g, np.full(_scaled(n_reads, scale), L), 0.01, 0.0, seed + 1)
    return Workload(f"batch{i}", b, o, k=k, m=7, n_bins=64)


# ------------------------------------------------------------- file formats

def to_fastq(bases: np.ndarray, offsets: np.ndarray, seed: int = BASE_SEED, crlf: bool = False) -> bytes:
    """The reads as a FASTQ file: "@r<i>" headers, "+" lines, and seeded
    quality strings drawn from '!'..'J' (they contain letters that are also
    bases)."""
    rng = np.random.default_rng(seed)
    nl = b"\r\n" if crlf else b"\n"
    parts = []
    off = np.asarray(offsets, dtype=np.int64)
    raw = np.asarray(bases, dtype=np.uint8)
    for i in range(off.size - 1):
        a, e = int(off[i]), int(off[i + 1])
        q = (rng.integers(33, 75, e - a)).astype(np.uint8).tobytes()
        parts += [b"@r%d" % i, nl, raw[a:e].tobytes(), nl, b"+", nl, q, nl]
    return b"".join(parts)


def to_fasta(bases: np.ndarray, offsets: np.ndarray, width: int = 60) -> bytes:
    """The reads as a multi-FASTA file: ">s<i>" headers, sequences wrapped at
    `width` bases per line."""
    parts = []
    off = np.asarray(offsets, dtype=np.int64)
    raw = np.asarray(bases, dtype=np.uint8)
    for i in range(off.size - 1):
        a, e = int(off[i]), int(off[i + 1])
        parts += [b">s%d\n" % i]
        for j in range(a, e, width):
            parts += [raw[j:min(e, j + width)].tobytes(), b"\n"]
    return b"".join(parts)


def batch_sets(n: int, scale: float = 1.0, threads: int = 0, first: int = 0):
    """Sets first..first+n-1 of the batched workload, built on `threads`
    threads (0: all cores); the bytes are those of batch_set(i, scale)."""
    import concurrent.futures as cf
    nt = threads or min(16, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        return list(ex.map(lambda i: batch_set(i, scale), range(first, first + n)))


SERVED_POOLS = 16
SERVED_LARGE_READS = 10_000_000


@dataclass
class ReadPool:
    bases: np.ndarray   # uint8, n_reads * L bytes
    L: int
    n_reads: int
    offsets: np.ndarray  # uint64 arange(n_reads + 1) * L: the offsets of any window of it


def served_pools(scale: float = 1.0, threads: int = 0):
    """The 16 read pools of the served workload: pool p is n = 10 M * scale
    reads (the largest request) of length L_p in {100, 150, 250} from its own
    order-3 Markov genome of 1-20 Mbp (scaled), 1 % substitutions, no N."""
    import concurrent.futures as cf
    n = _scaled(SERVED_LARGE_READS, scale)

    def one(p):
        rng = np.random.Generator(np.random.PCG64(BASE_SEED + 14_000 + p))
        genome = int(rng.integers(1_000_000, 20_000_001))
        L = int(rng.choice([100, 150, 250]))
        seed = BASE_SEED + 14_000 + p
        g = genome_markov3(max(_scaled(genome, scale, 1000), L), seed)
        b, o = reads(g, np.full(n, L), 0.01, 0.0, seed + 1)
        return ReadPool(b, L, n, o)

    nt = threads or min(16, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        return list(ex.map(one, range(SERVED_POOLS)))


def served_request(i: int, pools, scale: float = 1.0):
    """Request i of the served workload: (bases view, offsets view, k, n_reads).
    Sizes as batch_set_params, but 10 M reads with probability 0.05; the reads
    are a seeded window of one pool (views: nothing is copied)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 15_000 + i))
    if rng.random() < 0.05:
        nr = SERVED_LARGE_READS
    else:
        nr = int(np.clip(round(math.exp(math.log(200_000) + 1.0 * rng.standard_normal())), 10_000, 5_000_000))
    k = int(rng.choice([21, 28, 31]))
    pool = pools[int(rng.integers(0, len(pools)))]
    nr = min(_scaled(nr, scale), pool.n_reads)
    first = int(rng.integers(0, pool.n_reads - nr + 1))
    L = pool.L
    return pool.bases[first * L:(first + nr) * L], pool.offsets[:nr + 1], k, nr

