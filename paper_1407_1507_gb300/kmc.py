"""Thin ctypes binding of libkmc (include/kmc.h): same names, argument
marshalling only.  Every step of the counting runs in the library's CUDA
kernels; there is no CPU fallback.  If libkmc.so is missing or cannot be
loaded, import-time calls raise.

Host inputs are numpy arrays (or anything exposing the buffer protocol);
device inputs are torch CUDA tensors (only their data pointers are used).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KMC_OK = 0
KMC_EINVAL = -1
KMC_ESTATE = -2
KMC_ENOMEM = -3
KMC_ECUDA = -4
KMC_EOVERFLOW = -5
KMC_ETRUNC = -6
KMC_ETIMEOUT = -7
KMC_EAGAIN = -8
KMC_EINPUT = -9
KMC_EIO = -10
KMC_ECANCELED = -11
KMC_AUTO = 0xFFFFFFFF
KMC_DEBUG_KEEP_SUPERKMERS = 1
KMC_DEBUG_KEEP_KEYS = 2
KMC_DEBUG_NARROW_SORT = 4
KMC_DEBUG_SIG_TILE = 8
KMC_DEBUG_MINIMIZER = 16
KMC_DEBUG_WAIT_TIMEOUT = 32
KMC_FORMAT_FASTQ = 1
KMC_FORMAT_FASTA = 2


class kmc_params(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_uint32), ("m", ctypes.c_uint32), ("n_bins", ctypes.c_uint32),
        ("x", ctypes.c_uint32), ("cutoff_min", ctypes.c_uint64), ("cutoff_max", ctypes.c_uint64),
        ("canonical", ctypes.c_uint32), ("device", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
        ("debug_flags", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
        ("piece_bytes", ctypes.c_uint64), ("device_budget", ctypes.c_uint64),
        ("counter_max", ctypes.c_uint64),
    ]


class kmc_stats(ctypes.Structure):
    _fields_ = [
        ("n_reads", ctypes.c_uint64), ("n_bases", ctypes.c_uint64),
        ("n_kmer_positions", ctypes.c_uint64), ("n_superkmers", ctypes.c_uint64),
        ("n_sorted_keys", ctypes.c_uint64), ("n_distinct", ctypes.c_uint64),
        ("n_out", ctypes.c_uint64), ("max_bin_kmers", ctypes.c_uint64),
        ("bin_bytes", ctypes.c_uint64), ("x_used", ctypes.c_uint32), ("m_used", ctypes.c_uint32),
        ("n_tiles", ctypes.c_uint32), ("n_big_tiles", ctypes.c_uint32),
        ("ms_distribute", ctypes.c_float), ("ms_sort", ctypes.c_float),
        ("ms_order", ctypes.c_float), ("ms_total", ctypes.c_float),
        ("ms_stage", ctypes.c_float * 12), ("n_launches", ctypes.c_uint64),
        ("spilled_bytes", ctypes.c_uint64), ("n_waves", ctypes.c_uint32), ("reserved_s", ctypes.c_uint32),
        ("n_fused_keys", ctypes.c_uint64),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved_s"}
        d["ms_stage"] = {STAGES[i]: float(self.ms_stage[i]) for i in range(len(STAGES))}
        return d


# kmc_stats.ms_stage indices (KMC_STAGE_* in include/kmc.h)
STAGES = ["pack", "signature", "bin_scatter", "bin_map", "kx_count", "plan", "kx_scatter",
          "tile_sort", "big_sort", "order", "other"]


class kmc_batch_stats(ctypes.Structure):
    _fields_ = [
        ("ms_device", ctypes.c_float), ("ms_wall", ctypes.c_float),
        ("n_sub_batches", ctypes.c_uint32), ("n_single", ctypes.c_uint32),
        ("tuning_runs", ctypes.c_uint32), ("bins_per_set", ctypes.c_uint32),
        ("tile_keys", ctypes.c_uint32), ("bucket_keys", ctypes.c_uint32),
        ("n_kmers_out", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class kmc_server_cfg(ctypes.Structure):
    _fields_ = [
        ("base", kmc_params), ("batch_bases", ctypes.c_uint64), ("batch_reads", ctypes.c_uint64),
        ("batch_sets", ctypes.c_uint32), ("n_workers", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
        ("batch_flags", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
        ("warm_k_mask", ctypes.c_uint64),
    ]


class kmc_server_stats(ctypes.Structure):
    _fields_ = [
        ("jobs_done", ctypes.c_uint64), ("jobs_queued", ctypes.c_uint64), ("batches", ctypes.c_uint64),
        ("max_batch_jobs", ctypes.c_uint64), ("max_inflight_jobs", ctypes.c_uint64),
        ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
        ("wall_s", ctypes.c_double), ("error", ctypes.c_int32), ("reserved0", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved0"}


KMC_BATCH_AUTOTUNE = 1
KMC_BATCH_NO_GRAPH = 2


class kmc_db_info(ctypes.Structure):
    _fields_ = [
        ("kmer_length", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("counter_size", ctypes.c_uint32),
        ("lut_prefix_length", ctypes.c_uint32), ("signature_length", ctypes.c_uint32),
        ("min_count", ctypes.c_uint32), ("max_count", ctypes.c_uint32), ("total_kmers", ctypes.c_uint64),
        ("kmc_ver", ctypes.c_uint32), ("n_arrays", ctypes.c_uint32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class KmcError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p

# (name, restype, argtypes) of every exported symbol of include/kmc.h
SIGNATURES = [
    ("kmc_default_params", None, [ctypes.POINTER(kmc_params)]),
    ("kmc_open", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(kmc_params)]),
    ("kmc_add_reads", ctypes.c_int, [_vp, _vp, _u64p, ctypes.c_uint64]),
    ("kmc_add_reads_device", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_uint64, ctypes.c_uint64]),
    ("kmc_add_file_bytes", ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.c_uint32]),
    ("kmc_add_file_bytes_device", ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.c_uint32]),
    ("kmc_count", ctypes.c_int, [_vp]),
    ("kmc_result_size", ctypes.c_int, [_vp, _u64p]),
    ("kmc_result", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_uint64, _u64p]),
    ("kmc_result_device", ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _u64p]),
    ("kmc_stats_get", ctypes.c_int, [_vp, ctypes.POINTER(kmc_stats)]),
    ("kmc_reset", ctypes.c_int, [_vp]),
    ("kmc_close", None, [_vp]),
    ("kmc_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("kmc_set_bin_map", ctypes.c_int, [_vp, _u32p, ctypes.c_uint64]),
    ("kmc_get_bin_map", ctypes.c_int, [_vp, _u32p, ctypes.c_uint64]),
    ("kmc_debug_superkmers", ctypes.c_int, [_vp, _u64p, _u32p, _u32p, _u32p, ctypes.c_uint64, _u64p]),
    ("kmc_debug_bin_keys", ctypes.c_int, [_vp, ctypes.c_uint32, _u64p, ctypes.c_uint64, _u64p, _u32p]),
    ("kmc_batch_open", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(kmc_params), ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]),
    ("kmc_batch_run", ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     _u64p, _u32p]),
    ("kmc_batch_result", ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                        _u64p]),
    ("kmc_batch_stats_get", ctypes.c_int, [_vp, ctypes.POINTER(kmc_batch_stats)]),
    ("kmc_batch_close", None, [_vp]),
    ("kmc_server_open", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(kmc_server_cfg)]),
    ("kmc_server_submit", ctypes.c_int, [_vp, ctypes.c_uint32, _vp, _u64p, ctypes.c_uint64, _u64p]),
    ("kmc_server_submit_ref", ctypes.c_int, [_vp, ctypes.c_uint32, _vp, _u64p, ctypes.c_uint64, _u64p]),
    ("kmc_server_wait", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double]),
    ("kmc_server_result", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                         _u64p, ctypes.POINTER(ctypes.c_double)]),
    ("kmc_server_release", ctypes.c_int, [_vp, ctypes.c_uint64]),
    ("kmc_server_cancel", ctypes.c_int, [_vp, ctypes.c_uint64]),
    ("kmc_server_stats_get", ctypes.c_int, [_vp, ctypes.POINTER(kmc_server_stats)]),
    ("kmc_server_close", None, [_vp]),
    ("kmc_db_write", ctypes.c_int, [_vp, ctypes.c_char_p]),
    ("kmc_db_open", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_char_p, ctypes.c_int]),
    ("kmc_db_info_get", ctypes.c_int, [_vp, ctypes.POINTER(kmc_db_info)]),
    ("kmc_db_lookup", ctypes.c_int, [_vp, _vp, ctypes.c_uint64, _vp, _vp]),
    ("kmc_db_close", None, [_vp]),
    ("kmc_debug_fail_alloc", ctypes.c_int, [ctypes.c_int64]),
    ("kmc_count_small_noalloc", ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint64, ctypes.c_uint64, _vp, _vp, ctypes.c_uint64,
                                               _vp, _vp]),
]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libkmc.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libkmc.so not built ({path}); run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def strerror(code: int) -> str:
    return load().kmc_strerror(code).decode()


def _check(rc, what):
    if rc != KMC_OK:
        raise KmcError(rc, what)


def _ptr(a, ct=ctypes.c_uint8):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ----------------------------------------------------------- C-ABI mirror

def kmc_default_params() -> kmc_params:
    p = kmc_params()
    load().kmc_default_params(ctypes.byref(p))
    return p


def kmc_open(p: kmc_params) -> int:
    h = _vp()
    _check(load().kmc_open(ctypes.byref(h), ctypes.byref(p)), "kmc_open")
    return h.value


def kmc_add_reads(h, bases: np.ndarray, offsets: np.ndarray):
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    _check(load().kmc_add_reads(h, bases.ctypes.data if bases.size else None, _ptr(offsets, ctypes.c_uint64),
                                offsets.size - 1), "kmc_add_reads")


def kmc_add_reads_ptr(h, bases_ptr: int, offsets_ptr: int, n_reads: int):
    """kmc_add_reads on raw host pointers (e.g. pinned torch tensors)."""
    _check(load().kmc_add_reads(h, bases_ptr, ctypes.cast(offsets_ptr, _u64p), n_reads), "kmc_add_reads")


def kmc_add_reads_device(h, d_bases_ptr: int, d_offsets_ptr: int, n_reads: int, n_bases: int):
    _check(load().kmc_add_reads_device(h, d_bases_ptr, d_offsets_ptr, n_reads, n_bases),
           "kmc_add_reads_device")


def kmc_add_file_bytes(h, data, fmt: int):
    """FASTQ (KMC_FORMAT_FASTQ) or FASTA (KMC_FORMAT_FASTA) file contents in
    host memory (bytes or a uint8 array); parsed on the device."""
    buf = np.frombuffer(data, dtype=np.uint8) if isinstance(data, (bytes, bytearray)) else \
        np.ascontiguousarray(data, dtype=np.uint8)
    _check(load().kmc_add_file_bytes(h, buf.ctypes.data if buf.size else None, buf.size, fmt),
           "kmc_add_file_bytes")


def kmc_add_file_bytes_device(h, d_bytes_ptr: int, n_bytes: int, fmt: int):
    _check(load().kmc_add_file_bytes_device(h, d_bytes_ptr, n_bytes, fmt), "kmc_add_file_bytes_device")


def kmc_count(h):
    _check(load().kmc_count(h), "kmc_count")


def kmc_result_size(h) -> int:
    n = ctypes.c_uint64()
    _check(load().kmc_result_size(h, ctypes.byref(n)), "kmc_result_size")
    return n.value


def kmc_result(h, k: int):
    n = kmc_result_size(h)
    words = (k + 31) // 32
    kms = np.empty((n, words), dtype=np.uint64)
    cnt = np.empty(n, dtype=np.uint32)
    nout = ctypes.c_uint64()
    _check(load().kmc_result(h, kms.ctypes.data if n else None, cnt.ctypes.data if n else None, n,
                             ctypes.byref(nout)), "kmc_result")
    return kms, cnt


def kmc_result_into(h, k: int, kms_buf: np.ndarray, cnt_buf: np.ndarray):
    """kmc_result into caller arrays (e.g. pinned host memory): kms_buf uint64
    with at least n * ceil(k/32) elements, cnt_buf uint32 with at least n;
    returns views of the first n k-mers and counts."""
    n = kmc_result_size(h)
    words = (k + 31) // 32
    if kms_buf.size < n * words or cnt_buf.size < n:
        raise ValueError("result buffers too small")
    nout = ctypes.c_uint64()
    _check(load().kmc_result(h, kms_buf.ctypes.data if n else None, cnt_buf.ctypes.data if n else None,
                             n, ctypes.byref(nout)), "kmc_result")
    return kms_buf[:n * words].reshape(n, words), cnt_buf[:n]


def kmc_result_device(h):
    dk, dc, n = _vp(), _vp(), ctypes.c_uint64()
    _check(load().kmc_result_device(h, ctypes.byref(dk), ctypes.byref(dc), ctypes.byref(n)),
           "kmc_result_device")
    return dk.value, dc.value, n.value


def kmc_stats_get(h) -> dict:
    s = kmc_stats()
    _check(load().kmc_stats_get(h, ctypes.byref(s)), "kmc_stats_get")
    return s.as_dict()


def kmc_reset(h):
    _check(load().kmc_reset(h), "kmc_reset")


def kmc_close(h):
    if h:
        load().kmc_close(h)


def kmc_set_bin_map(h, mp: np.ndarray):
    mp = np.ascontiguousarray(mp, dtype=np.uint32)
    _check(load().kmc_set_bin_map(h, _ptr(mp, ctypes.c_uint32), mp.size), "kmc_set_bin_map")


def kmc_get_bin_map(h, n_entries: int) -> np.ndarray:
    mp = np.empty(n_entries, dtype=np.uint32)
    _check(load().kmc_get_bin_map(h, _ptr(mp, ctypes.c_uint32), n_entries), "kmc_get_bin_map")
    return mp


def kmc_debug_superkmers(h):
    n = ctypes.c_uint64()
    rc = load().kmc_debug_superkmers(h, None, None, None, None, 0, ctypes.byref(n))
    if rc not in (KMC_OK, KMC_ETRUNC):
        _check(rc, "kmc_debug_superkmers")
    cap = n.value
    rd = np.empty(max(cap, 1), np.uint64)
    ps = np.empty(max(cap, 1), np.uint32)
    nk = np.empty(max(cap, 1), np.uint32)
    sg = np.empty(max(cap, 1), np.uint32)
    _check(load().kmc_debug_superkmers(h, _ptr(rd, ctypes.c_uint64), _ptr(ps, ctypes.c_uint32),
                                       _ptr(nk, ctypes.c_uint32), _ptr(sg, ctypes.c_uint32), cap,
                                       ctypes.byref(n)), "kmc_debug_superkmers")
    return rd[:cap], ps[:cap], nk[:cap], sg[:cap]


def kmc_debug_bin_keys(h, b: int):
    n = ctypes.c_uint64()
    w = ctypes.c_uint32()
    rc = load().kmc_debug_bin_keys(h, b, None, 0, ctypes.byref(n), ctypes.byref(w))
    if rc not in (KMC_OK, KMC_ETRUNC):
        _check(rc, "kmc_debug_bin_keys")
    keys = np.empty((max(n.value, 1), max(w.value, 1)), np.uint64)
    _check(load().kmc_debug_bin_keys(h, b, _ptr(keys, ctypes.c_uint64), n.value, ctypes.byref(n),
                                     ctypes.byref(w)), "kmc_debug_bin_keys")
    return keys[:n.value]


def kmc_db_write(h, path: str):
    """Writes <path>.kmc_pre and <path>.kmc_suf from the counted result."""
    _check(load().kmc_db_write(h, os.fsencode(path)), "kmc_db_write")


def kmc_db_open(path: str, device: int = 0) -> int:
    db = _vp()
    _check(load().kmc_db_open(ctypes.byref(db), os.fsencode(path), device), "kmc_db_open")
    return db.value


def kmc_db_info_get(db) -> dict:
    info = kmc_db_info()
    _check(load().kmc_db_info_get(db, ctypes.byref(info)), "kmc_db_info_get")
    return info.as_dict()


def kmc_db_lookup(db, d_kmers_ptr: int, n: int, d_counts_ptr: int, stream=None):
    """Counts of n device-resident query k-mers into a device uint32 array;
    asynchronous on `stream` (a cudaStream_t value, None: legacy default)."""
    _check(load().kmc_db_lookup(db, d_kmers_ptr, n, d_counts_ptr, stream), "kmc_db_lookup")


def kmc_db_close(db):
    if db:
        load().kmc_db_close(db)


KMC_NOALLOC_MAX_BASES = 1 << 20


def kmc_count_small_noalloc(d_bases_ptr, d_offsets_ptr, n_reads, n_bases, k, cutoff_min,
                            cutoff_max, d_kmers_ptr, d_counts_ptr, capacity, d_n_out_ptr,
                            stream=None):
    """Allocation-free count of a small device-resident read set into caller
    device arrays (see include/kmc.h); asynchronous on `stream`."""
    _check(load().kmc_count_small_noalloc(d_bases_ptr, d_offsets_ptr, n_reads, n_bases, k,
                                          cutoff_min, cutoff_max, d_kmers_ptr, d_counts_ptr,
                                          capacity, d_n_out_ptr, stream), "kmc_count_small_noalloc")


def kmc_batch_open(p: kmc_params, max_bases: int, max_reads: int, max_sets: int, flags: int = 0) -> int:
    h = _vp()
    _check(load().kmc_batch_open(ctypes.byref(h), ctypes.byref(p), max_bases, max_reads, max_sets, flags),
           "kmc_batch_open")
    return h.value


def kmc_batch_run(b, sets, ks):
    """sets: list of (bases uint8 array, offsets uint64 array); ks: k per set."""
    n = len(sets)
    keep = [(np.ascontiguousarray(bs, dtype=np.uint8), np.ascontiguousarray(of, dtype=np.uint64))
            for bs, of in sets]
    bp = (_vp * max(n, 1))(*[x[0].ctypes.data for x in keep])
    op = (_vp * max(n, 1))(*[x[1].ctypes.data for x in keep])
    nr = np.array([x[1].size - 1 for x in keep] or [0], dtype=np.uint64)
    kk = np.array(list(ks) or [0], dtype=np.uint32)
    _check(load().kmc_batch_run(b, n, bp, op, _ptr(nr, ctypes.c_uint64), _ptr(kk, ctypes.c_uint32)),
           "kmc_batch_run")


def kmc_batch_result(b, s: int, copy: bool = True):
    """Set s's (k-mers uint64[n, 1], counts uint32[n]); copy=False returns views
    of the handle's arrays, valid until the next kmc_batch_run or close."""
    dk, dc, n = _vp(), _vp(), ctypes.c_uint64()
    _check(load().kmc_batch_result(b, s, ctypes.byref(dk), ctypes.byref(dc), ctypes.byref(n)),
           "kmc_batch_result")
    if n.value == 0:
        return np.zeros((0, 1), np.uint64), np.zeros(0, np.uint32)
    kms = np.ctypeslib.as_array(ctypes.cast(dk.value, _u64p), shape=(n.value,)).reshape(-1, 1)
    cnt = np.ctypeslib.as_array(ctypes.cast(dc.value, _u32p), shape=(n.value,))
    return (kms.copy(), cnt.copy()) if copy else (kms, cnt)


def kmc_batch_stats_get(b) -> dict:
    s = kmc_batch_stats()
    _check(load().kmc_batch_stats_get(b, ctypes.byref(s)), "kmc_batch_stats_get")
    return s.as_dict()


def kmc_batch_close(b):
    if b:
        load().kmc_batch_close(b)


def kmc_server_open(base: kmc_params, batch_bases=0, batch_reads=0, batch_sets=0, n_workers=0,
                    mem_budget=0, batch_flags=0, warm_k=()) -> int:
    c = kmc_server_cfg()
    c.base = base
    c.batch_bases, c.batch_reads, c.batch_sets = batch_bases, batch_reads, batch_sets
    c.n_workers, c.mem_budget, c.batch_flags = n_workers, mem_budget, batch_flags
    c.warm_k_mask = sum(1 << k for k in warm_k)
    h = _vp()
    _check(load().kmc_server_open(ctypes.byref(h), ctypes.byref(c)), "kmc_server_open")
    return h.value


def kmc_server_submit(s, k: int, bases: np.ndarray, offsets: np.ndarray) -> int:
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    jid = ctypes.c_uint64()
    _check(load().kmc_server_submit(s, k, bases.ctypes.data if bases.size else None,
                                    _ptr(offsets, ctypes.c_uint64), offsets.size - 1, ctypes.byref(jid)),
           "kmc_server_submit")
    return jid.value


def kmc_server_submit_ref(s, k: int, bases: np.ndarray, offsets: np.ndarray) -> int:
    """Zero-copy submission: the server reads `bases` and `offsets` (contiguous
    uint8 / uint64 arrays) in place; the caller keeps them alive and unchanged
    until the job has finished."""
    if bases.dtype != np.uint8 or offsets.dtype != np.uint64 or not bases.flags.c_contiguous \
            or not offsets.flags.c_contiguous:
        raise ValueError("kmc_server_submit_ref needs contiguous uint8 bases and uint64 offsets")
    jid = ctypes.c_uint64()
    _check(load().kmc_server_submit_ref(s, k, bases.ctypes.data if bases.size else None,
                                        _ptr(offsets, ctypes.c_uint64), offsets.size - 1, ctypes.byref(jid)),
           "kmc_server_submit_ref")
    return jid.value


def kmc_server_wait(s, job_id: int, timeout_s: float = -1.0) -> bool:
    rc = load().kmc_server_wait(s, job_id, timeout_s)
    if rc == KMC_EAGAIN:
        return False
    _check(rc, "kmc_server_wait")
    return True


def kmc_server_result(s, job_id: int, copy: bool = True):
    """(k-mers uint64[n, 1], counts uint32[n], latency ms) of a finished job;
    copy=False returns views valid until kmc_server_release."""
    dk, dc, n, lat = _vp(), _vp(), ctypes.c_uint64(), ctypes.c_double()
    _check(load().kmc_server_result(s, job_id, ctypes.byref(dk), ctypes.byref(dc), ctypes.byref(n),
                                    ctypes.byref(lat)), "kmc_server_result")
    if n.value == 0:
        return np.zeros((0, 1), np.uint64), np.zeros(0, np.uint32), lat.value
    kms = np.ctypeslib.as_array(ctypes.cast(dk.value, _u64p), shape=(n.value,)).reshape(-1, 1)
    cnt = np.ctypeslib.as_array(ctypes.cast(dc.value, _u32p), shape=(n.value,))
    if copy:
        kms, cnt = kms.copy(), cnt.copy()
    return kms, cnt, lat.value


def kmc_server_release(s, job_id: int):
    _check(load().kmc_server_release(s, job_id), "kmc_server_release")


def kmc_server_cancel(s, job_id: int):
    """Removes a queued job (it ends with KMC_ECANCELED); KmcError(KMC_ESTATE)
    once it has been admitted to a batch."""
    _check(load().kmc_server_cancel(s, job_id), "kmc_server_cancel")


def kmc_debug_fail_alloc(after: int):
    """Test hook: the allocation after `after` more successful ones fails once
    (after < 0 cancels)."""
    _check(load().kmc_debug_fail_alloc(after), "kmc_debug_fail_alloc")


def kmc_server_stats_get(s) -> dict:
    st = kmc_server_stats()
    _check(load().kmc_server_stats_get(s, ctypes.byref(st)), "kmc_server_stats_get")
    return st.as_dict()


def kmc_server_close(s):
    if s:
        load().kmc_server_close(s)


# ----------------------------------------------------------- convenience

def make_params(k, m=7, n_bins=512, x=KMC_AUTO, cutoff_min=2, cutoff_max=10**9, device=0,
                stream=None, debug_flags=0, piece_bytes=0, device_budget=0, canonical=1,
                counter_max=0) -> kmc_params:
    p = kmc_default_params()
    p.k, p.m, p.n_bins = k, m, n_bins
    p.x = KMC_AUTO if x is None else x
    p.cutoff_min, p.cutoff_max = cutoff_min, cutoff_max
    p.device = device
    p.cuda_stream = stream
    p.debug_flags = debug_flags
    p.piece_bytes = piece_bytes
    p.device_budget = device_budget
    p.canonical = canonical
    p.counter_max = counter_max
    return p


class Counter:
    """One counting job: open -> add reads -> count -> result -> close."""

    def __init__(self, k, **kw):
        self.k = k
        self.params = make_params(k, **kw)
        self.h = kmc_open(self.params)

    def add(self, bases, offsets):
        kmc_add_reads(self.h, bases, offsets)
        return self

    def add_file(self, data, fmt):
        """FASTQ / FASTA file contents (host bytes, or a torch CUDA uint8 tensor)."""
        if hasattr(data, "data_ptr"):
            kmc_add_file_bytes_device(self.h, data.data_ptr(), data.numel(), fmt)
        else:
            kmc_add_file_bytes(self.h, data, fmt)
        return self

    def add_device(self, d_bases, d_offsets):
        """Reads already on the device (torch CUDA tensors: uint8 bases, int64 offsets)."""
        kmc_add_reads_device(self.h, d_bases.data_ptr(), d_offsets.data_ptr(),
                             d_offsets.numel() - 1, d_bases.numel())
        return self

    def count(self):
        kmc_count(self.h)
        return self

    def result(self):
        return kmc_result(self.h, self.k)

    def size(self):
        return kmc_result_size(self.h)

    def stats(self):
        return kmc_stats_get(self.h)

    def bin_map(self):
        return kmc_get_bin_map(self.h, 4 ** self.stats()["m_used"] + 1)

    def write_db(self, path):
        """KMC 2 database files <path>.kmc_pre / <path>.kmc_suf of the result."""
        kmc_db_write(self.h, path)
        return self

    def close(self):
        kmc_close(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def count(bases, offsets, k, **kw):
    """Counts canonical k-mers of host reads; returns (kmers uint64[n, words], counts uint32[n])."""
    with Counter(k, **kw) as c:
        return c.add(bases, offsets).count().result()
