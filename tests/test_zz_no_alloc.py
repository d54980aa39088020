"""The allocation-free entry point (kmc_count_small_noalloc).

It is for callers that must not allocate GPU memory (for example code running
while a CUDA graph is captured, or a service whose device memory belongs to its
own allocator).  Its scratch is a fixed array inside the library, shared by
all calls, so this test checks that two calls in a row, on different read
sets, each give exactly the result of the regular entry points
(kmc_open / kmc_add_reads / kmc_count / kmc_result) and of the CPU oracle:
the second call must not see anything the first one left in the scratch.
Further cases: cutoff_min = 0, k = 32, an empty read set, a capacity below
the result size (nothing written past it) and malformed offsets.  This file
is collected last so that a stop at the first failure has already run every
other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu

SENTINEL_K = np.int64(0x5A5A5A5A5A5A5A5A)
SENTINEL_C = np.int32(0x3C3C3C3C)


def _reads(scale, seed_shift):
    w = synth.tiny(scale=scale)
    if seed_shift:  # a different read set: drop the first reads
        n = w.n_reads // 3
        o = w.offsets[n:] - w.offsets[n]
        return w.bases[int(w.offsets[n]):], o
    return w.bases, w.offsets


def _run(torch, dev, stream, bases, offsets, k, ci, cx, cap, pad=8):
    """One call; returns (n_out, kmers[:min(n, cap)], counts[:...], untouched tail ok)."""
    db = torch.from_numpy(bases if bases.size else np.zeros(1, np.uint8)).to(dev)
    do = torch.from_numpy(offsets.view(np.int64)).to(dev)
    out_k = torch.full((cap + pad,), int(SENTINEL_K), dtype=torch.int64, device=dev)
    out_c = torch.full((cap + pad,), int(SENTINEL_C), dtype=torch.int32, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    kmc.kmc_count_small_noalloc(db.data_ptr(), do.data_ptr(), offsets.size - 1, bases.size, k, ci,
                                cx, out_k.data_ptr(), out_c.data_ptr(), cap, n_out.data_ptr(),
                                stream.cuda_stream)
    torch.cuda.synchronize(dev)
    n = int(n_out.cpu().numpy().view(np.uint64)[0])
    hk = out_k.cpu().numpy()
    hc = out_c.cpu().numpy()
    m = min(n, cap)
    tail_ok = bool(np.all(hk[m:] == SENTINEL_K) and np.all(hc[m:] == SENTINEL_C))
    return n, hk[:m].view(np.uint64), hc[:m].view(np.uint32), tail_ok


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    return torch, dev, torch.cuda.current_stream(dev)


def test_noalloc_matches_regular_entry_points_and_oracle_twice(cuda):
    torch, dev, stream = cuda
    for call, (scale, shift, k, ci) in enumerate([(0.04, False, 28, 2), (0.03, True, 21, 1)]):
        bases, offsets = _reads(scale, shift)
        assert bases.size <= kmc.KMC_NOALLOC_MAX_BASES
        want_k, want_c = kmc.count(bases, offsets, k, m=7, n_bins=64, cutoff_min=ci)
        ok_, oc_ = oracle.count(bases, offsets, k, ci, 10**9)
        assert np.array_equal(want_k, ok_) and np.array_equal(want_c, oc_)
        n, got_k, got_c, tail_ok = _run(torch, dev, stream, bases, offsets, k, ci, 10**9,
                                        want_k.shape[0] + 16)
        assert n == want_k.shape[0], f"call {call}: {n} k-mers, expected {want_k.shape[0]}"
        assert np.array_equal(got_k, want_k[:, 0]), f"call {call}: k-mers differ"
        assert np.array_equal(got_c, want_c), f"call {call}: counts differ"
        assert tail_ok


def test_noalloc_edge_cases_against_the_oracle(cuda):
    torch, dev, stream = cuda
    bases, offsets = _reads(0.01, False)
    # cutoff_min = 0 keeps every k-mer (each has count >= 1); k = 32 fills the word
    for k, ci, cx in ((28, 0, 10**9), (32, 1, 10**9), (32, 2, 3), (1, 1, 2**32 - 1)):
        ok_, oc_ = oracle.count(bases, offsets, k, ci, cx)
        n, gk, gc, tail_ok = _run(torch, dev, stream, bases, offsets, k, ci, cx, ok_.shape[0])
        assert n == ok_.shape[0] and np.array_equal(gk, ok_[:, 0]) and np.array_equal(gc, oc_), (k, ci, cx)
        assert tail_ok
    # capacity below the result: n_out is the full size, only `cap` entries written
    ok_, oc_ = oracle.count(bases, offsets, 28, 1, 10**9)
    cap = ok_.shape[0] // 3
    n, gk, gc, tail_ok = _run(torch, dev, stream, bases, offsets, 28, 1, 10**9, cap)
    assert n == ok_.shape[0] and tail_ok
    assert np.array_equal(gk, ok_[:cap, 0]) and np.array_equal(gc, oc_[:cap])
    # an empty read set, and reads all shorter than k
    empty_o = np.zeros(1, np.uint64)
    n, _, _, tail_ok = _run(torch, dev, stream, np.zeros(0, np.uint8), empty_o, 28, 1, 10**9, 4)
    assert n == 0 and tail_ok
    sb, so = oracle.as_reads(["ACGT", "", "ACGTNACGTACGTACGTACGTACGTACG"])
    n, _, _, tail_ok = _run(torch, dev, stream, sb, so, 28, 1, 10**9, 4)
    assert n == 0 and tail_ok
    # malformed offsets (the last one is not n_bases): UINT64_MAX, nothing written
    bad = offsets.copy()
    bad[-1] = bad[-1] + np.uint64(5)
    n, _, _, tail_ok = _run(torch, dev, stream, bases, bad, 28, 1, 10**9, 0)
    assert n == 2**64 - 1 and tail_ok


def test_noalloc_rejects_inputs_above_its_scratch():
    lib = kmc.load()
    rc = lib.kmc_count_small_noalloc(None, ctypes.c_void_p(1), 1, kmc.KMC_NOALLOC_MAX_BASES + 1, 28,
                                     2, 10**9, None, None, 0, ctypes.c_void_p(1), None)
    assert rc == kmc.KMC_EINVAL
    for k in (0, 33):
        rc = lib.kmc_count_small_noalloc(None, ctypes.c_void_p(1), 0, 0, k, 1, 10, None, None, 0,
                                         ctypes.c_void_p(1), None)
        assert rc == kmc.KMC_EINVAL
