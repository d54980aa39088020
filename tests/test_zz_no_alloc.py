"""The allocation-free entry point (kmc_count_small_noalloc).

It is for callers that must not allocate GPU memory (for example code running
while a CUDA graph is captured, or a service whose device memory belongs to its
own allocator).  Its scratch is a fixed array inside the library, shared by
all calls, so this test checks that two calls in a row, on different read
sets, each give exactly the result of the regular entry points
(kmc_open / kmc_add_reads / kmc_count / kmc_result): the second call must not
see anything the first one left in the scratch.  This file is collected last
so that a stop at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu


def _reads(scale, seed_shift):
    w = synth.tiny(scale=scale)
    if seed_shift:  # a different read set: drop the first reads
        n = w.n_reads // 3
        o = w.offsets[n:] - w.offsets[n]
        return w.bases[int(w.offsets[n]):], o
    return w.bases, w.offsets


def test_noalloc_matches_regular_entry_points_twice():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    for call, (scale, shift, k, ci) in enumerate([(0.04, False, 28, 2), (0.03, True, 21, 1)]):
        bases, offsets = _reads(scale, shift)
        assert bases.size <= kmc.KMC_NOALLOC_MAX_BASES
        want_k, want_c = kmc.count(bases, offsets, k, m=7, n_bins=64, cutoff_min=ci)
        db = torch.from_numpy(bases).to(dev)
        do = torch.from_numpy(offsets.view(np.int64)).to(dev)
        cap = want_k.shape[0] + 16
        out_k = torch.empty(cap, dtype=torch.int64, device=dev)
        out_c = torch.empty(cap, dtype=torch.int32, device=dev)
        n_out = torch.zeros(1, dtype=torch.int64, device=dev)
        kmc.kmc_count_small_noalloc(db.data_ptr(), do.data_ptr(), offsets.size - 1, bases.size, k, ci,
                                    10**9, out_k.data_ptr(), out_c.data_ptr(), cap, n_out.data_ptr(),
                                    stream.cuda_stream)
        torch.cuda.synchronize(dev)
        n = int(n_out.item())
        assert n == want_k.shape[0], f"call {call}: {n} k-mers, expected {want_k.shape[0]}"
        got_k = out_k[:n].cpu().numpy().view(np.uint64)
        got_c = out_c[:n].cpu().numpy().view(np.uint32)
        assert np.array_equal(got_k, want_k[:, 0]), f"call {call}: k-mers differ"
        assert np.array_equal(got_c, want_c), f"call {call}: counts differ"


def test_noalloc_rejects_inputs_above_its_scratch():
    lib = kmc.load()
    rc = lib.kmc_count_small_noalloc(None, ctypes.c_void_p(1), 1, kmc.KMC_NOALLOC_MAX_BASES + 1, 28,
                                     2, 10**9, None, None, 0, ctypes.c_void_p(1), None)
    assert rc == kmc.KMC_EINVAL
