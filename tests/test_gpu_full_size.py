"""The benchmark's workload at its full size and in the benchmark's launch
configuration (mid: 20 M reads x 150 bp, k=28, m=7, 512 bins, cutoffs
[2, 1e9], reads resident in device memory): the result restricted to a
prefix class of k-mers (about 1/65,536 of them) equals the plain
definition's counts of that class (oracle/windows.py), the whole result is
sorted, distinct and inside the cutoffs, and with cutoff_min = 1 the counts
add up to the number of valid k-mer positions."""
import ctypes

import numpy as np
import pytest

from oracle import windows as WN
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu

PREFIX = "ACCTGATG"


def check_prefix_class(vals, cnt, k, prefix, want_vals, want_counts, ci, cx):
    """The result's k-mers with the given first symbols equal the definition's."""
    keep = (want_counts >= ci) & (want_counts <= cx)
    m = (vals >> np.uint64(2 * (k - len(prefix)))) == np.uint64(WN._value(prefix))
    assert int(m.sum()) == int(keep.sum()) > 0
    assert np.array_equal(vals[m], want_vals[keep])
    assert np.array_equal(cnt[m].astype(np.int64), want_counts[keep])


def test_mid_workload_full_size():
    torch = pytest.importorskip("torch")
    w = synth.mid(scale=1.0)
    k = w.k
    dev = torch.device("cuda", 0)
    d_b = torch.from_numpy(w.bases).to(dev)
    d_o = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    with kmc.Counter(k, m=w.m, n_bins=w.n_bins, cutoff_min=w.cutoff_min, cutoff_max=w.cutoff_max) as c:
        kms, cnt = c.add_device(d_b, d_o).count().result()
    vals = kms[:, 0]
    assert vals.size > 50_000_000
    assert np.all(vals[1:] > vals[:-1])
    assert int(cnt.min()) >= w.cutoff_min and int(cnt.max()) <= w.cutoff_max
    want_vals, want_counts, npos = WN.prefix_class_counts(w.bases, w.offsets, k, PREFIX)
    check_prefix_class(vals, cnt, k, PREFIX, want_vals, want_counts, w.cutoff_min, w.cutoff_max)
    del kms, cnt, vals
    # every valid position is one occurrence: with no lower cutoff the counts add up
    with kmc.Counter(k, m=w.m, n_bins=w.n_bins, cutoff_min=1, cutoff_max=w.cutoff_max) as c:
        c.add_device(d_b, d_o).count()
        n = c.size()
        counts = np.empty(n, dtype=np.uint32)
        nn = ctypes.c_uint64()
        assert kmc.load().kmc_result(c.h, None, counts.ctypes.data, n, ctypes.byref(nn)) == kmc.KMC_OK
    assert int(counts.sum(dtype=np.uint64)) == npos == 2_392_029_849


# ------------------------------------------------- the large workload at size
# 300 Mbp order-3 Markov genome with the mid workload's repeats; 20 M reads of
# 150 bp, 1 % substitutions, 0.1 % N; m = 9, 2048 bins, cutoffs [2, 1e9];
# k = 28 (64-bit keys) and k = 55 (128-bit keys); and the same counts with the
# device budget at a quarter of the bins' bytes, so that most bins are moved
# to pinned host memory and the sort runs in waves.

def _lex_increasing(vals):
    if vals.ndim == 1:
        return bool(np.all(vals[1:] > vals[:-1]))
    hi, lo = vals[:, 0], vals[:, 1]
    return bool(np.all((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))))


def _class_mask(vals, k, prefix):
    q = len(prefix)
    if vals.ndim == 1:
        return (vals >> np.uint64(2 * (k - q))) == np.uint64(WN._value(prefix))
    h = k - 32
    assert q <= h
    return (vals[:, 0] >> np.uint64(2 * (h - q))) == np.uint64(WN._value(prefix))


@pytest.fixture(scope="module")
def large_reads():
    torch = pytest.importorskip("torch")
    w = synth.large(k=28, scale=1.0)
    dev = torch.device("cuda", 0)
    d_b = torch.from_numpy(w.bases).to(dev)
    d_o = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    yield w, d_b, d_o
    del d_b, d_o
    torch.cuda.empty_cache()


@pytest.mark.parametrize("k", [28, 55])
def test_large_workload_full_size(large_reads, k):
    w, d_b, d_o = large_reads
    want_vals, want_counts, npos = WN.prefix_class_counts(w.bases, w.offsets, k, PREFIX)
    keep = (want_counts >= w.cutoff_min) & (want_counts <= w.cutoff_max)
    assert int(keep.sum()) > 0
    bin_bytes = 0
    for budget in (0, None):  # everything on the device; then a quarter of the bins' bytes
        kw = dict(m=w.m, n_bins=w.n_bins, cutoff_min=w.cutoff_min, cutoff_max=w.cutoff_max)
        if budget is None:
            kw["device_budget"] = max(1, bin_bytes // 4)
        with kmc.Counter(k, **kw) as c:
            kms, cnt = c.add_device(d_b, d_o).count().result()
            st = c.stats()
        assert st["n_kmer_positions"] == npos
        if budget is None:
            assert st["spilled_bytes"] > bin_bytes // 2 and st["n_waves"] > 1, st
        bin_bytes = st["bin_bytes"]
        vals = kms[:, 0] if k <= 32 else kms
        assert vals.shape[0] > 100_000_000
        assert _lex_increasing(vals)
        assert int(cnt.min()) >= w.cutoff_min and int(cnt.max()) <= w.cutoff_max
        m = _class_mask(vals, k, PREFIX)
        assert np.array_equal(vals[m], want_vals[keep]), budget
        assert np.array_equal(cnt[m].astype(np.int64), want_counts[keep]), budget
        del kms, cnt, vals
    # with no lower cutoff the counts add up to the valid positions
    with kmc.Counter(k, m=w.m, n_bins=w.n_bins, cutoff_min=1, cutoff_max=w.cutoff_max) as c:
        c.add_device(d_b, d_o).count()
        n = c.size()
        counts = np.empty(n, dtype=np.uint32)
        nn = ctypes.c_uint64()
        assert kmc.load().kmc_result(c.h, None, counts.ctypes.data, n, ctypes.byref(nn)) == kmc.KMC_OK
    assert int(counts.sum(dtype=np.uint64)) == npos
