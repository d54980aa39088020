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
