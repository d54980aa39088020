"""Failure paths, made to happen without faulting the GPU.

* Host side: an allocation (device pool or pinned host memory) is made to fail
  through the library's test hook; the call returns KMC_ENOMEM, the handle
  closes cleanly, and the next job counts correctly.
* Device side: a bounded mbarrier wait is pointed at a barrier that nothing
  arrives on; it gives up after its limit, the kernel waits for its own copy
  in flight, reports the timeout and returns; kmc_count returns KMC_ETIMEOUT
  and the CUDA context stays usable.
* Server: a queued job is cancelled and ends with KMC_ECANCELED, while the
  jobs around it still give the oracle's counts.
* A single set with more bins than the per-CTA shared-memory histograms hold.
"""
import numpy as np
import pytest

import oracle
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reads():
    w = synth.mid(scale=0.002)  # 40 k reads of 150 bp
    return w.bases, w.offsets


def _count_expect(b, o, k, **kw):
    """(rc, result): the count through the C ABI, or the error code it raised."""
    try:
        return kmc.KMC_OK, kmc.count(b, o, k, **kw)
    except kmc.KmcError as e:
        return e.code, None


def test_injected_allocation_failures_return_enomem(reads):
    b, o = reads
    want = oracle.count(b, o, 28, 2, 10**9, threads=8)
    failed = 0
    try:
        # successive allocation sites: the handle's first buffers, the pinned
        # staging of pageable input, the distribution, the sort scratch
        for after in (0, 1, 2, 4, 8, 16, 32, 64):
            kmc.kmc_debug_fail_alloc(after)
            rc, got = _count_expect(b, o, 28, m=7, n_bins=64)
            kmc.kmc_debug_fail_alloc(-1)
            assert rc in (kmc.KMC_OK, kmc.KMC_ENOMEM), (after, rc)
            if rc == kmc.KMC_ENOMEM:
                failed += 1
            else:  # the injection came after the last allocation of the job
                assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
            # the library is still usable after the failure
            got = kmc.count(b, o, 28, m=7, n_bins=64)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), after
    finally:
        kmc.kmc_debug_fail_alloc(-1)
    assert failed >= 4


def test_bounded_device_wait_times_out_and_reports(reads):
    b, o = reads
    k = 40  # wide keys: the tile kernel with bulk copies and mbarrier waits
    rc, _ = _count_expect(b, o, k, m=9, n_bins=64, debug_flags=kmc.KMC_DEBUG_WAIT_TIMEOUT)
    assert rc == kmc.KMC_ETIMEOUT
    # the context is usable: the same count without the flag equals the oracle
    got = kmc.count(b, o, k, m=9, n_bins=64)
    want = oracle.count(b, o, k, 2, 10**9, threads=8)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_server_cancels_a_queued_job():
    jobs = []
    for i in range(6):
        g = synth.genome_markov3(200_000, 4100 + i)
        nr = 150_000 if i == 0 else 3_000  # the first job keeps the worker busy
        bb, oo = synth.reads(g, np.full(nr, 150), 0.01, 0.0, 4200 + i)
        jobs.append((bb, oo, 28))
    s = kmc.kmc_server_open(kmc.make_params(28, m=7, n_bins=64), batch_bases=64 << 20,
                            batch_reads=400_000, batch_sets=1, n_workers=1)
    try:
        ids = [kmc.kmc_server_submit(s, k, bb, oo) for bb, oo, k in jobs]
        kmc.kmc_server_cancel(s, ids[4])  # behind four jobs that run one at a time
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_server_wait(s, ids[4], 60.0)
        assert e.value.code == kmc.KMC_ECANCELED
        for i, jid in enumerate(ids):
            if i == 4:
                continue
            assert kmc.kmc_server_wait(s, jid, 120.0)
            gk, gc, _ = kmc.kmc_server_result(s, jid)
            bb, oo, k = jobs[i]
            wk, wc = oracle.count(bb, oo, k, 2, 10**9, threads=8)
            assert np.array_equal(gk, wk) and np.array_equal(gc, wc), i
        # a finished job cannot be cancelled; a cancelled one can be released
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_server_cancel(s, ids[0])
        assert e.value.code == kmc.KMC_ESTATE
        kmc.kmc_server_release(s, ids[4])
        assert kmc.kmc_server_stats_get(s)["jobs_done"] == 5
    finally:
        kmc.kmc_server_close(s)


@pytest.mark.parametrize("n_bins", [2049, 4096, 65536])
def test_more_bins_than_shared_memory_histograms(reads, n_bins):
    b, o = reads
    want = oracle.count(b, o, 28, 2, 10**9, threads=8)
    for m in (7, 9):
        got = kmc.count(b, o, 28, m=m, n_bins=n_bins)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (m, n_bins)
