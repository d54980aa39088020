"""Served counting (kmc_server_*): jobs submitted while others run are batched
together (continuous batching), and each job's result is exactly the oracle's
count of its reads alone, whatever it was batched with."""
import random
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu


def _job(i):
    rng = random.Random(700 + i)
    g = synth.genome_markov3(rng.randint(5_000, 40_000), 900 + i)
    L = rng.choice([100, 150])
    b, o = synth.reads(g, np.full(rng.randint(10, 2500), L), 0.01, 0.0, 1300 + i)
    return b, o, rng.choice([21, 28, 31])


def test_served_results_match_oracle_alone_and_mixed():
    jobs = [_job(i) for i in range(48)]
    s = kmc.kmc_server_open(kmc.make_params(28, m=7, n_bins=64), batch_bases=2 << 20,
                            batch_reads=20_000, batch_sets=16, n_workers=2)
    try:
        ids = []
        # a burst, then arrivals spread over time while batches run
        for i, (b, o, k) in enumerate(jobs):
            ids.append(kmc.kmc_server_submit(s, k, b, o))
            if i >= 16:
                time.sleep(0.002)
        for jid in ids:
            assert kmc.kmc_server_wait(s, jid, 120.0)
        for jid, (b, o, k) in zip(ids, jobs):
            gk, gc, lat = kmc.kmc_server_result(s, jid)
            wk, wc = oracle.count(b, o, k, 2, 10**9, threads=8)
            assert np.array_equal(gk, wk) and np.array_equal(gc, wc), f"job {jid}"
            assert lat > 0
            kmc.kmc_server_release(s, jid)
        st = kmc.kmc_server_stats_get(s)
        assert st["jobs_done"] == len(jobs) and st["error"] == 0
        assert st["max_batch_jobs"] > 1          # jobs were batched together
        assert st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        kmc.kmc_server_close(s)


def test_served_job_alone_equals_job_in_mix():
    b, o, k = _job(3)
    s = kmc.kmc_server_open(kmc.make_params(28, m=7, n_bins=64), batch_bases=2 << 20,
                            batch_reads=20_000, batch_sets=16, n_workers=1)
    try:
        alone = kmc.kmc_server_submit(s, k, b, o)
        assert kmc.kmc_server_wait(s, alone, 60.0)
        a_k, a_c, _ = kmc.kmc_server_result(s, alone)
        others = [_job(100 + i) for i in range(12)]
        ids = [kmc.kmc_server_submit(s, kk, bb, oo) for bb, oo, kk in others[:6]]
        mixed = kmc.kmc_server_submit(s, k, b, o)
        ids += [kmc.kmc_server_submit(s, kk, bb, oo) for bb, oo, kk in others[6:]]
        assert kmc.kmc_server_wait(s, mixed, 60.0)
        m_k, m_c, _ = kmc.kmc_server_result(s, mixed)
        assert np.array_equal(a_k, m_k) and np.array_equal(a_c, m_c)
        for jid in ids:
            assert kmc.kmc_server_wait(s, jid, 60.0)
    finally:
        kmc.kmc_server_close(s)
