"""Batched counting (kmc_batch_*): every set's result equals the oracle's count
of that set alone, whatever the other sets of the sub-batch, with and without
the CUDA graph, with the autotuner, and for sets larger than the capacity."""
import random

import numpy as np
import pytest

import oracle
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu


def _sets(n, seed, max_reads=3000):
    rng = random.Random(seed)
    out = []
    for i in range(n):
        g = synth.genome_markov3(rng.randint(2_000, 50_000), seed * 1000 + i)
        L = rng.choice([100, 150, 250])
        nr = rng.randint(0, max_reads)
        if g.size < L:
            L = g.size
        b, o = synth.reads(g, np.full(nr, L), 0.01, rng.choice([0.0, 0.001]), seed * 7 + i)
        out.append((b, o, rng.choice([21, 28, 31])))
    return out


def _check(b, sets, ci):
    for s, (bs, of, k) in enumerate(sets):
        got = kmc.kmc_batch_result(b, s)
        wk, wc = oracle.count(bs, of, k, ci, 10**9, threads=8)
        assert got[0].shape == wk.shape and np.array_equal(got[0], wk), f"set {s}"
        assert np.array_equal(got[1], wc), f"set {s}"


@pytest.mark.parametrize("flags", [0, kmc.KMC_BATCH_NO_GRAPH, kmc.KMC_BATCH_AUTOTUNE])
def test_batch_sets_match_oracle(flags):
    sets = _sets(40, 3)
    p = kmc.make_params(28, m=7, n_bins=64)
    b = kmc.kmc_batch_open(p, 4 << 20, 40_000, 16, flags)
    try:
        kmc.kmc_batch_run(b, [(x[0], x[1]) for x in sets], [x[2] for x in sets])
        st = kmc.kmc_batch_stats_get(b)
        assert st["n_sub_batches"] >= 3
        _check(b, sets, 2)
        # a second run reuses the captured graph
        kmc.kmc_batch_run(b, [(x[0], x[1]) for x in sets], [x[2] for x in sets])
        _check(b, sets, 2)
    finally:
        kmc.kmc_batch_close(b)


def test_batch_large_sets_take_single_path_and_ci1():
    sets = _sets(6, 9, max_reads=30_000)
    p = kmc.make_params(21, m=7, n_bins=64, cutoff_min=1)
    b = kmc.kmc_batch_open(p, 1 << 20, 10_000, 8, 0)
    try:
        kmc.kmc_batch_run(b, [(x[0], x[1]) for x in sets], [x[2] for x in sets])
        st = kmc.kmc_batch_stats_get(b)
        assert st["n_single"] >= 1
        _check(b, sets, 1)
    finally:
        kmc.kmc_batch_close(b)


def test_batch_sets_of_several_mb_run_in_two_lanes():
    # sets of 4 MiB of bases or more are counted on the single-set path, two
    # at a time on their own streams, between small sets that are batched;
    # page-locked and pageable input mixed; results written into the pinned
    # arena from both lanes (with a growth in between)
    rng = random.Random(21)
    sets = []
    for i in range(9):
        g = synth.genome_markov3(rng.randint(200_000, 2_000_000), 5000 + i)
        nr = 40_000 if i % 3 == 0 else rng.randint(100, 3000)
        b_, o_ = synth.reads(g, np.full(nr, 150), 0.01, 0.001, 6000 + i)
        sets.append((b_, o_, rng.choice([21, 28, 31])))
    torch = pytest.importorskip("torch")
    pinned = torch.from_numpy(sets[3][0]).pin_memory().numpy()
    sets[3] = (pinned, sets[3][1], sets[3][2])
    p = kmc.make_params(28, m=7, n_bins=64)
    b = kmc.kmc_batch_open(p, 64 << 20, 500_000, 32, 0)
    try:
        for _ in range(2):
            kmc.kmc_batch_run(b, [(x[0], x[1]) for x in sets], [x[2] for x in sets])
            st = kmc.kmc_batch_stats_get(b)
            assert st["n_single"] == 3
            _check(b, sets, 2)
    finally:
        kmc.kmc_batch_close(b)
