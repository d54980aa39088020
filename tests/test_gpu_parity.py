"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is element by element and exact: the result is a list of
integers (canonical k-mers and counts), so the bar is bit-exact equality.
Inputs are seeded and synthetic; the oracle never sees anything produced by
the CUDA path.
"""
import random

import numpy as np
import pytest

import oracle
from oracle import strings as S
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu


def gpu_count(bases, offsets, k, **kw):
    return kmc.count(bases, offsets, k, **kw)


def oracle_count(bases, offsets, k, ci=2, cx=10**9):
    return oracle.count(bases, offsets, k, ci, cx, threads=8)


def assert_same(got, want):
    gk, gc = got
    wk, wc = want
    assert gk.shape == wk.shape, (gk.shape, wk.shape)
    assert np.array_equal(gk, wk)
    assert np.array_equal(gc, wc)


def rand_reads(rng, n, lo, hi, p_n=0.0, alphabet="ACGT"):
    out = []
    for _ in range(n):
        L = rng.randint(lo, hi)
        out.append("".join(rng.choice(alphabet) if rng.random() >= p_n else "N" for _ in range(L)))
    return out


@pytest.mark.parametrize("seed", range(16))
def test_random_small_inputs(seed):
    rng = random.Random(1000 + seed)
    k = rng.choice([1, 2, 4, 7, 12, 15, 21, 27, 28, 31, 32, 33, 40, 55, 63, 64])
    m = rng.choice([3, 4, 5, 7, 9, 11])
    B = rng.choice([1, 3, 64, 512, 2048])
    reads = rand_reads(rng, rng.randint(1, 300), 0, rng.choice([40, 150, 400]),
                       p_n=rng.choice([0.0, 0.01, 0.05]), alphabet=rng.choice(["ACGT", "ACGT", "AC"]))
    ci = rng.choice([1, 2])
    b, o = oracle.as_reads(reads)
    want = oracle_count(b, o, k, ci)
    for flags in (0, kmc.KMC_DEBUG_SIG_TILE):
        assert_same(gpu_count(b, o, k, m=m, n_bins=B, cutoff_min=ci, debug_flags=flags), want)


def test_tiny_workload_full_size():
    w = synth.tiny()
    got = gpu_count(w.bases, w.offsets, w.k, m=w.m, n_bins=w.n_bins)
    want = oracle_count(w.bases, w.offsets, w.k)
    assert want[0].shape[0] > 100_000
    assert_same(got, want)


@pytest.mark.parametrize("k", [21, 28, 31, 32, 55, 64])
def test_mid_workload_scaled(k):
    w = synth.mid(scale=0.004)
    got = gpu_count(w.bases, w.offsets, k, m=w.m, n_bins=w.n_bins)
    assert_same(got, oracle_count(w.bases, w.offsets, k))


@pytest.mark.parametrize("k,ci,B", [(31, 1, 16), (25, 1, 16), (32, 1, 16), (28, 2, 16), (28, 1, 2), (21, 1, 3),
                                    (40, 1, 16)])
def test_mostly_distinct_keys_fill_the_tiles(k, ci, B):
    # iid random reads: nearly every k-mer is distinct, so the hashed tiles
    # run close to their load limit (and k=32 takes the grouping kernel);
    # with 2 or 3 bins each bin holds millions of distinct keys, so the
    # super buckets counted in one shared-memory pass overflow their table
    # and are counted again in several passes; with ci = 1 the result holds
    # over 10 M k-mers, which the global order sorts by its two-level radix
    # partition (64-bit keys, and 128-bit ones for k = 40)
    rng = np.random.default_rng(77)
    n_reads, L = 120_000, 150
    bases = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, n_reads * L)]
    offsets = np.arange(0, (n_reads + 1) * L, L, dtype=np.uint64)
    got = gpu_count(bases, offsets, k, m=7, n_bins=B, cutoff_min=ci)
    assert_same(got, oracle_count(bases, offsets, k, ci))


@pytest.mark.parametrize("n_reads", [96_000, 100_000, 104_000, 108_000])
def test_super_buckets_split_into_passes_mid_way(n_reads):
    # iid random reads in 4 bins: each super bucket holds about 12 k distinct
    # keys, about twice what one pass of the shared-memory table takes, so
    # buckets are counted in two passes and some overflow in the second one
    # after the first was emitted; the split must not count a key twice
    rng = np.random.default_rng(91)
    L = 150
    bases = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, n_reads * L)]
    offsets = np.arange(0, (n_reads + 1) * L, L, dtype=np.uint64)
    for ci in (1, 2):
        got = gpu_count(bases, offsets, 28, m=7, n_bins=4, cutoff_min=ci)
        assert_same(got, oracle_count(bases, offsets, 28, ci))


def test_one_bin_takes_the_wide_digit_path():
    # ~19 M k-mers in one bin need 14 digit bits, more than a unit
    # histogram holds: the partition then reserves places per warp and digit
    w = synth.mid(scale=0.008)
    for k in (28, 40):
        with kmc.Counter(k, m=w.m, n_bins=1) as c:
            got = c.add(w.bases, w.offsets).count().result()
        assert_same(got, oracle_count(w.bases, w.offsets, k))


@pytest.mark.parametrize("k", [28, 40])
def test_device_budget_spills_bins_and_sorts_in_waves(k):
    # a budget of a quarter of the bins' bytes: most pieces' bins go to
    # pinned host memory, and the bins are sorted in many waves
    w = synth.mid(scale=0.002)
    want = oracle_count(w.bases, w.offsets, k)
    with kmc.Counter(k, m=7, n_bins=64, piece_bytes=1 << 20) as c:
        c.add(w.bases, w.offsets)
        bin_bytes = c.stats()["bin_bytes"]
        assert_same(c.count().result(), want)
        assert c.stats()["n_waves"] == 1 and c.stats()["spilled_bytes"] == 0
    with kmc.Counter(k, m=7, n_bins=64, piece_bytes=1 << 20, device_budget=bin_bytes // 4) as c:
        c.add(w.bases, w.offsets)
        st = c.stats()
        assert st["spilled_bytes"] > bin_bytes // 2
        assert_same(c.count().result(), want)
        assert c.stats()["n_waves"] > 4
        assert_same(c.count().result(), want)  # recount from the spilled bins


def test_large_workload_scaled_m9():
    w = synth.large(k=28, scale=0.002)
    for k in (28, 55):
        got = gpu_count(w.bases, w.offsets, k, m=9, n_bins=2048)
        assert_same(got, oracle_count(w.bases, w.offsets, k))


def test_result_independent_of_bins_and_signature_length():
    w = synth.mid(scale=0.002)
    want = oracle_count(w.bases, w.offsets, 28)
    for B in (1, 64, 512, 2048):
        assert_same(gpu_count(w.bases, w.offsets, 28, m=7, n_bins=B), want)
    for m in (3, 5, 9, 11):
        assert_same(gpu_count(w.bases, w.offsets, 28, m=m, n_bins=256), want)


def test_cutoffs_inclusive_and_ci1():
    w = synth.tiny(scale=0.02)
    for ci, cx in [(1, 2**32 - 1), (2, 3), (3, 3), (5, 10**9), (1, 1)]:
        got = gpu_count(w.bases, w.offsets, 25, m=7, n_bins=16, cutoff_min=ci, cutoff_max=cx)
        assert_same(got, oracle_count(w.bases, w.offsets, 25, ci, cx))


def test_total_count_is_number_of_positions():
    w = synth.mid(scale=0.002)
    with kmc.Counter(28, m=7, n_bins=64, cutoff_min=1, cutoff_max=2**32 - 1) as c:
        kms, cnt = c.add(w.bases, w.offsets).count().result()
        st = c.stats()
    _, _, npos = oracle.count(w.bases, w.offsets, 28, 1, 2**32 - 1, threads=8, return_npos=True)
    assert int(cnt.astype(np.uint64).sum()) == npos == st["n_kmer_positions"]


def test_heavy_repeats_take_the_big_tile_path():
    # one read repeated 30k times: each of its k-mers has 30k copies, far above
    # a tile.  k = 21: the small bins are counted straight from their super
    # buckets, where copies of a key meet in one hash slot whatever their
    # number; k = 32 (64-bit keys, no hashing): the copies fill buckets larger
    # than a tile, which take the big-tile path
    rng = random.Random(5)
    r = "".join(rng.choice("ACGT") for _ in range(60))
    reads = [r] * 30000 + ["A" * 80] * 2000 + rand_reads(rng, 500, 20, 120)
    b, o = oracle.as_reads(reads)
    for k in (21, 32):
        with kmc.Counter(k, m=7, n_bins=8) as c:
            got = c.add(b, o).count().result()
            st = c.stats()
        if k == 32:
            assert st["n_big_tiles"] > 0
        assert_same(got, oracle_count(b, o, k))


def test_poly_a_and_low_complexity():
    reads = ["A" * 200, "T" * 150, "AC" * 80, "ACGT" * 40, "AAAAAAAAAAAAAAAAAAAAAAAAAAAAAC" * 3]
    b, o = oracle.as_reads(reads * 3)
    for k in (5, 28, 33):
        assert_same(gpu_count(b, o, k, m=7, n_bins=4, cutoff_min=1), oracle_count(b, o, k, 1))


def test_empty_and_short_inputs():
    for reads in ([], [""], ["ACG"], ["", "", "ACGTACGTAC"], ["NNNN", "ACGTNACGT"]):
        b, o = oracle.as_reads(reads)
        got = gpu_count(b, o, 5, m=3, n_bins=4, cutoff_min=1)
        assert_same(got, oracle_count(b, o, 5, 1))


def test_multiple_add_calls_append():
    w = synth.tiny(scale=0.01)
    n = w.n_reads
    h1 = n // 3
    with kmc.Counter(28, m=7, n_bins=64) as c:
        c.add(w.bases[: int(w.offsets[h1])], w.offsets[: h1 + 1])
        o2 = w.offsets[h1:] - w.offsets[h1]
        c.add(w.bases[int(w.offsets[h1]):], o2)
        got = c.count().result()
    assert_same(got, oracle_count(w.bases, w.offsets, 28))


def test_recount_is_identical():
    w = synth.tiny(scale=0.01)
    with kmc.Counter(28, m=7, n_bins=64) as c:
        c.add(w.bases, w.offsets)
        a = c.count().result()
        b = c.count().result()
    assert_same(a, b)


def test_device_input_equals_host_input():
    torch = pytest.importorskip("torch")
    w = synth.mid(scale=0.002)
    want = oracle_count(w.bases, w.offsets, 28)
    db = torch.from_numpy(w.bases).cuda()
    do = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    # an unaligned start exercises the stream alignment
    with kmc.Counter(28, m=7, n_bins=512, stream=torch.cuda.current_stream().cuda_stream) as c:
        got = c.add_device(db, do).count().result()
    assert_same(got, want)
    pad = torch.zeros(w.bases.size + 3, dtype=torch.uint8, device="cuda")
    pad[3:] = db
    with kmc.Counter(28, m=7, n_bins=512) as c:
        kmc.kmc_add_reads_device(c.h, pad.data_ptr() + 3, do.data_ptr(), w.n_reads, w.bases.size)
        got = c.count().result()
    assert_same(got, want)


@pytest.mark.parametrize("k,m,flags", [(28, 7, 0), (28, 7, 8), (21, 9, 0), (64, 7, 0), (64, 7, 8),
                                        (12, 7, 0), (40, 11, 0), (32, 5, 0), (28, 7, 16), (28, 7, 24),
                                        (55, 5, 16), (12, 7, 16)])
def test_superkmers_match_oracle_split(k, m, flags):
    # flags 8 = KMC_DEBUG_SIG_TILE (tile-doubling signature kernel); k=12, m=7
    # (window of 6 m-mers) takes that kernel in any case; 16 =
    # KMC_DEBUG_MINIMIZER (canonical minimizers, no Sect. 2.2 filter)
    w = synth.mid(scale=0.0005)
    use_minimizer = bool(flags & kmc.KMC_DEBUG_MINIMIZER)
    flags |= kmc.KMC_DEBUG_KEEP_SUPERKMERS
    with kmc.Counter(k, m=m, n_bins=64, debug_flags=flags) as c:
        c.add(w.bases, w.offsets)
        rd, ps, nk, sg = kmc.kmc_debug_superkmers(c.h)
    got = sorted(zip(rd.tolist(), ps.tolist(), nk.tolist(), sg.tolist()))
    want = []
    for r in range(w.n_reads):
        a, e = int(w.offsets[r]), int(w.offsets[r + 1])
        for st, n, g in oracle.superkmers(bytes(w.bases[a:e]), k, m, use_minimizer=use_minimizer, cut_every=128):
            want.append((r, st, n, g))
    assert got == sorted(want)


@pytest.mark.parametrize("k,m", [(28, 7), (55, 9), (21, 5)])
def test_minimizer_bins_keep_the_counts(k, m):
    w = synth.mid(scale=0.002)
    got = gpu_count(w.bases, w.offsets, k, m=m, n_bins=512, debug_flags=kmc.KMC_DEBUG_MINIMIZER)
    assert_same(got, oracle_count(w.bases, w.offsets, k))


def test_bin_map_matches_oracle_reading():
    w = synth.mid(scale=0.001)
    k, m, B = 28, 7, 64
    with kmc.Counter(k, m=m, n_bins=B) as c:
        c.add(w.bases, w.offsets)
        got = kmc.kmc_get_bin_map(c.h, 4 ** m + 1)
        largest = c.stats()["max_bin_kmers"]
    ps = oracle.position_sigs(w.bases, w.offsets, k, m)
    ps = ps[ps != oracle.NO_KMER]
    weights = np.bincount(ps, minlength=4 ** m + 1).astype(np.uint64)
    want = oracle.bin_map(weights, B)
    assert np.array_equal(got, want)
    # the largest bin's k-mer positions (the statistic of the paper's
    # signatures-versus-minimizers table)
    assert largest == int(np.bincount(want[ps], minlength=B).max())


def test_user_bin_map_does_not_change_result():
    w = synth.tiny(scale=0.01)
    want = oracle_count(w.bases, w.offsets, 28)
    mp = np.random.default_rng(3).integers(0, 5, size=4 ** 7 + 1).astype(np.uint32)
    with kmc.Counter(28, m=7, n_bins=5) as c:
        kmc.kmc_set_bin_map(c.h, mp)
        got = c.add(w.bases, w.offsets).count().result()
    assert_same(got, want)


def test_errors_are_reported():
    b, o = oracle.as_reads(["ACGTACGTAC", "ACGT"])
    with kmc.Counter(5, m=3, n_bins=2) as c:
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_result_size(c.h)
        assert e.value.code == kmc.KMC_ESTATE
        bad = o.copy()
        bad[1], bad[2] = bad[2], bad[1]
        with pytest.raises(kmc.KmcError) as e:
            c.add(b, bad)
        assert e.value.code == kmc.KMC_EINPUT


@pytest.mark.parametrize("piece_bytes", [1 << 12, 100_000, 1 << 20])
def test_many_pieces_host_and_device(piece_bytes):
    torch = pytest.importorskip("torch")
    w = synth.mid(scale=0.002)
    want = oracle_count(w.bases, w.offsets, 28)
    got = gpu_count(w.bases, w.offsets, 28, m=7, n_bins=128, piece_bytes=piece_bytes)
    assert_same(got, want)
    db = torch.from_numpy(w.bases).cuda()
    do = torch.from_numpy(w.offsets.astype(np.int64)).cuda()
    with kmc.Counter(28, m=7, n_bins=128, piece_bytes=piece_bytes) as c:
        assert_same(c.add_device(db, do).count().result(), want)
    # pinned host input: pieces copied on a second stream, one ahead
    pb = torch.from_numpy(w.bases).pin_memory()
    po = torch.from_numpy(w.offsets.astype(np.int64)).pin_memory()
    with kmc.Counter(28, m=7, n_bins=128, piece_bytes=piece_bytes) as c:
        for _ in range(2):  # twice: the second call reuses the buffers and events
            kmc.kmc_add_reads_ptr(c.h, pb.data_ptr(), po.data_ptr(), w.n_reads)
        got2 = c.count().result()
    want2 = oracle_count(np.concatenate([w.bases, w.bases]),
                         np.concatenate([w.offsets, w.offsets[1:] + w.offsets[-1]]), 28)
    assert_same(got2, want2)


@pytest.mark.parametrize("k", [21, 28, 40])
def test_narrow_tile_sort_regroups_colliding_keys(k):
    # 8 sorted bits: many distinct keys share them, so runs must be regrouped
    w = synth.mid(scale=0.002)
    got = gpu_count(w.bases, w.offsets, k, m=7, n_bins=64, cutoff_min=1,
                    debug_flags=kmc.KMC_DEBUG_NARROW_SORT)
    assert_same(got, oracle_count(w.bases, w.offsets, k, 1))


# ------------------------------------------------------------------ (k,x)-mers

@pytest.mark.parametrize("x", [1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_kx_random_small_inputs(x, seed):
    rng = random.Random(5000 + 10 * x + seed)
    k = rng.choice([1, 3, 9, 15, 21, 28, 29, 31, 32, 33, 55, 60, 63])
    m = rng.choice([3, 5, 7, 9])
    reads = rand_reads(rng, rng.randint(1, 250), 0, rng.choice([60, 150, 300]),
                       p_n=rng.choice([0.0, 0.02]), alphabet=rng.choice(["ACGT", "AC"]))
    ci = rng.choice([1, 2])
    b, o = oracle.as_reads(reads)
    got = gpu_count(b, o, k, m=m, n_bins=rng.choice([1, 16, 512]), x=x, cutoff_min=ci)
    assert_same(got, oracle_count(b, o, k, ci))


@pytest.mark.parametrize("k,x", [(21, 3), (28, 1), (28, 2), (28, 3), (31, 3), (55, 3)])
def test_kx_mid_workload_scaled(k, x):
    w = synth.mid(scale=0.003)
    with kmc.Counter(k, m=7, n_bins=512, x=x) as c:
        got = c.add(w.bases, w.offsets).count().result()
        st = c.stats()
    assert st["x_used"] == x
    assert st["n_sorted_keys"] < st["n_kmer_positions"]  # fewer strings to sort (Sect. 2.3)
    assert_same(got, oracle_count(w.bases, w.offsets, k))


def test_kx_big_and_narrow_paths():
    rng = random.Random(11)
    r = "".join(rng.choice("ACGT") for _ in range(70))
    reads = [r] * 20000 + ["A" * 90] * 500 + rand_reads(rng, 400, 30, 150)
    b, o = oracle.as_reads(reads)
    for flags in (0, kmc.KMC_DEBUG_NARROW_SORT):
        got = gpu_count(b, o, 25, m=7, n_bins=4, x=3, debug_flags=flags)
        assert_same(got, oracle_count(b, o, 25))


def _kx_key(value, xp, k, x):
    return (xp << (2 * (k + x))) | (value << (2 * (x - xp)))


@pytest.mark.parametrize("k,x", [(28, 3), (21, 1), (40, 2)])
def test_kx_keys_per_bin_match_oracle_split(k, x):
    # the bins' (k,x)-mer multisets equal the oracle's Sect. 2.3 split of the
    # oracle's super k-mers (same 128-position cut), binned by the same map
    w = synth.mid(scale=0.0004)
    m, B = 7, 8
    mp = (np.arange(4 ** m + 1) % B).astype(np.uint32)
    with kmc.Counter(k, m=m, n_bins=B, x=x, debug_flags=kmc.KMC_DEBUG_KEEP_KEYS) as c:
        kmc.kmc_set_bin_map(c.h, mp)
        c.add(w.bases, w.offsets).count()
        got = {b: sorted(oracle.kmers_to_int(kmc.kmc_debug_bin_keys(c.h, b))) for b in range(B)}
    want = {b: [] for b in range(B)}
    for r in range(w.n_reads):
        a, e = int(w.offsets[r]), int(w.offsets[r + 1])
        read = bytes(w.bases[a:e]).decode()
        for st, n, g in oracle.superkmers(read, k, m, cut_every=128):
            sk = read[st:st + n + k - 1]
            for _, xp, _, v in oracle.kxmers(sk, k, x):
                want[int(mp[g])].append(_kx_key(v, xp, k, x))
    for b in range(B):
        assert got[b] == sorted(want[b]), f"bin {b}"


@pytest.mark.parametrize("k", [1, 5, 21, 28, 32, 55, 64])
def test_noncanonical_counts(k):
    # Suppl. S1 -b: k-mers as read, no canonical form
    w = synth.mid(scale=0.002)
    got = gpu_count(w.bases, w.offsets, k, m=w.m, n_bins=w.n_bins, canonical=0)
    want = oracle.count(w.bases, w.offsets, k, 2, 10 ** 9, threads=8, canonical=False)
    assert want[0].shape[0] > 0
    assert_same(got, want)


@pytest.mark.parametrize("k,cmax,x", [(28, 40, kmc.KMC_AUTO), (28, 255, 0), (31, 3, 0), (55, 10, 0), (25, 7, 2),
                                      (21, 1, 3)])
def test_counter_max_saturates(k, cmax, x):
    # Suppl. S1 -cs: counts above the counter's maximal value are reported as it
    w = synth.mid(scale=0.002)
    got = gpu_count(w.bases, w.offsets, k, m=w.m, n_bins=w.n_bins, x=x, counter_max=cmax)
    want = oracle.count(w.bases, w.offsets, k, 2, 10 ** 9, threads=8, counter_max=cmax)
    exact = oracle.count(w.bases, w.offsets, k, 2, 10 ** 9, threads=8)
    assert int(want[1].max()) == min(cmax, int(exact[1].max()))
    assert_same(got, want)
