"""KMC 2 database files written on the GPU and batched GPU lookups, against
the oracle's writer and counts (oracle/kmc_db.py, pinned to the supplement's
format section).  Files are compared byte for byte; lookups element by
element."""
import random

import numpy as np
import pytest

import oracle
from oracle import kmc_db as DB
from oracle import strings as S
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reads(seed, n, L, genome_len, p_err=0.01):
    rng = random.Random(seed)
    g = "".join(rng.choice("ACGT") for _ in range(genome_len))
    out = []
    for _ in range(n):
        p = rng.randrange(0, genome_len - L)
        r = list(g[p:p + L])
        for j in range(L):
            if rng.random() < p_err:
                r[j] = rng.choice("ACGTN")
        out.append("".join(r))
    return out


def _write_both(tmp_path, reads, k, m, B, ci, cx=10 ** 9):
    b, o = oracle.as_reads(reads)
    with kmc.Counter(k, m=m, n_bins=B, cutoff_min=ci, cutoff_max=cx) as c:
        c.add(b, o).count()
        kms, cnt = c.result()
        mp = c.bin_map()
        m_used = c.stats()["m_used"]
        base = str(tmp_path / f"db_k{k}")
        c.write_db(base)
    got = (open(base + ".kmc_pre", "rb").read(), open(base + ".kmc_suf", "rb").read())
    vals = oracle.kmers_to_int(kms)
    # the counts themselves are the oracle's (checked elsewhere too)
    wk, wc = oracle.count(b, o, k, ci, cx, threads=8)
    assert oracle.kmers_to_int(wk) == vals and np.array_equal(wc, cnt)
    want = DB.write(k, m_used, vals, [int(x) for x in cnt], [int(x) for x in mp], B, ci, cx)
    return base, got, want, dict(zip(vals, [int(x) for x in cnt]))


@pytest.mark.parametrize("k,m,B,ci", [(28, 7, 64, 2), (25, 7, 7, 1), (31, 7, 512, 2), (12, 5, 1, 1),
                                      (32, 7, 64, 1), (55, 9, 16, 2), (64, 11, 3, 1)])
def test_db_files_match_oracle(tmp_path, k, m, B, ci):
    reads = _reads(k * 7 + m, 1500, 150, 20_000)
    base, got, want, _ = _write_both(tmp_path, reads, k, m, B, ci)
    assert len(got[0]) == len(want[0]) and got[0] == want[0]
    assert len(got[1]) == len(want[1]) and got[1] == want[1]


def test_db_empty_result(tmp_path):
    # every k-mer occurs once and the cutoff keeps counts >= 2: no records
    base, got, want, counts = _write_both(tmp_path, ["ACGTACGGTCATTGCA"], 8, 3, 4, 2)
    assert not counts and got == want


def _to_words(vals, k):
    words = (k + 31) // 32
    a = np.zeros((len(vals), words), dtype=np.uint64)
    for i, v in enumerate(vals):
        for w in range(words):
            a[i, words - 1 - w] = (v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF
    return a


@pytest.mark.parametrize("k,m,B", [(28, 7, 64), (21, 7, 512), (55, 9, 16), (15, 5, 2)])
def test_db_lookup_matches_oracle(tmp_path, k, m, B):
    reads = _reads(k + 3 * m, 1200, 150, 15_000)
    base, got, want, counts = _write_both(tmp_path, reads, k, m, B, 2)
    assert got == want
    rng = random.Random(k)
    present = list(counts)
    queries, expect = [], []
    for v in present:  # both strands of every stored k-mer
        s = S.from_value(v, k)
        queries += [v, S.value(S.revcomp(s))]
        expect += [counts[v], counts[v]]
    n_abs = 0
    while n_abs < 2000:  # k-mers not in the database (absent or below the cutoff)
        s = "".join(rng.choice("ACGT") for _ in range(k))
        if S.value(S.canonical(s)) not in counts:
            queries.append(S.value(s))
            expect.append(0)
            n_abs += 1
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(_to_words(queries, k).view(np.int64)).to(dev)
    out = torch.full((len(queries),), 0xDEAD, dtype=torch.int32, device=dev)
    db = kmc.kmc_db_open(base, 0)
    try:
        info = kmc.kmc_db_info_get(db)
        assert info["total_kmers"] == len(counts) and info["kmer_length"] == k and info["kmc_ver"] == 0x200
        assert info["n_arrays"] == B
        stream = torch.cuda.current_stream(dev)
        kmc.kmc_db_lookup(db, q.data_ptr(), len(queries), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
    finally:
        kmc.kmc_db_close(db)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), np.array(expect, dtype=np.uint32))


def test_db_mid_workload_scaled(tmp_path):
    w = synth.mid(scale=0.002)
    with kmc.Counter(w.k, m=w.m, n_bins=w.n_bins) as c:
        c.add(w.bases, w.offsets).count()
        kms, cnt = c.result()
        mp = c.bin_map()
        base = str(tmp_path / "mid")
        c.write_db(base)
    vals = oracle.kmers_to_int(kms)
    pre, suf = DB.write(w.k, w.m, vals, [int(x) for x in cnt], [int(x) for x in mp], w.n_bins, 2, 10 ** 9)
    assert open(base + ".kmc_pre", "rb").read() == pre
    assert open(base + ".kmc_suf", "rb").read() == suf


def test_db_write_refuses_minimizer_bins(tmp_path):
    b, o = oracle.as_reads(["ACGTACGGTCATTGCAACGTACGGTCATTGCA"] * 3)
    with kmc.Counter(12, m=5, n_bins=4, debug_flags=kmc.KMC_DEBUG_MINIMIZER) as c:
        c.add(b, o).count()
        with pytest.raises(kmc.KmcError) as e:
            c.write_db(str(tmp_path / "x"))
        assert e.value.code == kmc.KMC_EINVAL


def test_db_write_refuses_noncanonical_counts(tmp_path):
    b, o = oracle.as_reads(["ACGTACGGTCATTGCAACGTACGGTCATTGCA"] * 3)
    with kmc.Counter(12, m=5, n_bins=4, canonical=0) as c:
        c.add(b, o).count()
        with pytest.raises(kmc.KmcError) as e:
            c.write_db(str(tmp_path / "x"))
        assert e.value.code == kmc.KMC_EINVAL
