"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

The oracle (oracle/kmc_oracle.c) is trusted only after these pass.  Each test
checks it against something other than itself: a worked example printed in the
paper (tests/golden/paper_examples.json), a closed form, an invariant, or brute
force with a different method (Python strings and collections.Counter instead
of 2-bit numbers and a hash table).
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from oracle import strings as S


# ----------------------------------------------------------- worked examples

def test_encoding_example(golden):
    g = golden["encoding"]
    assert S.value(g["string"]) == g["value"]
    # the C oracle's per-symbol code agrees (A0 C1 G2 T3, first symbol most significant)
    lib = oracle._load()
    v = 0
    for c in g["string"]:
        v = 4 * v + lib.oracle_code(ord(c))
    assert v == g["value"]
    assert lib.oracle_code(ord("N")) < 0 and lib.oracle_code(ord("a")) < 0


def test_suffix_packing_example(golden):
    g = golden["suffix_packing"]
    v = S.value(g["string"])
    n = len(g["string"]) // 4
    assert list(v.to_bytes(n, "big")) == g["bytes"]


def test_signature_example(golden):
    g = golden["signature"]
    sig = oracle.signature_of(g["kmer"], g["m"])
    assert S.from_value(sig, g["m"]) == g["signature"]
    assert S.signature(g["kmer"], g["m"]) == g["signature"]
    # the plain minimiser of the same k-mer is AAATG: the filter matters here
    assert min(g["kmer"][i:i + 5] for i in range(len(g["kmer"]) - 4)) == "AAATG"


def test_superkmer_split_example(golden):
    g = golden["superkmer_split"]
    read, k, m = g["read"], g["k"], g["m"]
    for mode, use_min in (("signatures", False), ("minimizers", True)):
        want = g[mode]
        got = oracle.superkmers(read, k, m, use_minimizer=use_min)
        assert len(got) == len(want), mode
        for (start, nk, sig), (sub, sig_str) in zip(got, want):
            assert read[start:start + nk + k - 1] == sub
            assert S.from_value(sig, m) == sig_str
        got_s = S.superkmers(read, k, m, use_minimizer=use_min)
        assert [(a, b) for a, b in got_s] == [tuple(w) for w in want]


def test_kx_split_example(golden):
    g = golden["kx_split"]
    sk, k, x = g["superkmer"], g["k"], g["x"]
    got = oracle.kxmers(sk, k, x)
    strs = [S.from_value(v, k + xp) for (_, xp, _, v) in got]
    assert strs == g["successive"]
    # Fig. 2 sorted order: k-mers first, then (k+1)-mers, each lexicographic
    srt = sorted(zip([xp for (_, xp, _, _) in got], strs))
    assert [s for _, s in srt] == g["sorted"]
    sorted_strs = [s for _, s in srt]
    for name, (a, b) in g["ranges"].items():
        seg = sorted_strs[a:b]
        if name == "R0":
            assert all(len(s) == k for s in seg)
        elif name == "R1":
            assert all(len(s) == k + 1 for s in seg) and b - a == sum(len(s) == k + 1 for s in sorted_strs)
        else:
            assert all(len(s) == k + 1 and s[0] == name[1] for s in seg)
            assert len(seg) == sum(len(s) == k + 1 and s[0] == name[1] for s in sorted_strs)
    assert [s for _, s in S.kxmers(sk, k, x)] == g["successive"]


# ----------------------------------------------------------- closed forms

def _allowed_closed_form(m):
    """Number of allowed m-mers: s0 free, no AA among s1..s(m-1) (this also
    excludes the AAA start), minus the ACA starts.  a(n) counts AA-free strings
    of length n, e(n) those ending (equivalently starting) with A."""
    e, f = 1, 3  # length 1
    a = {1: 4}
    ev = {1: 1}
    for n in range(2, m + 1):
        e, f = f, 3 * (e + f)
        a[n] = e + f
        ev[n] = e
    return 4 * a[m - 1] - (ev[m - 2] if m >= 3 else 0)


@pytest.mark.parametrize("m", [3, 4, 5, 6, 7, 8, 9])
def test_allowed_mmer_count_closed_form(m):
    lib = oracle._load()
    n = sum(lib.oracle_mmer_allowed(v, m) for v in range(4 ** m))
    assert n == _allowed_closed_form(m)
    if m == 7:
        assert n == 12249


def test_poly_a_closed_form():
    for L, k in [(50, 28), (100, 31), (200, 55), (28, 28), (27, 28)]:
        b, o = oracle.as_reads(["A" * L])
        kms, cnt = oracle.count(b, o, k)
        if L < k:
            assert kms.shape[0] == 0
        else:
            assert kms.shape[0] == 1 and int(cnt[0]) == L - k + 1
            assert oracle.kmers_to_int(kms) == [0]  # A^k has value 0


def _de_bruijn(k):
    """Linear de Bruijn sequence over ACGT of order k (every k-mer exactly once)."""
    a = [0] * (4 * k)
    seq = []

    def db(t, p):
        if t > k:
            if k % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, 4):
                a[t] = j
                db(t + 1, t)
    db(1, 1)
    s = "".join("ACGT"[i] for i in seq)
    return s + s[:k - 1]


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_de_bruijn_closed_form(k):
    seq = _de_bruijn(k)
    b, o = oracle.as_reads([seq])
    kms, cnt = oracle.count(b, o, k)
    vals = oracle.kmers_to_int(kms)
    # every canonical k-mer appears; count 1 for palindromes, 2 otherwise
    n_pal = 4 ** (k // 2) if k % 2 == 0 else 0
    assert len(vals) == (4 ** k + n_pal) // 2
    for v, c in zip(vals, cnt):
        s = S.from_value(v, k)
        assert s == S.canonical(s)
        assert int(c) == (1 if s == S.revcomp(s) else 2)
    assert vals == sorted(vals)


# ----------------------------------------------------------- brute force

def _rand_reads(rng, n, lo, hi, alphabet="ACGT", p_n=0.0):
    out = []
    for _ in range(n):
        L = rng.randint(lo, hi)
        r = "".join(rng.choice(alphabet) if rng.random() >= p_n else rng.choice("NnX.")
                    for _ in range(L))
        out.append(r)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_count_matches_brute_force(seed):
    rng = random.Random(seed)
    k = rng.choice([1, 2, 3, 5, 8, 12, 16, 21, 28, 31, 32, 33, 40, 55, 63, 64])
    alphabet = rng.choice(["ACGT", "AC", "AT", "ACGT"])
    reads = _rand_reads(rng, rng.randint(0, 40), 0, 90, alphabet, p_n=rng.choice([0, 0.02, 0.1]))
    ci = rng.choice([1, 1, 2, 3])
    cx = rng.choice([2**32 - 1, 4, 2])
    want = S.count_brute(reads, k, ci, cx)
    b, o = oracle.as_reads(reads)
    kms, cnt = oracle.count(b, o, k, ci, cx, threads=rng.choice([1, 3]), passes=rng.choice([1, 2]))
    got = {S.from_value(v, k): int(c) for v, c in zip(oracle.kmers_to_int(kms), cnt)}
    assert got == want
    vals = oracle.kmers_to_int(kms)
    assert vals == sorted(vals) and len(set(vals)) == len(vals)


def test_count_exhaustive_small_alphabet():
    # every read over {A,C} of length 6, k = 3: compare with brute force
    reads = ["".join(p) for p in itertools.product("AC", repeat=6)]
    want = S.count_brute(reads, 3)
    b, o = oracle.as_reads(reads)
    kms, cnt = oracle.count(b, o, 3)
    assert {S.from_value(v, 3): int(c) for v, c in zip(oracle.kmers_to_int(kms), cnt)} == want


# ----------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def medium_reads():
    from paper_1407_1507_gb300 import synth
    g = synth.genome_markov3(20000, 99)
    b, o = synth.reads(g, np.full(3000, 100), 0.01, 0.002, 1234)
    return b, o


def _npos(b, o, k):
    """Valid k-mer positions counted with numpy run lengths (independent of the oracle)."""
    ok = np.isin(b, np.frombuffer(b"ACGT", np.uint8))
    total = 0
    for r in range(o.size - 1):
        seg = ok[int(o[r]):int(o[r + 1])]
        run = 0
        for v in seg:
            run = run + 1 if v else 0
            total += run >= k
    return total


def test_total_count_equals_positions(medium_reads):
    b, o = medium_reads
    for k in (21, 28, 40):
        kms, cnt, npos = oracle.count(b, o, k, return_npos=True)
        assert int(cnt.astype(np.uint64).sum()) == npos == _npos(b, o, k)


def _revcomp_reads(b, o):
    table = np.arange(256, dtype=np.uint8)
    for x, y in zip(b"ACGT", b"TGCA"):
        table[x] = y
    out = np.empty_like(b)
    for r in range(o.size - 1):
        a, e = int(o[r]), int(o[r + 1])
        out[a:e] = table[b[a:e][::-1]]
    return out


def test_reverse_complement_symmetry(medium_reads):
    b, o = medium_reads
    rb = _revcomp_reads(b, o)
    for k in (15, 28, 33):
        k1, c1 = oracle.count(b, o, k)
        k2, c2 = oracle.count(rb, o, k)
        assert np.array_equal(k1, k2) and np.array_equal(c1, c2)


def test_union_doubles_counts(medium_reads):
    b, o = medium_reads
    b2 = np.concatenate([b, b])
    o2 = np.concatenate([o, o[1:] + o[-1]])
    rb = _revcomp_reads(b, o)
    b3 = np.concatenate([b, rb])
    for k in (19, 28):
        k1, c1 = oracle.count(b, o, k)
        k2, c2 = oracle.count(b2, o2, k)
        k3, c3 = oracle.count(b3, o2, k)
        assert np.array_equal(k1, k2) and np.array_equal(c2, 2 * c1)
        assert np.array_equal(k1, k3) and np.array_equal(c3, 2 * c1)


def test_cutoff_boundaries():
    # k-mers with exactly 1..6 occurrences (distinct, non-overlapping, no palindromes)
    rng = random.Random(7)
    reads = []
    want_counts = {}
    for n in range(1, 7):
        while True:
            s = "".join(rng.choice("ACGT") for _ in range(12))
            c = S.canonical(s)
            if c != S.revcomp(c) and c not in want_counts:
                break
        want_counts[c] = n
        reads += [s] * n
    for ci, cx in [(1, 6), (2, 5), (3, 3), (4, 2), (6, 6), (7, 100)]:
        b, o = oracle.as_reads(reads)
        kms, cnt = oracle.count(b, o, 12, ci, cx)
        got = {S.from_value(v, 12): int(c) for v, c in zip(oracle.kmers_to_int(kms), cnt)}
        assert got == {s: n for s, n in want_counts.items() if ci <= n <= cx}


# ----------------------------------------------------------- signatures

def test_signature_is_strand_symmetric():
    rng = random.Random(3)
    for _ in range(2000):
        k = rng.choice([8, 12, 21, 28, 31, 55])
        m = rng.choice([4, 5, 7, 9])
        s = "".join(rng.choice("ACGT") for _ in range(k))
        assert oracle.signature_of(s, m) == oracle.signature_of(S.revcomp(s), m)


def test_signature_occurs_and_is_allowed():
    rng = random.Random(4)
    for _ in range(1000):
        k, m = rng.choice([(12, 5), (28, 7), (31, 9), (55, 9)])
        s = "".join(rng.choice("ACGT") for _ in range(k))
        sig = oracle.signature_of(s, m)
        if sig == 4 ** m:
            assert all(not S.allowed(S.canonical(s[i:i + m])) for i in range(k - m + 1))
            continue
        t = S.from_value(sig, m)
        assert S.allowed(t) and (t in s or S.revcomp(t) in s)


def test_signature_sentinel_for_poly_a():
    # every canonical m-mer of A^k is A^m, which starts with AAA
    assert oracle.signature_of("A" * 28, 7) == 4 ** 7
    assert oracle.signature_of("T" * 28, 7) == 4 ** 7


def test_position_sigs_consistent_with_superkmers(medium_reads):
    b, o = medium_reads
    k, m = 28, 7
    ps = oracle.position_sigs(b[: int(o[200])], o[:201], k, m)
    for r in range(200):
        a, e = int(o[r]), int(o[r + 1])
        read = bytes(b[a:e]).decode()
        sk = oracle.superkmers(read, k, m)
        seen = np.full(e - a, oracle.NO_KMER, dtype=np.uint64)
        for start, nk, sig in sk:
            seen[start:start + nk] = sig
        assert np.array_equal(seen, ps[a:e].astype(np.uint64))
        # consecutive super k-mers that touch have different signatures (maximal runs)
        for (s1, n1, g1), (s2, n2, g2) in zip(sk, sk[1:]):
            if s1 + n1 == s2:
                assert g1 != g2


# ----------------------------------------------------------- (k,x)-mers

@pytest.mark.parametrize("x", [0, 1, 2, 3])
def test_kx_split_covers_each_kmer_once_minimally(x):
    rng = random.Random(10 + x)
    for _ in range(300):
        k = rng.choice([5, 9, 15, 28])
        n = rng.randint(1, 40)
        sk = "".join(rng.choice("ACGT") for _ in range(n + k - 1))
        groups = oracle.kxmers(sk, k, x)
        covered = []
        for (start, xp, rev, v) in groups:
            assert 0 <= xp <= x
            s = S.from_value(v, k + xp)
            for j in range(xp + 1):
                km = s[j:j + k]
                assert km == S.canonical(km)  # every k-mer inside is canonical
            covered += [S.canonical(sk[start + j:start + j + k]) for j in range(xp + 1)]
            orig = sk[start:start + k + xp]
            assert s == (S.revcomp(orig) if rev else orig)
        assert covered == [S.canonical(sk[i:i + k]) for i in range(n)]
        # as few as possible: each orientation run of length r needs ceil(r/(x+1)) groups
        d = [sk[i:i + k] <= S.revcomp(sk[i:i + k]) for i in range(n)]
        runs = [len(list(g)) for _, g in itertools.groupby(d)]
        assert len(groups) == sum(-(-r // (x + 1)) for r in runs)


# ----------------------------------------------------------- bin map

def test_bin_map_properties():
    rng = np.random.default_rng(5)
    m, B = 5, 16
    w = rng.integers(0, 1000, size=4 ** m + 1).astype(np.uint64)
    w[rng.integers(0, w.size, 200)] = 0
    w[17] = 50_000  # one heavy signature
    mp = oracle.bin_map(w, B)
    assert mp.max() < B
    loads = np.bincount(mp, weights=w.astype(np.float64), minlength=B)
    total = float(w.sum())
    assert loads.max() <= total / B + float(w.max())
    # the heavy signature shares its bin with nothing heavier than the rest
    assert loads[mp[17]] <= 50_000 + total / B
    # unseen signatures are spread round-robin
    z = np.flatnonzero(w == 0)
    assert np.array_equal(mp[z], z % B)
    # uniform weights: equal group sizes
    mp2 = oracle.bin_map(np.ones(1024, np.uint64), 16)
    assert np.array_equal(np.bincount(mp2, minlength=16), np.full(16, 64))


# ----------------------------------------------- -b and -cs (Suppl. S1 options)

@pytest.mark.parametrize("seed", range(6))
def test_noncanonical_count_is_the_forward_kmers(seed):
    rng = random.Random(500 + seed)
    k = rng.choice([1, 3, 8, 21, 32, 33, 50])
    reads = ["".join(rng.choice("ACGTN") for _ in range(rng.randint(0, 120))) for _ in range(40)]
    b, o = oracle.as_reads(reads)
    kms, cnt = oracle.count(b, o, k, 1, canonical=False)
    got = dict(zip(oracle.kmers_to_int(kms), cnt.tolist()))
    from collections import Counter
    want = Counter(S.value(s) for r in reads for s in S.kmers(r, k))
    assert got == dict(want)
    # the canonical count of c is the forward count of c plus that of its
    # reverse complement (once for a palindrome)
    ck, cc = oracle.count(b, o, k, 1)
    for v, n in zip(oracle.kmers_to_int(ck), cc.tolist()):
        s = S.from_value(v, k)
        r = S.value(S.revcomp(s))
        assert n == got.get(v, 0) + (got.get(r, 0) if r != v else 0)


def test_counter_max_saturates_after_the_cutoffs():
    reads = ["ACGT" * 30, "TTTTTTTTTTTT", "ACGTACGTAC"]
    b, o = oracle.as_reads(reads)
    full_k, full_c = oracle.count(b, o, 4, 1)
    sat_k, sat_c = oracle.count(b, o, 4, 1, counter_max=5)
    assert np.array_equal(full_k, sat_k) and np.array_equal(sat_c, np.minimum(full_c, 5))
    assert full_c.max() > 5
    # the cutoffs look at the true count: cx = 10 drops k-mers seen more often
    # even though their reported count would be 5
    cut_k, cut_c = oracle.count(b, o, 4, 1, cutoff_max=10, counter_max=5)
    keep = full_c <= 10
    assert np.array_equal(cut_k, full_k[keep]) and np.array_equal(cut_c, np.minimum(full_c[keep], 5))


def test_sampled_count_is_a_hash_class_of_the_full_count():
    # the sample oracle (one pass of the hash-partitioned count) equals the
    # full count restricted to its class; the classes partition the k-mers
    from paper_1407_1507_gb300 import synth
    w = synth.mid(scale=0.001)
    for k in (28, 55):
        fk, fc, npos = oracle.count(w.bases, w.offsets, k, 2, 10 ** 9, threads=4, return_npos=True)
        seen = np.zeros(fk.shape[0], dtype=np.int64)
        for which in range(4):
            sk, sc, spos = oracle.count_sample(w.bases, w.offsets, k, 2, 10 ** 9, 4, which, threads=3)
            m = oracle.in_sample(fk, k, 4, which, threads=3)
            assert np.array_equal(fk[m], sk) and np.array_equal(fc[m], sc) and spos == npos
            seen += m
        assert np.all(seen == 1)


@pytest.mark.parametrize("k,prefix", [(28, "ACCTG"), (21, "TT"), (32, "ACGTA"), (5, "C"), (28, "AAAAAAAA"),
                                      (31, "GATTACA"), (55, "ACCTG"), (33, "GT"), (40, "CAGTCAGT"),
                                      (64, "A"), (55, "AAAAAAAA"), (34, "TTT")])
def test_prefix_class_counts_match_the_full_count(k, prefix):
    # the numpy prefix-class counter (used on the full-size workload) against
    # the C oracle's complete count and valid-position total
    from oracle import windows as WN
    from paper_1407_1507_gb300 import synth
    w = synth.mid(scale=0.001)
    fk, fc, npos = oracle.count(w.bases, w.offsets, k, 1, threads=4, return_npos=True)
    v, n, np_ = WN.prefix_class_counts(w.bases, w.offsets, k, prefix, chunk_reads=7_000)
    top = np.array([x >> (2 * (k - len(prefix))) for x in oracle.kmers_to_int(fk)], dtype=object)
    m = np.array([t == S.value(prefix) for t in top], dtype=bool)
    assert np_ == npos and m.sum() > 0
    want = fk[m, 0] if k <= 32 else fk[m]
    assert np.array_equal(v, want) and np.array_equal(n, fc[m].astype(np.int64))


# ------------------------------- signatures and splits against brute force
# The C oracle finds signatures with 2-bit numbers (value and reverse-
# complement value of each m-mer, the Sect. 2.2 rule as bit tests); the
# string module enumerates substrings, canonicalises them as strings and
# filters them with str.startswith / "AA" in.  Random k-mers and reads with
# N, reads close to k long and low-complexity runs (A-rich, short periods,
# poly-A with rare changes) exercise the rule's every branch: a minimum
# taken before the filter, a wrong orientation or a lost sentinel would each
# fail here.

def _low_complexity(rng, n):
    kind = rng.randrange(5)
    if kind == 0:
        return "".join(rng.choice("ACGT") for _ in range(n))
    if kind == 1:  # A-rich
        return "".join(rng.choice("AAAAAAACGT") for _ in range(n))
    if kind == 2:  # short period
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(1, 4)))
        return (p * (n // len(p) + 1))[:n]
    if kind == 3:  # poly-A / poly-T with a few changes
        s = list(rng.choice("AT") * n)
        for _ in range(rng.randint(0, 3)):
            s[rng.randrange(n)] = rng.choice("ACGT")
        return "".join(s)
    return "".join(rng.choice("AC") for _ in range(n))  # AA / ACA starts everywhere


_SIG_CASES = [(k, m) for m in (3, 5, 7, 9, 11) for k in (8, 21, 28, 31, 55) if m < k]


@pytest.mark.parametrize("k,m", _SIG_CASES)
def test_signature_matches_brute_force_strings(k, m):
    rng = random.Random(1000 * k + m)
    for _ in range(150):
        s = _low_complexity(rng, k)
        want = S.signature(s, m)
        got = oracle.signature_of(s, m)
        assert got == (4 ** m if want is None else S.value(want)), (s, m)


@pytest.mark.parametrize("k,m", [(8, 3), (8, 5), (21, 5), (21, 7), (28, 7), (28, 9), (31, 9), (31, 11),
                                 (55, 9), (55, 11)])
def test_superkmers_match_brute_force_strings(k, m):
    rng = random.Random(77 * k + m)
    for _ in range(100):
        L = rng.choice([k - 1, k, k + 1, k + rng.randint(2, 10), rng.randint(k, 3 * k + 20)])
        read = list(_low_complexity(rng, L))
        for _ in range(rng.choice([0, 0, 1, 3])):  # N breaks the read into segments
            read[rng.randrange(L)] = "N"
        read = "".join(read)
        for use_min in (False, True):
            got = oracle.superkmers(read, k, m, use_minimizer=use_min)
            want = S.superkmers(read, k, m, use_minimizer=use_min)
            assert len(got) == len(want), (read, use_min)
            for (start, nk, sig), (sub, sig_s) in zip(got, want):
                assert read[start:start + nk + k - 1] == sub
                assert sig == (4 ** m if sig_s is None else S.value(sig_s))
            # the per-position signatures agree with the split
            if not use_min:
                b, o = oracle.as_reads([read])
                ps = oracle.position_sigs(b, o, k, m)
                for p in range(L):
                    kmer = read[p:p + k]
                    if len(kmer) < k or "N" in kmer:
                        assert ps[p] == oracle.NO_KMER
                    else:
                        sg = S.signature(kmer, m)
                        assert ps[p] == (4 ** m if sg is None else S.value(sg))
