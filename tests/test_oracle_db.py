"""Pins of the oracle's KMC database writer / reader (oracle/kmc_db.py) to the
supplement's "Database format" section: its worked example (signature,
prefix value, array position, suffix), its file-structure rules (markers,
header position, byte packing), and lookups equal to brute-force string
counts."""
import random
import struct

import numpy as np
import pytest

import oracle
from oracle import kmc_db as DB
from oracle import strings as S


def _packed(s):
    """Symbols four per byte, first symbol in the top bits (computed from the string value)."""
    return S.value(s).to_bytes(len(s) // 4, "big")


def test_db_walk_example(golden):
    g = golden["db_walk"]
    k, m = len(g["kmer"]), g["m"]
    assert oracle.signature_of(g["kmer"], m) == g["signature_value"]
    assert S.value(g["prefix"]) == g["prefix_value"]
    n_arrays = 4 ** m + 1
    ident = list(range(n_arrays))  # the example reads array 97 for signature 97
    # the example k-mer, a k-mer sharing its signature and prefix, and others
    kms = [g["kmer"], "ATACGACAAATC", "CCCCCCCCCCCC", "ACGTACGTACGA"]
    kms = [S.canonical(x) for x in kms]
    counts = [7, 3, 2, 300]
    pre, suf = DB.write(k, m, [S.value(x) for x in kms], counts, ident, n_arrays, 2, 10 ** 9)
    db = DB.read(pre, suf)
    assert db["header"]["lut_prefix_length"] == g["lut_prefix_length"]
    # element 49 of array 97 is the first record of prefix ATAC, element 50 one past the last
    a0 = g["array_start_byte"]
    first, end = struct.unpack_from("<2Q", pre, a0 + 8 * g["prefix_value"])
    same = [x for x in kms if oracle.signature_of(x, m) == 97 and x[:4] == g["prefix"]]
    assert end - first == len(same) == 2
    # the records of that range hold the suffixes in order; the example's is GACAAATG
    rec = db["record_bytes"]
    sufs = [db["data"][i * rec:i * rec + 2] for i in range(first, end)]
    assert sufs == sorted(sufs) and _packed(g["suffix"]) in sufs
    i = first + sufs.index(_packed(g["suffix"]))
    assert int.from_bytes(db["data"][i * rec + 2:(i + 1) * rec], "little") == 7
    assert DB.lookup(db, g["kmer"]) == 7
    assert DB.lookup(db, S.revcomp(g["kmer"])) == 7


def test_db_file_structure(golden):
    reads = ["ACGTTGCAACGGTTACGATCGATCGGATCCA", "TTGCAACGGTTACGATCGAT"]
    k, m, B = 8, 3, 5
    cnt = S.count_brute(reads, k, 1)
    vals = [S.value(x) for x in cnt]
    rng = random.Random(3)
    mp = [rng.randrange(B) for _ in range(4 ** m + 1)]
    pre, suf = DB.write(k, m, vals, list(cnt.values()), mp, B, 1, 10 ** 9)
    # markers at both ends of both files
    assert pre[:4] == pre[-4:] == b"KMCP" and suf[:4] == suf[-4:] == b"KMCS"
    # the header sits x + 8 bytes before the end, x being the 4 bytes before the end marker
    x = struct.unpack("<I", pre[-8:-4])[0]
    hdr = pre[len(pre) - 8 - x:len(pre) - 8]
    assert x == len(hdr) == 68
    f = struct.unpack("<7IQ7II", hdr)
    assert f[0] == k and f[1] == 0 and f[4] == m and f[7] == len(cnt) and f[15] == 0x200
    lut, csize = f[3], f[2]
    assert (k - lut) % 4 == 0
    # sizes: prefixes (one array per bin plus the guard), map, header; records
    assert len(pre) == 4 + 8 * (B * 4 ** lut + 1) + 4 * (4 ** m + 1) + 68 + 8
    assert len(suf) == 8 + len(cnt) * ((k - lut) // 4 + csize)
    # the map region holds the map, least significant byte first
    moff = 4 + 8 * (B * 4 ** lut + 1)
    assert list(struct.unpack_from("<%dI" % len(mp), pre, moff)) == mp
    # the guard is the total
    assert struct.unpack_from("<Q", pre, moff - 8)[0] == len(cnt)


def test_db_suffix_packing_example(golden):
    g = golden["suffix_packing"]
    # a k-mer whose suffix (after a 4-symbol prefix) is the example string
    assert list(DB.suffix_bytes("ACGT" + g["string"], 4)) == g["bytes"]


def test_db_rules():
    assert [DB.counter_size(c) for c in (0, 255, 256, 65535, 65536, 2 ** 24 - 1, 2 ** 24, 2 ** 32 - 1)] == \
        [1, 1, 2, 2, 3, 3, 4, 4]
    assert DB.lut_prefix_length(28, 512) == 4
    assert DB.lut_prefix_length(25, 512) == 5
    assert DB.lut_prefix_length(31, 512) == 7
    assert DB.lut_prefix_length(55, 2048) == 3  # 2048 * 4^7 > 2^24
    assert DB.lut_prefix_length(3, 1) == 3
    for k in range(1, 65):
        assert (k - DB.lut_prefix_length(k, 512)) % 4 == 0


@pytest.mark.parametrize("k,m,B,ci", [(12, 5, 7, 1), (21, 7, 64, 2), (31, 7, 16, 2), (25, 6, 1, 1)])
def test_db_lookup_matches_brute_force(k, m, B, ci):
    rng = random.Random(k * 100 + m)
    genome = "".join(rng.choice("ACGT") for _ in range(600))
    reads = []
    for _ in range(60):
        p = rng.randrange(0, len(genome) - 80)
        r = list(genome[p:p + 80])
        for j in range(len(r)):
            if rng.random() < 0.02:
                r[j] = rng.choice("ACGTN")
        reads.append("".join(r))
    cnt = S.count_brute(reads, k, ci)
    w = np.array([rng.randrange(0, 50) for _ in range(4 ** m + 1)], dtype=np.uint64)
    mp = oracle.bin_map(w, B)
    pre, suf = DB.write(k, m, [S.value(x) for x in cnt], list(cnt.values()), list(mp), B, ci, 10 ** 9)
    db = DB.read(pre, suf)
    for km, c in cnt.items():
        assert DB.lookup(db, km) == c
        assert DB.lookup(db, S.revcomp(km)) == c
    absent = 0
    while absent < 50:
        q = "".join(rng.choice("ACGT") for _ in range(k))
        if S.canonical(q) not in cnt:
            assert DB.lookup(db, q) == 0
            absent += 1
