"""FASTQ / FASTA input read on the device (kmc_add_file_bytes[_device]):
the counts equal the oracle's counts of the reads that the oracle's format
readers (oracle/formats.py) find in the same bytes."""
import random

import numpy as np
import pytest

import oracle
from oracle import formats as F
from paper_1407_1507_gb300 import kmc, synth

pytestmark = pytest.mark.gpu


def oracle_count_reads(reads, k, ci=2):
    b, o = oracle.as_reads(reads)
    return oracle.count(b, o, k, ci, 10 ** 9, threads=8)


def assert_same(got, want):
    assert got[0].shape == want[0].shape
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def count_file(data, fmt, k, device=False, **kw):
    with kmc.Counter(k, **kw) as c:
        if device:
            import torch
            t = torch.from_numpy(np.frombuffer(data, dtype=np.uint8).copy()).to("cuda")
            c.add_file(t, fmt)
        else:
            c.add_file(data, fmt)
        st = c.stats()
        return c.count().result(), st


@pytest.mark.parametrize("crlf,device", [(False, False), (True, False), (False, True)])
def test_fastq_of_the_mid_workload(crlf, device):
    w = synth.mid(scale=0.002)
    data = synth.to_fastq(w.bases, w.offsets, crlf=crlf)
    got, st = count_file(data, kmc.KMC_FORMAT_FASTQ, w.k, device=device, m=w.m, n_bins=w.n_bins)
    assert st["n_reads"] == w.n_reads and st["n_bases"] == w.bases.size
    assert_same(got, oracle.count(w.bases, w.offsets, w.k, 2, 10 ** 9, threads=8))


@pytest.mark.parametrize("width,device", [(60, False), (7, False), (1000, True)])
def test_multi_fasta_joins_lines(width, device):
    w = synth.mid(scale=0.001)
    data = synth.to_fasta(w.bases, w.offsets, width=width)
    got, st = count_file(data, kmc.KMC_FORMAT_FASTA, 31, device=device, m=7, n_bins=64)
    assert st["n_reads"] == w.n_reads and st["n_bases"] == w.bases.size
    assert_same(got, oracle.count(w.bases, w.offsets, 31, 2, 10 ** 9, threads=8))


def test_fasta_genome_on_one_line_and_wrapped():
    rng = random.Random(5)
    g = "".join(rng.choice("ACGT") for _ in range(300_000))
    g = g[:150_000] + g[20_000:60_000] + g[150_000:]  # repeated stretch: counts >= 2
    want = oracle_count_reads([g], 25)
    for data in (b">genome\n" + g.encode() + b"\n",
                 b">genome description\r\n" + b"\r\n".join(g[i:i + 70].encode() for i in range(0, len(g), 70))):
        assert F.parse_fasta(data) == [g]
        got, st = count_file(data, kmc.KMC_FORMAT_FASTA, 25, m=7, n_bins=16)
        assert st["n_reads"] == 1 and st["n_bases"] == len(g)
        assert_same(got, want)


HAND_FASTQ = (b"@r1 first\nACGTNACGTACGTAC\n+\nACGTACGTACGTACG\n"
              b"@r2\nGGGGACGTACGTAC\n+r2\nCCCCCCCCCCCCCC\n"
              b"@\n\n+\n\n"
              b"@r4\r\nTTACGTACGTAC\r\n+\r\n!!!!!!!!!!!!\r\n"
              b"@r5\nACGTACGTAC\n+\nIIIIIIIIII")
HAND_FASTA = (b">chr1 a genome\nACGTAC\nGTACGT\n\nAC\n"
              b">chr2\r\nTTTT\r\nGG\r\n"
              b">empty\n"
              b">last\nNNACGTACGTAC")


@pytest.mark.parametrize("data,fmt,parse", [(HAND_FASTQ, kmc.KMC_FORMAT_FASTQ, F.parse_fastq),
                                            (HAND_FASTA, kmc.KMC_FORMAT_FASTA, F.parse_fasta)])
def test_hand_worked_files(data, fmt, parse):
    reads = parse(data)
    for k in (3, 4, 6):
        got, st = count_file(data, fmt, k, m=3, n_bins=4, cutoff_min=1)
        assert st["n_reads"] == len(reads) and st["n_bases"] == sum(len(r) for r in reads)
        assert_same(got, oracle_count_reads(reads, k, ci=1))


@pytest.mark.parametrize("data,fmt", [(b"@a\nAC\n+\n", kmc.KMC_FORMAT_FASTQ),
                                      (b"@a\nAC\n+\nII\n\n", kmc.KMC_FORMAT_FASTQ),
                                      (b"a\nAC\n+\nII\n", kmc.KMC_FORMAT_FASTQ),
                                      (b"@a\nAC\n-\nII\n", kmc.KMC_FORMAT_FASTQ),
                                      (b"ACGT\n>x\nAC\n", kmc.KMC_FORMAT_FASTA),
                                      (b"\n>x\nAC\n", kmc.KMC_FORMAT_FASTA)])
def test_malformed_files_are_rejected(data, fmt):
    parse = F.parse_fastq if fmt == kmc.KMC_FORMAT_FASTQ else F.parse_fasta
    with pytest.raises(ValueError):
        parse(data)
    with kmc.Counter(4, m=3, n_bins=4) as c:
        with pytest.raises(kmc.KmcError) as e:
            c.add_file(data, fmt)
        assert e.value.code == kmc.KMC_EINPUT


def test_files_and_reads_add_up():
    w = synth.tiny(scale=0.01)
    n = w.n_reads
    half = n // 2
    fq = synth.to_fastq(w.bases, w.offsets[:half + 1])
    fa = synth.to_fasta(w.bases[w.offsets[half]:], w.offsets[half:] - w.offsets[half], width=50)
    with kmc.Counter(w.k, m=w.m, n_bins=w.n_bins) as c:
        c.add_file(fq, kmc.KMC_FORMAT_FASTQ).add_file(fa, kmc.KMC_FORMAT_FASTA)
        c.add_file(b"", kmc.KMC_FORMAT_FASTQ)
        got = c.count().result()
    assert_same(got, oracle.count(w.bases, w.offsets, w.k, 2, 10 ** 9, threads=8))
