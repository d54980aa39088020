"""Pins of the oracle's FASTQ / FASTA readers (oracle/formats.py) on
hand-worked files: which bytes are reads, where records end, which files are
malformed.  The expected reads are written out by hand in each test."""
import pytest

from oracle import formats as F


def test_fastq_records_are_the_sequence_lines():
    # quality lines full of letters that are also bases must not become reads
    data = (b"@r1 first\nACGTNACGT\n+\nACGTACGTA\n"
            b"@r2\nGGGG\n+r2\nCCCC\n"
            b"@\n\n+\n\n"                 # an empty read
            b"@r4\r\nTTAC\r\n+\r\n!!!!\r\n")  # CRLF lines
    assert F.parse_fastq(data) == ["ACGTNACGT", "GGGG", "", "TTAC"]


def test_fastq_final_newline_may_be_missing():
    assert F.parse_fastq(b"@a\nAC\n+\nII") == ["AC"]
    assert F.parse_fastq(b"@a\nAC\n+\nII\n") == ["AC"]
    assert F.parse_fastq(b"") == []


@pytest.mark.parametrize("bad", [b"@a\nAC\n+\n",            # three lines
                                 b"@a\nAC\n+\nII\n\n",      # an empty fifth line
                                 b"a\nAC\n+\nII\n",         # no '@'
                                 b"@a\nAC\n-\nII\n"])       # no '+'
def test_fastq_malformed(bad):
    with pytest.raises(ValueError):
        F.parse_fastq(bad)


def test_fasta_records_join_their_lines():
    data = (b">chr1 a genome\nACGTAC\nGTACGT\n\nAC\n"
            b">chr2\r\nTTTT\r\nGG\r\n"
            b">empty\n"
            b">last\nNNAC")
    assert F.parse_fasta(data) == ["ACGTACGTACGTAC", "TTTTGG", "", "NNAC"]
    assert F.parse_fasta(b"") == []
    assert F.parse_fasta(b">x\n") == [""]


def test_fasta_must_start_with_a_header():
    with pytest.raises(ValueError):
        F.parse_fasta(b"ACGT\n>x\nAC\n")
    with pytest.raises(ValueError):
        F.parse_fasta(b"\n>x\nAC\n")


def test_generator_files_read_back_as_the_reads():
    # the seeded FASTQ / FASTA writers used by the GPU tests produce files that
    # the readers turn back into exactly the generator's reads
    import oracle
    from paper_1407_1507_gb300 import synth
    w = synth.tiny(scale=0.002)
    reads = [bytes(w.bases[w.offsets[i]:w.offsets[i + 1]]).decode() for i in range(w.n_reads)]
    assert F.parse_fastq(synth.to_fastq(w.bases, w.offsets)) == reads
    assert F.parse_fastq(synth.to_fastq(w.bases, w.offsets, crlf=True)) == reads
    for width in (1, 7, 60, 1000):
        assert F.parse_fasta(synth.to_fasta(w.bases, w.offsets, width=width)) == reads
    b, o = oracle.as_reads(reads)
    assert bytes(b) == bytes(w.bases) and list(o) == list(w.offsets)
