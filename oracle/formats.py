"""Read files in the two input formats of KMC 2 (Sect. 2.4: reads come from
FASTQ or FASTA files; Suppl. S1 options -fq, -fa, -fm) -- TEST INFRASTRUCTURE
ONLY.  Plain Python on the file's lines; the reads come out as strings, in
file order, ready for the oracle's counting (``oracle.as_reads``).

Readings (the paper names the formats but does not define them):

* FASTQ: records of four lines -- "@" header, sequence, "+" line, quality.
  The read is the sequence line as it stands (a byte other than A/C/G/T
  breaks it, as everywhere); one "\\r" at a line end is dropped; a final
  newline ends the last line and may be missing.  A record whose first line
  does not start with "@" or whose third line does not start with "+", or a
  last record with fewer than four lines (an empty line after the last
  record counts as one), is an error (ValueError).
* FASTA and multi-FASTA: a record is a ">" header line followed by any
  number of sequence lines up to the next ">" line or the end; the read is
  the concatenation of its sequence lines without the line breaks ("\\r"
  dropped, empty lines contribute nothing).  A non-empty file must start
  with ">".

Parity status: pinned by tests/test_oracle_formats.py (hand-worked examples).
"""
from __future__ import annotations

from typing import List


def _lines(data: bytes) -> List[bytes]:
    lines = data.split(b"\n")
    if lines and lines[-1] == b"":
        lines.pop()  # the final newline ends the last line; it does not start one
    return [ln[:-1] if ln.endswith(b"\r") else ln for ln in lines]


def parse_fastq(data: bytes) -> List[str]:
    lines = _lines(data)
    if len(lines) % 4:
        raise ValueError("FASTQ: the last record has fewer than four lines")
    reads = []
    for i in range(0, len(lines), 4):
        if not lines[i].startswith(b"@"):
            raise ValueError(f"FASTQ: record {i // 4} does not start with '@'")
        if not lines[i + 2].startswith(b"+"):
            raise ValueError(f"FASTQ: record {i // 4} has no '+' line")
        reads.append(lines[i + 1].decode("latin-1"))
    return reads


def parse_fasta(data: bytes) -> List[str]:
    if data and not data.startswith(b">"):
        raise ValueError("FASTA: the file does not start with a '>' header")
    reads: List[str] = []
    cur = None
    for ln in _lines(data):
        if ln.startswith(b">"):
            if cur is not None:
                reads.append("".join(cur))
            cur = []
        else:
            cur.append(ln.decode("latin-1"))
    if cur is not None:
        reads.append("".join(cur))
    return reads
