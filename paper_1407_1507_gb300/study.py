"""Signatures versus canonical minimizers (the paper's comparison table,
Sect. 3 / "signatures and minimizers"): for k = 28 and 55 and signature
lengths m = 5..9, the average number of super k-mers per read, the number of
k-mers in the largest bin and the memory needed to sort that bin, on the
seeded mid workload (reads resident in device memory, 512 bins).

    python -m paper_1407_1507_gb300.study [--scale S] [--bins B] [--ks 28 55] [--ms 5 6 7 8 9]

Prints one JSON object per (k, m) and a table.  "Minimizers" are canonical
minimizers (the smallest canonical m-mer, no Sect. 2.2 filter; the binning is
strand-symmetric, so the counts are unchanged); "signatures" add the
Sect. 2.2 filter.  Sorting memory for the largest bin = its k-mers x the key
size (8 bytes for k <= 32, 16 above) x 2 (the sort's two key arrays).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import kmc, synth


def measure(d_bases, d_offs, n_reads, k, m, bins, minimizer):
    flags = kmc.KMC_DEBUG_MINIMIZER if minimizer else 0
    with kmc.Counter(k, m=m, n_bins=bins, debug_flags=flags) as c:
        c.add_device(d_bases, d_offs)
        st = c.stats()
    key_bytes = 8 if k <= 32 else 16
    return {
        "superkmers_per_read": st["n_superkmers"] / max(n_reads, 1),
        "largest_bin_kmers": int(st["max_bin_kmers"]),
        "largest_bin_sort_gb": st["max_bin_kmers"] * key_bytes * 2 / 1e9,
        "kmer_positions": int(st["n_kmer_positions"]),
    }


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--bins", type=int, default=512)
    ap.add_argument("--ks", type=int, nargs="+", default=[28, 55])
    ap.add_argument("--ms", type=int, nargs="+", default=[5, 6, 7, 8, 9])
    args = ap.parse_args(argv)
    w = synth.mid(scale=args.scale)
    dev = torch.device("cuda", 0)
    d_bases = torch.from_numpy(w.bases).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    rows = []
    for k in args.ks:
        for m in args.ms:
            r = {"k": k, "m": m, "reads": int(w.n_reads), "bins": args.bins,
                 "minimizers": measure(d_bases, d_offs, w.n_reads, k, m, args.bins, True),
                 "signatures": measure(d_bases, d_offs, w.n_reads, k, m, args.bins, False)}
            rows.append(r)
            print(json.dumps(r), flush=True)
    print(f"{'k':>3} {'m':>2} | {'min: sk/read':>12} {'largest bin':>12} {'sort GB':>8} | "
          f"{'sig: sk/read':>12} {'largest bin':>12} {'sort GB':>8}")
    for r in rows:
        a, b = r["minimizers"], r["signatures"]
        print(f"{r['k']:>3} {r['m']:>2} | {a['superkmers_per_read']:12.3f} {a['largest_bin_kmers']:12,d} "
              f"{a['largest_bin_sort_gb']:8.2f} | {b['superkmers_per_read']:12.3f} "
              f"{b['largest_bin_kmers']:12,d} {b['largest_bin_sort_gb']:8.2f}")
    return rows


if __name__ == "__main__":
    main()
