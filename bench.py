#!/usr/bin/env python
"""Benchmark of the GB300 k-mer counter on the mid-size workload.

One step = the whole hot path over one read set: 2-bit packing, signature
scan, super k-mer binning, (k,x)-mer construction, radix sort, run-length
counting with the cutoffs and the global order of the result
(kmc_add_reads_device + kmc_count).  Workload: 50 Mbp order-3 Markov genome
(GC 0.41) with 2,000 repeat copies of 5 kbp at 10 % divergence, 20 M reads
of 150 bp, 0.5 % substitutions, 0.1 % N; k=28, m=7, 512 bins, cutoffs
[2, 1e9].  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank counts its own copy of the workload
(replicas; the path has no exchange step), value = all ranks' k-mers / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "k-mers counted/s at k=28 & % HBM roofline; batched/served vs plain; p99 latency"
UNIT = "k-mers/s"
WORKLOAD = ("mid: 50 Mbp order-3 Markov genome (GC 0.41) + 2,000 repeat copies of 5 kbp at 10% "
            "divergence; 20M reads x 150 bp, 0.5% substitutions, 0.1% N; k=28, m=7, 512 bins, "
            "cutoffs [2, 1e9]")
CPU_SAMPLE_READS = 400_000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--bins", type=int, default=0,
                    help="bin count override (profiling a scaled workload at full-size bins)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the batched / served comparisons")
    ap.add_argument("--batch-sets", type=int, default=300)
    ap.add_argument("--batch-scale", type=float, default=0.02)
    ap.add_argument("--served-jobs", type=int, default=300)
    ap.add_argument("--served-rho", type=float, nargs="+", default=[0.8, 2.0],
                    help="loads relative to the serial plain path's capacity")
    return ap.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Largest value of x over the ranks (the slowest replica sets the step time)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units all replicas processed over the (max) time."""
    return units_per_rank * world / (ms / 1e3)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def workload(scale):
    from paper_1407_1507_gb300 import synth
    return synth.mid(scale=scale)


def cpu_baseline(w, k, ci, cx):
    """The oracle as it stands on a bounded sample of the workload (host cores)."""
    import oracle
    n = min(CPU_SAMPLE_READS, w.n_reads)
    b = w.bases[: int(w.offsets[n])]
    o = w.offsets[: n + 1]
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    _, _, npos = oracle.count(b, o, k, ci, cx, threads=cores, return_npos=True)
    dt = time.perf_counter() - t
    return {"value": npos / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n:,} reads of the workload ({npos:,} k-mer positions), "
                      f"{dt:.1f} s on {cores} host threads"}


# Algorithmic bytes per launch of each stage (minimum traffic of the method:
# every input read once, every output written once).
# DRAM bytes (read + written) per key of the two sweeps (kx0_sweep_kernel on
# 64-bit keys, both modes), from one ncu capture of the 1 M-read case
# (--scale 0.05: 3,747.6 MB for 119,586,137 keys); the sweeps' traffic grows
# with the keys, so it is scaled by this run's keys.
SWEEP_DRAM_BYTES_PER_KEY_U64 = 3747.6e6 / 119586137


def stage_bytes(st, k):
    nb = st["n_bases"]
    npos = st["n_kmer_positions"]
    nrec = st["n_superkmers"]
    binb = st["bin_bytes"]
    nout = st["n_out"]
    kw = 8 * ((k + 31) // 32)
    return {
        "pack": nb * 1.0 + nb / 4 + nb / 4,            # ASCII in; 2-bit codes + 2 masks out
        "signature": nb / 4 + nb / 4 + 8 * nrec,        # codes + masks in; records out
        "bin_scatter": 8 * nrec + binb / 2 + binb,      # records + bases in; bins out
        "kx_count": binb + kw * npos,                   # bins in; keys out (built once)
        "kx_scatter": 4 * kw * npos,                    # two sweeps: keys in and out, each
        "tile_sort": kw * npos + (kw + 4) * nout,       # keys in; survivors out
        "order": 2 * (kw + 4) * nout,                   # survivors in and out
    }


def run_ours(args, rank, local_rank, world):
    import torch
    from paper_1407_1507_gb300 import kmc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workload(args.scale)
    k, m, B, ci, cx = w.k, w.m, args.bins or w.n_bins, w.cutoff_min, w.cutoff_max
    d_bases = torch.from_numpy(w.bases).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)
    p = kmc.make_params(k, m=m, n_bins=B, cutoff_min=ci, cutoff_max=cx, device=local_rank,
                        stream=stream.cuda_stream)
    h = kmc.kmc_open(p)

    def step():
        kmc.kmc_reset(h)
        kmc.kmc_add_reads_device(h, d_bases.data_ptr(), d_offs.data_ptr(), w.n_reads, w.bases.size)
        kmc.kmc_count(h)

    for _ in range(max(args.warmup, 0)):
        step()
    st0 = kmc.kmc_stats_get(h)
    npos = st0["n_kmer_positions"]

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = Clocks(local_rank)
    clocks.start()
    stage_ms = {s: 0.0 for s in kmc.STAGES}
    launches = 0
    barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        st = kmc.kmc_stats_get(h)
        for s, v in st["ms_stage"].items():
            stage_ms[s] += v
        launches += st["n_launches"]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    value = job_rate(npos, world, ms)

    # roofline of the dominant kernel stage
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    per = {s: stage_ms[s] / args.steps for s in stage_ms}
    alg = stage_bytes(st0, k)
    dom = max((s for s in alg), key=lambda s: per.get(s, 0.0))
    stages = {}
    for s, t in per.items():
        if t <= 0:
            continue
        stages[s] = {"ms": round(t, 4)}
        if s in alg:
            gbs = alg[s] / (t / 1e3) / 1e9
            stages[s].update({"alg_bytes": int(alg[s]), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)})
    stages["sum_ms"] = round(sum(per.values()), 3)
    achieved = stages[dom]["gbs"]
    traffic = None
    if dom == "kx_scatter" and k <= 32 and st0.get("x_used", 0) == 0:
        traffic = int(SWEEP_DRAM_BYTES_PER_KEY_U64 * st0["n_kmer_positions"])
    roofline = {"bound": "hbm", "kernel_stage": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"}

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not args.no_e2e:
        hb = torch.from_numpy(w.bases).pin_memory()
        ho = torch.from_numpy(w.offsets.view(np.int64)).pin_memory()
        nout = st0["n_out"]
        words = (k + 31) // 32
        rk = torch.empty(max(nout, 1) * words, dtype=torch.int64).pin_memory()
        rc = torch.empty(max(nout, 1), dtype=torch.int32).pin_memory()
        import ctypes
        lib = kmc.load()

        def e2e_step():
            kmc.kmc_reset(h)
            kmc.kmc_add_reads_ptr(h, hb.data_ptr(), ho.data_ptr(), w.n_reads)
            kmc.kmc_count(h)
            n = ctypes.c_uint64()
            r = lib.kmc_result(h, rk.data_ptr(), rc.data_ptr(), max(nout, 1), ctypes.byref(n))
            if r != 0:
                raise RuntimeError(kmc.strerror(r))

        for _ in range(2):
            e2e_step()
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        laps = []
        for _ in range(args.steps):
            t1 = time.perf_counter()
            e2e_step()  # ends with the result read back into host memory
            laps.append((time.perf_counter() - t1) * 1e3)
        torch.cuda.synchronize(dev)
        barrier()
        e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world, dev)
        e2e = {"value": job_rate(npos, world, e_ms), "unit": UNIT, "ms_per_step": round(e_ms, 3),
               "ms_per_step_median": round(float(np.median(laps)), 3), "ms_per_step_max": round(max(laps), 3),
               "h2d_bytes_per_step": int(w.bases.size + w.offsets.size * 8),
               "d2h_bytes_per_step": int(nout * (8 * words + 4))}
    kmc.kmc_close(h)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, k, ci, cx)
    modes = None
    if rank == 0 and world == 1 and not args.no_modes:
        modes = {}
        for name, fn in (("batched", run_batched), ("served", run_served)):
            try:
                modes[name] = fn(args, local_rank)
            except Exception as e:  # reported, never hides the main line
                modes[name] = {"error": f"{type(e).__name__}: {e}"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reads": w.n_reads, "bases": int(w.bases.size),
                   "kmer_positions": npos, "result_kmers": st0["n_out"],
                   "distinct_kmers": st0["n_distinct"], "super_kmers": st0["n_superkmers"],
                   "x": st0["x_used"], "l2": "inputs (3 GB of reads, 19 GB of keys) exceed L2; no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "scale": args.scale, "n_bins": B},
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "stages": stages,
        "cpu_baseline": cpu, "clocks": clk, "modes": modes,
        "bases_per_s": job_rate(int(w.bases.size), world, ms),
    }
    return out


# ------------------------------------------------------------ batched / served

def _mode_sets(n, scale, seed_base=0):
    """Sets shaped like the batched workload (log-normal read counts with median
    200 k, genomes 1-20 Mbp, L in {100,150,250}, k in {21,28,31}, 1 % errors, no
    N), with read counts and genome sizes multiplied by `scale`."""
    from paper_1407_1507_gb300 import synth
    out = []
    for i in range(n):
        n_reads, genome, L, k = synth.batch_set_params(seed_base + i)
        nr = max(1, int(n_reads * scale))
        g = synth.genome_markov3(max(int(genome * scale), L + 1), synth.BASE_SEED + 10_000 + seed_base + i)
        b, o = synth.reads(g, np.full(nr, L), 0.01, 0.0, synth.BASE_SEED + 20_000 + seed_base + i)
        out.append((b, o, k, nr * (L - k + 1)))
    return out


def run_batched(args, local_rank):
    """Batched mode (kmc_batch_run, one graph-replayed launch sequence per
    sub-batch, autotuned) against the plain loop of one kmc_open / add /
    count / result per set, both through the public API from host memory."""
    import torch
    from paper_1407_1507_gb300 import kmc
    sets = _mode_sets(args.batch_sets, args.batch_scale)
    pos = sum(x[3] for x in sets)
    # plain per-set loop
    torch.cuda.synchronize()
    t = time.perf_counter()
    plain = []
    for b, o, k, _ in sets:
        with kmc.Counter(k, m=7, n_bins=64, device=local_rank) as c:
            plain.append(c.add(b, o).count().result())
    t_plain = time.perf_counter() - t
    p = kmc.make_params(28, m=7, n_bins=64, device=local_rank)
    bh = kmc.kmc_batch_open(p, 256 << 20, 2_000_000, 512, kmc.KMC_BATCH_AUTOTUNE)
    try:
        kmc.kmc_batch_run(bh, [(x[0], x[1]) for x in sets], [x[2] for x in sets])  # tunes + captures
        t = time.perf_counter()
        kmc.kmc_batch_run(bh, [(x[0], x[1]) for x in sets], [x[2] for x in sets])
        t_batch = time.perf_counter() - t
        st = kmc.kmc_batch_stats_get(bh)
        same = all(np.array_equal(kmc.kmc_batch_result(bh, i)[0], plain[i][0]) and
                   np.array_equal(kmc.kmc_batch_result(bh, i)[1], plain[i][1]) for i in range(len(sets)))
    finally:
        kmc.kmc_batch_close(bh)
    return {"workload": f"{len(sets)} sets shaped like the batched workload, read counts and genomes x{args.batch_scale}",
            "kmer_positions": pos, "plain_kmers_per_s": pos / t_plain, "batched_kmers_per_s": pos / t_batch,
            "speedup": t_plain / t_batch, "identical_to_plain": bool(same), "sub_batches": st["n_sub_batches"],
            "single_path_sets": st["n_single"], "tuning": {"bins_per_set": st["bins_per_set"],
                                                          "tile_keys": st["tile_keys"],
                                                          "bucket_keys": st["bucket_keys"]}}


def run_served(args, local_rank):
    """Served mode: Poisson arrivals at load rho (relative to the serial plain
    path's capacity), continuous batching, p50/p99 latency and aggregate
    throughput, against serial plain execution of the same arrivals (one job at
    a time, FIFO; its latencies follow from the measured service times)."""
    from paper_1407_1507_gb300 import kmc
    rng = np.random.default_rng(20140715)
    jobs = _mode_sets(args.served_jobs, args.batch_scale, seed_base=5000)
    # 5 % large jobs (10 M reads at full scale)
    for i in range(0, len(jobs), 20):
        b, o, k, _ = jobs[i]
        from paper_1407_1507_gb300 import synth
        L = int(o[1] - o[0]) if o.size > 1 else 150
        nr = max(1, int(10_000_000 * args.batch_scale))
        g = synth.genome_markov3(max(int(5_000_000 * args.batch_scale), L + 1), 31337 + i)
        b2, o2 = synth.reads(g, np.full(nr, L), 0.01, 0.0, 4242 + i)
        jobs[i] = (b2, o2, k, nr * (L - k + 1))
    pos = sum(x[3] for x in jobs)
    # serial plain: service times one job at a time
    svc = []
    for b, o, k, _ in jobs:
        t = time.perf_counter()
        with kmc.Counter(k, m=7, n_bins=64, device=local_rank) as c:
            c.add(b, o).count().result()
        svc.append(time.perf_counter() - t)
    mean_svc = float(np.mean(svc))
    out = {"workload": f"{len(jobs)} Poisson requests, sizes and k as the batched sets x{args.batch_scale}, "
                       "5% large jobs", "kmer_positions": pos,
           "serial_plain_mean_service_ms": mean_svc * 1e3}
    for rho in args.served_rho:
        out[f"rho={rho}"] = _served_run(kmc, jobs, svc, rho, rng, local_rank, pos)
    return out


def _served_run(kmc, jobs, svc, rho, rng, local_rank, pos):
    lam = rho / float(np.mean(svc))
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(jobs)))
    done, lat_serial = 0.0, []
    for a, sv in zip(arrivals, svc):
        start = max(a, done)
        done = start + sv
        lat_serial.append((done - a) * 1e3)
    serial_wall = done - arrivals[0]
    s = kmc.kmc_server_open(kmc.make_params(28, m=7, n_bins=64, device=local_rank),
                            batch_bases=128 << 20, batch_reads=1_000_000, batch_sets=256, n_workers=2,
                            warm_k=(21, 28, 31))
    try:
        st0 = kmc.kmc_server_stats_get(s)
        t0 = time.perf_counter()
        ids = []
        for (b, o, k, _), a in zip(jobs, arrivals - arrivals[0]):
            d = t0 + a - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids.append(kmc.kmc_server_submit(s, k, b, o))
        lat = []
        for jid in ids:
            kmc.kmc_server_wait(s, jid, 600.0)
            lat.append(kmc.kmc_server_result(s, jid)[2])
        wall = time.perf_counter() - t0
        st = kmc.kmc_server_stats_get(s)
    finally:
        kmc.kmc_server_close(s)
    return {"arrival_rate_per_s": lam,
            "served_kmers_per_s": pos / wall, "serial_plain_kmers_per_s": pos / serial_wall,
            "served_p50_ms": float(np.percentile(lat, 50)), "served_p99_ms": float(np.percentile(lat, 99)),
            "serial_plain_p50_ms": float(np.percentile(lat_serial, 50)),
            "serial_plain_p99_ms": float(np.percentile(lat_serial, 99)),
            "batches": st["batches"] - st0["batches"], "max_batch_jobs": st["max_batch_jobs"],
            "max_inflight_jobs": st["max_inflight_jobs"]}


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step counts a bounded
    sample of the same workload."""
    if rank != 0:
        return None
    w = workload(args.scale)
    import oracle
    n = min(CPU_SAMPLE_READS, w.n_reads)
    b = w.bases[: int(w.offsets[n])]
    o = w.offsets[: n + 1]
    cores = os.cpu_count() or 1
    for _ in range(max(args.warmup, 0)):
        oracle.count(b, o, w.k, w.cutoff_min, w.cutoff_max, threads=cores)
    t = time.perf_counter()
    npos = 0
    for _ in range(args.steps):
        _, _, npos = oracle.count(b, o, w.k, w.cutoff_min, w.cutoff_max, threads=cores, return_npos=True)
    dt = (time.perf_counter() - t) / args.steps
    v = npos / dt
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_reads": n, "kmer_positions": npos},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {n:,} reads of the workload per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank, local_rank, world = dist_info()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, local_rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
