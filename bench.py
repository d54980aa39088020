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
    ap.add_argument("--no-modes", action="store_true",
                    help="skip the other workloads (large, x sweep, batched, served)")
    ap.add_argument("--modes", nargs="+", default=["large", "x_sweep", "batched", "served"],
                    choices=["large", "x_sweep", "batched", "served"])
    ap.add_argument("--large-scale", type=float, default=1.0)
    ap.add_argument("--large-steps", type=int, default=3)
    ap.add_argument("--batch-sets", type=int, default=1000)
    ap.add_argument("--batch-scale", type=float, default=0.1,
                    help="read counts and genomes of the batched sets (1.0: the full workload)")
    ap.add_argument("--served-jobs", type=int, default=1000)
    ap.add_argument("--served-scale", type=float, default=0.02,
                    help="request sizes of the served workload (1.0 with 5000 jobs: the full workload)")
    ap.add_argument("--served-mem-gb", type=float, default=96.0,
                    help="predicted device memory the served jobs in flight may take")
    ap.add_argument("--served-rho", type=float, nargs="+", default=[0.5, 0.8, 0.95, 1.2],
                    help="loads relative to the serial plain path's capacity")
    ap.add_argument("--cpu-sample-reads", type=int, default=CPU_SAMPLE_READS)
    return ap.parse_args()


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:8.1f} s] {msg}\n")
    sys.stderr.flush()


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


_CPU_CHILD = r"""
import json, os, resource, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
b = np.load(sys.argv[2]); o = np.load(sys.argv[3])
k, ci, cx, threads, nr = (int(x) for x in sys.argv[4:9])
o = o[:nr + 1]
b = b[:int(o[-1])]
t = time.perf_counter()
_, _, npos = oracle.count(b, o, k, ci, cx, threads=threads, passes=1, return_npos=True)
dt = time.perf_counter() - t
print(json.dumps({"s": dt, "npos": npos, "rss_kb": resource.getrusage(resource.RUSAGE_SELF).ru_maxrss}))
"""


def cpu_baseline(w, k, ci, cx, n_reads=CPU_SAMPLE_READS):
    """The oracle as it stands on a bounded sample of the workload, on all host
    cores and on one, each in a child process of its own (its peak RSS is the
    child's own); one hash-partition pass (the sample fits in memory)."""
    n = min(n_reads, w.n_reads)
    cores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as td:
        bp, op = os.path.join(td, "b.npy"), os.path.join(td, "o.npy")
        np.save(bp, w.bases[: int(w.offsets[n])])
        np.save(op, w.offsets[: n + 1])
        runs = {}
        for th, nr in ((cores, n), (1, max(1, n // 4))):
            r = subprocess.run([sys.executable, "-c", _CPU_CHILD, ROOT, bp, op, str(k), str(ci), str(cx),
                                str(th), str(nr)], capture_output=True, text=True, check=True)
            runs[th] = json.loads(r.stdout.strip().splitlines()[-1])
    a, one = runs[cores], runs[1]
    return {"value": a["npos"] / a["s"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n:,} reads of the workload ({a['npos']:,} k-mer positions), "
                      f"{a['s']:.1f} s on {cores} host threads",
            "single_thread_kmers_per_s": one["npos"] / one["s"],
            "single_thread_sample": f"first {max(1, n // 4):,} reads, {one['s']:.1f} s on 1 thread",
            "peak_rss_mb": round(max(a["rss_kb"], one["rss_kb"]) / 1024, 1), "hash_passes": 1,
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


# Algorithmic bytes per launch of each stage (minimum traffic of the method:
# every input read once, every output written once).
# DRAM bytes (read + written) per k-mer position of a stage's kernels, from one
# ncu capture of the 1 M-read case of the mid workload (the kernels' traffic
# grows with the keys, so it is scaled by this run's positions); filled in for
# the stages whose kernels were captured after their last change.
# kx_scatter: the upper sweep (every key) and the lower sweep (keys of the bins
# that are not counted straight from their super buckets), captured separately:
# 1,863.8 MB for 119,586,137 keys (upper, 512 bins) and 2,808.7 MB for the same
# keys all in the lower sweep (8 bins: its histogram pass reads the super
# buckets once more where they outgrow L2).  tile_sort: 992.2 MB (super-bucket
# count, 512 bins) and 992.8 MB (tile count, 8 bins) for the same keys.
STAGE_DRAM_BYTES_PER_KEY = {
    "kx_scatter": (1863.8e6 / 119586137, 2808.7e6 / 119586137),
    "tile_sort": (992.2e6 / 119586137, 992.8e6 / 119586137),
}
# Signature scan: warp instructions per base of a piece (ncu sm__inst_executed
# of one piece's launch: 552.0 M for 150 M bases), against the issue peak of
# 4 warp instructions per SM and clock.
SIG_WARP_INST_PER_BASE = 552.0e6 / 150e6


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
        # upper sweep over every key; lower sweep over the keys not counted
        # straight from their super buckets: keys in and out, each
        "kx_scatter": 2 * kw * npos + 2 * kw * (npos - st.get("n_fused_keys", 0)),
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
    log(f"main: {ms:.2f} ms per step")
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
    if dom in STAGE_DRAM_BYTES_PER_KEY and k <= 32 and st0.get("x_used", 0) == 0:
        fused = st0.get("n_fused_keys", 0)
        a, b = STAGE_DRAM_BYTES_PER_KEY[dom]
        traffic = int(a * (st0["n_kmer_positions"] if dom == "kx_scatter" else fused)
                      + b * (st0["n_kmer_positions"] - fused))
    if "signature" in stages and clk.get("sm_mhz"):
        peak_inst = 4 * torch.cuda.get_device_properties(dev).multi_processor_count * clk["sm_mhz"] * 1e6
        got_inst = SIG_WARP_INST_PER_BASE * st0["n_bases"] / (stages["signature"]["ms"] / 1e3)
        stages["signature"]["alu_frac"] = round(got_inst / peak_inst, 4)
        stages["signature"]["alu_bound"] = "warp-instruction issue (4 per SM and clock)"
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
               "value_median": job_rate(npos, world, float(np.median(laps))),
               "h2d_bytes_per_step": int(w.bases.size + w.offsets.size * 8),
               "d2h_bytes_per_step": int(nout * (8 * words + 4))}
    kmc.kmc_close(h)

    modes = None
    if rank == 0 and world == 1 and not args.no_modes:
        modes = {}
        if "x_sweep" in args.modes:
            try:
                modes["x_sweep"] = run_x_sweep(args, local_rank, w, d_bases, d_offs)
            except Exception as e:  # reported, never hides the main line
                modes["x_sweep"] = {"error": f"{type(e).__name__}: {e}"}
    del d_bases, d_offs
    torch.cuda.empty_cache()
    if modes is not None:
        for name, fn in (("large", run_large), ("batched", run_batched), ("served", run_served)):
            if name not in args.modes:
                continue
            try:
                t = time.perf_counter()
                log(f"mode {name} ...")
                modes[name] = fn(args, local_rank)
                modes[name]["mode_wall_s"] = round(time.perf_counter() - t, 1)
                log(f"mode {name} done in {modes[name]['mode_wall_s']} s")
            except Exception as e:  # reported, never hides the main line
                modes[name] = {"error": f"{type(e).__name__}: {e}"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, k, ci, cx, args.cpu_sample_reads)
        log("cpu baseline done")

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

def digest(kms, cnt):
    """Size and CRC-32s of a result's k-mers and counts: equal results give equal
    tuples; a changed, moved or missing entry changes them (up to 2^-64)."""
    import zlib
    k = np.ascontiguousarray(kms)
    c = np.ascontiguousarray(cnt)
    return (int(c.size), zlib.crc32(memoryview(k).cast("B")) if k.size else 0,
            zlib.crc32(memoryview(c).cast("B")) if c.size else 0)


def host_register(arrays):
    """Page-locks the arrays' host memory in place (cudaHostRegister): the
    library then copies them to the device without staging.  Returns the
    arrays it registered."""
    import torch
    rt = torch._C._cudart
    done = []
    for a in arrays:
        if a.nbytes:
            r = rt.cudaHostRegister(a.ctypes.data, a.nbytes, 0)
            if int(getattr(r, "value", r)) == 0:
                done.append(a)
    return done


def host_unregister(arrays):
    import torch
    for a in arrays:
        torch._C._cudart.cudaHostUnregister(a.ctypes.data)


class PinnedOut:
    """Reused pinned host buffers for results read back with kmc_result."""

    def __init__(self):
        self.k = self.c = None

    def get(self, kmc, h, k):
        import torch
        n = kmc.kmc_result_size(h)
        words = (k + 31) // 32
        if self.k is None or self.k.size < n * words or self.c.size < n:
            m = max(n, 1) * 2
            self.tk = torch.empty(m * 2, dtype=torch.int64).pin_memory()
            self.tc = torch.empty(m, dtype=torch.int32).pin_memory()
            self.k = self.tk.numpy().view(np.uint64)
            self.c = self.tc.numpy().view(np.uint32)
        return kmc.kmc_result_into(h, k, self.k, self.c)


def run_batched(args, local_rank):
    """Batched mode (kmc_batch_run: sub-batches replayed as one captured CUDA
    graph, autotuned) against the plain per-set loop (kmc_reset / kmc_add_reads
    / kmc_count / kmc_result on one open handle per k).  Both read the same host
    arrays and copy every result back; both get one untimed warm-up pass over all
    sets (allocations, staging buffers, tuning, graph capture), so the timed
    passes compare counting, not set-up."""
    from paper_1407_1507_gb300 import kmc, synth
    t0 = time.perf_counter()
    sets = synth.batch_sets(args.batch_sets, args.batch_scale)
    gen_s = time.perf_counter() - t0
    log(f"batched: {len(sets)} sets generated in {gen_s:.1f} s")
    t0 = time.perf_counter()
    pinned = host_register([w.bases for w in sets])  # both paths read page-locked input
    log(f"batched: {len(pinned)} sets page-locked in {time.perf_counter() - t0:.1f} s")
    pos = sum(w.n_reads * max(0, int(w.offsets[1] - w.offsets[0]) - w.k + 1) for w in sets)
    bases = sum(int(w.bases.size) for w in sets)
    handles = {}
    try:
        for w in sets:
            if w.k not in handles:
                handles[w.k] = kmc.kmc_open(kmc.make_params(w.k, m=7, n_bins=64, device=local_rank))

        po = PinnedOut()

        stage_sum = {}

        def plain_pass():
            out, busy = [], 0.0
            stage_sum.clear()
            for w in sets:
                h = handles[w.k]
                t = time.perf_counter()
                kmc.kmc_reset(h)
                kmc.kmc_add_reads(h, w.bases, w.offsets)
                kmc.kmc_count(h)
                res = po.get(kmc, h, w.k)
                busy += time.perf_counter() - t
                out.append(digest(*res))  # outside the timed part
                for x, v in kmc.kmc_stats_get(h)["ms_stage"].items():
                    stage_sum[x] = stage_sum.get(x, 0.0) + v
            return out, busy

        plain_pass()
        plain, t_plain = plain_pass()
        log("batched: plain stage ms " + json.dumps({x: round(v, 1) for x, v in stage_sum.items() if v}))
        log(f"batched: plain pass {t_plain:.2f} s")
    finally:
        for h in handles.values():
            kmc.kmc_close(h)
    # the batched calls take groups of sets of up to 4 GB of reads; each
    # group's results are checked (untimed) before the next call reuses them
    groups, g, gb = [], [], 0
    for i, w in enumerate(sets):
        if g and gb + w.bases.size > (4 << 30):
            groups.append(g)
            g, gb = [], 0
        g.append(i)
        gb += w.bases.size
    if g:
        groups.append(g)
    p = kmc.make_params(28, m=7, n_bins=64, device=local_rank)
    bh = kmc.kmc_batch_open(p, 256 << 20, 2_000_000, 512, kmc.KMC_BATCH_AUTOTUNE)
    try:
        def batch_pass():
            busy, ok = 0.0, True
            for g in groups:
                t = time.perf_counter()
                kmc.kmc_batch_run(bh, [(sets[i].bases, sets[i].offsets) for i in g], [sets[i].k for i in g])
                busy += time.perf_counter() - t
                ok &= all(digest(*kmc.kmc_batch_result(bh, j, copy=False)) == plain[i] for j, i in enumerate(g))
            return busy, ok

        batch_pass()  # tunes, captures, sizes the result arena
        t_batch, same = batch_pass()
        log(f"batched: batched pass {t_batch:.2f} s")
        st = kmc.kmc_batch_stats_get(bh)
    finally:
        kmc.kmc_batch_close(bh)
        host_unregister(pinned)
    return {"workload": f"{len(sets)} sets of the batched workload, read counts and genomes x{args.batch_scale}",
            "kmer_positions": pos, "bases": bases, "generation_s": round(gen_s, 2),
            "plain_s": round(t_plain, 4), "batched_s": round(t_batch, 4),
            "plain_kmers_per_s": pos / t_plain, "batched_kmers_per_s": pos / t_batch,
            "plain_device_stage_ms": {x: round(v, 1) for x, v in stage_sum.items() if v},
            "speedup": t_plain / t_batch, "identical_to_plain": bool(same),
            "plain": "one open handle per k, reset per set, page-locked host input, result read back into "
                     "reused pinned buffers; time of those calls only",
            "batched": f"{len(groups)} kmc_batch_run calls (groups of sets up to 4 GB of reads, page-locked "
                       "host input, results in the handle's pinned arena); time of those calls only",
            "sub_batches_last_call": st["n_sub_batches"], "single_path_sets_last_call": st["n_single"],
            "tuning": {"bins_per_set": st["bins_per_set"], "tile_keys": st["tile_keys"],
                       "bucket_keys": st["bucket_keys"]}}


def run_served(args, local_rank):
    """Served mode: Poisson arrivals at load rho (relative to the serial plain
    path's capacity, from its measured service times), continuous batching,
    p50/p99 latency and aggregate throughput, against serial plain execution of
    the same arrivals (one job at a time in arrival order on open handles; its
    latencies follow from the measured service times).  Every served result is
    compared with the plain result of the same request (64-bit digests)."""
    from paper_1407_1507_gb300 import kmc, synth
    t0 = time.perf_counter()
    pools = synth.served_pools(args.served_scale)
    reqs = [synth.served_request(i, pools, args.served_scale) for i in range(args.served_jobs)]
    gen_s = time.perf_counter() - t0
    log(f"served: pools and {len(reqs)} requests in {gen_s:.1f} s")
    pinned = host_register([pl.bases for pl in pools])  # both paths read page-locked input
    pos = sum(nr * max(0, int(o[1] - o[0]) - k + 1) for b, o, k, nr in reqs)
    handles = {}
    svc, plain = [], []
    po = PinnedOut()
    try:
        big = max(range(len(reqs)), key=lambda i: reqs[i][3])
        for k in (21, 28, 31):
            handles[k] = kmc.kmc_open(kmc.make_params(k, m=7, n_bins=64, device=local_rank))
            b, o, _, _ = reqs[big]
            kmc.kmc_add_reads(handles[k], b, o)  # staging and device buffers at their largest
            kmc.kmc_count(handles[k])
            po.get(kmc, handles[k], k)
        for b, o, k, _ in reqs:
            h = handles[k]
            t = time.perf_counter()
            kmc.kmc_reset(h)
            kmc.kmc_add_reads(h, b, o)
            kmc.kmc_count(h)
            res = po.get(kmc, h, k)
            svc.append(time.perf_counter() - t)
            plain.append(digest(*res))  # outside the service time
    finally:
        for h in handles.values():
            kmc.kmc_close(h)
    out = {"workload": f"{len(reqs)} Poisson requests, sizes and k as the batched sets (5% of 10 M reads) "
                       f"x{args.served_scale}, reads from 16 pools", "kmer_positions": pos,
           "bases": int(sum(b.size for b, _, _, _ in reqs)), "generation_s": round(gen_s, 2),
           "serial_plain_total_s": round(float(np.sum(svc)), 3),
           "serial_plain_mean_service_ms": float(np.mean(svc)) * 1e3,
           "serial_plain_kmers_per_s": pos / float(np.sum(svc))}
    log(f"served: serial plain {np.sum(svc):.2f} s")
    rng = np.random.default_rng(20140715)
    try:
        for rho in args.served_rho:
            out[f"rho={rho}"] = _served_run(kmc, reqs, svc, plain, rho, rng, local_rank, pos,
                                            int(args.served_mem_gb * (1 << 30)))
            log(f"served: rho={rho} done")
    finally:
        host_unregister(pinned)
    out["input"] = "page-locked host memory (the read pools registered once), zero-copy submission"
    out["mem_budget_gb"] = args.served_mem_gb
    return out


def _served_run(kmc, reqs, svc, plain, rho, rng, local_rank, pos, mem_budget):
    lam = rho / float(np.mean(svc))
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(reqs)))
    arrivals -= arrivals[0]
    done, lat_serial = 0.0, []
    for a, sv in zip(arrivals, svc):
        done = max(a, done) + sv
        lat_serial.append((done - a) * 1e3)
    serial_wall = done
    # predicted device bytes in flight (32 per input byte): mem_budget of the GPU's memory
    s = kmc.kmc_server_open(kmc.make_params(28, m=7, n_bins=64, device=local_rank),
                            batch_bases=64 << 20, batch_reads=500_000, batch_sets=256, n_workers=4,
                            mem_budget=mem_budget, warm_k=(21, 28, 31))
    lat, same = [None] * len(reqs), [False] * len(reqs)
    ids = [None] * len(reqs)
    have = threading.Semaphore(0)
    err = []

    got = [0]
    stop_mon = threading.Event()

    def monitor():  # progress every 10 s on stderr
        while not stop_mon.wait(10.0):
            try:
                q = kmc.kmc_server_stats_get(s)
                rss = next((ln.split()[1] for ln in open("/proc/self/status") if ln.startswith("VmRSS")), "?")
                log(f"served rho={rho}: submitted {sum(x is not None for x in ids)}, collected {got[0]}, "
                    f"done {q['jobs_done']}, queued {q['jobs_queued']}, rss {int(rss) // 1024} MB")
            except Exception:
                pass

    import concurrent.futures as cf

    def check(i):  # compares job i with the serial result and releases it
        kms, cnt, lat[i] = kmc.kmc_server_result(s, ids[i], copy=False)
        same[i] = digest(kms, cnt) == plain[i]
        del kms, cnt
        kmc.kmc_server_release(s, ids[i])
        got[0] += 1

    def collect():  # waits for the jobs in submission order; checks run on 4 threads
        try:
            with cf.ThreadPoolExecutor(max_workers=4) as ex:
                futs = []
                for i in range(len(reqs)):
                    have.acquire()
                    if not kmc.kmc_server_wait(s, ids[i], 600.0):
                        raise TimeoutError(f"request {i} not done after 600 s")
                    futs.append(ex.submit(check, i))
                for f in futs:
                    f.result()
        except Exception as e:  # reported below
            err.append(f"{type(e).__name__}: {e}")

    try:
        st0 = kmc.kmc_server_stats_get(s)
        col = threading.Thread(target=collect)
        col.start()
        mon = threading.Thread(target=monitor, daemon=True)
        mon.start()
        late = 0.0
        t0 = time.perf_counter()
        for i, ((b, o, k, _), a) in enumerate(zip(reqs, arrivals)):
            d = t0 + a - time.perf_counter()
            if d > 0:
                time.sleep(d)
            else:
                late = max(late, -d)
            ids[i] = kmc.kmc_server_submit_ref(s, k, b, o)
            have.release()
        col.join()
        wall = time.perf_counter() - t0
        stop_mon.set()
        st = kmc.kmc_server_stats_get(s)
    finally:
        kmc.kmc_server_close(s)
    if err:
        return {"error": err[0]}
    # throughput over the server's own clock (first submission to last
    # completion); the checks of the results run beside it, on the host
    swall = st["wall_s"] if st["wall_s"] > 0 else wall
    return {"arrival_rate_per_s": lam, "served_wall_s": round(swall, 3), "checked_wall_s": round(wall, 3),
            "served_kmers_per_s": pos / swall, "serial_plain_kmers_per_s": pos / serial_wall,
            "served_p50_ms": float(np.percentile(lat, 50)), "served_p99_ms": float(np.percentile(lat, 99)),
            "serial_plain_p50_ms": float(np.percentile(lat_serial, 50)),
            "serial_plain_p99_ms": float(np.percentile(lat_serial, 99)),
            "identical_to_plain": bool(all(same)), "max_submit_lag_ms": round(late * 1e3, 3),
            "batches": st["batches"] - st0["batches"], "max_batch_jobs": st["max_batch_jobs"],
            "max_inflight_jobs": st["max_inflight_jobs"]}


def _time_counts(kmc, torch, dev, stream, d_b, d_o, n_reads, n_bases, k, steps, **kw):
    """Device-timed kmc_reset + kmc_add_reads_device + kmc_count on a resident
    read set: (ms per step, per-stage ms, stats)."""
    p = kmc.make_params(k, stream=stream.cuda_stream, device=dev.index, **kw)
    h = kmc.kmc_open(p)
    try:
        def step():
            kmc.kmc_reset(h)
            kmc.kmc_add_reads_device(h, d_b.data_ptr(), d_o.data_ptr(), n_reads, n_bases)
            kmc.kmc_count(h)
        step()
        st = kmc.kmc_stats_get(h)
        stage = {x: 0.0 for x in kmc.STAGES}
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
            for x, v in kmc.kmc_stats_get(h)["ms_stage"].items():
                stage[x] += v
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps, {x: v / steps for x, v in stage.items()}, st
    finally:
        kmc.kmc_close(h)


def run_large(args, local_rank):
    """The large workload at full size (300 Mbp genome, 20 M reads x 150 bp,
    1 % errors, 0.1 % N, m = 9, 2048 bins): k = 28 (64-bit keys) and k = 55
    (128-bit keys) with the reads resident in HBM, and the spill run (device
    budget a quarter of the bins' bytes: bins in pinned host memory, sort in
    waves)."""
    import torch
    from paper_1407_1507_gb300 import kmc, synth
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = synth.large(k=28, scale=args.large_scale)
    d_b = torch.from_numpy(w.bases).to(dev)
    d_o = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    out = {"workload": f"large x{args.large_scale}: 300 Mbp order-3 Markov genome + repeats; 20M reads x 150 bp, "
                       "1% substitutions, 0.1% N; m=9, 2048 bins, cutoffs [2, 1e9]"}
    try:
        for k in (28, 55):
            ms, stage, st = _time_counts(kmc, torch, dev, stream, d_b, d_o, w.n_reads, int(w.bases.size), k,
                                         args.large_steps, m=w.m, n_bins=w.n_bins, cutoff_min=w.cutoff_min,
                                         cutoff_max=w.cutoff_max)
            alg = stage_bytes(st, k)
            a46 = sum(stage.get(x, 0.0) for x in ("kx_count", "kx_scatter", "tile_sort", "big_sort"))
            minb = st["bin_bytes"] + 4 * 8 * ((k + 31) // 32) * st["n_kmer_positions"]
            out[f"k={k}"] = {
                "kmers_per_s": st["n_kmer_positions"] / (ms / 1e3), "ms_per_step": round(ms, 3),
                "kmer_positions": st["n_kmer_positions"], "result_kmers": st["n_out"],
                "distinct_kmers": st["n_distinct"], "key_bytes": 8 * ((k + 31) // 32),
                "stages_ms": {x: round(v, 3) for x, v in stage.items() if v > 0},
                "a4_a6_ms": round(a46, 3),
                "a4_a6_frac_method_min": round(minb / (a46 / 1e3) / 1e9 / peak, 4) if a46 else None,
                "a4_a6_frac_pass_bytes": round((alg["kx_count"] + alg["kx_scatter"] + alg["tile_sort"])
                                               / (a46 / 1e3) / 1e9 / peak, 4) if a46 else None}
            if k == 28:
                bin_bytes = st["bin_bytes"]
            log(f"large: k={k} {ms:.1f} ms per step")
        ms, stage, st = _time_counts(kmc, torch, dev, stream, d_b, d_o, w.n_reads, int(w.bases.size), 28, 1,
                                     m=w.m, n_bins=w.n_bins, cutoff_min=w.cutoff_min, cutoff_max=w.cutoff_max,
                                     device_budget=max(1, bin_bytes // 4))
        out["spill_k=28"] = {"device_budget": bin_bytes // 4, "spilled_bytes": st["spilled_bytes"],
                             "waves": st["n_waves"], "ms_per_step": round(ms, 3),
                             "kmers_per_s": st["n_kmer_positions"] / (ms / 1e3)}
    finally:
        del d_b, d_o
        torch.cuda.empty_cache()
    return out


def run_x_sweep(args, local_rank, w, d_b, d_o):
    """Sect. 2.3's (k,x)-mers on the mid workload: sorted fraction (keys sorted
    per k-mer position) and stage times for x = 0..3 at k = 28."""
    import torch
    from paper_1407_1507_gb300 import kmc
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for x in (0, 1, 2, 3):
        ms, stage, st = _time_counts(kmc, torch, dev, stream, d_b, d_o, w.n_reads, int(w.bases.size), w.k,
                                     2, m=w.m, n_bins=w.n_bins, x=x, cutoff_min=w.cutoff_min,
                                     cutoff_max=w.cutoff_max)
        log(f"x sweep: x={x} {ms:.1f} ms per step")
        out[f"x={x}"] = {"ms_per_step": round(ms, 3), "kmers_per_s": st["n_kmer_positions"] / (ms / 1e3),
                         "sorted_fraction": round(st["n_sorted_keys"] / max(1, st["n_kmer_positions"]), 4),
                         "stages_ms": {s: round(v, 3) for s, v in stage.items() if v > 0}}
    return out


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
