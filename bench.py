#!/usr/bin/env python
"""Benchmark of the gDP2d hot path on GB300: Steiner points inserted per second.

One step = the whole hot path on one synthetic PSLG: the GPU CDT (the first step of
Algorithm 1) and the refinement loop (the rest of Algorithm 1).  The default
workload is the paper-shaped one, the largest single-GPU configuration:
1,000,164 FP64 points (uniform, Gaussian clusters, circles), 10,000 random
segments plus 20 fans of 8 segments 5 degrees apart, B = sqrt 2.

  value     Steiner points / (CDT + refine) device time, inputs resident in HBM,
            un-instrumented steps
  e2e       the same through the C ABI with pinned host buffers: create (H2D
            inside), refine and export (D2H) all in the timed region
  roofline  the cavity-growth kernel (the largest refinement kernel), timed by
            CUDA events inside the graph in separate instrumented steps:
            algorithmic bytes per launch / launch time vs the HBM peak, plus its
            FP64 rate vs the measured FP64 peak and its L2 traffic
  cpu_baseline  the sequential C oracle on the machine's host cores
  batched / served  (N=1) the 4,096-PSLG batch and a 10 s Poisson request
            trace, each against the plain per-mesh loop on the same GPU, run
            after the headline step and summarised in its line

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SQ2 = math.sqrt(2.0)
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
L2_NOTE = "flushed between steps (512 MB write)"
WORKLOAD_NAMES = {
    "paper_shaped": "paper-shaped: 1,000,164 FP64 points (500k uniform, 300k in 100 Gaussian clusters, "
                    "200k on 50 circles), 10,000 random segments + 20 fans of 8 segments 5 deg apart, "
                    "B=sqrt(2)",
    "mid": "mid: unit square + 100,000 uniform FP64 points + 1,000 random segments, B=sqrt(2)",
    "contours": "contours: unit square + 20 families x 25 nested closed polylines x 200 vertices "
                "(100,004 points and segments)",
}
# the reference arm's bounded sample: the same recipe at a quarter of the size
REF_SAMPLE = {"n_uniform": 125_000, "n_gauss": 75_000, "n_circle": 50_000, "n_seg": 2_500, "n_fans": 5}

# Algorithmic bytes of the dominant step of the refinement, cavity growth
# (the pre-pass k_pre, then k_grow_w<0>, or k_grow_b above 32,768 candidates;
# Sec. 5.2-5.3), per unit of
# work the library counts on the device:
#   per cavity of k triangles: the k cavity triangles and the k + 2 triangles
#   across its boundary edges are read, each 12 B of vertex ids + 48 B of FP64
#   coordinates, (2k + 2) * 60 B, and each cavity triangle gets an 8 B mark
#   written and read back, 16 k B:  120 B per grown candidate + 136 B per cavity
#   triangle;
#   per point-location walk step: one triangle and its neighbours, 76 B;
#   per candidate set up by the pre-pass (k_pre): its own triangle, 12 B of ids
#   + 48 B of coordinates, and its key put on its start triangles and their
#   first ring (4 marks of 8 B on average), 92 B.
GROW_BYTES = {"candidate": 120, "cavity_tri": 136, "walk_step": 76, "setup": 92}
GROW_SOURCES = ("gdp_core.cuh", "gdp_pred.cuh", "gdp_kernels.cuh")
# the kernels of one refinement iteration (launched once per iteration, so an ncu
# launch list counts them in every step and their shares compare directly)
GROW_KERNELS = ("k_pre", "k_grow_w<0>", "k_grow_b", "k_grow_g<0>", "k_grow_t<0>")
REFINE_KERNELS = ("k_scan_eval", "k_scan_count", "k_scan_write") + GROW_KERNELS + (
    "k_grow_big<0>", "k_survive", "k_depend", "k_offsets", "k_insert_w<0>", "k_insert_g<0>", "k_insert_t<0>",
    "k_link<0>")
# ncu counters of the cavity-growth kernels over one whole refine of the bench
# workload, per grown candidate (DRAM and L2 bytes, FP64 flops, FP64 pipe)
COUNTERS_FILE = os.path.join(ROOT, "profiles", "cavity_growth_paper_shaped_counters.md")


def grow_bytes(st) -> float:
    return (GROW_BYTES["candidate"] * st["grown"] + GROW_BYTES["cavity_tri"] * st["cavity_tris"] +
            GROW_BYTES["walk_step"] * st["walk_steps"] + GROW_BYTES["setup"] * st.get("setups", 0))


def grow_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in GROW_SOURCES:
        with open(os.path.join(ROOT, "paper_2007_00324_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_counters():
    """per-grown-candidate ncu counters of the cavity-growth kernels from the
    committed summary, or {} when the kernels' sources changed since"""
    try:
        kv = {}
        with open(COUNTERS_FILE) as f:
            for line in f:
                if line.startswith("counter:"):
                    k, v = line[len("counter:"):].split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source-hash") != grow_source_hash():
            return {}
        return {k: float(v) for k, v in kv.items() if k != "source-hash"}
    except Exception:
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdp", choices=["gdp", "reference"])
    ap.add_argument("--B", type=float, default=SQ2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="paper_shaped",
                    choices=["paper_shaped", "mid", "contours", "batched", "served"],
                    help="paper_shaped: the headline line; mid / contours (with --max-len): the same "
                         "step on those inputs; batched / served: the batching and serving "
                         "configurations (one JSON line each)")
    ap.add_argument("--roof-steps", type=int, default=2,
                    help="instrumented steps (cavity growth timed inside the graph) for the roofline")
    ap.add_argument("--measure-step", action="store_true",
                    help="run exactly one CDT + refine of the workload and print its counters "
                         "(the command the ncu counter captures run)")
    ap.add_argument("--count", type=int, default=4096, help="batched: number of PSLGs")
    ap.add_argument("--rate", type=float, default=200.0, help="served: requests per second")
    ap.add_argument("--duration", type=float, default=10.0, help="served: seconds of arrivals")
    ap.add_argument("--no-systems", action="store_true",
                    help="paper_shaped at N=1: skip the batched and served runs that follow the "
                         "headline step (sub-objects 'batched' and 'served' of its line)")
    ap.add_argument("--cand-cap", type=int, default=0, help="per-mesh candidate cap (Rule 2), 0 = none")
    ap.add_argument("--cand-block", type=int, default=0, help="threads per block of the per-candidate kernels")
    ap.add_argument("--graph-iters", type=int, default=0, help="iterations per graph replay, -1 = no graph")
    ap.add_argument("--max-len", type=float, default=0.0, help="edge-length bound l, 0 = none")
    return ap.parse_args()


def refine_kwargs(args):
    return {"cand_cap": args.cand_cap, "cand_block": args.cand_block, "graph_iters": args.graph_iters,
            "max_len": args.max_len}


# ---------------------------------------------------------------- batched / served
def _gen_square(job):
    from paper_2007_00324_gb300 import workloads
    n, m, seed = job
    p = workloads.square_pslg(n, m, seed)
    return p.xy, p.seg


def _generate(jobs, workers=None):
    """square PSLGs in a spawn process pool (before any GPU call)"""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_square, jobs, chunksize=max(1, len(jobs) // (4 * workers))))


def _oracle_run(job):
    from oracle import oracle
    xy, seg, B = job
    t0 = time.perf_counter()
    m = oracle.Mesh(xy, seg)
    st = m.refine(B)
    return st, m.n_steiner, time.perf_counter() - t0


def _oracle_pool(jobs):
    """the oracle as independent processes over all host cores"""
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import oracle
    oracle.build()
    workers = max(1, os.cpu_count() or 1)
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        out = list(ex.map(_oracle_run, jobs))
    return out, time.perf_counter() - t0, workers


def _pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


def run_batched(args):
    """4,096 PSLGs (log-uniform 200-50,000 uniform points, 2% segments,
    B = sqrt 2): the plain per-mesh loop against one batch (default launch
    parameters and autotuned ones) on the same GPU."""
    from paper_2007_00324_gb300 import workloads
    sizes = workloads.batched_sizes(args.count)
    seed = workloads.SEED_BASE + 3
    jobs = [(int(n), int(round(0.02 * n)), seed * 7919 + i) for i, n in enumerate(sizes)]
    t_gen = time.perf_counter()
    pslgs = _generate(jobs)
    t_gen = time.perf_counter() - t_gen
    cpu = None
    if not args.no_cpu_baseline:
        sample = pslgs[::max(1, len(pslgs) // 64)][:64]
        out, dt, workers = _oracle_pool([(xy, seg, args.B) for xy, seg in sample])
        cpu = {"value": len(sample) / dt, "unit": "meshes/s", "cores": workers, "kind": "oracle",
               "sample": f"{len(sample)} PSLGs of the batch (every {max(1, len(pslgs) // 64)}th), "
                         f"one process per core, {dt:.1f} s",
               "steiner_per_s": sum(o[1] for o in out) / dt}
    import torch
    from paper_2007_00324_gb300 import gdp
    gdp.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    tot_pts = int(sum(len(xy) for xy, _ in pslgs))
    # autotune on a sample (every 32nd PSLG)
    sample = pslgs[::32]
    t_tune = time.perf_counter()
    best, trials = gdp.autotune(sample, args.B, stream=stream)
    t_tune = time.perf_counter() - t_tune

    def batch_run(opts):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = gdp.Batch(pslgs, stream=stream)
        s = b.refine(args.B, **opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        info = b.info()
        ok = int((info["status"] == 0).sum())
        b.close()
        return {"ms": 1000 * dt, "meshes_per_s": len(pslgs) / dt, "steiner": int(s["n_steiner"]),
                "steiner_per_s": s["n_steiner"] / dt, "cdt_ms": s["cdt_ms"], "refine_ms": s["refine_ms"],
                "iterations": s["iterations"], "ok": ok}

    batch_run({})   # warm-up (allocator, graph paths)
    default = batch_run({})
    tuned = batch_run(best)
    # the plain per-mesh loop: one gdp_mesh per PSLG, one after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_plain = 0
    for xy, seg in pslgs:
        m = gdp.Mesh(xy, seg, stream=stream)
        st_plain += m.refine(args.B)["n_steiner"]
        m.close()
    torch.cuda.synchronize()
    dt_plain = time.perf_counter() - t0
    plain = {"ms": 1000 * dt_plain, "meshes_per_s": len(pslgs) / dt_plain, "steiner": st_plain,
             "steiner_per_s": st_plain / dt_plain}
    line = {"metric": "batched meshes/s (CDT + refine, host inputs, wall clock)",
            "value": tuned["meshes_per_s"], "unit": "meshes/s", "n_gpus": 1, "steps": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched: {len(pslgs)} PSLGs, uniform points log-uniform in "
                                   f"[200, 50000] ({tot_pts} points), 2% segments, B=sqrt(2)"},
            "batched_tuned": tuned, "batched_default": default, "plain_loop": plain,
            "speedup_vs_plain_loop": tuned["meshes_per_s"] / plain["meshes_per_s"],
            "autotune": {"best": best, "seconds": t_tune, "sample_meshes": len(sample),
                         "trials": [{"cand_block": int(t[0]), "cand_cap": int(t[1]),
                                     "refine_ms": round(t[2], 3), "steiner": int(t[3])} for t in trials]},
            "generate_s": t_gen}
    if cpu:
        line["cpu_baseline"] = cpu
    return line


def run_served(args):
    """Poisson arrivals (seeded, --rate per second for --duration s) of PSLGs
    with log-uniform 1,000-500,000 points, 1-5% segments, B in {1.5, sqrt 2}:
    the continuous-batching server against the plain loop (one request at a
    time, in arrival order) on the same trace and GPU."""
    from paper_2007_00324_gb300 import workloads
    trace = workloads.served_trace(rate=args.rate, duration=args.duration, build=False)
    # the same per-request draws as served_trace(build=True), generated in parallel
    rng_jobs = []
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(workloads.SEED_BASE + 4))
    t = 0.0
    i = 0
    meta = []
    while True:
        t += float(rng.exponential(1.0 / args.rate))
        if t > args.duration:
            break
        n = int(math.exp(rng.uniform(math.log(1000), math.log(500_000))))
        frac = int(rng.integers(1, 6)) / 100.0
        B = 1.5 if rng.random() < 0.5 else SQ2
        rng_jobs.append((n, int(round(frac * n)), (workloads.SEED_BASE + 4) * 104729 + i))
        meta.append((t, B))
        i += 1
    assert len(meta) == len(trace) and all(abs(a[0] - r.t_arrival) < 1e-12 for a, r in zip(meta, trace))
    t_gen = time.perf_counter()
    pslgs = _generate(rng_jobs)
    t_gen = time.perf_counter() - t_gen
    tot_pts = int(sum(len(xy) for xy, _ in pslgs))
    cpu = None
    if not args.no_cpu_baseline:
        k = min(len(pslgs), 32)
        out, dt, workers = _oracle_pool([(pslgs[j][0], pslgs[j][1], meta[j][1]) for j in range(k)])
        cpu = {"value": k / dt, "unit": "meshes/s", "cores": workers, "kind": "oracle",
               "sample": f"the first {k} requests of the trace, one process per core, all at once, "
                         f"{dt:.1f} s", "steiner_per_s": sum(o[1] for o in out) / dt}
    import torch
    from paper_2007_00324_gb300 import gdp
    gdp.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    # warm-up of both paths on a small request
    w = workloads.square_pslg(2000, 40, 1)
    gdp.Mesh(w.xy, w.seg, stream=stream).refine(SQ2)
    free, _ = torch.cuda.mem_get_info()
    tri_slots = int(min((1 << 29) - 1, 0.35 * free / 64))

    def serve():
        srv = gdp.Server(tri_slots, tri_slots // 2, 1 << 23, 2048, stream=stream)
        srv.submit(w.xy, w.seg, SQ2)
        while True:
            nw, nl, _ = srv.step()
            if nw == 0 and nl == 0:
                break
        srv.results()
        lat, steiner, done_at = {}, 0, {}
        nxt = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = {}
        while len(done_at) < len(pslgs):
            now = time.perf_counter() - t0
            while nxt < len(pslgs) and meta[nxt][0] <= now:
                tickets[srv.submit(pslgs[nxt][0], pslgs[nxt][1], meta[nxt][1])] = nxt
                nxt += 1
            if nxt < len(pslgs) and not tickets.keys() - done_at.keys():
                time.sleep(max(0.0, min(0.002, meta[nxt][0] - now)))
            srv.step()
            for info, xy, tri, sub in srv.results():
                j = tickets[info["ticket"]]
                done_at[info["ticket"]] = time.perf_counter() - t0
                lat[j] = 1000 * (done_at[info["ticket"]] - meta[j][0])
                steiner += info["n_steiner"]
                assert info["status"] == 0, info
        span = max(done_at.values())
        srv.close()
        return lat, steiner, span

    def plain():
        lat, steiner = {}, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j, (xy, seg) in enumerate(pslgs):
            now = time.perf_counter() - t0
            if meta[j][0] > now:
                time.sleep(meta[j][0] - now)
            m = gdp.Mesh(xy, seg, stream=stream)
            steiner += m.refine(meta[j][1])["n_steiner"]
            m.export()
            m.close()
            lat[j] = 1000 * (time.perf_counter() - t0 - meta[j][0])
        return lat, steiner, time.perf_counter() - t0

    lat_s, st_s, span_s = serve()
    lat_p, st_p, span_p = plain()

    def summary(lat, steiner, span):
        v = list(lat.values())
        return {"p50_ms": _pct(v, 50), "p99_ms": _pct(v, 99), "mean_ms": sum(v) / len(v),
                "meshes_per_s": len(v) / span, "steiner_per_s": steiner / span, "makespan_s": span}

    served, pl = summary(lat_s, st_s, span_s), summary(lat_p, st_p, span_p)
    line = {"metric": "served meshes/s and p50/p99 latency (Poisson arrivals, wall clock)",
            "value": served["meshes_per_s"], "unit": "meshes/s", "n_gpus": 1, "steps": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"served: {len(pslgs)} requests, Poisson {args.rate:g}/s for "
                                   f"{args.duration:g} s, 1,000-500,000 points ({tot_pts} in all), "
                                   f"1-5% segments, B in {{1.5, sqrt 2}}",
                       "pool_tri_slots": tri_slots},
            "served": served, "plain_loop": pl,
            "p99_speedup_vs_plain": pl["p99_ms"] / served["p99_ms"],
            "throughput_speedup_vs_plain": served["meshes_per_s"] / pl["meshes_per_s"],
            "generate_s": t_gen}
    if cpu:
        line["cpu_baseline"] = cpu
    return line


def systems_summary(args):
    """The batched and served configurations run after the headline step, in
    the same process, summarised as sub-objects of the headline line."""
    out = {}
    b = run_batched(args)
    out["batched"] = {"config": b["config"]["workload"], "meshes_per_s": b["value"],
                      "batched_tuned": b["batched_tuned"], "batched_default": b["batched_default"],
                      "plain_loop": b["plain_loop"], "speedup_vs_plain_loop": b["speedup_vs_plain_loop"],
                      "autotune_best": b["autotune"]["best"], "cpu_baseline": b.get("cpu_baseline")}
    v = run_served(args)
    out["served"] = {"config": v["config"]["workload"], "meshes_per_s": v["value"], "served": v["served"],
                     "plain_loop": v["plain_loop"], "p99_speedup_vs_plain": v["p99_speedup_vs_plain"],
                     "throughput_speedup_vs_plain": v["throughput_speedup_vs_plain"],
                     "cpu_baseline": v.get("cpu_baseline")}
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.
    The sampler is started before the warm-up steps and the timed steps wait
    for its first sample: starting nvidia-smi initialises NVML, which can stall
    the CUDA calls of other processes for tens of milliseconds."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([time.perf_counter()] + [x.strip() for x in line.split(",")])

    def wait_first(self, timeout=15.0):
        t0 = time.perf_counter()
        while self.proc and not self.rows and time.perf_counter() - t0 < timeout:
            time.sleep(0.05)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t_lo=None, t_hi=None):
        """the samples taken in [t_lo, t_hi] (plus the last one before t_lo,
        the state when the window opened); all samples without a window"""
        rows = self.rows
        if t_lo is not None:
            before = [r for r in rows if r[0] < t_lo]
            rows = before[-1:] + [r for r in rows if t_lo <= r[0] <= t_hi]
        rows = [r[1:] for r in rows]
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def load_workload(name):
    from paper_2007_00324_gb300 import workloads
    return {"mid": workloads.mid, "paper_shaped": workloads.paper_shaped, "contours": workloads.contours}[name]()


def workload_config(args, p):
    config = {"workload": WORKLOAD_NAMES[args.workload], "points": p.n, "segments": p.m, "B": args.B,
              "l2": L2_NOTE}
    if args.max_len > 0:
        config["max_len"] = args.max_len
    for k in ("cand_cap", "cand_block", "graph_iters"):
        if getattr(args, k):
            config[k] = getattr(args, k)
    return config


def cpu_baseline(p, B, reps=1, max_len=0.0, name="paper_shaped"):
    """the oracle as it stands: CDT + sequential Ruppert on the host, one thread"""
    from oracle import oracle
    oracle.build()
    t0 = time.perf_counter()
    steiner = 0
    for _ in range(reps):
        m = oracle.Mesh(p.xy, p.seg)
        assert m.refine_len(B, max_len) == 0
        steiner += m.n_steiner
    dt = time.perf_counter() - t0
    return {"value": steiner / dt, "unit": "Steiner pts/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} full run(s) of the {name} workload (CDT + refine, {steiner // reps} "
                      f"Steiner points each), {dt:.2f} s"}


def replica_totals(ms, steiner, world, device):
    """Replicas (one independent mesh per rank, no data-path collective): the
    job's time is the slowest rank's, its work the sum over ranks."""
    if world <= 1:
        return float(ms), float(steiner)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([float(steiner)], dtype=torch.float64, device=device)
    dist.all_reduce(s)
    return float(t.item()), float(s.item())


def run_reference(args):
    """The oracle (the sequential CPU program the GPU path is checked against)
    timed on the host: every step is a bounded sample of the workload, the
    same recipe at a quarter of its size, so that K + W steps take minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2007_00324_gb300 import workloads
    from oracle import oracle
    oracle.build()
    if args.workload == "paper_shaped":
        p = workloads.paper_shaped(**REF_SAMPLE)
        sample = (f"paper-shaped recipe at a quarter of the size ({p.n:,} points, {p.m:,} segments incl. "
                  f"{p.meta['fans']} fans), one full CDT + refine per step")
    else:
        p = load_workload(args.workload)
        sample = f"one full run of the {args.workload} workload per step"
    for _ in range(args.warmup):
        m = oracle.Mesh(p.xy, p.seg)
        m.refine_len(args.B, args.max_len)
    times, steiner = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        m = oracle.Mesh(p.xy, p.seg)
        assert m.refine_len(args.B, args.max_len) == 0
        times.append(time.perf_counter() - t0)
        steiner += m.n_steiner
    tot = sum(times)
    v = steiner / tot
    config = workload_config(args, load_workload(args.workload))   # the GPU arm's config
    line = {"metric": f"Steiner points inserted per second (CDT + refine, {args.workload} workload)",
            "value": v, "unit": "Steiner pts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "Steiner pts/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "Steiner pts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_measure_step(args):
    """exactly one CDT + refine of the workload (the ncu counter captures run
    this), then its work counters"""
    import torch
    from paper_2007_00324_gb300 import gdp
    gdp.load()
    p = load_workload(args.workload)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    m = gdp.Mesh(p.xy, p.seg, stream=stream)
    s = m.refine(args.B, **refine_kwargs(args))
    keys = ("n_steiner", "iterations", "candidates", "setups", "grown", "cavity_tris", "cavity_edges",
            "walk_steps")
    print(json.dumps({"workload": args.workload, "source_hash": grow_source_hash(),
                      **{k: s[k] for k in keys}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched", "served"):
        line = (run_batched if args.workload == "batched" else run_served)(args)
        print(json.dumps(line), flush=True)
        return
    if args.measure_step:
        return run_measure_step(args)
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2007_00324_gb300 import gdp
    gdp.load()
    p = load_workload(args.workload)
    config = workload_config(args, p)
    stream = torch.cuda.current_stream(dev)
    xy_d = torch.from_numpy(p.xy).to(dev)
    seg_d = torch.from_numpy(p.seg).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(flags=0):
        m = gdp.Mesh(xy_d, seg_d, stream=stream, device=True)
        s = m.refine(args.B, flags=flags, **refine_kwargs(args))
        return m, s

    clk = ClockSampler(local).__enter__()   # started early: see ClockSampler
    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clk.wait_first()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # the timed steps: nothing instrumented
    times, steiner, launches = [], 0, 0
    stats = None
    barrier()
    t_lo = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)              # L2 flush, outside the timed region
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m, stats = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        steiner += stats["n_steiner"]
        launches += stats["launches"]
        del m
    barrier()
    t_hi = time.perf_counter()
    clk.__exit__()
    clocks = clk.summary(t_lo, t_hi)
    tot_ms, steiner_all = replica_totals(sum(times), steiner, world, dev)
    value = steiner_all / (tot_ms / 1000.0)

    # end to end through the C ABI with pinned host buffers: the inputs, and
    # the export's destination (allocated once, sized from the timed steps'
    # counts with a margin, outside the timed region)
    xy_h = torch.from_numpy(p.xy).pin_memory()
    seg_h = torch.from_numpy(p.seg).pin_memory()
    room = 1.25
    out_h = (torch.empty((int(room * (p.n + stats["n_steiner"] + 16)), 2), dtype=torch.float64).pin_memory().numpy(),
             torch.empty((int(room * stats["n_tris"]) + 64, 3), dtype=torch.int32).pin_memory().numpy(),
             torch.empty((int(room * stats["n_subsegs"]) + 64, 3), dtype=torch.int32).pin_memory().numpy())
    e2e_ms, e2e_steiner, d2h = [], 0, 0
    for k in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = gdp.Mesh(xy_h.numpy(), seg_h.numpy(), stream=stream)
        s2 = m.refine(args.B, **refine_kwargs(args))
        xy_o, tri_o, sub_o = m.export(out=out_h)
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_steiner += s2["n_steiner"]
        d2h = xy_o.nbytes + tri_o.nbytes + sub_o.nbytes
        del m
    e2e = {"value": e2e_steiner / (sum(e2e_ms) / 1000.0), "unit": "Steiner pts/s",
           "h2d_bytes_per_step": int(p.xy.nbytes + p.seg.nbytes), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": sum(e2e_ms) / len(e2e_ms)}

    # roofline of the cavity growth, from separate instrumented steps: the
    # growth launch pair of the first iteration of every graph replay is
    # bracketed by CUDA events inside the graph (the events stall the graph,
    # which is why the timed steps above run without them)
    grow = {"grow_ms": 0.0, "grow_launches": 0, "timed_grown": 0, "timed_walk_steps": 0,
            "timed_cavity_tris": 0, "timed_cavity_edges": 0, "timed_setups": 0}
    for _ in range(max(1, args.roof_steps)):
        flush.fill_(1.0)
        m, rs = step(gdp.REFINE_TIME_GROW)
        for k in grow:
            grow[k] += rs[k]
        del m

    # per-kernel device times of one more step, every launch bracketed by events
    os.environ["GDP_PROFILE"] = "1"
    flush.fill_(1.0)
    m, ps = step()
    kt = m.kernel_times()
    del os.environ["GDP_PROFILE"]
    del m
    # the same step with Flip-Flop insertion (Sec. 4.3), for the A/B against cavity insertion
    ff_ms, ff, ff_err = [], None, None
    for _ in range(2):
        flush.fill_(1.0)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        try:
            m, ff = step(gdp.REFINE_FLIPFLOP)
        except gdp.GdpError as e:   # reported in the line, never fatal to it
            ff_err = str(e)
            break
        f1.record(stream)
        f1.synchronize()
        ff_ms.append(f0.elapsed_time(f1))
        del m
    if ff_err:
        flipflop = {"error": ff_err}
    else:
        flipflop = {"value": ff["n_steiner"] / (min(ff_ms) / 1000.0), "unit": "Steiner pts/s",
                    "ms_per_step": min(ff_ms), "refine_ms": ff["refine_ms"], "steiner_per_step": ff["n_steiner"],
                    "iterations": ff["iterations"], "inserted": ff["inserted"], "flips": ff["flips"],
                    "flops": ff["flops"], "redundant_removed": ff["redundant_removed"],
                    "note": "the same step with GDP_REFINE_FLIPFLOP (host-driven passes, no CUDA graph); "
                            "best of 2 steps"}
    tot_k = sum(v[0] for v in kt.values())
    top = max(kt.items(), key=lambda kv: kv[1][0])
    peak, peak_kind = peaks()
    fp64_peak = gdp.measure_fp64_peak(stream)
    n_l = max(grow["grow_launches"], 1)
    timed = {k[len("timed_"):]: v for k, v in grow.items() if k.startswith("timed_")}
    by = grow_bytes(timed)
    sec = grow["grow_ms"] / 1000.0
    gbs = by / sec / 1e9 if sec > 0 else None
    cnt = measured_counters()
    per_launch = timed["grown"] / n_l
    traffic = cnt["dram_bytes_per_grown"] * per_launch if "dram_bytes_per_grown" in cnt else None
    fp64 = {"peak": fp64_peak, "unit": "TFLOP/s", "peak_source": "measured (gdp_measure_fp64_peak)"}
    if "fp64_flops_per_grown" in cnt and sec > 0:
        a = cnt["fp64_flops_per_grown"] * timed["grown"] / sec / 1e12
        fp64.update({"achieved": a, "frac": a / fp64_peak if fp64_peak > 0 else None,
                     "flops_per_grown_candidate": cnt["fp64_flops_per_grown"],
                     "pipe_busy_ncu": cnt.get("fp64_pipe_busy")})
    l2 = None
    if "l2_bytes_per_grown" in cnt and sec > 0:
        l2 = {"bytes_per_launch": cnt["l2_bytes_per_grown"] * per_launch,
              "achieved": cnt["l2_bytes_per_grown"] * timed["grown"] / sec / 1e9, "unit": "GB/s"}
    share = sum(kt.get(k, (0.0, 0))[0] for k in GROW_KERNELS)
    grow_names = " + ".join(k for k in GROW_KERNELS if k in kt) or "k_grow_w<0>"
    roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": (gbs / peak) if gbs else None, "traffic": traffic,
            "kernel": f"cavity growth: {grow_names}", "algorithmic_bytes_per_launch": by / n_l,
            "kernel_ms_per_launch": grow["grow_ms"] / n_l, "launches": grow["grow_launches"],
            "grown_candidates_per_launch": per_launch,
            "setup_candidates_per_launch": timed["setups"] / n_l,
            "share_of_kernel_time": share / tot_k,
            "share_of_refine_kernel_time": share / max(sum(kt.get(k, (0.0, 0))[0] for k in REFINE_KERNELS), 1e-9),
            "largest_kernel": top[0],
            "peak_source": "measured (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "timed_launches": f"the first iteration of every graph replay, {args.roof_steps} instrumented steps",
            "mean_cavity_tris": timed["cavity_tris"] / max(timed["grown"], 1),
            "mean_walk_steps": timed["walk_steps"] / max(timed["setups"], 1),
            "fp64": fp64, "l2": l2}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {"metric": f"Steiner points inserted per second (CDT + refine, {args.workload} workload)",
            "value": value, "unit": "Steiner pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config, parallelism=f"replicas x{world}"),
            "refine_ms": stats["refine_ms"], "cdt_ms": stats["cdt_ms"],
            "steiner_per_step": stats["n_steiner"], "iterations": stats["iterations"],
            "cdt_rounds": stats["cdt_rounds"],
            "refine_only_steiner_per_s": stats["n_steiner"] / (stats["refine_ms"] / 1000.0),
            "work_per_step": {"candidates": stats["candidates"], "set_up": stats["setups"],
                              "grown": stats["grown"], "inserted": stats["inserted"]},
            "gpu_launches": launches, "e2e": e2e, "roofline": roof, "clocks": clocks,
            "step_ms": [round(t, 3) for t in times],
            "flipflop": flipflop,
            "kernels_ms": {k: round(v[0], 4) for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.B, 1 if args.workload == "paper_shaped" else 3,
                                            args.max_len, args.workload)
    if args.workload == "paper_shaped" and world == 1 and not args.no_systems:
        torch.cuda.empty_cache()
        line.update(systems_summary(args))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
