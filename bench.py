#!/usr/bin/env python
"""Benchmark of the gDP2d hot path on GB300: Steiner points inserted per second.

One step = the whole hot path on one synthetic PSLG: the GPU CDT (Algorithm 1
line 1) and the refinement loop (lines 2-9) of the mid workload
(unit square + 100,000 uniform points + 1,000 random segments, B = sqrt 2).

  value   Steiner points / (CDT + refine) device time, inputs resident in HBM
  e2e     the same through the C ABI with host buffers: create (H2D inside),
          refine and export (D2H) all in the timed region
  roofline  dominant kernel: algorithmic bytes / average launch time vs HBM peak
  cpu_baseline  the sequential C oracle on the machine's host cores

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
CONFIG = {"workload": "mid: unit square + 100,000 uniform FP64 points + 1,000 random "
                      "segments, B=sqrt(2)", "points": 100_004, "segments": 1_004, "B": SQ2,
          "l2": "flushed between steps (512 MB write)"}

# Algorithmic bytes of the dominant kernel, k_grow<0> (cavity growth of the
# refinement, Sec. 5.2): what each grown candidate must read and write once,
# from the device layout (triangle T/N 16 B each, vertex 16 B FP64 + 8 B FP32
# copy, marks 8 B), with the work counters the library reports:
#   per candidate  134 = element id 4 + element triangle 16 + its 3 vertices 48
#                        + candidate record written 66
#   per walk step   56 = T 16 + N 16 + one new vertex 24
#   per cavity tri  84 = T + N 32 + neighbour test (T 16 + apex 24) + list 4 + mark 8
#   per boundary edge 56 = neighbour test 40 + boundary record 16
GROW_BYTES = {"candidate": 134, "walk_step": 56, "cavity_tri": 84, "boundary_edge": 56}
GROW_SOURCES = ("gdp_core.cuh", "gdp_pred.cuh", "gdp_kernels.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_grow0_mid_traffic.md")


def grow_bytes(st) -> float:
    return (GROW_BYTES["candidate"] * st["grown"] + GROW_BYTES["walk_step"] * st["walk_steps"] +
            GROW_BYTES["cavity_tri"] * st["cavity_tris"] + GROW_BYTES["boundary_edge"] * st["cavity_edges"])


def grow_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in GROW_SOURCES:
        with open(os.path.join(ROOT, "paper_2007_00324_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic():
    """DRAM bytes per k_grow<0> launch from the committed ncu summary, or None
    when the kernel's sources changed since it was captured."""
    try:
        with open(TRAFFIC_FILE) as f:
            kv = dict(line.split(":", 1) for line in f
                      if line.startswith(("source-hash:", "dram-bytes-per-launch:")))
        if kv["source-hash"].strip() != grow_source_hash():
            return None
        return float(kv["dram-bytes-per-launch"])
    except Exception:
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdp", choices=["gdp", "reference"])
    ap.add_argument("--B", type=float, default=SQ2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region"""

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
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def cpu_baseline(p, B, reps=3):
    """the oracle as it stands: CDT + sequential Ruppert on the host, one thread"""
    from oracle import oracle
    oracle.build()
    t0 = time.perf_counter()
    steiner = 0
    for _ in range(reps):
        m = oracle.Mesh(p.xy, p.seg)
        assert m.refine(B) == 0
        steiner += m.n_steiner
    dt = time.perf_counter() - t0
    return {"value": steiner / dt, "unit": "Steiner pts/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} full runs of the mid workload (CDT + refine, {steiner // reps} "
                      f"Steiner points each), {dt:.2f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2007_00324_gb300 import workloads
    from oracle import oracle
    oracle.build()
    p = workloads.mid()
    for _ in range(args.warmup):
        m = oracle.Mesh(p.xy, p.seg)
        m.refine(args.B)
    times, steiner = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        m = oracle.Mesh(p.xy, p.seg)
        assert m.refine(args.B) == 0
        times.append(time.perf_counter() - t0)
        steiner += m.n_steiner
    tot = sum(times)
    v = steiner / tot
    line = {"metric": "Steiner points inserted per second (CDT + refine, mid workload)",
            "value": v, "unit": "Steiner pts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "Steiner pts/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full runs of the mid workload"},
            "e2e": {"value": v, "unit": "Steiner pts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2007_00324_gb300 import gdp, workloads
    gdp.load()
    p = workloads.mid()
    stream = torch.cuda.current_stream(dev)
    xy_d = torch.from_numpy(p.xy).to(dev)
    seg_d = torch.from_numpy(p.seg).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        m = gdp.Mesh(xy_d, seg_d, stream=stream, device=True)
        s = m.refine(args.B, flags=gdp.REFINE_TIME_GROW)
        return m, s

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    times, steiner, launches = [], 0, 0
    stats = None
    grow = {"grow_ms": 0.0, "grow_launches": 0, "grown": 0, "walk_steps": 0, "cavity_tris": 0,
            "cavity_edges": 0}
    barrier()
    with ClockSampler(local) as clk:
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
            for k in grow:
                grow[k] += stats[k]
            del m
        barrier()
    tot_ms = sum(times)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        s = torch.tensor([float(steiner)], device=dev)
        dist.all_reduce(s)
        steiner_all = float(s.item())
    else:
        steiner_all = float(steiner)
    value = steiner_all / (tot_ms / 1000.0)

    # end to end through the C ABI with pinned host buffers
    xy_h = torch.from_numpy(p.xy).pin_memory()
    seg_h = torch.from_numpy(p.seg).pin_memory()
    e2e_ms, e2e_steiner, d2h = [], 0, 0
    for k in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = gdp.Mesh(xy_h.numpy(), seg_h.numpy(), stream=stream)
        s2 = m.refine(args.B)
        xy_o, tri_o, sub_o = m.export()
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_steiner += s2["n_steiner"]
        d2h = xy_o.nbytes + tri_o.nbytes + sub_o.nbytes
        del m
    e2e = {"value": e2e_steiner / (sum(e2e_ms) / 1000.0), "unit": "Steiner pts/s",
           "h2d_bytes_per_step": int(p.xy.nbytes + p.seg.nbytes), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": sum(e2e_ms) / len(e2e_ms)}

    # per-kernel device times of one more step, every launch bracketed by events
    os.environ["GDP_PROFILE"] = "1"
    flush.fill_(1.0)
    m, ps = step()
    kt = m.kernel_times()
    del os.environ["GDP_PROFILE"]
    del m
    tot_k = sum(v[0] for v in kt.values())
    top = max(kt.items(), key=lambda kv: kv[1][0])
    peak, peak_kind = peaks()
    # roofline of k_grow<0> over the timed steps: algorithmic bytes from the
    # work counters / device time from the events recorded around each launch
    n_l = max(grow["grow_launches"], 1)
    by = grow_bytes(grow)
    gbs = by / (grow["grow_ms"] / 1000.0) / 1e9 if grow["grow_ms"] > 0 else None
    tr = measured_traffic()
    roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": (gbs / peak) if gbs else None, "traffic": tr,
            "kernel": "k_grow<0>", "algorithmic_bytes_per_launch": by / n_l,
            "kernel_ms_per_launch": grow["grow_ms"] / n_l, "launches": grow["grow_launches"],
            "share_of_kernel_time": kt.get("k_grow<0>", (0.0, 0))[0] / tot_k,
            "largest_kernel": top[0],
            "peak_source": "measured (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "mean_cavity_tris": grow["cavity_tris"] / max(grow["grown"], 1),
            "mean_boundary_edges": grow["cavity_edges"] / max(grow["grown"], 1),
            "mean_walk_steps": grow["walk_steps"] / max(grow["grown"], 1)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {"metric": "Steiner points inserted per second (CDT + refine, mid workload)",
            "value": value, "unit": "Steiner pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(CONFIG, parallelism=f"replicas x{world}"),
            "refine_ms": stats["refine_ms"], "cdt_ms": stats["cdt_ms"],
            "steiner_per_step": stats["n_steiner"], "iterations": stats["iterations"],
            "cdt_rounds": stats["cdt_rounds"],
            "refine_only_steiner_per_s": stats["n_steiner"] / (stats["refine_ms"] / 1000.0),
            "gpu_launches": launches, "e2e": e2e, "roofline": roof, "clocks": clk.summary(),
            "kernels_ms": {k: round(v[0], 4) for k, v in sorted(kt.items(), key=lambda kv: -kv[1][0])}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.B)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
