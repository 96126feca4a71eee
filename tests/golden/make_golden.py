"""Writes tests/golden/oracle_counts.json: the sequential oracle's Steiner
counts (and output sizes) for the seeded workloads, so that GPU tests at full
size compare against them without rerunning the oracle.  Calls only oracle/
and the input generators.

    python tests/golden/make_golden.py
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_2007_00324_gb300 import workloads  # noqa: E402


def main():
    out = {}
    cases = [("tiny", workloads.tiny, math.sqrt(2)), ("tiny", workloads.tiny, 1.5),
             ("mid", workloads.mid, math.sqrt(2)), ("mid", workloads.mid, 1.5),
             ("paper_shaped", workloads.paper_shaped, math.sqrt(2))]
    cache = {}
    for name, gen, B in cases:
        if name not in cache:
            cache[name] = gen()
        p = cache[name]
        t0 = time.time()
        m = oracle.Mesh(p.xy, p.seg)
        xy, tri, _ = m.export()
        n_cdt_tri = len(tri)
        st = m.refine(B)
        xy, tri, sub = m.export()
        out[f"{name}/B={B:.6f}"] = {"status": st, "n_in": p.n, "n_seg": p.m, "cdt_triangles": n_cdt_tri,
                                    "steiner": m.n_steiner, "triangles": len(tri),
                                    "subsegments": len(sub), "seconds": round(time.time() - t0, 2)}
        print(name, B, out[f"{name}/B={B:.6f}"], flush=True)
    with open(os.path.join(HERE, "oracle_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
