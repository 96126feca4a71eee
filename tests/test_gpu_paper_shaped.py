"""The full-size workload shaped like the paper's synthetic inputs (Section 6:
about a million points in a unit square, one percent as many constraining
segments, plus narrow fans of segments that create small input angles).

The initial CDT is compared with the oracle's triangle for triangle; the
refined mesh is validated by the oracle's checker and its Steiner count is
compared with the oracle's, stored in tests/golden/oracle_counts.json by
tests/golden/make_golden.py (which calls only the oracle)."""
import json
import math
import os

import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_counts.json")


def golden(name, B):
    with open(GOLDEN) as f:
        return json.load(f)[f"{name}/B={B:.6f}"]


@pytest.fixture(scope="module")
def workload():
    from paper_2007_00324_gb300 import workloads as W
    return W.paper_shaped()


def test_paper_shaped_cdt_bit_exact(oracle, workload):
    gdp = need_gpu()
    p = workload
    g = gdp.Mesh(p.xy, p.seg)
    assert all(v == 0 for v in g.check().values()), g.check()
    gxy, gtri, gsub = g.export()
    ref = golden("paper_shaped", SQ2)
    assert len(gtri) == ref["cdt_triangles"]
    o = oracle.Mesh(p.xy, p.seg)
    oxy, otri, osub = o.export()
    assert np.array_equal(gxy, oxy)
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)
    norm = lambda S: sorted((min(a, b), max(a, b), s) for a, b, s in S.tolist())
    assert norm(gsub) == norm(osub)


def test_paper_shaped_refine(oracle, workload):
    gdp = need_gpu()
    p = workload
    ref = golden("paper_shaped", SQ2)
    g = gdp.Mesh(p.xy, p.seg)
    stats = g.refine(SQ2)
    assert all(v == 0 for v in g.check().values()), g.check()
    xy, tri, sub = g.export()
    assert np.array_equal(xy[:p.n], p.xy)
    assert len(xy) == p.n + stats["n_steiner"]
    rep = oracle.check(xy, tri, sub, p.seg, p.n, B=SQ2)
    assert_valid(rep)
    assert math.isclose(rep["area_sum"], 1.0, rel_tol=1e-9)
    n_ref = ref["steiner"]
    assert abs(stats["n_steiner"] - n_ref) <= 0.10 * n_ref, (stats["n_steiner"], n_ref)
