"""Small input angles on the GPU (Sec. 4.1: bad triangles next to input angles
below 60 degrees are unavoidable and accepted), element by element against the
oracle's pinned rules:

* concentric-shell split points (C6): subsegments at fan apexes are split on
  both sides in the same fixed batches; the triangulations, and so every
  split point's coordinates, must be identical;
* the exemption (C10) and the bad-triangle test (C1): on a mesh with many
  triangles at fan apexes, the GPU's scan must flag as bad exactly the
  triangles the oracle flags, and accept as exempt exactly the ones the
  oracle's rule accepts.
"""
import math

import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fans():
    from paper_2007_00324_gb300 import workloads as W
    p = W.paper_shaped(n_uniform=3000, n_gauss=1500, n_circle=1000, n_seg=60, n_fans=6, seed=4711)
    assert p.meta["fans"] == 6
    return p


def apexes(p):
    """input vertices where two segments meet below 60 degrees (cos > 1/2)"""
    inc = {}
    for s, (a, b) in enumerate(p.seg.tolist()):
        inc.setdefault(a, []).append(b)
        inc.setdefault(b, []).append(a)
    out = set()
    for o, ends in inc.items():
        for i in range(len(ends)):
            for j in range(i + 1, len(ends)):
                u, w = p.xy[ends[i]] - p.xy[o], p.xy[ends[j]] - p.xy[o]
                if np.dot(u, w) > 0.5 * np.linalg.norm(u) * np.linalg.norm(w):
                    out.add(o)
    return out


def apex_subsegments(xy, sub, apx):
    """endpoint coordinates of the subsegments with exactly one end at an apex"""
    rows = [(a, b) for a, b, _ in sub.tolist() if (a in apx) != (b in apx)]
    return np.array([[*xy[a], *xy[b]] for a, b in rows], np.float64)


def scan_sets(xy, kind, verts):
    def canon(t):
        pts = [tuple(xy[i].tolist()) for i in t]
        k = min(range(3), key=lambda i: pts[i])
        return (pts[k], pts[(k + 1) % 3], pts[(k + 2) % 3])
    bad = {canon(verts[k]) for k in range(len(kind)) if kind[k] == 0}
    ex = {canon(verts[k]) for k in range(len(kind)) if kind[k] == 2}
    return bad, ex


def oracle_sets(oracle, xy, tri, sub, p, B):
    def canon(t):
        pts = [tuple(xy[i].tolist()) for i in t]
        k = min(range(3), key=lambda i: pts[i])
        return (pts[k], pts[(k + 1) % 3], pts[(k + 2) % 3])
    bad, _, _ = oracle.eval_tris(xy, tri, B * B)
    ex = oracle.eval_exempt(xy, tri, sub, p.seg, p.n, B * B)
    return ({canon(tri[i]) for i in np.nonzero(bad & (ex == 0))[0]},
            {canon(tri[i]) for i in np.nonzero(ex)[0]})


def test_shell_splits_match_oracle(oracle, fans):
    gdp = need_gpu()
    p = fans
    apx = apexes(p)
    assert len(apx) == 6
    g = gdp.Mesh(p.xy, p.seg)
    o = oracle.Mesh(p.xy, p.seg)
    for rnd in range(3):   # each round splits the apex-adjacent halves again (shells)
        oxy, _, osub = o.export()
        abxy = apex_subsegments(oxy, osub, apx)
        assert len(abxy) >= 6 * 8
        g.split_subsegments(abxy)
        assert o.split_subsegments(abxy) == 0
        gxy, gtri, gsub = g.export()
        oxy, otri, osub = o.export()
        assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri), rnd
        assert_valid(oracle.check(gxy, gtri, gsub, p.seg, p.n), refined=False)
    # the new vertices next to the apexes sit on shells: a power of two from the apex
    dist = set()
    for a, b, _ in gsub.tolist():
        for u, v in ((a, b), (b, a)):
            if u in apx and v >= p.n:
                dist.add(float(np.hypot(*(gxy[v] - gxy[u]))))
    assert dist and all(abs(math.log2(d) - round(math.log2(d))) < 1e-12 for d in dist), sorted(dist)


@pytest.mark.parametrize("B", [SQ2, 1.5])
def test_bad_and_exempt_match_oracle_before_refinement(oracle, fans, B):
    """the CDT after shell splits has many bad triangles at the fans"""
    gdp = need_gpu()
    p = fans
    apx = apexes(p)
    g = gdp.Mesh(p.xy, p.seg)
    o = oracle.Mesh(p.xy, p.seg)
    for _ in range(2):
        oxy, _, osub = o.export()
        abxy = apex_subsegments(oxy, osub, apx)
        g.split_subsegments(abxy)
        assert o.split_subsegments(abxy) == 0
    xy, tri, sub = g.export()
    kind, verts, _, _ = g.scan(B)
    got_bad, got_ex = scan_sets(xy, kind, verts)
    want_bad, want_ex = oracle_sets(oracle, xy, tri, sub, p, B)
    assert len(want_ex) >= 6 and len(want_bad) > 100
    assert got_ex == want_ex
    assert got_bad == want_bad


def test_bad_and_exempt_match_oracle_after_refinement(oracle, fans):
    gdp = need_gpu()
    p = fans
    g = gdp.Mesh(p.xy, p.seg)
    g.refine(SQ2)
    xy, tri, sub = g.export()
    assert_valid(oracle.check(xy, tri, sub, p.seg, p.n, B=SQ2))
    kind, verts, _, _ = g.scan(SQ2)
    got_bad, got_ex = scan_sets(xy, kind, verts)
    want_bad, want_ex = oracle_sets(oracle, xy, tri, sub, p, SQ2)
    assert not want_bad and not got_bad
    assert want_ex and got_ex == want_ex
