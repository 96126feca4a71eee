"""Pins for the oracle's CDT (Sec. 4 definition; the first step of Algorithm 1)."""
import math
import random

import numpy as np
import pytest

from tests import exact_ref as X

SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
BOUNDARY = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)


def pslg(n, segs=(), seed=0):
    rng = np.random.default_rng(seed)
    pts = 0.02 + 0.96 * rng.random((n, 2))
    xy = np.concatenate([SQUARE, pts])
    seg = np.concatenate([BOUNDARY, np.asarray(segs, np.int32).reshape(-1, 2)])
    return xy, seg


def brute_cdt_check(xy, tri, sub):
    """independent exact check (fractions): CCW triangles, and no vertex
    visible from a triangle's interior inside its circumcircle (SoS)"""
    subs = [(int(u), int(v)) for u, v, _ in sub]

    def crosses(g, w, p, q):
        o1 = X.sign(X.orient(g, w, p)) * X.sign(X.orient(g, w, q))
        o2 = X.sign(X.orient(p, q, g)) * X.sign(X.orient(p, q, w))
        return o1 < 0 and o2 < 0

    used = set(int(i) for i in tri.ravel())
    for t in tri:
        a, b, c = (tuple(xy[i]) for i in t)
        assert X.orient(a, b, c) > 0
        g = ((a[0] + b[0] + c[0]) / 3, (a[1] + b[1] + c[1]) / 3)
        for w in used:
            if w in t:
                continue
            p = tuple(xy[w])
            if X.incircle_sos(a, b, c, p) <= 0:
                continue
            assert any(crosses(g, p, tuple(xy[u]), tuple(xy[v])) for u, v in subs), (t, w)


def test_empty_square_two_triangles(oracle):
    m = oracle.Mesh(SQUARE, BOUNDARY)
    xy, tri, sub = m.export()
    assert len(tri) == 2 and len(sub) == 4
    brute_cdt_check(xy, tri, sub)


def test_square_plus_centre(oracle):
    xy = np.concatenate([SQUARE, [[0.5, 0.5]]])
    m = oracle.Mesh(xy, BOUNDARY)
    xy2, tri, sub = m.export()
    assert len(tri) == 4
    for t in tri:
        assert 4 in t   # every triangle uses the centre: 4 right isosceles triangles
        a, b, c = (xy2[i] for i in t)
        assert abs(0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])) - 0.25) < 1e-15


def test_matches_qhull_without_interior_segments(oracle):
    """With only the square boundary as segments the CDT is the Delaunay
    triangulation of the points; for random points it is unique and Qhull
    computes it independently."""
    from scipy.spatial import Delaunay
    for seed in range(3):
        xy, seg = pslg(300, seed=seed)
        m = oracle.Mesh(xy, seg)
        xy2, tri, sub = m.export()
        mine = oracle.triangle_set(xy2, tri)
        q = Delaunay(xy)
        simp = q.simplices.copy()
        # orient Qhull's simplices CCW
        for k, s in enumerate(simp):
            a, b, c = xy[s]
            if (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]) < 0:
                simp[k] = [s[0], s[2], s[1]]
        theirs = oracle.triangle_set(xy, simp)
        # the 4 corners are cocircular only if no point is inside their circle;
        # with interior points that cannot happen, so the triangulations agree
        assert mine == theirs


def test_euler_and_brute_force_with_segments(oracle):
    rng = random.Random(3)
    for seed in range(4):
        xy, _ = pslg(40, seed=seed)
        n = len(xy)
        # a few non-crossing short segments
        segs = []
        for _ in range(200):
            i, j = rng.randrange(4, n), rng.randrange(4, n)
            if i == j or any(i in s or j in s for s in segs):
                continue
            if math.dist(xy[i], xy[j]) > 0.3:
                continue
            ok = True
            for a, b in segs:
                p, q, r, s = xy[i], xy[j], xy[a], xy[b]
                if X.orient(p, q, r) * X.orient(p, q, s) <= 0 and X.orient(r, s, p) * X.orient(r, s, q) <= 0:
                    ok = False
            if ok:
                segs.append((i, j))
            if len(segs) == 5:
                break
        seg = np.concatenate([BOUNDARY, np.array(segs, np.int32).reshape(-1, 2)])
        m = oracle.Mesh(xy, seg)
        xy2, tri, sub = m.export()
        # Euler for a triangulated square with no extra boundary vertices
        assert len(tri) == 2 * len(xy2) - 4 - 2
        rep = oracle.check(xy2, tri, sub, seg, len(xy), brute=True)
        assert rep["bad_orient"] == 0 and rep["not_locally_cd"] == 0
        assert rep["seg_not_covered"] == 0 and rep["bf_cd_violations"] == 0
        brute_cdt_check(xy2, tri, sub)
        # every input segment is an edge
        edges = {tuple(sorted((int(t[k]), int(t[(k + 1) % 3])))) for t in tri for k in range(3)}
        for a, b in seg:
            assert tuple(sorted((int(a), int(b)))) in edges


def test_invalid_inputs(oracle):
    xy = np.concatenate([SQUARE, [[0.25, 0.5], [0.75, 0.5], [0.5, 0.25], [0.5, 0.75]]])
    crossing = np.concatenate([BOUNDARY, [[4, 5], [6, 7]]])
    with pytest.raises(ValueError):
        oracle.Mesh(xy, crossing)
    dup = np.concatenate([xy, [[0.25, 0.5]]])
    with pytest.raises(ValueError):
        oracle.Mesh(dup, BOUNDARY)
    through = np.concatenate([SQUARE, [[0.25, 0.25], [0.5, 0.5], [0.75, 0.75]]])
    with pytest.raises(ValueError):
        oracle.Mesh(through, np.concatenate([BOUNDARY, [[4, 6]]]))
    with pytest.raises(ValueError):
        oracle.Mesh(xy, np.concatenate([BOUNDARY, [[0, 99]]]))


def test_tiny_config_cdt(oracle):
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    m = oracle.Mesh(p.xy, p.seg)
    xy, tri, sub = m.export()
    assert len(tri) == 2 * len(xy) - 6
    rep = oracle.check(xy, tri, sub, p.seg, p.n, brute=True)
    for k in ("bad_orient", "bad_adjacency", "open_not_sub", "sub_not_edge", "seg_not_covered",
              "not_locally_cd", "bf_cd_violations", "euler_defect", "inputs_missing"):
        assert rep[k] == 0, k
    assert abs(rep["area_sum"] - 1.0) < 1e-12
