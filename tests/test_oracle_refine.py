"""Pins for the oracle's refinement (Algorithm 1 run sequentially: Ruppert's
algorithm with the paper's rules, Sec. 4.1-4.3)."""
import math

import numpy as np
import pytest

from tests import exact_ref as X

SQ2 = math.sqrt(2.0)
SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
BOUNDARY = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)


def min_angles(xy, tri):
    P = xy[tri]                                  # (t, 3, 2)
    out = np.full(len(tri), 180.0)
    for k in range(3):
        a, b, c = P[:, k], P[:, (k + 1) % 3], P[:, (k + 2) % 3]
        u, v = b - a, c - a
        cosang = np.sum(u * v, 1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
        out = np.minimum(out, np.degrees(np.arccos(np.clip(cosang, -1, 1))))
    return out


def encroached_exact(xy, tri, sub):
    """independent: apex of an adjacent triangle strictly inside the
    diametral circle of a subsegment (fractions)"""
    apex = {}
    for t in tri:
        for k in range(3):
            apex[(int(t[k]), int(t[(k + 1) % 3]))] = int(t[(k + 2) % 3])
    n = 0
    for u, v, _ in sub:
        for e in ((u, v), (v, u)):
            w = apex.get((int(e[0]), int(e[1])))
            if w is not None and X.dot(tuple(xy[u]), tuple(xy[v]), tuple(xy[w])) < 0:
                n += 1
    return n


def test_empty_square_needs_no_steiner_points(oracle):
    m = oracle.Mesh(SQUARE, BOUNDARY)
    assert m.refine(SQ2) == 0
    assert m.n_steiner == 0


def test_thin_triangle_gets_refined(oracle):
    xy = np.concatenate([SQUARE, [[0.5, 0.01]]])
    m = oracle.Mesh(xy, BOUNDARY)
    xy0, tri0, _ = m.export()
    assert min_angles(xy0, tri0).min() < 2.0
    assert m.refine(SQ2) == 0
    assert m.n_steiner > 0
    xy1, tri1, sub1 = m.export()
    rep = oracle.check(xy1, tri1, sub1, BOUNDARY, 5, B=SQ2, brute=True)
    assert rep["bad_quality"] == 0 and rep["encroached"] == 0 and rep["bf_cd_violations"] == 0
    # B = sqrt 2 <=> smallest angle >= arcsin(1 / (2 sqrt 2)) = 20.705 deg
    assert min_angles(xy1, tri1).min() >= math.degrees(math.asin(1 / (2 * SQ2))) - 1e-9


@pytest.mark.parametrize("B", [SQ2, 1.5])
def test_tiny_config_refinement_invariants(oracle, B):
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    m = oracle.Mesh(p.xy, p.seg)
    assert m.refine(B) == 0
    xy, tri, sub = m.export()
    rep = oracle.check(xy, tri, sub, p.seg, p.n, B=B, brute=True)
    for k in ("bad_orient", "bad_adjacency", "open_not_sub", "sub_not_edge", "seg_not_covered",
              "not_locally_cd", "bf_cd_violations", "bad_quality", "encroached", "euler_defect",
              "inputs_missing"):
        assert rep[k] == 0, (k, rep[k])
    assert abs(rep["area_sum"] - 1.0) < 1e-12
    assert min_angles(xy, tri).min() >= math.degrees(math.asin(1 / (2 * B))) - 1e-9
    assert encroached_exact(xy, tri, sub) == 0
    # input points keep their ids and coordinates
    assert np.array_equal(xy[:p.n], p.xy)
    assert len(xy) == p.n + m.n_steiner


def test_queue_order_spread_is_small(oracle):
    """sequential Ruppert is order dependent; the spread across queue orders
    bounds what 'within 10%' can mean for a parallel refinement"""
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    counts = []
    for order in (0, 1, 2):
        m = oracle.Mesh(p.xy, p.seg)
        assert m.refine(SQ2, order=order) == 0
        counts.append(m.n_steiner)
    assert max(counts) <= 1.10 * min(counts), counts


def test_small_input_angle_fan_terminates(oracle):
    """segments meeting at 10 degrees: refinement must terminate; the only
    bad triangles left are the exempt ones at the apex (Sec. 4.1)"""
    apex = np.array([[0.5, 0.5]])
    ends = np.array([[0.5 + 0.3 * math.cos(math.radians(a)), 0.5 + 0.3 * math.sin(math.radians(a))]
                     for a in (0, 10, 20)])
    xy = np.concatenate([SQUARE, apex, ends])
    seg = np.concatenate([BOUNDARY, [[4, 5], [4, 6], [4, 7]]])
    m = oracle.Mesh(xy, seg)
    assert m.refine(SQ2, max_steiner=200_000) == 0
    xy1, tri1, sub1 = m.export()
    rep = oracle.check(xy1, tri1, sub1, seg, len(xy), B=SQ2)
    assert rep["bad_quality"] == 0 and rep["encroached"] == 0 and rep["not_locally_cd"] == 0
    assert rep["exempt_bad"] > 0
    assert m.n_steiner < 20_000


def test_step_limit_reports_and_keeps_a_valid_cdt(oracle):
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    m = oracle.Mesh(p.xy, p.seg)
    assert m.refine(SQ2, max_steiner=100) == oracle.LIMIT
    assert m.n_steiner == 100
    xy, tri, sub = m.export()
    rep = oracle.check(xy, tri, sub, p.seg, p.n, brute=True)
    assert rep["bad_orient"] == 0 and rep["not_locally_cd"] == 0 and rep["bf_cd_violations"] == 0


def test_fixed_batch_equals_fresh_cdt(oracle):
    """inserting a batch of free points into a CDT gives the CDT of the
    enlarged point set (uniqueness under simulation of simplicity)"""
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(300, 6, 77)
    rng = np.random.default_rng(5)
    extra = 0.05 + 0.9 * rng.random((200, 2))
    m = oracle.Mesh(p.xy, p.seg)
    assert m.insert_points(extra) == 0
    xy1, tri1, _ = m.export()
    fresh = oracle.Mesh(np.concatenate([p.xy, extra]), p.seg)
    xy2, tri2, _ = fresh.export()
    assert oracle.triangle_set(xy1, tri1) == oracle.triangle_set(xy2, tri2)
