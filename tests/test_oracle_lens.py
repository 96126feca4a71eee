"""Pins for the oracle's diametral-lens encroachment (Chew's rule, Sec. 4.2).

Reading: a point encroaches a subsegment under Chew's rule when it lies
strictly inside the diametral lens, the region from which the subsegment
subtends an angle above 120 degrees.  The pins below come from the geometry,
not from the oracle's formula: the lens apex on the bisector, angles measured
with atan2 away from the boundary, containment in the diametral circle, exact
symmetries, and a hand-worked mesh where the two rules differ."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O


def test_bisector_closed_form():
    # a = (-1, 0), b = (1, 0): the lens meets the bisector at height
    # tan(30 deg) = 1/sqrt(3), so (0, h) is inside iff h^2 < 1/3
    a, b = (-1.0, 0.0), (1.0, 0.0)
    hs = [0.0, 0.1, 0.5, 0.57, 0.5773, 0.57735, 0.577350269, 0.5773502691896257,
          0.5773502691896258, 0.57735027, 0.578, 0.6, 1.0, 10.0]
    for h in hs:
        for sgn in (1.0, -1.0):
            inside = Fraction(h) ** 2 < Fraction(1, 3)
            assert O.lens_sign(a, b, (0.0, sgn * h)) == (-1 if inside else 1), h


def test_endpoints_and_midpoint():
    a, b = (0.25, -3.0), (7.5, 2.0)
    assert O.lens_sign(a, b, a) == 0
    assert O.lens_sign(a, b, b) == 0
    mid = ((a[0] + b[0]) / 2, (a[1] + b[1]) / 2)
    assert O.lens_sign(a, b, mid) == -1
    # beyond an endpoint on the segment's line: angle 0
    assert O.lens_sign(a, b, (2 * b[0] - a[0], 2 * b[1] - a[1])) == 1


def test_angle_against_atan2():
    rng = np.random.default_rng(20070324)
    checked = 0
    for _ in range(4000):
        a = tuple(rng.uniform(-1, 1, 2))
        b = tuple(rng.uniform(-1, 1, 2))
        p = tuple(rng.uniform(-1, 1, 2))
        ux, uy = a[0] - p[0], a[1] - p[1]
        wx, wy = b[0] - p[0], b[1] - p[1]
        ang = abs(math.atan2(ux * wy - uy * wx, ux * wx + uy * wy))
        if abs(ang - 2 * math.pi / 3) < 1e-6:
            continue
        assert O.lens_sign(a, b, p) == (-1 if ang > 2 * math.pi / 3 else 1)
        checked += 1
    assert checked > 3900


def test_lens_inside_diametral_circle():
    # the lens is a subset of the diametral circle: inside the lens implies
    # encroachment under Ruppert's rule; the two differ between 90 and 120 deg
    rng = np.random.default_rng(7)
    n_lens = n_circle_only = 0
    for _ in range(4000):
        a = tuple(rng.uniform(0, 1, 2))
        b = tuple(rng.uniform(0, 1, 2))
        p = tuple(rng.uniform(0, 1, 2))
        lz, dz = O.lens_sign(a, b, p), O.dot_sign(a, b, p)
        if lz < 0:
            assert dz < 0
            n_lens += 1
        elif dz < 0:
            n_circle_only += 1
    assert n_lens > 50 and n_circle_only > 50


def test_symmetries_exact():
    # swapping the endpoints, reflecting in an axis and rotating by 90 degrees
    # are exact in binary64 and leave the answer unchanged, near the boundary too
    rng = np.random.default_rng(11)
    base = [((-1.0, 0.0), (1.0, 0.0), (0.0, h)) for h in
            (0.5773502691896257, 0.5773502691896258, 0.57735026918962573)]
    for _ in range(300):
        base.append(tuple(tuple(rng.uniform(-4, 4, 2)) for _ in range(3)))
    for a, b, p in base:
        s = O.lens_sign(a, b, p)
        assert O.lens_sign(b, a, p) == s
        ref = lambda q: (q[0], -q[1])
        assert O.lens_sign(ref(a), ref(b), ref(p)) == s
        rot = lambda q: (-q[1], q[0])
        assert O.lens_sign(rot(a), rot(b), rot(p)) == s


def test_filter_agrees_with_exact():
    # the floating-point filter never changes an answer of the exact path
    rng = np.random.default_rng(3)
    pts = [tuple(rng.uniform(-1, 1, 2)) for _ in range(600)]
    # points on the upper arc of the lens of (-1, 0)-(1, 0), rounded to binary64:
    # the circle through both ends centred at (0, -1/sqrt 3)
    r = 2 / math.sqrt(3)
    near = [((-1.0, 0.0), (1.0, 0.0), (x, -1 / math.sqrt(3) + math.sqrt(r * r - x * x)))
            for x in np.linspace(-0.95, 0.95, 77)]
    cases = [(pts[i], pts[i + 1], pts[i + 2]) for i in range(0, 597, 3)] + near
    want = [O.lens_sign(a, b, p) for a, b, p in cases]
    O.set_filter(False)
    try:
        got = [O.lens_sign(a, b, p) for a, b, p in cases]
    finally:
        O.set_filter(True)
    assert got == want


SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
BOUNDARY = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)


@pytest.mark.parametrize("h, circle, lens", [(0.35, 1, 0), (0.2, 1, 1), (0.5, 0, 0), (0.7, 1, 0)])
def test_rules_differ_on_one_mesh(h, circle, lens):
    # the square plus one point (0.5, h); its CDT has four triangles, each side's
    # apex being that point.  It sees the bottom side at 2 atan(0.5 / h): 110 deg
    # at h = 0.35 (circle only), 136 deg at h = 0.2 (both); the top side at
    # 2 atan(0.5 / (1 - h)): 118 deg at h = 0.7 (circle only); the left and right
    # sides at atan(2 h) + atan(2 (1 - h)), below 90 deg here.  At h = 0.5 it lies
    # on all four diametral circles (dot product exactly 0): neither rule
    xy = np.vstack([SQUARE, [[0.5, h]]])
    m = O.Mesh(xy, BOUNDARY)
    gxy, tri, sub = m.export()
    rc = O.check(gxy, tri, sub, BOUNDARY, len(xy))
    rl = O.check(gxy, tri, sub, BOUNDARY, len(xy), lens=True)
    assert rc["encroached"] == circle
    assert rl["encroached"] == lens
    # the scan helper (per subsegment) agrees with the checker's count
    assert int(O.eval_subs(gxy, tri, sub)[0].sum()) == circle
    assert int(O.eval_subs(gxy, tri, sub, lens=True)[0].sum()) == lens


@pytest.mark.parametrize("lens", [False, True])
def test_refine_mode_invariants(lens):
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    m = O.Mesh(p.xy, p.seg)
    assert m.refine_mode(math.sqrt(2), lens=lens) == 0
    xy, tri, sub = m.export()
    rep = O.check(xy, tri, sub, p.seg, p.n, B=math.sqrt(2), brute=True, lens=lens)
    for k in ("bad_orient", "bad_adjacency", "open_not_sub", "sub_not_edge", "seg_not_covered",
              "not_locally_cd", "bf_cd_violations", "bad_quality", "encroached", "euler_defect",
              "inputs_missing"):
        assert rep[k] == 0, (k, rep)


def test_lens_mode_splits_fewer_subsegments():
    # fewer points encroach under the lens: on the same input the lens mode ends
    # with no more subsegments than the circle mode (a property of these inputs,
    # checked on three of them, not a theorem)
    from paper_2007_00324_gb300 import workloads as W
    for p in (W.tiny(), W.square_pslg(3000, 60, 5), W.square_pslg(3000, 60, 6)):
        subs = []
        for lens in (False, True):
            m = O.Mesh(p.xy, p.seg)
            assert m.refine_mode(math.sqrt(2), lens=lens) == 0
            xy, tri, sub = m.export()
            subs.append(len(sub))
        assert subs[1] <= subs[0], subs
