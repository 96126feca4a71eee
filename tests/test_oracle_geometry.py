"""Pins for the oracle's FP64 geometry: the bad-triangle test (radius-edge
ratio, Sec. 4.1 / Sec. 5.1), circumcentre and midpoint (splitting points,
Sec. 4.2) and the priority measure (Sec. 4.3)."""
import math
import random
from fractions import Fraction as F

import pytest

SQ2 = math.sqrt(2.0)


def tri_with_min_angle(deg):
    """isosceles triangle whose two equal angles are `deg`: its smallest angle
    is min(deg, 180 - 2 deg)"""
    t = math.radians(deg)
    return (0.0, 0.0), (1.0, 0.0), (0.5, 0.5 * math.tan(t))


def ratio_closed_form(a, b, c):
    """R / l_min from the law of sines: R = l / (2 sin(opposite angle))"""
    L = [math.dist(b, c), math.dist(a, c), math.dist(a, b)]
    s = 0.5 * sum(L)
    area = math.sqrt(max(s * (s - L[0]) * (s - L[1]) * (s - L[2]), 0.0))
    R = L[0] * L[1] * L[2] / (4 * area)
    return R / min(L)


def test_equilateral_and_right_isosceles(oracle):
    eq = ((0.0, 0.0), (1.0, 0.0), (0.5, math.sqrt(3) / 2))
    assert abs(ratio_closed_form(*eq) - 1 / math.sqrt(3)) < 1e-12
    assert not oracle.is_bad(*eq, 2.0)
    ri = ((0.0, 0.0), (1.0, 0.0), (0.0, 1.0))
    assert abs(ratio_closed_form(*ri) - 1 / SQ2) < 1e-12
    assert not oracle.is_bad(*ri, 2.0)


@pytest.mark.parametrize("deg,B,bad", [
    (20.0, SQ2, True),      # 20 deg < 20.705 deg -> bad at B = sqrt 2
    (21.0, SQ2, False),
    (19.0, 1.5, True),      # 19 deg < 19.47 deg
    (20.0, 1.5, False),
    (1.0, SQ2, True),
    (60.0, 0.5774, True),   # equilateral ratio 0.57735 > 0.5774? no: just below
])
def test_threshold(oracle, deg, B, bad):
    a, b, c = tri_with_min_angle(deg)
    want = ratio_closed_form(a, b, c) > B
    if deg != 60.0:
        assert want == bad
    assert oracle.is_bad(a, b, c, B * B) == want


def test_rotation_and_orientation_invariance(oracle):
    rng = random.Random(7)
    for _ in range(500):
        pts = [(rng.random(), rng.random()) for _ in range(3)]
        if (pts[1][0] - pts[0][0]) * (pts[2][1] - pts[0][1]) - (pts[1][1] - pts[0][1]) * (pts[2][0] - pts[0][0]) < 0:
            pts[1], pts[2] = pts[2], pts[1]
        a, b, c = pts
        r = ratio_closed_form(a, b, c)
        if abs(r - SQ2) < 1e-9:
            continue
        v = oracle.is_bad(a, b, c, 2.0)
        assert v == (r > SQ2)
        # canonical form: every rotation gives the same bits
        assert oracle.is_bad(b, c, a, 2.0) == v and oracle.is_bad(c, a, b, 2.0) == v
        cc = oracle.circumcenter(a, b, c)
        assert oracle.circumcenter(b, c, a) == cc and oracle.circumcenter(c, a, b) == cc


def exact_circumcenter(a, b, c):
    ax, ay, bx, by, cx, cy = map(F, (*a, *b, *c))
    d = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
    return ux, uy


def test_circumcenter_accuracy(oracle):
    rng = random.Random(8)
    for _ in range(300):
        a, b, c = [(rng.random(), rng.random()) for _ in range(3)]
        if (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]) < 0:
            b, c = c, b
        ux, uy = exact_circumcenter(a, b, c)
        x, y = oracle.circumcenter(a, b, c)
        # relative to the circumradius, the FP64 formula is accurate to ~1e-12
        # unless the triangle is nearly degenerate
        R = math.dist((float(ux), float(uy)), a)
        area2 = abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        if area2 < 1e-6:
            continue
        assert abs(x - float(ux)) <= 1e-10 * (1 + R) and abs(y - float(uy)) <= 1e-10 * (1 + R)


def test_circumcenter_closed_forms(oracle):
    # right triangle: circumcentre is the hypotenuse midpoint
    assert oracle.circumcenter((0.0, 0.0), (2.0, 0.0), (0.0, 2.0)) == (1.0, 1.0)
    x, y = oracle.circumcenter((0.0, 0.0), (1.0, 0.0), (0.5, math.sqrt(3) / 2))
    assert abs(x - 0.5) < 1e-15 and abs(y - 1 / (2 * math.sqrt(3))) < 1e-15


def test_midpoint(oracle):
    assert oracle.midpoint((0.0, 0.0), (1.0, 0.0)) == (0.5, 0.0)
    assert oracle.midpoint((1.0, 0.5), (1.0, 0.75)) == (1.0, 0.625)
    rng = random.Random(9)
    for _ in range(100):
        a, b = (rng.random(), rng.random()), (rng.random(), rng.random())
        m = oracle.midpoint(a, b)
        assert m == oracle.midpoint(b, a)
        assert abs(F(m[0]) - (F(a[0]) + F(b[0])) / 2) <= F(math.ulp(m[0]))


def test_measure_bits_monotone(oracle):
    vals = sorted(random.Random(10).random() * 10 ** random.Random(11).randint(-8, 3) for _ in range(200))
    bits = [oracle.measure_bits(v) for v in vals]
    assert bits == sorted(bits)
    assert oracle.measure_bits(1.0) == 0x3F800000
    assert oracle.measure_bits(0.0) == 0
