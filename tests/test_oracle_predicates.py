"""Pins for the oracle's exact predicates (Sec. 7: exact arithmetic +
simulation of simplicity) against exact rational arithmetic."""
import math
import random

import numpy as np
import pytest

from tests import exact_ref as X


def _near_degenerate(rng, k):
    """points on a line / circle, nudged by a few ulps"""
    out = []
    for _ in range(k):
        t = rng.random()
        a = (rng.random(), rng.random())
        b = (rng.random(), rng.random())
        c = (a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1]))
        c = (c[0] + rng.choice([-1, 0, 1]) * math.ulp(c[0]) * rng.randint(0, 3),
             c[1] + rng.choice([-1, 0, 1]) * math.ulp(c[1]) * rng.randint(0, 3))
        out.append((a, b, c))
    return out


def _cocircular(rng, k):
    out = []
    for _ in range(k):
        cx, cy, r = rng.random(), rng.random(), 0.1 + rng.random()
        ang = [rng.random() * 2 * math.pi for _ in range(4)]
        ang[:3] = sorted(ang[:3])
        pts = [(cx + r * math.cos(t), cy + r * math.sin(t)) for t in ang]
        d = pts[3]
        d = (d[0] + rng.choice([-1, 0, 1]) * math.ulp(d[0]), d[1])
        out.append((pts[0], pts[1], pts[2], d))
    return out


@pytest.mark.parametrize("filt", [True, False])
def test_orient_matches_rationals(oracle, filt):
    oracle.set_filter(filt)
    rng = random.Random(1)
    cases = [tuple((rng.random(), rng.random()) for _ in range(3)) for _ in range(300)]
    cases += _near_degenerate(rng, 300)
    # exactly collinear, incl. dyadic boundary points
    cases += [((0, 0), (0.5, 0), (1, 0)), ((0, 0), (1, 1), (0.25, 0.25)), ((1, 0), (1, 0.5), (1, 1))]
    try:
        for a, b, c in cases:
            assert oracle.orient(a, b, c) == X.sign(X.orient(a, b, c)), (a, b, c)
    finally:
        oracle.set_filter(True)


@pytest.mark.parametrize("filt", [True, False])
def test_incircle_matches_rationals(oracle, filt):
    oracle.set_filter(filt)
    rng = random.Random(2)
    cases = [tuple((rng.random(), rng.random()) for _ in range(4)) for _ in range(200)]
    cases += _cocircular(rng, 300)
    cases += [((0, 0), (1, 0), (1, 1), (0, 1)), ((0, 0), (2, 0), (2, 2), (1, 1 + 2 ** 0.5))]
    try:
        for a, b, c, d in cases:
            assert oracle.incircle(a, b, c, d) == X.sign(X.incircle(a, b, c, d)), (a, b, c, d)
    finally:
        oracle.set_filter(True)


def test_incircle_extreme_magnitudes(oracle):
    """exact path over wide exponent ranges (no overflow / underflow errors)"""
    rng = random.Random(3)
    for _ in range(200):
        s = 10.0 ** rng.randint(-150, 150)
        pts = [(s * rng.random(), s * rng.random()) for _ in range(4)]
        assert oracle.incircle(*pts) == X.sign(X.incircle(*pts))
    tiny = [(1e-300, 0.0), (0.0, 1e-300), (-1e-300, 0.0), (0.0, -1e-300)]
    assert oracle.incircle(*tiny) == 0
    huge = [(1e150, 0.0), (0.0, 1e150), (-1e150, 0.0), (0.0, -1e150 * (1 + 2 ** -52))]
    assert oracle.incircle(*huge) == X.sign(X.incircle(*huge))


def test_dot_sign_matches_rationals(oracle):
    rng = random.Random(4)
    for _ in range(300):
        a, b = (rng.random(), rng.random()), (rng.random(), rng.random())
        # points near the diametral circle of ab
        cx, cy = 0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[1])
        r = 0.5 * math.hypot(b[0] - a[0], b[1] - a[1])
        t = rng.random() * 2 * math.pi
        p = (cx + r * math.cos(t), cy + r * math.sin(t))
        assert oracle.dot_sign(a, b, p) == X.sign(X.dot(a, b, p))
    # closed forms: centre encroaches, endpoints and the circle itself do not
    assert oracle.dot_sign((0, 0), (1, 0), (0.5, 0)) == -1
    assert oracle.dot_sign((0, 0), (2, 0), (1, 1)) == 0
    assert oracle.dot_sign((0, 0), (1, 0), (0.5, 0.6)) == 1


def test_closed_forms(oracle):
    assert oracle.orient((0, 0), (1, 0), (0, 1)) == 1
    assert oracle.orient((0, 0), (0, 1), (1, 0)) == -1
    assert oracle.orient((0, 0), (0.5, 0), (1, 0)) == 0
    assert oracle.incircle((0, 0), (1, 0), (0, 1), (0.1, 0.1)) == 1
    assert oracle.incircle((0, 0), (1, 0), (0, 1), (2, 2)) == -1
    assert oracle.incircle((0, 0), (1, 0), (1, 1), (0, 1)) == 0


def test_sos_matches_rational_definition(oracle):
    rng = random.Random(5)
    cases = [((0, 0), (1, 0), (1, 1), (0, 1)), ((1, 0), (1, 1), (0, 1), (0, 0)),
             ((0, 0), (0.5, 0), (0.5, 1), (0, 1))]
    # exactly cocircular dyadic rectangles in random rotations of roles
    for _ in range(50):
        x0, x1 = sorted(rng.randint(0, 8) / 8 for _ in range(2))
        y0, y1 = sorted(rng.randint(0, 8) / 8 for _ in range(2))
        if x0 == x1 or y0 == y1:
            continue
        pts = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        rng.shuffle(pts)
        a, b, c, d = pts
        if X.orient(a, b, c) < 0:
            a, b = b, a
        cases.append((a, b, c, d))
    for a, b, c, d in cases:
        if X.orient(a, b, c) == 0:
            continue
        s = oracle.incircle_sos(a, b, c, d)
        assert s != 0
        assert s == X.incircle_sos(a, b, c, d), (a, b, c, d)


def test_sos_consistency_of_square_diagonal(oracle):
    """For 4 cocircular points exactly one diagonal is locally Delaunay under
    the perturbation: (a,b,c | d) and (a,c,d | b) can't both say 'inside'."""
    sq = [(0, 0), (1, 0), (1, 1), (0, 1)]
    a, b, c, d = sq
    s1 = oracle.incircle_sos(a, b, c, d)   # diagonal ac: is d inside abc?
    s2 = oracle.incircle_sos(b, c, d, a)   # diagonal bd: is a inside bcd?
    assert s1 != 0 and s2 != 0
    assert (s1 > 0) != (s2 > 0)
