"""Pins for the oracle's small-input-angle rules (Sec. 4.1: bad triangles
near input angles below 60 degrees are unavoidable and accepted).

* C6, concentric shells: a subsegment with exactly one end at an apex (an
  input vertex where two segments meet below 60 degrees) is split at the
  power-of-two distance from that end nearest to half its length, nearest in
  ratio (on a log scale).  Each expected point below is worked out here from
  that rule with exact powers of two, not by calling the oracle.
* C10, the exemption: a bad triangle is accepted when its shortest edge joins
  vertices lying on two segments that meet at a small input angle (an apex
  lies on every segment incident to it; a Steiner vertex on the segment it
  was placed on).  The cases below are literal triangles beside a fan, each
  decided here from that rule.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
BOUNDARY = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)


def shell_distance(L):
    """the power of two d nearest to L/2 in ratio: |log2 d - log2(L/2)| smallest"""
    half = Fraction(L) / 2
    k = math.floor(math.log2(half))
    lo, hi = Fraction(2) ** k, Fraction(2) ** (k + 1)
    while lo > half:
        lo, hi = lo / 2, lo
    while hi <= half:
        lo, hi = hi, hi * 2
    # half / lo vs hi / half, compared exactly: lo is nearer iff half^2 < lo * hi
    return float(lo) if half * half < lo * hi else float(hi)


@pytest.mark.parametrize("L,d", [(3.0, 2.0), (5.0, 2.0), (0.7, 0.25), (1.0, 0.5), (0.3, 0.125),
                                 (6.0, 4.0), (0.09, 0.0625)])
def test_shell_distances_worked_by_hand(L, d):
    """the table is the rule worked by hand (e.g. L = 3: L/2 = 1.5 lies between
    1 and 2, and 1.5^2 = 2.25 > 1 * 2, so 2 is nearer in ratio); the helper
    used for the other cases must agree with it"""
    assert shell_distance(L) == d


@pytest.mark.parametrize("L", [3.0, 5.0, 0.7, 1.0, 0.3, 6.0, 0.09, 1.3e-3, 7.77])
def test_shell_point_on_axis(oracle, L):
    d = shell_distance(L)
    # apex at a: the point is d from a along ab
    px, py = oracle.split_point((0.0, 0.0), (L, 0.0), apex_a=True)
    assert py == 0.0 and abs(px - d) <= 4e-16 * d
    # apex at b: d from b towards a
    px, py = oracle.split_point((0.0, 0.0), (L, 0.0), apex_b=True)
    assert py == 0.0 and abs((L - px) - d) <= 1e-15 * L


@pytest.mark.parametrize("L,deg", [(3.0, 30.0), (5.0, 117.0), (0.7, 200.0), (1.0, 301.0)])
def test_shell_point_off_axis(oracle, L, deg):
    ox, oy = 0.25, -0.5
    qx, qy = ox + L * math.cos(math.radians(deg)), oy + L * math.sin(math.radians(deg))
    px, py = oracle.split_point((ox, oy), (qx, qy), apex_a=True)
    Lq = math.hypot(qx - ox, qy - oy)
    d = shell_distance(Lq)
    assert abs(math.hypot(px - ox, py - oy) - d) <= 1e-14 * d
    # on the segment: the cross product with the direction vanishes to rounding
    cross = (px - ox) * (qy - oy) - (py - oy) * (qx - ox)
    assert abs(cross) <= 1e-14 * L * L


@pytest.mark.parametrize("apex_a,apex_b", [(False, False), (True, True)])
def test_no_single_apex_gives_the_midpoint(oracle, apex_a, apex_b):
    a, b = (0.1, 0.2), (0.7, 0.5)
    assert oracle.split_point(a, b, apex_a, apex_b) == ((0.1 + 0.7) * 0.5, (0.2 + 0.5) * 0.5)


def test_shell_never_the_midpoint_distance_unless_a_power_of_two(oracle):
    """a plausible slip -- the arithmetic midpoint of the two candidate powers
    instead of the ratio rule -- differs at L/2 = 1.45 (between 1 and 2: ratio
    rule gives 2 since 1.45^2 = 2.1025 > 2; the arithmetic rule would give 1)"""
    px, _ = oracle.split_point((0.0, 0.0), (2.9, 0.0), apex_a=True)
    assert px == pytest.approx(2.0, rel=1e-15)
    px, _ = oracle.split_point((0.0, 0.0), (2.8, 0.0), apex_a=True)   # 1.4^2 = 1.96 < 2
    assert px == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("deg,small", [(10.0, True), (45.0, True), (59.5, True), (60.5, False),
                                       (90.0, False), (170.0, False)])
def test_small_angle_threshold(oracle, deg, small):
    r = math.radians(deg)
    assert oracle.small_angle((0.3, 0.4), (1.3, 0.4), (0.3 + 2 * math.cos(r), 0.4 + 2 * math.sin(r))) == small
    # symmetric in the two directions
    assert oracle.small_angle((0.3, 0.4), (0.3 + 2 * math.cos(r), 0.4 + 2 * math.sin(r)), (1.3, 0.4)) == small


def fan_mesh(oracle):
    """unit square; apex O = (0.5, 0.5) with segments to A at 0 deg, B at
    10 deg, C at 20 deg (radius 0.3) and D at 90 deg; a free point P; then the
    subsegments OA and OB split once each (concentric shells: 0.125 from O)"""
    O = (0.5, 0.5)
    ends = [(O[0] + 0.3 * math.cos(math.radians(a)), O[1] + 0.3 * math.sin(math.radians(a)))
            for a in (0.0, 10.0, 20.0, 90.0)]
    xy = np.concatenate([SQUARE, [O], ends, [[0.64, 0.45]]])
    seg = np.concatenate([BOUNDARY, [[4, 5], [4, 6], [4, 7], [4, 8]]])
    m = oracle.Mesh(xy, seg)
    assert m.split_subsegments(np.array([[*O, *ends[0]], [*O, *ends[1]]])) == 0
    xy1, _, _ = m.export()
    return m, xy1


def test_fan_split_points_are_shell_points(oracle):
    m, xy = fan_mesh(oracle)
    assert len(xy) == 12
    for k, deg in ((10, 0.0), (11, 10.0)):
        assert math.hypot(xy[k][0] - 0.5, xy[k][1] - 0.5) == pytest.approx(0.125, rel=1e-14)
        assert math.degrees(math.atan2(xy[k][1] - 0.5, xy[k][0] - 0.5)) == pytest.approx(deg, abs=1e-9)


# vertex ids: 0-3 corners, 4 = O, 5 = A (0 deg), 6 = B (10 deg), 7 = C (20 deg),
# 8 = D (90 deg), 9 = P (0.64, 0.45), 10 = S1 on OA, 11 = S2 on OB.
# Each case: (triangle, exempt?, why)
FAN_CASES = [
    ((4, 10, 11), True, "shortest S1-S2: on OA and OB, 10 deg at O"),
    ((10, 11, 7), True, "shortest S1-S2 again; the third vertex does not matter"),
    ((4, 10, 1), True, "shortest O-S1: O lies on OB, S1 on OA, 10 deg at O"),
    ((5, 7, 2), True, "shortest A-C: on OA and OC, 20 deg at O"),
    ((4, 10, 9), False, "shortest S1-P (0.052): P lies on no segment; the longer O-S1 would qualify"),
    ((10, 8, 2), False, "shortest S1-D: on OA and OD, 90 deg at O"),
    ((5, 8, 2), False, "shortest A-D (0.42; both other edges 0.54): on OA and OD, 90 deg at O"),
    ((0, 1, 4), False, "shortest edges O-0 and O-1 (a tie): corners lie on boundary segments only"),
    ((1, 2, 5), False, "shortest A-1 and A-2 (a tie): 1, 2 on boundary segments, A on OA, no shared end"),
]


def _seg_sets(xy):
    """the segments each vertex lies on, from the construction above"""
    s = {0: {0, 3}, 1: {0, 1}, 2: {1, 2}, 3: {2, 3}, 4: {4, 5, 6, 7}, 5: {4}, 6: {5}, 7: {6}, 8: {7},
         9: set(), 10: {4}, 11: {5}}
    return s


def _rule(xy, tri, segsets, seg):
    """C10 written out: every shortest edge, every pair of segments of its ends"""
    def l2(a, b):
        return (xy[a][0] - xy[b][0]) ** 2 + (xy[a][1] - xy[b][1]) ** 2
    edges = [(tri[(e + 1) % 3], tri[(e + 2) % 3]) for e in range(3)]
    ls = [l2(a, b) for a, b in edges]
    for (a, b), l in zip(edges, ls):
        if l != min(ls):
            continue
        for s1 in segsets[a]:
            for s2 in segsets[b]:
                if s1 == s2:
                    continue
                shared = set(seg[s1]) & set(seg[s2])
                if not shared:
                    continue
                o = shared.pop()
                p = seg[s1][0] if seg[s1][1] == o else seg[s1][1]
                q = seg[s2][0] if seg[s2][1] == o else seg[s2][1]
                u = np.subtract(xy[p], xy[o])
                w = np.subtract(xy[q], xy[o])
                ang = math.degrees(math.acos(np.dot(u, w) / (np.linalg.norm(u) * np.linalg.norm(w))))
                if ang < 60.0:
                    return True
    return False


@pytest.mark.parametrize("tri,want,why", FAN_CASES)
def test_exemption_beside_a_fan(oracle, tri, want, why):
    m, xy = fan_mesh(oracle)
    seg = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (4, 6), (4, 7), (4, 8)]
    assert _rule(xy, tri, _seg_sets(xy), seg) == want, why   # the table is the rule
    for r in range(3):   # and the oracle agrees in every rotation
        t = tri[r:] + tri[:r]
        assert m.exempt(*t) == (1 if want else 0), (t, why)


def test_exemption_tie_is_independent_of_rotation(oracle):
    """triangle A B C with |AB| = |BC| exactly (both shortest): AB joins two
    segments meeting at 26.6 deg (exempt), BC joins B to a point on no segment.
    With ties every shortest edge is tried, so all three rotations agree."""
    xy = np.concatenate([SQUARE, [[0.5, 0.5], [0.75, 0.5], [0.75, 0.625], [0.875, 0.625]]])
    seg = np.concatenate([BOUNDARY, [[4, 5], [4, 6]]])
    m = oracle.Mesh(xy, seg)
    for t in ((5, 7, 6), (7, 6, 5), (6, 5, 7)):
        assert m.exempt(*t) == 1, t
    # a triangle whose only shortest edge is BC is not exempt
    assert m.exempt(6, 7, 2) == 0


def test_eval_exempt_agrees_with_the_mesh_query(oracle):
    """the array form (used against the GPU) gives the per-triangle query's
    answer on every bad triangle of a refined fan"""
    m, _ = fan_mesh(oracle)
    assert m.refine(math.sqrt(2.0), max_steiner=100_000) == 0
    xy, tri, sub = m.export()
    seg = np.concatenate([BOUNDARY, [[4, 5], [4, 6], [4, 7], [4, 8]]])
    ex = oracle.eval_exempt(xy, tri, sub, seg, 10, 2.0)
    assert ex.sum() > 0
    for k, t in enumerate(tri):
        bad = oracle.is_bad(tuple(xy[t[0]]), tuple(xy[t[1]]), tuple(xy[t[2]]), 2.0)
        assert ex[k] == (1 if bad and m.exempt(*map(int, t)) == 1 else 0)
