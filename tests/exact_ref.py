"""Exact rational reference predicates (Python fractions), used to pin the
oracle's predicates.  Each is the determinant written out directly."""
from fractions import Fraction as F


def orient(a, b, c):
    ax, ay, bx, by, cx, cy = map(F, (*a, *b, *c))
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)


def incircle(a, b, c, d):
    rows = []
    for p in (a, b, c, d):
        x, y = F(p[0]), F(p[1])
        rows.append([x, y, x * x + y * y, F(1)])
    return det4(rows)


def det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def det4(m):
    s = F(0)
    for j in range(4):
        minor = [row[:j] + row[j + 1:] for row in m[1:]]
        s += (-1) ** j * m[0][j] * det3(minor)
    return s


def dot(a, b, p):
    ax, ay, bx, by, px, py = map(F, (*a, *b, *p))
    return (ax - px) * (bx - px) + (ay - py) * (by - py)


def sign(v):
    return (v > 0) - (v < 0)


def incircle_sos(a, b, c, d):
    """lift perturbation: lexicographically larger points get larger eps"""
    s = sign(incircle(a, b, c, d))
    if s:
        return s
    pts = [a, b, c, d]
    order = sorted(range(4), key=lambda i: (pts[i][0], pts[i][1]), reverse=True)
    for i in order:
        rows = []
        for j in range(4):
            x, y = F(pts[j][0]), F(pts[j][1])
            # derivative of the 4x4 determinant w.r.t. the lift of row i
            rows.append([x, y, F(1) if j == i else F(0), F(1)])
        c_i = det4(rows)
        if c_i:
            return sign(c_i)
    return 0
