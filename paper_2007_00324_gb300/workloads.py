"""Seeded synthetic PSLG workloads.

These stand in for the paper's contour-map inputs (Sec. 7, Table 1), which
are not available.  The module only draws inputs; it holds none of the
refinement arithmetic, and both the CUDA path and the CPU oracle read what
it produces.

Every PSLG lives in the unit square: the four corners are input points 0..3
and the four boundary edges are segments 0..3, so the domain is the square.
Interior constraint segments are drawn by seeded rejection sampling: the
first endpoint is a uniform random input point, the second a uniform pick
among its 16 nearest neighbours; a candidate is rejected if it comes within
1e-6 of an existing segment (so it neither crosses nor touches one), shares
an endpoint with one, or passes within 1e-6 of any other input point.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20070324
MARGIN = 1e-6
SQRT2 = math.sqrt(2.0)


@dataclass
class PSLG:
    xy: np.ndarray                 # (n, 2) float64
    seg: np.ndarray                # (m, 2) int32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.xy)

    @property
    def m(self) -> int:
        return len(self.seg)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _uniform_interior(rng, n):
    out = np.empty((0, 2))
    while len(out) < n:
        p = rng.random((n - len(out) + 16, 2))
        ok = np.all((p > MARGIN) & (p < 1.0 - MARGIN), axis=1)
        out = np.concatenate([out, p[ok]])[:n]
    return out


def _seg_point_dist(a, b, p):
    """distance from points p (k,2) to segment ab"""
    ab = b - a
    L2 = float(ab @ ab)
    t = np.clip(((p - a) @ ab) / L2, 0.0, 1.0) if L2 > 0 else np.zeros(len(p))
    q = a + t[:, None] * ab
    return np.sqrt(np.sum((p - q) ** 2, axis=1))


def _seg_seg_dist(a, b, c, d):
    def orient(p, q, r):
        return (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])
    o1, o2 = orient(a, b, c), orient(a, b, d)
    o3, o4 = orient(c, d, a), orient(c, d, b)
    if o1 * o2 < 0 and o3 * o4 < 0:
        return 0.0
    return float(min(_seg_point_dist(a, b, np.array([c, d])).min(),
                     _seg_point_dist(c, d, np.array([a, b])).min()))


class _SegGrid:
    """uniform grid over accepted segments (for the crossing / touching test)"""

    def __init__(self, cell):
        self.cell = cell
        self.g = {}
        self.segs = []

    def _cells(self, a, b):
        lo = np.floor((np.minimum(a, b) - MARGIN) / self.cell).astype(int)
        hi = np.floor((np.maximum(a, b) + MARGIN) / self.cell).astype(int)
        for i in range(lo[0], hi[0] + 1):
            for j in range(lo[1], hi[1] + 1):
                yield (i, j)

    def near(self, a, b):
        seen = set()
        for c in self._cells(a, b):
            for k in self.g.get(c, ()):
                if k not in seen:
                    seen.add(k)
                    yield self.segs[k]

    def add(self, a, b):
        k = len(self.segs)
        self.segs.append((a, b))
        for c in self._cells(a, b):
            self.g.setdefault(c, []).append(k)


def _sample_segments(rng, xy, n_seg, first, used_ends, grid, tree, knn=16, max_tries=None):
    """rejection-sample n_seg segments among points xy[first:]"""
    n = len(xy)
    out = []
    tries = 0
    max_tries = max_tries or 200 * n_seg + 1000
    k = min(knn, n - first - 1)
    while len(out) < n_seg and tries < max_tries:
        tries += 1
        i = int(rng.integers(first, n))
        if i in used_ends:
            continue
        _, nb = tree.query(xy[i], k=k + 1)
        nb = [int(x) for x in np.atleast_1d(nb) if int(x) != i and int(x) >= first]
        if not nb:
            continue
        j = nb[int(rng.integers(0, len(nb)))]
        if j in used_ends:
            continue
        a, b = xy[i], xy[j]
        mid = 0.5 * (a + b)
        r = 0.5 * float(np.hypot(*(b - a))) + MARGIN
        close = [int(q) for q in tree.query_ball_point(mid, r) if int(q) not in (i, j)]
        if close and _seg_point_dist(a, b, xy[close]).min() < MARGIN:
            continue
        if any(_seg_seg_dist(a, b, c, d) < MARGIN for c, d in grid.near(a, b)):
            continue
        grid.add(a, b)
        used_ends.update((i, j))
        out.append((i, j))
    return out


def square_pslg(n_pts: int, n_seg: int, seed: int, name: str = "") -> PSLG:
    """Unit-square boundary + n_pts uniform interior points + n_seg random
    interior segments (the tiny / mid / batched / served recipe)."""
    from scipy.spatial import cKDTree
    rng = _rng(seed)
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    pts = _uniform_interior(rng, n_pts)
    xy = np.concatenate([corners, pts])
    tree = cKDTree(xy)
    grid = _SegGrid(cell=max(4.0 / math.sqrt(max(n_pts, 1)), 1e-3))
    segs = [(0, 1), (1, 2), (2, 3), (3, 0)]
    for a, b in segs:
        grid.add(xy[a], xy[b])
    segs += _sample_segments(rng, xy, n_seg, 4, set(), grid, tree)
    return PSLG(xy=np.ascontiguousarray(xy, np.float64),
                seg=np.ascontiguousarray(np.array(segs, np.int32).reshape(-1, 2)),
                name=name or f"square_{n_pts}_{n_seg}", meta={"seed": seed})


def tiny() -> PSLG:
    """1,000 uniform points + 20 segments in the unit square (B = sqrt 2)."""
    return square_pslg(1000, 20, SEED_BASE + 0, "tiny")


def mid() -> PSLG:
    """100,000 uniform points + 1,000 segments in the unit square (B = sqrt 2, 1.5)."""
    return square_pslg(100_000, 1000, SEED_BASE + 1, "mid")


def paper_shaped(n_uniform=500_000, n_gauss=300_000, n_circle=200_000, n_seg=10_000,
                 n_fans=20, seed=SEED_BASE + 2) -> PSLG:
    """Mixed distribution standing in for contour maps: 50% uniform, 30% in
    100 Gaussian clusters (sigma 0.01), 20% on 50 circles; 10,000 random
    segments plus 20 fans of 8 segments 5 degrees apart at a shared apex
    (small input angles)."""
    from scipy.spatial import cKDTree
    rng = _rng(seed)
    uni = _uniform_interior(rng, n_uniform)
    centres = 0.05 + 0.9 * rng.random((100, 2))
    g = np.empty((0, 2))
    while len(g) < n_gauss:
        k = n_gauss - len(g)
        c = centres[rng.integers(0, 100, k)]
        p = c + 0.01 * rng.standard_normal((k, 2))
        ok = np.all((p > MARGIN) & (p < 1 - MARGIN), axis=1)
        g = np.concatenate([g, p[ok]])
    cc = 0.1 + 0.8 * rng.random((50, 2))
    rad = 0.02 + 0.08 * rng.random(50)
    ci = rng.integers(0, 50, n_circle)
    ang = 2 * math.pi * rng.random(n_circle)
    circ = cc[ci] + rad[ci, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    circ = circ[np.all((circ > MARGIN) & (circ < 1 - MARGIN), axis=1)]
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    xy = np.concatenate([corners, uni, g, circ])
    _, first = np.unique(xy, axis=0, return_index=True)
    xy = xy[np.sort(first)]
    tree = cKDTree(xy)
    grid = _SegGrid(cell=0.01)
    segs = [(0, 1), (1, 2), (2, 3), (3, 0)]
    for a, b in segs:
        grid.add(xy[a], xy[b])
    used = set()
    segs += _sample_segments(rng, xy, n_seg, 4, used, grid, tree)
    # fans: apex = an existing input point, 8 new endpoints at radius 0.01
    fan_pts, fan_segs = [], []
    n0 = len(xy)
    fans = 0
    tries = 0
    while fans < n_fans and tries < 200 * n_fans:
        tries += 1
        apex = int(rng.integers(4, n0))
        if apex in used:
            continue
        phi0 = 2 * math.pi * rng.random()
        ends = np.array([[xy[apex, 0] + 0.01 * math.cos(phi0 + k * math.radians(5)),
                          xy[apex, 1] + 0.01 * math.sin(phi0 + k * math.radians(5))]
                         for k in range(8)])
        if np.any(ends <= MARGIN) or np.any(ends >= 1 - MARGIN):
            continue
        ok = True
        for e in ends:
            a, b = xy[apex], e
            close = [int(q) for q in tree.query_ball_point(0.5 * (a + b), 0.005 + MARGIN)
                     if int(q) != apex]
            if close and _seg_point_dist(a, b, xy[close]).min() < MARGIN:
                ok = False
                break
            if tree.query(e)[0] < MARGIN:
                ok = False
                break
            if any(_seg_seg_dist(a, b, c, d) < MARGIN for c, d in grid.near(a, b)):
                ok = False
                break
        if not ok:
            continue
        base = n0 + len(fan_pts)
        for k, e in enumerate(ends):
            grid.add(xy[apex], e)
            fan_pts.append(e)
            fan_segs.append((apex, base + k))
        used.add(apex)
        fans += 1
    if fan_pts:
        xy = np.concatenate([xy, np.array(fan_pts)])
    segs += fan_segs
    return PSLG(xy=np.ascontiguousarray(xy, np.float64),
                seg=np.ascontiguousarray(np.array(segs, np.int32)),
                name="paper_shaped", meta={"seed": seed, "fans": fans})


def contours(n_hills=20, levels=25, per_curve=200, seed=SEED_BASE + 5) -> PSLG:
    """Contour-map-like input (the paper's inputs are contour maps, Sec. 7.1):
    the unit square plus n_hills families of nested closed polylines (levels
    each, per_curve vertices per curve).  A family is r(theta) = r_k * f(theta)
    around its centre with a common shape f > 0 and r_k = R k / (levels + 1),
    so its curves never cross; families are placed apart.  No other points."""
    rng = _rng(seed)
    centres, radii = [], []
    tries = 0
    while len(centres) < n_hills and tries < 10000:
        tries += 1
        R = 0.03 + 0.07 * rng.random()
        c = 0.02 + R * 1.3 + (1 - 2 * (0.02 + R * 1.3)) * rng.random(2)
        if all(np.hypot(*(c - c2)) > 1.3 * (R + R2) + 0.01 for c2, R2 in zip(centres, radii)):
            centres.append(c)
            radii.append(R)
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    pts = [corners]
    segs = [(0, 1), (1, 2), (2, 3), (3, 0)]
    n = 4
    th = 2 * math.pi * np.arange(per_curve) / per_curve
    for c, R in zip(centres, radii):
        a, k, ph = 0.1 + 0.15 * rng.random(), int(rng.integers(2, 6)), 2 * math.pi * rng.random()
        f = 1.0 + a * np.sin(k * th + ph)
        for lv in range(1, levels + 1):
            r = R * lv / (levels + 1) * f
            pts.append(np.stack([c[0] + r * np.cos(th), c[1] + r * np.sin(th)], 1))
            segs += [(n + j, n + (j + 1) % per_curve) for j in range(per_curve)]
            n += per_curve
    return PSLG(xy=np.ascontiguousarray(np.concatenate(pts), np.float64),
                seg=np.ascontiguousarray(np.array(segs, np.int32)),
                name="contours", meta={"seed": seed, "hills": len(centres)})


def batched_sizes(count=4096, lo=200, hi=50_000, seed=SEED_BASE + 3):
    """point counts, log-uniform in [lo, hi]"""
    rng = _rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)


def batched(count=4096, lo=200, hi=50_000, seed=SEED_BASE + 3, limit=None):
    """independent PSLGs for one batched launch (segments = 2% of points)"""
    sizes = batched_sizes(count, lo, hi, seed)
    if limit is not None:
        sizes = sizes[:limit]
    out = []
    for i, n in enumerate(sizes):
        out.append(square_pslg(int(n), int(round(0.02 * n)), seed * 7919 + i, f"batch_{i}"))
    return out


@dataclass
class Request:
    t_arrival: float
    pslg: PSLG
    B: float


def served_trace(rate=200.0, duration=60.0, lo=1000, hi=500_000, seed=SEED_BASE + 4,
                 max_requests=None, build=True):
    """Poisson request stream: point counts log-uniform in [lo, hi], 1-5%
    segments, B drawn from {1.5, sqrt 2} with equal probability."""
    rng = _rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration or (max_requests is not None and i >= max_requests):
            break
        n = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        frac = int(rng.integers(1, 6)) / 100.0
        B = 1.5 if rng.random() < 0.5 else SQRT2
        p = square_pslg(n, int(round(frac * n)), seed * 104729 + i, f"req_{i}") if build else None
        out.append(Request(t, p, B))
        i += 1
    return out
