"""The seeded input generators: determinism and the sampler's rules."""
import numpy as np

from tests import exact_ref as X


def test_deterministic_and_valid():
    from paper_2007_00324_gb300 import workloads as W
    a, b = W.tiny(), W.tiny()
    assert np.array_equal(a.xy, b.xy) and np.array_equal(a.seg, b.seg)
    assert a.n == 1004 and a.m == 24
    assert np.array_equal(a.xy[:4], [[0, 0], [1, 0], [1, 1], [0, 1]])
    assert np.all((a.xy[4:] > 0) & (a.xy[4:] < 1))
    assert len(np.unique(a.xy, axis=0)) == a.n
    inner = a.seg[4:]
    # no shared endpoints among interior segments
    assert len(np.unique(inner.ravel())) == 2 * len(inner)
    # pairwise non-crossing (exact)
    for i in range(len(inner)):
        for j in range(i + 1, len(inner)):
            p, q = a.xy[inner[i, 0]], a.xy[inner[i, 1]]
            r, s = a.xy[inner[j, 0]], a.xy[inner[j, 1]]
            o1 = X.sign(X.orient(p, q, r)) * X.sign(X.orient(p, q, s))
            o2 = X.sign(X.orient(r, s, p)) * X.sign(X.orient(r, s, q))
            assert not (o1 <= 0 and o2 <= 0)


def test_batched_sizes_log_uniform():
    from paper_2007_00324_gb300 import workloads as W
    s = W.batched_sizes()
    assert len(s) == 4096 and s.min() >= 200 and s.max() <= 50_000
    assert 7_000 < s.mean() < 11_000


def test_served_trace_shape():
    from paper_2007_00324_gb300 import workloads as W
    tr = W.served_trace(duration=2.0, build=False)
    assert 300 < len(tr) < 500
    assert all(r.B in (1.5, W.SQRT2) for r in tr)
    assert all(tr[i].t_arrival < tr[i + 1].t_arrival for i in range(len(tr) - 1))
