"""Edge-length criterion on the GPU (Sec. 4.1): refined meshes whose longest
edge is at most l and that pass every invariant, Steiner counts within 10% of
the oracle's with the same l, and batched meshes equal to their alone runs."""
import math

import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


def longest(xy, tri):
    e = np.concatenate([xy[tri[:, (k + 1) % 3]] - xy[tri[:, k]] for k in range(3)])
    return float(np.sqrt((e ** 2).sum(1).max()))


@pytest.mark.parametrize("l", [0.1, 0.03])
def test_contours_refined_to_length(oracle, l):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.contours(5, 8, 60, 21)
    g = gdp.Mesh(p.xy, p.seg)
    s = g.refine(1.462, max_len=l)
    xy, tri, sub = g.export()
    assert longest(xy, tri) <= l
    assert_valid(oracle.check(xy, tri, sub, p.seg, p.n, B=1.462))
    o = oracle.Mesh(p.xy, p.seg)
    assert o.refine_len(1.462, l) == 0
    assert abs(s["n_steiner"] - o.n_steiner) <= 0.10 * o.n_steiner, (s["n_steiner"], o.n_steiner)


def test_random_pslg_length_and_batch(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    ps = [W.square_pslg(n, n // 50, 800 + n) for n in (500, 3000, 1500)]
    b = gdp.Batch([(p.xy, p.seg) for p in ps])
    b.refine(SQ2, max_len=0.05)
    for i, p in enumerate(ps):
        a = gdp.Mesh(p.xy, p.seg)
        a.refine(SQ2, max_len=0.05)
        axy, atri, asub = a.export()
        bxy, btri, _ = b.export(i)
        assert np.array_equal(axy, bxy)
        assert oracle.triangle_set(axy, atri) == oracle.triangle_set(bxy, btri)
        assert longest(axy, atri) <= 0.05
        assert_valid(oracle.check(axy, atri, asub, p.seg, p.n, B=SQ2))
