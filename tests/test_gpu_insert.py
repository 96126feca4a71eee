"""The parallel cavity insertion (Sec. 5.2: grow, atomic priority marks,
dependence check, fan re-triangulation) gives exactly the CDT that the
oracle's sequential Bowyer-Watson insertion gives for the same batch."""
import numpy as np
import pytest

from tests.gpu_util import assert_valid, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_extra,seed", [(50, 1), (2000, 2), (20000, 3)])
def test_fixed_free_point_batch(oracle, n_extra, seed):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(max(2000, n_extra // 2), 40, 1000 + seed)
    rng = np.random.default_rng(seed)
    extra = 0.001 + 0.998 * rng.random((n_extra, 2))
    g = gdp.Mesh(p.xy, p.seg)
    g.insert_points(extra)
    gxy, gtri, gsub = g.export()
    o = oracle.Mesh(p.xy, p.seg)
    assert o.insert_points(extra) == 0
    oxy, otri, osub = o.export()
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)
    assert_valid(oracle.check(gxy, gtri, gsub, p.seg, p.n), refined=False)


def test_oracle_steiner_batch(oracle):
    """the oracle's own first Steiner points (free ones), inserted on both sides"""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    o = oracle.Mesh(p.xy, p.seg)
    assert o.refine(2 ** 0.5) == 0
    oxy, _, osub = o.export()
    steiner = oxy[p.n:]
    on_seg = set(osub[:, :2].ravel().tolist())
    free = np.array([steiner[i] for i in range(len(steiner)) if (p.n + i) not in on_seg])
    batch = free[: max(1, len(free) // 10)]
    g = gdp.Mesh(p.xy, p.seg)
    g.insert_points(batch)
    o2 = oracle.Mesh(p.xy, p.seg)
    assert o2.insert_points(batch) == 0
    gxy, gtri, _ = g.export()
    oxy2, otri2, _ = o2.export()
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy2, otri2)


def test_subsegment_split_batch(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(1500, 30, 4242)
    g = gdp.Mesh(p.xy, p.seg)
    _, _, sub = g.export()
    xy = p.xy
    pick = sub[: len(sub) // 2]
    abxy = np.concatenate([xy[pick[:, 0]], xy[pick[:, 1]]], axis=1)
    g.split_subsegments(abxy)
    o = oracle.Mesh(p.xy, p.seg)
    assert o.split_subsegments(abxy) == 0
    gxy, gtri, gsub = g.export()
    oxy, otri, _ = o.export()
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)
    assert_valid(oracle.check(gxy, gtri, gsub, p.seg, p.n), refined=False)
