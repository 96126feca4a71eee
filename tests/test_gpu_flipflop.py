"""Flip-Flop insertion (the paper's gDP2d insertion step, Sec. 4.3;
GDP_REFINE_FLIPFLOP), an alternative to cavity insertion: survivors of the
cavity filter are split in, flips restore the constrained Delaunay property,
and points of one iteration joined by an edge (Delaunay dependent, Sec. 4.2)
are removed again by flips and a flop, the one with the lower priority.

The refined meshes must pass every oracle invariant (constrained Delaunay,
conforming, quality, no encroachment), with a Steiner count within 10% of the
oracle's sequential refinement; batches equal alone runs; runs repeat bit for
bit.
"""
import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


def refine_ff(gdp, p, B=SQ2, **kw):
    g = gdp.Mesh(p.xy, p.seg)
    st = g.refine(B, flags=gdp.REFINE_FLIPFLOP | kw.pop("flags", 0), **kw)
    assert all(v == 0 for v in g.check().values()), g.check()
    return g, st


@pytest.mark.parametrize("name,B", [("tiny", SQ2), ("tiny", 1.5), ("square20k", SQ2)])
def test_flipflop_invariants_and_count(oracle, name, B):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny() if name == "tiny" else W.square_pslg(20_000, 200, 2020)
    g, st = refine_ff(gdp, p, B)
    xy, tri, sub = g.export()
    assert len(xy) == p.n + st["n_steiner"]
    assert np.array_equal(xy[:p.n], p.xy)
    rep = oracle.check(xy, tri, sub, p.seg, p.n, B=B, brute=(name == "tiny"))
    assert_valid(rep, brute=(name == "tiny"))
    assert abs(rep["area_sum"] - 1.0) < 1e-12
    o = oracle.Mesh(p.xy, p.seg)
    assert o.refine(B) == 0
    assert abs(st["n_steiner"] - o.n_steiner) <= 0.10 * o.n_steiner, (st["n_steiner"], o.n_steiner)
    assert st["flips"] > 0


def test_flipflop_removes_redundant_points(oracle):
    """without the dependence check before insertion, points of one iteration
    end up joined by edges: the lower-priority ones are flopped out again"""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(20_000, 200, 2020)
    _, st = refine_ff(gdp, p)
    assert st["redundant_removed"] > 0 and st["flops"] == st["redundant_removed"]
    assert st["inserted"] - st["redundant_removed"] == st["n_steiner"]


def test_flipflop_small_angles_and_chew(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.paper_shaped(n_uniform=3000, n_gauss=1500, n_circle=1000, n_seg=60, n_fans=6, seed=4711)
    g, st = refine_ff(gdp, p)
    xy, tri, sub = g.export()
    assert_valid(oracle.check(xy, tri, sub, p.seg, p.n, B=SQ2))
    o = oracle.Mesh(p.xy, p.seg)
    assert o.refine(SQ2) == 0
    assert abs(st["n_steiner"] - o.n_steiner) <= 0.10 * o.n_steiner, (st["n_steiner"], o.n_steiner)
    # Chew's mode with Flip-Flop insertion
    c = W.contours(n_hills=5, levels=6, per_curve=80, seed=99)
    g2, st2 = refine_ff(gdp, c, flags=gdp.REFINE_CHEW)
    xy2, tri2, sub2 = g2.export()
    assert_valid(oracle.check(xy2, tri2, sub2, c.seg, c.n, B=SQ2, lens=True))
    o2 = oracle.Mesh(c.xy, c.seg)
    assert o2.refine_mode(SQ2, lens=True) == 0
    assert abs(st2["n_steiner"] - o2.n_steiner) <= 0.10 * o2.n_steiner + 5


def test_flipflop_deterministic_and_batch_equals_alone():
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    pslgs = [W.square_pslg(n, m, 900 + n) for n, m in ((500, 10), (4000, 80), (1500, 30))]
    alone = []
    for p in pslgs:
        g, _ = refine_ff(gdp, p)
        alone.append(g.export())
    g, _ = refine_ff(gdp, pslgs[1])
    again = g.export()
    assert all(np.array_equal(a, b) for a, b in zip(alone[1], again))
    b = gdp.Batch([(p.xy, p.seg) for p in pslgs])
    b.refine(SQ2, flags=gdp.REFINE_FLIPFLOP)
    assert (b.info()["status"] == 0).all()
    for k in range(len(pslgs)):
        assert all(np.array_equal(x, y) for x, y in zip(alone[k], b.export(k))), k
