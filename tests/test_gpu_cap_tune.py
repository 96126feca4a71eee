"""Per-mesh candidate cap (Rule 2) and the autotuner.  A capped refinement
still reaches a valid quality mesh; the cap is per mesh, so a mesh refined in
a batch equals the same mesh refined alone with the same cap; block shapes do
not change results."""
import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cap", [64, 1000])
def test_capped_refinement_is_valid(oracle, cap):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(20000, 300, 21)
    free = gdp.Mesh(p.xy, p.seg)
    s0 = free.refine(SQ2)
    g = gdp.Mesh(p.xy, p.seg)
    s1 = g.refine(SQ2, cand_cap=cap)
    xy, tri, sub = g.export()
    assert_valid(oracle.check(xy, tri, sub, p.seg, p.n, B=SQ2))
    assert s1["iterations"] > s0["iterations"]
    # never more grown candidates per iteration than the cap allows, up to one bucket
    assert s1["candidates"] <= s0["candidates"] * 1.5
    o = oracle.Mesh(p.xy, p.seg)
    assert o.refine(SQ2) == 0
    assert abs(s1["n_steiner"] - o.n_steiner) <= 0.10 * o.n_steiner


def test_cap_is_per_mesh_in_a_batch(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    ps = [W.square_pslg(n, n // 50, 500 + n) for n in (900, 4000, 2500)]
    b = gdp.Batch([(p.xy, p.seg) for p in ps])
    b.refine(SQ2, cand_cap=128)
    for i, p in enumerate(ps):
        a = gdp.Mesh(p.xy, p.seg)
        a.refine(SQ2, cand_cap=128)
        axy, atri, _ = a.export()
        bxy, btri, _ = b.export(i)
        assert np.array_equal(axy, bxy)
        assert oracle.triangle_set(axy, atri) == oracle.triangle_set(bxy, btri)


@pytest.mark.parametrize("block", [32, 128, 256])
def test_block_shape_does_not_change_results(oracle, block):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(8000, 120, 33)
    a = gdp.Mesh(p.xy, p.seg)
    a.refine(SQ2)
    b = gdp.Mesh(p.xy, p.seg)
    b.refine(SQ2, cand_block=block)
    axy, atri, _ = a.export()
    bxy, btri, _ = b.export()
    assert np.array_equal(axy, bxy)
    assert oracle.triangle_set(axy, atri) == oracle.triangle_set(bxy, btri)


def test_autotune_picks_from_its_grid():
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    ps = [W.square_pslg(n, n // 50, 600 + n) for n in (500, 3000, 1200, 7000)]
    best, trials = gdp.autotune([(p.xy, p.seg) for p in ps], SQ2)
    assert best["cand_block"] in (32, 64, 128, 256)
    assert best["cand_cap"] in (0, 16384, 4096, 1024, 256)
    assert len(trials) == 20 and all(t[2] > 0 and t[3] > 0 for t in trials)
    rates = {(int(t[0]), int(t[1])): t[3] / t[2] for t in trials}
    assert rates[(best["cand_block"], best["cand_cap"])] == max(rates.values())
