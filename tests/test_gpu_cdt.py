"""GPU initial CDT (first step of Algorithm 1) against the oracle: the CDT is unique
under simulation of simplicity, so the triangle sets must be identical."""
import numpy as np
import pytest

from tests.gpu_util import assert_valid, need_gpu

pytestmark = pytest.mark.gpu

SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
BOUNDARY = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)


def both(oracle, gdp, xy, seg):
    g = gdp.Mesh(xy, seg)
    gxy, gtri, gsub = g.export()
    o = oracle.Mesh(xy, seg)
    oxy, otri, osub = o.export()
    return (gxy, gtri, gsub), (oxy, otri, osub)


def test_empty_square(oracle):
    gdp = need_gpu()
    (gxy, gtri, gsub), (oxy, otri, _) = both(oracle, gdp, SQUARE, BOUNDARY)
    assert len(gtri) == 2 and len(gsub) == 4
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)


def test_square_plus_centre(oracle):
    gdp = need_gpu()
    xy = np.concatenate([SQUARE, [[0.5, 0.5]]])
    (gxy, gtri, _), (oxy, otri, _) = both(oracle, gdp, xy, BOUNDARY)
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)


@pytest.mark.parametrize("n,m,seed", [(50, 3, 1), (300, 10, 2), (1000, 20, 3), (3000, 60, 4)])
def test_random_square_pslgs_bit_exact(oracle, n, m, seed):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(n, m, seed)
    (gxy, gtri, gsub), (oxy, otri, osub) = both(oracle, gdp, p.xy, p.seg)
    assert np.array_equal(gxy, oxy)
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)
    rep = oracle.check(gxy, gtri, gsub, p.seg, p.n, brute=n <= 1000)
    assert_valid(rep, refined=False, brute=n <= 1000)
    norm = lambda S: sorted((min(a, b), max(a, b), s) for a, b, s in S.tolist())
    assert norm(gsub) == norm(osub)


def test_tiny_config_bit_exact(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny()
    (gxy, gtri, _), (oxy, otri, _) = both(oracle, gdp, p.xy, p.seg)
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)


def test_mid_config_bit_exact(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.mid()
    g = gdp.Mesh(p.xy, p.seg)
    # the device links, not only the exported triangle list, must be consistent
    assert all(v == 0 for v in g.check().values()), g.check()
    (gxy, gtri, gsub), (oxy, otri, _) = both(oracle, gdp, p.xy, p.seg)
    assert len(gtri) == len(otri)
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)
    assert_valid(oracle.check(gxy, gtri, gsub, p.seg, p.n), refined=False)


def test_dyadic_grid_degenerate(oracle):
    """many exactly cocircular / collinear points: the tie-break decides"""
    gdp = need_gpu()
    g = np.linspace(0, 1, 9)
    xx, yy = np.meshgrid(g, g)
    pts = np.stack([xx.ravel(), yy.ravel()], 1)
    corners = [0, 8, 80, 72]
    rest = [i for i in range(81) if i not in corners]
    xy = np.concatenate([pts[corners], pts[rest]])
    # boundary as chains of unit segments along the grid
    idx = {tuple(p): i for i, p in enumerate(xy.tolist())}
    segs = []
    for k in range(8):
        for a, b in (((g[k], 0), (g[k + 1], 0)), ((1, g[k]), (1, g[k + 1])),
                     ((g[k], 1), (g[k + 1], 1)), ((0, g[k]), (0, g[k + 1]))):
            segs.append((idx[a], idx[b]))
    seg = np.array(segs, np.int32)
    (gxy, gtri, _), (oxy, otri, _) = both(oracle, gdp, xy, seg)
    assert oracle.triangle_set(gxy, gtri) == oracle.triangle_set(oxy, otri)


def test_invalid_inputs_rejected():
    gdp = need_gpu()
    xy = np.concatenate([SQUARE, [[0.25, 0.5], [0.75, 0.5], [0.5, 0.25], [0.5, 0.75]]])
    for seg in (np.concatenate([BOUNDARY, [[4, 5], [6, 7]]]),      # crossing
                np.concatenate([BOUNDARY, [[0, 99]]]),              # bad index
                np.concatenate([BOUNDARY, [[4, 4]]])):              # degenerate
        with pytest.raises(gdp.GdpError) as e:
            gdp.Mesh(xy, seg)
        assert e.value.status in (gdp.ERR_INPUT,)
    with pytest.raises(gdp.GdpError):
        gdp.Mesh(np.concatenate([xy, [[0.25, 0.5]]]), BOUNDARY)   # duplicate point
    through = np.concatenate([SQUARE, [[0.25, 0.25], [0.5, 0.5], [0.75, 0.75]]])
    with pytest.raises(gdp.GdpError):
        gdp.Mesh(through, np.concatenate([BOUNDARY, [[4, 6]]]))
    with pytest.raises(gdp.GdpError):
        gdp.Mesh(np.array([[0, 0], [np.nan, 1], [1, 1], [0, 1]]), BOUNDARY)
