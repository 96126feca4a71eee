"""Batched refinement: many independent PSLGs share one pool and every kernel
launch processes all of them; each mesh must come out exactly as when it is
refined alone (same vertices, same triangles), and be valid."""
import math

import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


def pslgs(sizes, seed):
    from paper_2007_00324_gb300 import workloads as W
    return [W.square_pslg(n, max(1, int(round(0.02 * n))), seed + i) for i, n in enumerate(sizes)]


@pytest.mark.parametrize("Bs", [(SQ2,), (SQ2, 1.5)])
def test_batch_equals_alone(oracle, Bs):
    gdp = need_gpu()
    ps = pslgs([200, 1500, 400, 5000, 800, 2500, 300, 10000], 900)
    B = np.array([Bs[i % len(Bs)] for i in range(len(ps))])
    batch = gdp.Batch([(p.xy, p.seg) for p in ps])
    stats = batch.refine(B)
    info = batch.info()
    assert np.all(info["status"] == 0)
    for i, p in enumerate(ps):
        bxy, btri, bsub = batch.export(i)
        alone = gdp.Mesh(p.xy, p.seg)
        alone.refine(float(B[i]))
        axy, atri, asub = alone.export()
        assert np.array_equal(bxy, axy), i
        assert np.array_equal(btri, atri), i
        assert_valid(oracle.check(bxy, btri, bsub, p.seg, p.n, B=float(B[i])))
        assert info["n_steiner"][i] == len(bxy) - p.n
    assert stats["n_steiner"] == int(info["n_steiner"].sum())


def test_batch_cdt_bit_exact(oracle):
    gdp = need_gpu()
    ps = pslgs([100, 700, 3000, 50], 77)
    batch = gdp.Batch([(p.xy, p.seg) for p in ps])
    for i, p in enumerate(ps):
        bxy, btri, _ = batch.export(i)
        o = oracle.Mesh(p.xy, p.seg)
        oxy, otri, _ = o.export()
        assert oracle.triangle_set(bxy, btri) == oracle.triangle_set(oxy, otri)


def test_batch_with_a_bad_mesh_reports_it():
    gdp = need_gpu()
    ps = pslgs([300, 300], 5)
    xy = np.concatenate([ps[1].xy, ps[1].xy[4:5]])   # duplicate point
    with pytest.raises(gdp.GdpError):
        gdp.Batch([(ps[0].xy, ps[0].seg), (xy, ps[1].seg)])
