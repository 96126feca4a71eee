"""Chew's mode on the GPU (Sec. 4.2: under Chew's algorithm a subsegment is
encroached by a point strictly inside its diametral lens, where the
subsegment subtends more than 120 degrees, instead of its diametral circle).

* the scan's encroachment test by the lens is bit-exact against the oracle's
  (exact lens predicate, or_eval_subs_mode), subsegment by subsegment;
* refinement with GDP_REFINE_CHEW gives meshes that pass every oracle invariant
  with encroachment checked against the lens, with a Steiner count within 10%
  of the oracle's sequential refinement in the same mode.
"""
import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


def sub_key(xy, u, v):
    a, b = sorted([tuple(xy[u].tolist()), tuple(xy[v].tolist())])
    return (a, b)


@pytest.mark.parametrize("lens", [True, False])
def test_scan_encroachment_matches_oracle(oracle, lens):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(4000, 400, 2024)
    g = gdp.Mesh(p.xy, p.seg)
    xy, tri, sub = g.export()
    kind, verts, pt, meas = g.scan(SQ2, flags=gdp.REFINE_CHEW if lens else 0)
    got = {}
    for k in range(len(kind)):
        if kind[k] == 1:
            got[sub_key(xy, verts[k, 0], verts[k, 1])] = (tuple(pt[k].tolist()), int(meas[k]))
    enc, mid, smeas = oracle.eval_subs(xy, tri, sub, lens=lens)
    want = {sub_key(xy, sub[i, 0], sub[i, 1]): (tuple(mid[i].tolist()), int(smeas[i]))
            for i in np.nonzero(enc)[0]}
    assert len(want) > 20
    assert got == want
    if lens:   # the lens lies inside the circle: fewer subsegments, and some differ
        enc_c, _, _ = oracle.eval_subs(xy, tri, sub, lens=False)
        assert enc.sum() < enc_c.sum()


def small_contours():
    from paper_2007_00324_gb300 import workloads as W
    return W.contours(n_hills=5, levels=6, per_curve=80, seed=99)


@pytest.mark.parametrize("name", ["tiny", "contours"])
def test_chew_refinement_invariants_and_count(oracle, name):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.tiny() if name == "tiny" else small_contours()
    g = gdp.Mesh(p.xy, p.seg)
    st = g.refine(SQ2, flags=gdp.REFINE_CHEW)
    assert all(v == 0 for v in g.check().values()), g.check()
    xy, tri, sub = g.export()
    rep = oracle.check(xy, tri, sub, p.seg, p.n, B=SQ2, lens=True, brute=(name == "tiny"))
    assert_valid(rep, brute=(name == "tiny"))
    o = oracle.Mesh(p.xy, p.seg)
    assert o.refine_mode(SQ2, lens=True) == 0
    n_ref = o.n_steiner
    assert abs(st["n_steiner"] - n_ref) <= 0.10 * n_ref + 5, (st["n_steiner"], n_ref)


def test_chew_deterministic():
    gdp = need_gpu()
    p = small_contours()
    out = []
    for _ in range(2):
        g = gdp.Mesh(p.xy, p.seg)
        g.refine(SQ2, flags=gdp.REFINE_CHEW)
        xy, tri, _ = g.export()
        out.append((xy.tobytes(), tri.tobytes()))
    assert out[0] == out[1]
