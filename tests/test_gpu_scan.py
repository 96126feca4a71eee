"""Scan and splitting points (the scan and the splitting points of Algorithm 1): the bad-triangle
test, the circumcentre / midpoint and the priority measure bits are
bit-identical to the oracle's fixed-order FP64 formulas."""
import math

import numpy as np
import pytest

from tests.gpu_util import SQ2, need_gpu

pytestmark = pytest.mark.gpu


def canon_tri(xy, t):
    pts = [tuple(xy[i].tolist()) for i in t]
    k = min(range(3), key=lambda i: pts[i])
    return (pts[k], pts[(k + 1) % 3], pts[(k + 2) % 3])


@pytest.mark.parametrize("B", [SQ2, 1.5])
def test_scan_matches_oracle(oracle, B):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(3000, 80, 99)
    g = gdp.Mesh(p.xy, p.seg)
    xy, tri, sub = g.export()
    kind, verts, pt, meas = g.scan(B)
    # oracle on the same mesh
    bad, cc, tmeas = oracle.eval_tris(xy, tri, B * B)
    enc, mid, smeas = oracle.eval_subs(xy, tri, sub)
    want_t = {canon_tri(xy, tri[i]): (tuple(cc[i].tolist()), int(tmeas[i])) for i in np.nonzero(bad)[0]}
    want_s = {}
    for i in np.nonzero(enc)[0]:
        a, b = sorted([tuple(xy[sub[i, 0]].tolist()), tuple(xy[sub[i, 1]].tolist())])
        want_s[(a, b)] = (tuple(mid[i].tolist()), int(smeas[i]))
    got_t, got_s = {}, {}
    for k in range(len(kind)):
        if kind[k] == 0:
            got_t[canon_tri(xy, verts[k])] = (tuple(pt[k].tolist()), int(meas[k]))
        elif kind[k] == 1:
            a, b = sorted([tuple(xy[verts[k, 0]].tolist()), tuple(xy[verts[k, 1]].tolist())])
            got_s[(a, b)] = (tuple(pt[k].tolist()), int(meas[k]))
    assert len(want_t) > 100
    assert set(kind.tolist()) <= {0, 1}   # no small input angles here, so nothing exempt
    assert got_t == want_t
    assert got_s == want_s
