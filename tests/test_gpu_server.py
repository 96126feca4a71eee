"""Serving (continuous batching): requests submitted while others refine are
admitted into the resident pool as regions free up, and each result is the
mesh the request gives alone (bit for bit: same vertices in the same order,
same triangles)."""
import math

import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu


def alone(gdp, p, B):
    m = gdp.Mesh(p.xy, p.seg)
    m.refine(B)
    return m.export()


def same(oracle, a, b):
    axy, atri, asub = a
    bxy, btri, bsub = b
    assert np.array_equal(axy, bxy)
    assert oracle.triangle_set(axy, atri) == oracle.triangle_set(bxy, btri)
    norm = lambda S: sorted((min(x, y), max(x, y), s) for x, y, s in S.tolist())
    assert norm(asub) == norm(bsub)


def drain(srv, limit=100000):
    out = {}
    for _ in range(limit):
        w, l, d = srv.step()
        for info, xy, tri, sub in srv.results():
            out[info["ticket"]] = (info, (xy, tri, sub))
        if w == 0 and l == 0:
            for info, xy, tri, sub in srv.results():
                out[info["ticket"]] = (info, (xy, tri, sub))
            return out
    raise AssertionError("server did not drain")


def test_served_equals_alone_with_late_arrivals(oracle):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    ps = [W.square_pslg(n, m, 300 + i) for i, (n, m) in
          enumerate([(3000, 60), (800, 20), (12000, 200), (400, 8), (6000, 120), (1500, 45)])]
    Bs = [SQ2, 1.5, SQ2, 1.5, SQ2, SQ2]
    srv = gdp.Server(1 << 21, 1 << 20, 1 << 14, 64)
    tickets = {}
    for i in range(3):
        tickets[srv.submit(ps[i].xy, ps[i].seg, Bs[i])] = i
    srv.step()
    srv.step()
    for i in range(3, 6):   # arrive while the first ones refine
        tickets[srv.submit(ps[i].xy, ps[i].seg, Bs[i])] = i
    got = drain(srv)
    assert sorted(got) == sorted(tickets)
    for t, i in tickets.items():
        info, res = got[t]
        assert info["status"] == 0
        assert info["t_submit_ms"] <= info["t_admit_ms"] <= info["t_done_ms"]
        same(oracle, res, alone(gdp, ps[i], Bs[i]))
        assert_valid(oracle.check(*res, ps[i].seg, ps[i].n, B=Bs[i]))
    srv.close()


def test_admission_waits_for_memory(oracle):
    """A pool with room for about one request at a time still serves them all,
    one after another, with the same results."""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    ps = [W.square_pslg(2000, 40, 400 + i) for i in range(4)]
    # one 2000-point request needs 2 (n + 7 + 3n + 64 m + 1024) + 16 slots
    need = 2 * (2000 + 7 + 3 * 2000 + 64 * 44 + 1024) + 16
    srv = gdp.Server(need + need // 2, need, 256, 8)
    tickets = {srv.submit(p.xy, p.seg, SQ2): i for i, p in enumerate(ps)}
    w, l, d = srv.step()
    assert l <= 1 and w >= 2
    got = drain(srv)
    for t, i in tickets.items():
        assert got[t][0]["status"] == 0
        same(oracle, got[t][1], alone(gdp, ps[i], SQ2))
    srv.close()


def test_request_too_large_is_refused():
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(5000, 50, 9)
    srv = gdp.Server(1 << 12, 1 << 12, 64, 4)
    with pytest.raises(gdp.GdpError) as e:
        srv.submit(p.xy, p.seg, SQ2)
    assert e.value.status == gdp.ERR_NOMEM
    srv.close()


def test_invalid_request_fails_alone(oracle):
    """A request with an invalid input (crossing segments) fails with
    GDP_ERR_INPUT; requests staged with it are not affected."""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    good = [W.square_pslg(1500, 30, 700 + i) for i in range(3)]
    bad_xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [0.2, 0.2], [0.8, 0.8], [0.2, 0.8], [0.8, 0.2]], float)
    bad_seg = np.array([[0, 1], [1, 2], [2, 3], [3, 0], [4, 5], [6, 7]], np.int32)
    srv = gdp.Server(1 << 20, 1 << 19, 1 << 12, 16)
    tg = [srv.submit(good[0].xy, good[0].seg, SQ2), srv.submit(bad_xy, bad_seg, SQ2),
          srv.submit(good[1].xy, good[1].seg, SQ2), srv.submit(good[2].xy, good[2].seg, 1.5)]
    got = drain(srv)
    assert got[tg[1]][0]["status"] == gdp.ERR_INPUT
    for t, p, B in ((tg[0], good[0], SQ2), (tg[2], good[1], SQ2), (tg[3], good[2], 1.5)):
        assert got[t][0]["status"] == 0
        same(oracle, got[t][1], alone(gdp, p, B))
    srv.close()
