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
