"""Slots that run out during refinement (the loop of Algorithm 1 inserts as
many Steiner points as the bounds demand, which no starting capacity can
know): the pool is laid out again with more room for the mesh and the
refinement goes on, with the result it would have had with room from the
start; when no more room can be had the mesh stops with GDP_ERR_NOMEM and is
still a valid CDT."""
import numpy as np
import pytest

from tests.gpu_util import SQ2, assert_valid, need_gpu

pytestmark = pytest.mark.gpu

SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
BOUNDARY = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)


def test_unit_square_outgrows_its_slots(oracle):
    """4 points, 4 segments: room for 1,292 Steiner points at the start; the
    edge-length bound l = 0.01 (Sec. 4.1) needs about 25,000"""
    gdp = need_gpu()
    g = gdp.Mesh(SQUARE, BOUNDARY)
    st = g.refine(SQ2, max_len=0.01)
    assert st["grow_steps"] >= 4
    assert all(v == 0 for v in g.check().values()), g.check()
    xy, tri, sub = g.export()
    rep = oracle.check(xy, tri, sub, BOUNDARY, 4, B=SQ2)
    assert_valid(rep)
    assert abs(rep["area_sum"] - 1.0) < 1e-12
    assert max(np.hypot(*(xy[tri[:, (k + 1) % 3]] - xy[tri[:, k]]).T).max() for k in range(3)) <= 0.01
    # an empty square under a length bound is where the sequential order
    # matters most (worst ratio first: 24,965 points; FIFO and largest area
    # first, the paper's priority of Sec. 4.3: 33,021): compare with each
    counts = []
    for order in (0, 1, 2):
        o = oracle.Mesh(SQUARE, BOUNDARY)
        assert o.refine_len(SQ2, 0.01, order=order) == 0
        counts.append(o.n_steiner)
    assert min(abs(st["n_steiner"] - c) / c for c in counts) <= 0.10, (st["n_steiner"], counts)


def test_growth_does_not_change_the_result(monkeypatch):
    """the same PSLG refined with room from the start and with almost none:
    identical meshes (mesh-local slot order survives the moves)"""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(3000, 60, 31)
    out = []
    for per_point in ("3", "0"):
        monkeypatch.setenv("GDP_STEINER_PER_POINT", per_point)
        monkeypatch.setenv("GDP_STEINER_PER_SEGMENT", "64" if per_point == "3" else "0")
        g = gdp.Mesh(p.xy, p.seg)
        st = g.refine(SQ2)
        xy, tri, sub = g.export()
        out.append((st["grow_steps"], st["n_steiner"], xy.tobytes(), tri.tobytes(), sub.tobytes()))
    assert out[0][0] == 0 and out[1][0] >= 1
    assert out[0][1:] == out[1][1:]


def test_batch_with_growth_equals_alone_runs(monkeypatch):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    monkeypatch.setenv("GDP_STEINER_PER_POINT", "0")
    monkeypatch.setenv("GDP_STEINER_PER_SEGMENT", "0")
    pslgs = [W.square_pslg(n, m, 500 + n) for n, m in ((300, 6), (2000, 40), (800, 16))]
    pslgs.append(W.PSLG(xy=SQUARE.copy(), seg=BOUNDARY.copy(), name="square"))
    b = gdp.Batch([(p.xy, p.seg) for p in pslgs])
    st = b.refine(SQ2, max_len=0.03)
    assert st["grow_steps"] >= 1
    assert (b.info()["status"] == 0).all()
    for k, p in enumerate(pslgs):
        g = gdp.Mesh(p.xy, p.seg)
        g.refine(SQ2, max_len=0.03)
        xy1, tri1, sub1 = g.export()
        xy2, tri2, sub2 = b.export(k)
        assert np.array_equal(xy1, xy2) and np.array_equal(tri1, tri2) and np.array_equal(sub1, sub2), k


def test_no_room_is_nomem_and_a_valid_cdt(oracle, monkeypatch):
    """no Steiner room and growth switched off: GDP_ERR_NOMEM, and the mesh is
    still a valid CDT (not refined) that exports"""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    monkeypatch.setenv("GDP_STEINER_PER_POINT", "0")
    monkeypatch.setenv("GDP_STEINER_PER_SEGMENT", "0")
    monkeypatch.setenv("GDP_GROW_LIMIT", "0")
    p = W.square_pslg(2000, 40, 77)
    g = gdp.Mesh(p.xy, p.seg)
    status, st = g.refine(SQ2, check=False)
    assert status == gdp.ERR_NOMEM
    assert 0 < st["n_steiner"] <= 1024
    assert all(v == 0 for v in g.check().values()), g.check()
    xy, tri, sub = g.export()
    assert len(xy) == p.n + st["n_steiner"]
    assert_valid(oracle.check(xy, tri, sub, p.seg, p.n, B=SQ2), refined=False)
