"""gdp_scan_noalloc: the scan for callers that cannot allocate device memory
(see include/gdp.h).  Its output must equal gdp_mesh_scan's on the same
triangulation -- the same fixed-order FP64 formulas, so bit for bit -- on two
calls in a row that share the library's static scratch array.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import math

import numpy as np
import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def as_set(kind, verts, pt, meas):
    """entries as a sorted multiset (a subsegment encroached from both sides
    appears twice, once per side)"""
    out = []
    for k in range(len(kind)):
        v = tuple(int(x) for x in verts[k])
        if kind[k] == 1:
            v = (min(v[0], v[1]), max(v[0], v[1]), -1)
        out.append((int(kind[k]), v, float(pt[k][0]), float(pt[k][1]), int(meas[k]) & 0xffffffff))
    return sorted(out)


@pytest.mark.parametrize("B", [math.sqrt(2.0), 1.5])
def test_noalloc_scan_matches_mesh_scan(B):
    gdp = need_gpu()
    import torch
    from paper_2007_00324_gb300 import workloads as W
    p = W.square_pslg(3000, 80, 99)
    mesh = gdp.Mesh(p.xy, p.seg)
    xy, tri, sub = mesh.export()
    want = as_set(*mesh.scan(B))
    assert len(want) > 100
    # the caller's own device buffers: triangles with subsegment flags
    subs = {(min(a, b), max(a, b)) for a, b, _ in sub.tolist()}
    t4 = np.zeros((len(tri), 4), np.int32)
    t4[:, :3] = tri
    for e in range(3):
        u, v = tri[:, (e + 1) % 3], tri[:, (e + 2) % 3]
        flag = np.array([(min(a, b), max(a, b)) in subs for a, b in zip(u.tolist(), v.tolist())])
        t4[:, 3] |= flag.astype(np.int32) << e
    dev = torch.device("cuda", 0)
    xy_d = torch.from_numpy(np.ascontiguousarray(xy)).to(dev)
    t4_d = torch.from_numpy(t4).to(dev)
    cap = len(want) + 64
    for call in range(2):
        kind = torch.full((cap,), -7, dtype=torch.int32, device=dev)
        verts = torch.full((cap, 3), -7, dtype=torch.int32, device=dev)
        pt = torch.zeros((cap, 2), dtype=torch.float64, device=dev)
        meas = torch.zeros((cap,), dtype=torch.int32, device=dev)
        n = gdp.scan_noalloc(xy_d, t4_d, B, kind, verts, pt, meas)
        assert n == len(want), (call, n, len(want))
        got = as_set(kind[:n].cpu().numpy(), verts[:n].cpu().numpy(), pt[:n].cpu().numpy(),
                     meas[:n].cpu().numpy().view(np.uint32))
        assert got == want, call
        assert int(kind[n:].min()) == -7   # nothing written past the count


def test_noalloc_rejects_oversize_and_bad_ids():
    gdp = need_gpu()
    import torch
    dev = torch.device("cuda", 0)
    xy = torch.zeros((3, 2), dtype=torch.float64, device=dev)
    xy[1, 0] = 1.0
    xy[2, 1] = 1.0
    t4 = torch.tensor([[0, 1, 5, 0]], dtype=torch.int32, device=dev)   # vertex 5 out of range
    out_i = torch.zeros((4,), dtype=torch.int32, device=dev)
    out_v = torch.zeros((4, 3), dtype=torch.int32, device=dev)
    out_p = torch.zeros((4, 2), dtype=torch.float64, device=dev)
    with pytest.raises(gdp.GdpError) as e:
        gdp.scan_noalloc(xy, t4, 1.5, out_i, out_v, out_p, out_i)
    assert e.value.status == gdp.ERR_INPUT
    # a point buffer that is 8- but not 16-byte aligned: refused before any launch
    ok_t4 = torch.tensor([[0, 1, 2, 0]], dtype=torch.int32, device=dev)
    pbuf = torch.zeros((9,), dtype=torch.float64, device=dev)
    L = gdp.load()
    cnt = gdp.C.c_int64()
    st = L.gdp_scan_noalloc(gdp.C.c_void_p(xy.data_ptr()), 3, gdp.C.c_void_p(ok_t4.data_ptr()), 1, 1.5,
                            gdp.C.c_void_p(out_i.data_ptr()), gdp.C.c_void_p(out_v.data_ptr()),
                            gdp.C.c_void_p(pbuf.data_ptr() + 8), gdp.C.c_void_p(out_i.data_ptr()), 4,
                            gdp.C.byref(cnt), None)
    assert st == gdp.ERR_INPUT
    big = torch.zeros(((1 << 22) + 1, 4), dtype=torch.int32, device=dev)
    with pytest.raises(gdp.GdpError) as e:
        gdp.scan_noalloc(xy, big, 1.5, out_i, out_v, out_p, out_i)
    assert e.value.status == gdp.ERR_CAPACITY
