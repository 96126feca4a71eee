"""The cavity-growth and insertion kernels come in three forms that must give
the same mesh bit for bit (Sec. 5.3, the tuple-list expansion, and Sec. 4.3,
the retriangulation): one warp per candidate (k_grow_w / k_insert_w, the
default up to GDP_WARP_GROW_MAX candidates), groups of lanes above it (four
cavities per warp grown by groups of eight lanes, k_grow_g, and eight written
by groups of four, k_insert_g) and one thread per candidate (k_grow_t /
k_insert_t, GDP_GROW_GROUP=0); the warp-batched growth (k_grow_b,
GDP_GROW_GROUP=2) grows the cavities of a warp's 32 candidates from one
shared tuple list.  Setting
GDP_WARP_GROW_MAX=1 sends every iteration to the group or thread kernels, so
the small inputs here cover all of their paths: spill tiers, circumcentres
that give way to a subsegment's split point, Chew's lenses and Flip-Flop.
"""
import numpy as np
import pytest

from tests.gpu_util import SQ2, need_gpu

pytestmark = pytest.mark.gpu

KERNELS = (
    {},                                                   # warp per candidate
    {"GDP_WARP_GROW_MAX": "1"},                           # warp-batched growth (default)
    {"GDP_WARP_GROW_MAX": "1", "GDP_GROW_GROUP": "1"},    # lane groups
    {"GDP_WARP_GROW_MAX": "1", "GDP_GROW_GROUP": "0"},    # thread per candidate
)


def refine_with(monkeypatch, gdp, p, env, flags=0, B=SQ2):
    for k in ("GDP_WARP_GROW_MAX", "GDP_GROW_GROUP"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    g = gdp.Mesh(p.xy, p.seg)
    st = g.refine(B, flags=flags)
    assert all(v == 0 for v in g.check().values()), g.check()
    return g.export(), st


def inputs(W, name):
    if name == "square":
        return W.square_pslg(6_000, 120, 515)
    if name == "fans":
        return W.paper_shaped(n_uniform=3000, n_gauss=1500, n_circle=1000, n_seg=60, n_fans=6, seed=4711)
    return W.contours(n_hills=5, levels=6, per_curve=80, seed=99)


@pytest.mark.parametrize("name,flag", [("square", 0), ("fans", 0), ("contours", "chew"), ("fans", "flipflop")])
def test_growth_kernel_forms_agree(monkeypatch, name, flag):
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    p = inputs(W, name)
    flags = {0: 0, "chew": gdp.REFINE_CHEW, "flipflop": gdp.REFINE_FLIPFLOP}[flag]
    runs = [refine_with(monkeypatch, gdp, p, env, flags) for env in KERNELS]
    (xy0, tri0, sub0), st0 = runs[0]
    assert st0["n_steiner"] > 0
    for (xy, tri, sub), st in runs[1:]:
        assert st["n_steiner"] == st0["n_steiner"]
        assert st["grown"] == st0["grown"] and st["cavity_tris"] == st0["cavity_tris"]
        assert np.array_equal(xy, xy0)
        assert np.array_equal(tri, tri0)
        assert np.array_equal(sub, sub0)


def test_lockstep_groups_on_a_batch(monkeypatch):
    """a batch mixes meshes in one candidate list, so the four groups of a warp
    grow cavities of different meshes; each mesh must still equal its alone run"""
    gdp = need_gpu()
    from paper_2007_00324_gb300 import workloads as W
    monkeypatch.setenv("GDP_WARP_GROW_MAX", "1")
    pslgs = [W.square_pslg(n, m, 700 + n) for n, m in ((700, 12), (3000, 60), (1800, 40))]
    alone = []
    for p in pslgs:
        g = gdp.Mesh(p.xy, p.seg)
        g.refine(SQ2)
        alone.append(g.export())
    b = gdp.Batch([(p.xy, p.seg) for p in pslgs])
    b.refine(SQ2)
    assert (b.info()["status"] == 0).all()
    for k in range(len(pslgs)):
        assert all(np.array_equal(x, y) for x, y in zip(alone[k], b.export(k))), k
