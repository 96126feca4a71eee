"""Edge-length criterion of the oracle (Sec. 4.1: an edge-length bound l
beside the angle bound): closed forms of the test, and refined meshes whose
longest edge is at most l while every other invariant still holds."""
import math

import numpy as np
import pytest

SQ2 = math.sqrt(2.0)


def longest(xy, tri):
    e = np.concatenate([xy[tri[:, (k + 1) % 3]] - xy[tri[:, k]] for k in range(3)])
    return float(np.sqrt((e ** 2).sum(1).max()))


def test_is_long_closed_forms(oracle):
    # right isosceles triangle with unit legs: longest edge squared is exactly 2
    a, b, c = (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)
    assert oracle.is_long(a, b, c, 1.99) == 1
    assert oracle.is_long(a, b, c, 2.0) == 0      # strict: equal is not too long
    assert oracle.is_long(c, a, b, 1.99) == 1      # any vertex order
    # 3-4-5 triangle: 25
    assert oracle.is_long((0, 0), (4, 0), (0, 3), 24.999) == 1
    assert oracle.is_long((0, 0), (4, 0), (0, 3), 25.0) == 0


@pytest.mark.parametrize("l", [0.5, 0.2, 0.07])
def test_square_refined_to_length(oracle, l):
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    seg = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)
    m = oracle.Mesh(xy, seg)
    assert m.refine_len(SQ2, l) == 0
    oxy, tri, sub = m.export()
    assert longest(oxy, tri) <= l
    rep = oracle.check(oxy, tri, sub, seg, 4, B=SQ2)
    for k in ("bad_orient", "bad_adjacency", "not_locally_cd", "seg_not_covered", "bad_quality",
              "encroached", "euler_defect"):
        assert rep[k] == 0, (k, rep[k])
    assert math.isclose(rep["area_sum"], 1.0, rel_tol=1e-12)


def test_length_bound_monotone_and_inf_is_none(oracle):
    from paper_2007_00324_gb300 import workloads as W
    p = W.contours(3, 5, 40, 11)
    counts = []
    for l in (0.0, math.inf, 0.2, 0.1, 0.05):
        m = oracle.Mesh(p.xy, p.seg)
        assert m.refine_len(1.462, l if math.isfinite(l) else 1e300) == 0
        xy, tri, sub = m.export()
        if 0 < l < math.inf:
            assert longest(xy, tri) <= l
        counts.append(m.n_steiner)
    assert counts[0] == counts[1]                 # no bound == infinite bound
    assert counts[1] <= counts[2] <= counts[3] <= counts[4]


def test_contours_are_a_valid_pslg(oracle):
    from paper_2007_00324_gb300 import workloads as W
    p = W.contours(4, 6, 50, 3)
    m = oracle.Mesh(p.xy, p.seg)
    xy, tri, sub = m.export()
    rep = oracle.check(xy, tri, sub, p.seg, p.n, brute=True)
    for k in ("bad_orient", "bad_adjacency", "seg_not_covered", "not_locally_cd", "bf_cd_violations",
              "inputs_missing"):
        assert rep[k] == 0, (k, rep[k])
