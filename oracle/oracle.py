"""Python access to the sequential CPU oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg, never by the product package.  The oracle
shares no code with the CUDA path.

The oracle follows the paper's definitions (Sec. 4: PSLG, CDT, subsegment,
encroachment, bad triangle; Sec. 5.2: cavity insertion; Sec. 7: exact
predicates with simulation of simplicity) and runs plain sequential Ruppert
refinement.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["exact.c", "pred.c", "mesh.c", "ruppert.c", "check.c", "capi.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INPUT, NOMEM, LIMIT, INTERNAL = 0, 1, 2, 3, 5


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, no FP contraction: the FP64
    formulas are a bit-exact specification)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    hdrs = [os.path.join(_HERE, h) for h in ("oracle.h", "mesh_int.h")]
    if not force and os.path.exists(_LIB_PATH):
        mt = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= mt for s in srcs + hdrs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Report(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "n_tri", "n_vert", "n_sub", "bad_orient", "bad_adjacency", "open_not_sub",
        "sub_not_edge", "seg_not_covered", "not_locally_cd", "bf_cd_violations",
        "bad_quality", "exempt_bad", "encroached", "euler_defect", "inputs_missing")] + [
        ("min_angle_deg", C.c_double), ("area_sum", C.c_double), ("bad_area", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            d, i32, i64, vp = C.c_double, C.c_int32, C.c_int64, C.c_void_p
            L.or_set_filter.argtypes = [C.c_int]
            for n in ("or_orient",):
                getattr(L, n).argtypes = [d] * 6
                getattr(L, n).restype = C.c_int
            for n in ("or_incircle", "or_incircle_sos"):
                getattr(L, n).argtypes = [d] * 8
                getattr(L, n).restype = C.c_int
            L.or_dot_sign.argtypes = [d] * 6
            L.or_dot_sign.restype = C.c_int
            L.or_lens_sign.argtypes = [d] * 6
            L.or_lens_sign.restype = C.c_int
            L.or_is_bad.argtypes = [d] * 7
            L.or_is_bad.restype = C.c_int
            L.or_circumcenter.argtypes = [d] * 6 + [C.POINTER(d), C.POINTER(d)]
            L.or_midpoint.argtypes = [d] * 4 + [C.POINTER(d), C.POINTER(d)]
            L.or_measure_bits.argtypes = [d]
            L.or_measure_bits.restype = C.c_uint32
            L.or_cdt_create.argtypes = [vp, i64, vp, i64, C.POINTER(C.c_int)]
            L.or_cdt_create.restype = vp
            L.or_destroy.argtypes = [vp]
            L.or_refine.argtypes = [vp, d, i64, C.c_int]
            L.or_refine.restype = C.c_int
            L.or_refine_len.argtypes = [vp, d, d, i64, C.c_int]
            L.or_refine_len.restype = C.c_int
            L.or_refine_mode.argtypes = [vp, d, d, C.c_int, i64, C.c_int]
            L.or_refine_mode.restype = C.c_int
            L.or_is_long.argtypes = [d] * 7
            L.or_is_long.restype = C.c_int
            L.or_insert_points.argtypes = [vp, vp, i64]
            L.or_insert_points.restype = C.c_int
            L.or_split_subsegments.argtypes = [vp, vp, i64]
            L.or_split_subsegments.restype = C.c_int
            for n in ("or_n_vertices", "or_n_triangles", "or_n_subsegments", "or_n_steiner"):
                getattr(L, n).argtypes = [vp]
                getattr(L, n).restype = i64
            L.or_export.argtypes = [vp, vp, vp, vp]
            L.or_check.argtypes = [vp, i64, vp, i64, vp, i64, vp, i64, i64, d, C.c_int,
                                   C.POINTER(Report)]
            L.or_check.restype = C.c_int
            L.or_check_mode.argtypes = [vp, i64, vp, i64, vp, i64, vp, i64, i64, d, C.c_int, C.c_int,
                                        C.POINTER(Report)]
            L.or_check_mode.restype = C.c_int
            L.or_eval_tris.argtypes = [vp, vp, i64, d, vp, vp, vp]
            L.or_eval_subs.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp]
            L.or_eval_subs_mode.argtypes = [vp, vp, i64, vp, i64, C.c_int, vp, vp, vp]
            L.or_split_point.argtypes = [d, d, d, d, C.c_int, C.c_int, C.POINTER(d), C.POINTER(d)]
            L.or_small_angle.argtypes = [d] * 6
            L.or_small_angle.restype = C.c_int
            L.or_exempt_query.argtypes = [vp, i64, i64, i64]
            L.or_exempt_query.restype = C.c_int
            L.or_eval_exempt.argtypes = [vp, i64, vp, i64, vp, i64, vp, i64, i64, d, vp]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------- predicates ----------------
def set_filter(on: bool):
    lib().or_set_filter(1 if on else 0)


def orient(a, b, c):
    return lib().or_orient(*a, *b, *c)


def incircle(a, b, c, d):
    return lib().or_incircle(*a, *b, *c, *d)


def incircle_sos(a, b, c, d):
    return lib().or_incircle_sos(*a, *b, *c, *d)


def dot_sign(a, b, p):
    return lib().or_dot_sign(*a, *b, *p)


def lens_sign(a, b, p):
    """-1: p strictly inside the diametral lens of ab (Chew's rule, Sec. 4.2),
    0: p is a or b, +1: outside"""
    return lib().or_lens_sign(*a, *b, *p)


def is_bad(a, b, c, B2):
    return bool(lib().or_is_bad(*a, *b, *c, B2))


def circumcenter(a, b, c):
    x, y = C.c_double(), C.c_double()
    lib().or_circumcenter(*a, *b, *c, C.byref(x), C.byref(y))
    return x.value, y.value


def midpoint(a, b):
    x, y = C.c_double(), C.c_double()
    lib().or_midpoint(*a, *b, C.byref(x), C.byref(y))
    return x.value, y.value


def measure_bits(v):
    return lib().or_measure_bits(v)


def split_point(a, b, apex_a=False, apex_b=False):
    """C6: the midpoint of ab, or the concentric-shell point when exactly one
    endpoint is an apex (an input vertex with a small input angle)"""
    x, y = C.c_double(), C.c_double()
    lib().or_split_point(*a, *b, 1 if apex_a else 0, 1 if apex_b else 0, C.byref(x), C.byref(y))
    return x.value, y.value


def small_angle(o, p, q):
    """the angle at o between the directions to p and q is below 60 degrees"""
    return bool(lib().or_small_angle(*o, *p, *q))


def eval_exempt(xy, tri, sub, seg_in, n_in, B2):
    """per triangle: 1 if it is bad (C1) and accepted by the small-angle
    exemption (C10)"""
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
    sub = np.ascontiguousarray(sub, np.int32).reshape(-1, 3)
    seg_in = np.ascontiguousarray(seg_in, np.int32).reshape(-1, 2)
    out = np.zeros(len(tri), np.int32)
    lib().or_eval_exempt(_p(xy), len(xy), _p(tri), len(tri), _p(sub), len(sub), _p(seg_in), len(seg_in),
                         int(n_in), B2, _p(out))
    return out


# ---------------- meshes ----------------
class Mesh:
    """Oracle CDT of a PSLG; refine() runs sequential Ruppert refinement."""

    def __init__(self, xy, seg):
        self.xy_in = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self.seg_in = np.ascontiguousarray(seg, dtype=np.int32).reshape(-1, 2)
        st = C.c_int(0)
        self._h = lib().or_cdt_create(_p(self.xy_in), len(self.xy_in), _p(self.seg_in),
                                      len(self.seg_in), C.byref(st))
        self.status = st.value
        if not self._h:
            raise ValueError(f"oracle CDT failed with status {st.value}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def refine(self, B: float, max_steiner: int = 1 << 40, order: int = 0) -> int:
        return lib().or_refine(self._h, B, max_steiner, order)

    def refine_len(self, B: float, l: float, max_steiner: int = 1 << 40, order: int = 0) -> int:
        """refinement with the edge-length bound l as well (l <= 0: none)"""
        return lib().or_refine_len(self._h, B, l, max_steiner, order)

    def refine_mode(self, B: float, l: float = 0.0, lens: bool = False, max_steiner: int = 1 << 40,
                    order: int = 0) -> int:
        """refinement with the encroachment region chosen: the diametral circle
        (Ruppert's rule) or, with lens, the diametral lens (Chew's rule)"""
        return lib().or_refine_mode(self._h, B, l, 1 if lens else 0, max_steiner, order)

    def insert_points(self, xy) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        return lib().or_insert_points(self._h, _p(xy), len(xy))

    def exempt(self, a: int, b: int, c: int) -> int:
        """C10 on three vertices (export ids): 1 exempt, 0 not, -1 bad id"""
        return lib().or_exempt_query(self._h, a, b, c)

    def split_subsegments(self, abxy) -> int:
        abxy = np.ascontiguousarray(abxy, dtype=np.float64).reshape(-1, 4)
        return lib().or_split_subsegments(self._h, _p(abxy), len(abxy))

    @property
    def n_steiner(self) -> int:
        return lib().or_n_steiner(self._h)

    def export(self):
        L = lib()
        nv, nt, ns = L.or_n_vertices(self._h), L.or_n_triangles(self._h), L.or_n_subsegments(self._h)
        xy = np.zeros((nv, 2), np.float64)
        tri = np.zeros((nt, 3), np.int32)
        sub = np.zeros((ns, 3), np.int32)
        L.or_export(self._h, _p(xy), _p(tri), _p(sub))
        return xy, tri, sub


def is_long(a, b, c, L2):
    return lib().or_is_long(a[0], a[1], b[0], b[1], c[0], c[1], L2)


def check(xy, tri, sub, seg_in, n_in, B=None, brute=False, lens=False) -> dict:
    """Invariant report for any mesh (see oracle/check.c); lens: encroachment
    against the diametral lens (Chew's rule) instead of the diametral circle."""
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
    sub = np.ascontiguousarray(sub, np.int32).reshape(-1, 3)
    seg_in = np.ascontiguousarray(seg_in, np.int32).reshape(-1, 2)
    rep = Report()
    lib().or_check_mode(_p(xy), len(xy), _p(tri), len(tri), _p(sub), len(sub), _p(seg_in),
                        len(seg_in), int(n_in), (B * B) if B else 0.0, 1 if brute else 0,
                        1 if lens else 0, C.byref(rep))
    return rep.as_dict()


def eval_tris(xy, tri, B2):
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
    n = len(tri)
    bad = np.zeros(n, np.int32)
    cc = np.zeros((n, 2), np.float64)
    meas = np.zeros(n, np.uint32)
    lib().or_eval_tris(_p(xy), _p(tri), n, B2, _p(bad), _p(cc), _p(meas))
    return bad, cc, meas


def eval_subs(xy, tri, sub, lens=False):
    """per subsegment: encroached by an adjacent apex (diametral circle, or the
    diametral lens with lens), its midpoint and priority measure"""
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
    sub = np.ascontiguousarray(sub, np.int32).reshape(-1, 3)
    n = len(sub)
    enc = np.zeros(n, np.int32)
    mid = np.zeros((n, 2), np.float64)
    meas = np.zeros(n, np.uint32)
    lib().or_eval_subs_mode(_p(xy), _p(tri), len(tri), _p(sub), n, 1 if lens else 0, _p(enc), _p(mid),
                            _p(meas))
    return enc, mid, meas


def triangle_set(xy, tri):
    """Triangles as a set of coordinate triples (rotation-normalised, CCW kept),
    independent of vertex numbering."""
    xy = np.asarray(xy, np.float64).reshape(-1, 2)
    tri = np.asarray(tri).reshape(-1, 3)
    out = set()
    for t in tri:
        pts = [tuple(xy[i].tolist()) for i in t]
        k = min(range(3), key=lambda i: pts[i])
        out.add((pts[k], pts[(k + 1) % 3], pts[(k + 2) % 3]))
    return out
