"""Thin ctypes binding of libgdp.so (include/gdp.h), same names as the C ABI.

Only argument marshalling happens here; every step of the CDT and of the
refinement runs in the library's CUDA kernels.  There is no fallback: if the
library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_INPUT, ERR_NOMEM, ERR_ITER_LIMIT, ERR_WALK_LIMIT, ERR_CUDA, ERR_INTERNAL, ERR_CAPACITY = range(8)


class GdpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


class RefineOpts(C.Structure):
    _fields_ = [("B", C.c_double), ("max_len", C.c_double), ("max_iter", C.c_int32),
                ("cand_cap", C.c_int32), ("graph_iters", C.c_int32), ("flags", C.c_int32),
                ("cand_block", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_in_pts", C.c_int64), ("n_steiner", C.c_int64), ("n_tris", C.c_int64),
                ("n_subsegs", C.c_int64), ("iterations", C.c_int64), ("candidates", C.c_int64),
                ("inserted", C.c_int64), ("cdt_rounds", C.c_int64), ("refine_ms", C.c_double),
                ("cdt_ms", C.c_double), ("launches", C.c_int64), ("grown", C.c_int64),
                ("cavity_tris", C.c_int64), ("cavity_edges", C.c_int64), ("walk_steps", C.c_int64),
                ("grow_ms", C.c_double), ("grow_launches", C.c_int64), ("timed_grown", C.c_int64),
                ("timed_cavity_tris", C.c_int64), ("timed_cavity_edges", C.c_int64),
                ("timed_walk_steps", C.c_int64), ("grow_steps", C.c_int64), ("flips", C.c_int64),
                ("flops", C.c_int64), ("redundant_removed", C.c_int64), ("setups", C.c_int64),
                ("timed_setups", C.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


SYMBOLS = ["gdp_mesh_create", "gdp_mesh_create_device", "gdp_mesh_refine", "gdp_mesh_export",
           "gdp_mesh_insert_points", "gdp_mesh_split_subsegments", "gdp_mesh_scan", "gdp_mesh_scan_mode",
           "gdp_mesh_stats", "gdp_mesh_check", "gdp_mesh_profile", "gdp_mesh_kernel_time", "gdp_mesh_destroy",
           "gdp_batch_create", "gdp_batch_refine",
           "gdp_batch_info", "gdp_batch_export", "gdp_batch_destroy", "gdp_scan_noalloc",
           "gdp_autotune", "gdp_server_create", "gdp_server_submit", "gdp_server_step", "gdp_server_result",
           "gdp_server_destroy", "gdp_measure_fp64_peak", "gdp_status_str"]


def load(build_if_missing: bool = True):
    """Load libgdp.so (building it in-tree if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libgdp.so is missing: run paper_2007_00324_gb300.build")
            L = C.CDLL(path)
            vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            L.gdp_mesh_create.argtypes = [vp, i64, vp, i64, vp, C.POINTER(vp)]
            L.gdp_mesh_create_device.argtypes = [vp, i64, vp, i64, vp, C.POINTER(vp)]
            L.gdp_mesh_refine.argtypes = [vp, C.POINTER(RefineOpts), C.POINTER(Stats)]
            L.gdp_mesh_export.argtypes = [vp, vp, i64, vp, i64, vp, i64, C.POINTER(i64),
                                          C.POINTER(i64), C.POINTER(i64)]
            L.gdp_mesh_insert_points.argtypes = [vp, vp, i64]
            L.gdp_mesh_split_subsegments.argtypes = [vp, vp, i64]
            L.gdp_mesh_scan.argtypes = [vp, d, vp, vp, vp, vp, i64, C.POINTER(i64)]
            L.gdp_mesh_scan_mode.argtypes = [vp, d, i32, vp, vp, vp, vp, i64, C.POINTER(i64)]
            L.gdp_mesh_stats.argtypes = [vp, C.POINTER(Stats)]
            L.gdp_mesh_check.argtypes = [vp, vp]
            L.gdp_mesh_profile.argtypes = [vp, C.c_int]
            L.gdp_mesh_kernel_time.argtypes = [vp, i32, C.c_char_p, i64, C.POINTER(d), C.POINTER(i64)]
            L.gdp_mesh_destroy.argtypes = [vp]
            L.gdp_mesh_destroy.restype = None
            L.gdp_batch_create.argtypes = [vp, vp, vp, vp, i32, vp, C.POINTER(vp)]
            L.gdp_batch_refine.argtypes = [vp, vp, C.POINTER(RefineOpts), C.POINTER(Stats)]
            L.gdp_batch_info.argtypes = [vp, vp, vp, vp, vp, vp]
            L.gdp_batch_export.argtypes = [vp, i32, vp, i64, vp, i64, vp, i64, C.POINTER(i64),
                                           C.POINTER(i64), C.POINTER(i64)]
            L.gdp_batch_destroy.argtypes = [vp]
            L.gdp_batch_destroy.restype = None
            L.gdp_scan_noalloc.argtypes = [vp, i64, vp, i64, d, vp, vp, vp, vp, i64,
                                           C.POINTER(i64), vp]
            L.gdp_autotune.argtypes = [vp, vp, vp, vp, i32, vp, C.POINTER(RefineOpts), vp,
                                       C.POINTER(RefineOpts), vp, i32]
            L.gdp_server_create.argtypes = [i64, i64, i64, i32, C.POINTER(RefineOpts), vp, C.POINTER(vp)]
            L.gdp_server_submit.argtypes = [vp, vp, i64, vp, i64, d, C.POINTER(i64)]
            L.gdp_server_step.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
            L.gdp_server_result.argtypes = [vp, C.POINTER(ResultInfo), vp, i64, vp, i64, vp, i64]
            L.gdp_server_destroy.argtypes = [vp]
            L.gdp_server_destroy.restype = None
            L.gdp_measure_fp64_peak.argtypes = [vp, C.POINTER(d)]
            L.gdp_status_str.argtypes = [C.c_int]
            L.gdp_status_str.restype = C.c_char_p
            for n in SYMBOLS:
                if n not in ("gdp_mesh_destroy", "gdp_batch_destroy", "gdp_server_destroy", "gdp_status_str"):
                    getattr(L, n).restype = C.c_int
            _lib = L
    return _lib


def measure_fp64_peak(stream=None) -> float:
    """gdp_measure_fp64_peak: the device's FP64 FMA throughput in TFLOP/s"""
    t = C.c_double()
    st = load().gdp_measure_fp64_peak(_stream_handle(stream), C.byref(t))
    if st != OK:
        raise GdpError(st, "gdp_measure_fp64_peak")
    return t.value


def status_str(s: int) -> str:
    try:
        return load(False).gdp_status_str(s).decode()
    except Exception:
        return str(s)


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


REFINE_TIME_GROW = 1   # gdp_refine_opts.flags: time the first k_grow launch pair of each replay
REFINE_CHEW = 2        # gdp_refine_opts.flags: encroachment by the diametral lens (Chew's rule)
REFINE_FLIPFLOP = 4    # gdp_refine_opts.flags: Flip-Flop insertion instead of cavity insertion


def _opts(B=math.sqrt(2.0), max_iter=0, cand_cap=0, graph_iters=0, flags=0, cand_block=0, max_len=0.0):
    return RefineOpts(B=B, max_len=max_len, max_iter=max_iter, cand_cap=cand_cap,
                      graph_iters=graph_iters, flags=flags, cand_block=cand_block)


def _stream_handle(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Mesh:
    """gdp_mesh: CDT of a PSLG built on the GPU, refined by gdp_mesh_refine."""

    def __init__(self, xy, seg, stream=None, device=False):
        L = load()
        self._h = C.c_void_p()
        if device:
            # xy, seg: torch CUDA tensors (float64 (n,2), int32 (m,2))
            n, m = int(xy.shape[0]), int(seg.shape[0])
            st = L.gdp_mesh_create_device(C.c_void_p(xy.data_ptr()), n,
                                          C.c_void_p(seg.data_ptr()) if m else None, m,
                                          _stream_handle(stream), C.byref(self._h))
            self.n_in = n
        else:
            xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
            seg = np.ascontiguousarray(seg, np.int32).reshape(-1, 2)
            self.n_in = len(xy)
            st = L.gdp_mesh_create(_p(xy), len(xy), _p(seg) if len(seg) else None, len(seg),
                                   _stream_handle(stream), C.byref(self._h))
        if st != OK:
            self.close()
            raise GdpError(st, "gdp_mesh_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gdp_mesh_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refine(self, B=math.sqrt(2.0), max_iter=0, cand_cap=0, graph_iters=0, check=True, flags=0,
               cand_block=0, max_len=0.0):
        s = Stats()
        o = _opts(B, max_iter, cand_cap, graph_iters, flags, cand_block, max_len)
        st = load().gdp_mesh_refine(self._h, C.byref(o), C.byref(s))
        if check and st != OK:
            raise GdpError(st, "gdp_mesh_refine")
        return s.as_dict() if check else (st, s.as_dict())

    def stats(self):
        s = Stats()
        load().gdp_mesh_stats(self._h, C.byref(s))
        return s.as_dict()

    def check(self):
        """device-side consistency counts (all zero for a valid mesh)"""
        c = np.zeros(5, np.int64)
        st = load().gdp_mesh_check(self._h, _p(c))
        if st != OK:
            raise GdpError(st, "gdp_mesh_check")
        return dict(zip(("not_mutual", "edge_mismatch", "flag_mismatch", "not_ccw", "open_not_sub"),
                        c.tolist()))

    def profile(self, enable=True):
        st = load().gdp_mesh_profile(self._h, 1 if enable else 0)
        if st != OK:
            raise GdpError(st, "gdp_mesh_profile")

    def kernel_times(self):
        """{kernel name: (total ms, launches)} recorded since profile(True)"""
        L = load()
        out = {}
        i = 0
        buf = C.create_string_buffer(128)
        while True:
            ms, cnt = C.c_double(), C.c_int64()
            if L.gdp_mesh_kernel_time(self._h, i, buf, 128, C.byref(ms), C.byref(cnt)) != OK:
                break
            out[buf.value.decode()] = (ms.value, cnt.value)
            i += 1
        return out

    def export(self, out=None):
        """(xy, tri, sub) as numpy arrays.  out: optional (xy, tri, sub) host
        arrays of at least the mesh's sizes (C-contiguous float64 (n,2), int32
        (t,3), int32 (s,3), e.g. views of pinned memory) to copy into; the
        returned arrays are then views of their leading rows."""
        L = load()
        n_pts, n_tri, n_seg = C.c_int64(), C.c_int64(), C.c_int64()
        if out is not None:   # one call: the library checks the capacities
            xy, tri, sub = out
            for a, dt, w in ((xy, np.float64, 2), (tri, np.int32, 3), (sub, np.int32, 3)):
                if a.dtype != dt or a.ndim != 2 or a.shape[1] != w or not a.flags.c_contiguous:
                    raise ValueError(f"export: out array {a.dtype} {a.shape} is not a C-contiguous (n, {w}) {dt}")
        else:
            st = L.gdp_mesh_export(self._h, None, 0, None, 0, None, 0, C.byref(n_pts), C.byref(n_tri),
                                   C.byref(n_seg))
            if st != OK:
                raise GdpError(st, "gdp_mesh_export")
            xy = np.zeros((n_pts.value, 2), np.float64)
            tri = np.zeros((n_tri.value, 3), np.int32)
            sub = np.zeros((n_seg.value, 3), np.int32)
        st = L.gdp_mesh_export(self._h, _p(xy), len(xy), _p(tri), len(tri), _p(sub), len(sub),
                               C.byref(n_pts), C.byref(n_tri), C.byref(n_seg))
        if st != OK:
            raise GdpError(st, "gdp_mesh_export")
        return xy[:n_pts.value], tri[:n_tri.value], sub[:n_seg.value]

    def insert_points(self, xy):
        xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
        st = load().gdp_mesh_insert_points(self._h, _p(xy), len(xy))
        if st != OK:
            raise GdpError(st, "gdp_mesh_insert_points")

    def split_subsegments(self, abxy):
        abxy = np.ascontiguousarray(abxy, np.float64).reshape(-1, 4)
        st = load().gdp_mesh_split_subsegments(self._h, _p(abxy), len(abxy))
        if st != OK:
            raise GdpError(st, "gdp_mesh_split_subsegments")

    def scan(self, B=math.sqrt(2.0), cap=None, flags=0):
        L = load()
        cnt = C.c_int64()
        st = L.gdp_mesh_scan_mode(self._h, B, flags, None, None, None, None, 0, C.byref(cnt))
        if st != OK:
            raise GdpError(st, "gdp_mesh_scan")
        n = cnt.value if cap is None else min(cap, cnt.value)
        kind = np.zeros(n, np.int32)
        verts = np.zeros((n, 3), np.int32)
        pt = np.zeros((n, 2), np.float64)
        meas = np.zeros(n, np.uint32)
        st = L.gdp_mesh_scan_mode(self._h, B, flags, _p(kind), _p(verts), _p(pt), _p(meas), n, C.byref(cnt))
        if st != OK:
            raise GdpError(st, "gdp_mesh_scan")
        return kind, verts, pt, meas


class Batch:
    """gdp_batch: many independent PSLGs refined together, one launch per step."""

    def __init__(self, pslgs, stream=None):
        L = load()
        xys = [np.ascontiguousarray(p[0], np.float64).reshape(-1, 2) for p in pslgs]
        segs = [np.ascontiguousarray(p[1], np.int32).reshape(-1, 2) for p in pslgs]
        self.n = len(pslgs)
        pt_off = np.zeros(self.n + 1, np.int64)
        seg_off = np.zeros(self.n + 1, np.int64)
        pt_off[1:] = np.cumsum([len(x) for x in xys])
        seg_off[1:] = np.cumsum([len(s) for s in segs])
        xy = np.ascontiguousarray(np.concatenate(xys))
        seg = np.ascontiguousarray(np.concatenate(segs)) if seg_off[-1] else np.zeros((1, 2), np.int32)
        self._h = C.c_void_p()
        st = L.gdp_batch_create(_p(xy), _p(pt_off), _p(seg), _p(seg_off), self.n,
                                _stream_handle(stream), C.byref(self._h))
        if st != OK:
            self.close()
            raise GdpError(st, "gdp_batch_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gdp_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refine(self, B, max_iter=0, cand_cap=0, graph_iters=0, check=True, flags=0, cand_block=0,
               max_len=0.0):
        Bs = np.ascontiguousarray(np.broadcast_to(np.asarray(B, np.float64), (self.n,)))
        s = Stats()
        o = _opts(float(Bs[0]), max_iter, cand_cap, graph_iters, flags, cand_block, max_len)
        st = load().gdp_batch_refine(self._h, _p(Bs), C.byref(o), C.byref(s))
        if check and st != OK:
            raise GdpError(st, "gdp_batch_refine")
        return s.as_dict() if check else (st, s.as_dict())

    def info(self):
        status = np.zeros(self.n, np.int32)
        n_pts = np.zeros(self.n, np.int64)
        n_tri = np.zeros(self.n, np.int64)
        n_st = np.zeros(self.n, np.int64)
        st = load().gdp_batch_info(self._h, _p(status), _p(n_pts), _p(n_tri), None, _p(n_st))
        if st != OK:
            raise GdpError(st, "gdp_batch_info")
        return {"status": status, "n_pts": n_pts, "n_tri": n_tri, "n_steiner": n_st}

    def export(self, m):
        L = load()
        n_pts, n_tri, n_seg = C.c_int64(), C.c_int64(), C.c_int64()
        st = L.gdp_batch_export(self._h, m, None, 0, None, 0, None, 0, C.byref(n_pts),
                                C.byref(n_tri), C.byref(n_seg))
        if st != OK:
            raise GdpError(st, "gdp_batch_export")
        xy = np.zeros((n_pts.value, 2), np.float64)
        tri = np.zeros((n_tri.value, 3), np.int32)
        sub = np.zeros((n_seg.value, 3), np.int32)
        st = L.gdp_batch_export(self._h, m, _p(xy), len(xy), _p(tri), len(tri), _p(sub), len(sub),
                                C.byref(n_pts), C.byref(n_tri), C.byref(n_seg))
        if st != OK:
            raise GdpError(st, "gdp_batch_export")
        return xy, tri, sub


def _concat(pslgs):
    xys = [np.ascontiguousarray(p[0], np.float64).reshape(-1, 2) for p in pslgs]
    segs = [np.ascontiguousarray(p[1], np.int32).reshape(-1, 2) for p in pslgs]
    pt_off = np.zeros(len(pslgs) + 1, np.int64)
    seg_off = np.zeros(len(pslgs) + 1, np.int64)
    pt_off[1:] = np.cumsum([len(x) for x in xys])
    seg_off[1:] = np.cumsum([len(s) for s in segs])
    xy = np.ascontiguousarray(np.concatenate(xys))
    seg = np.ascontiguousarray(np.concatenate(segs)) if seg_off[-1] else np.zeros((1, 2), np.int32)
    return xy, pt_off, seg, seg_off


def autotune(pslgs, B, stream=None):
    """gdp_autotune on a sample [(xy, seg)]: returns ({"cand_block", "cand_cap"},
    [(cand_block, cand_cap, refine_ms, steiner) per trial])"""
    xy, pt_off, seg, seg_off = _concat(pslgs)
    Bs = np.ascontiguousarray(np.broadcast_to(np.asarray(B, np.float64), (len(pslgs),)))
    best = RefineOpts()
    trials = np.zeros((32, 4), np.float64)
    st = load().gdp_autotune(_p(xy), _p(pt_off), _p(seg), _p(seg_off), len(pslgs), _p(Bs),
                             C.byref(_opts(float(Bs[0]))), _stream_handle(stream), C.byref(best),
                             _p(trials), 32)
    if st != OK:
        raise GdpError(st, "gdp_autotune")
    n = 20
    return ({"cand_block": best.cand_block, "cand_cap": best.cand_cap},
            [tuple(trials[k]) for k in range(n)])


class ResultInfo(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("status", C.c_int32), ("n_in_pts", C.c_int64),
                ("n_steiner", C.c_int64), ("n_pts", C.c_int64), ("n_tri", C.c_int64),
                ("n_subseg", C.c_int64), ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double),
                ("t_done_ms", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Server:
    """gdp_server: continuous batching of refinement requests in one resident
    pool (capacities in triangle slots, vertices, segments and meshes)."""

    def __init__(self, tri_slots, vert_slots, seg_slots, max_meshes, cand_cap=0, cand_block=0,
                 graph_iters=0, stream=None, max_len=0.0):
        o = _opts(math.sqrt(2.0), 0, cand_cap, graph_iters, 0, cand_block, max_len)
        self._h = C.c_void_p()
        st = load().gdp_server_create(int(tri_slots), int(vert_slots), int(seg_slots), int(max_meshes),
                                      C.byref(o), _stream_handle(stream), C.byref(self._h))
        if st != OK:
            self.close()
            raise GdpError(st, "gdp_server_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gdp_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, xy, seg, B):
        xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
        seg = np.ascontiguousarray(seg, np.int32).reshape(-1, 2)
        t = C.c_int64()
        st = load().gdp_server_submit(self._h, _p(xy), len(xy), _p(seg) if len(seg) else None, len(seg),
                                      float(B), C.byref(t))
        if st != OK:
            raise GdpError(st, "gdp_server_submit")
        return t.value

    def step(self):
        w, l, d = C.c_int32(), C.c_int32(), C.c_int32()
        st = load().gdp_server_step(self._h, C.byref(w), C.byref(l), C.byref(d))
        if st != OK:
            raise GdpError(st, "gdp_server_step")
        return w.value, l.value, d.value

    def results(self):
        """every finished request: [(info dict, xy, tri, subseg)], oldest first"""
        L = load()
        out = []
        while True:
            info = ResultInfo()
            if L.gdp_server_result(self._h, C.byref(info), None, 0, None, 0, None, 0) != OK:
                return out
            xy = np.zeros((info.n_pts, 2), np.float64)
            tri = np.zeros((info.n_tri, 3), np.int32)
            sub = np.zeros((info.n_subseg, 3), np.int32)
            st = L.gdp_server_result(self._h, C.byref(info), _p(xy), len(xy), _p(tri), len(tri),
                                     _p(sub), len(sub))
            if st != OK:
                raise GdpError(st, "gdp_server_result")
            out.append((info.as_dict(), xy, tri, sub))


def scan_noalloc(xy, tri4, B, kind, verts, pt, meas, stream=None):
    """gdp_scan_noalloc on caller-owned torch CUDA tensors: xy (n,2) float64,
    tri4 (t,4) int32, outputs kind (cap,) int32, verts (cap,3) int32,
    pt (cap,2) float64, meas (cap,) int32.  Returns the entry count."""
    import torch
    cap = int(kind.shape[0])
    want = ((xy, torch.float64, (None, 2)), (tri4, torch.int32, (None, 4)), (kind, torch.int32, (cap,)),
            (verts, torch.int32, (cap, 3)), (pt, torch.float64, (cap, 2)), (meas, torch.int32, (cap,)))
    for t, dt, shape in want:
        if not (t.is_cuda and t.is_contiguous() and t.dtype == dt and t.dim() == len(shape) and
                all(w is None or w == g for w, g in zip(shape, t.shape))):
            raise ValueError(f"scan_noalloc: expected a contiguous CUDA {dt} tensor of shape {shape}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    cnt = C.c_int64()
    st = load().gdp_scan_noalloc(C.c_void_p(xy.data_ptr()), int(xy.shape[0]),
                                 C.c_void_p(tri4.data_ptr()), int(tri4.shape[0]), float(B),
                                 C.c_void_p(kind.data_ptr()), C.c_void_p(verts.data_ptr()),
                                 C.c_void_p(pt.data_ptr()), C.c_void_p(meas.data_ptr()),
                                 int(kind.shape[0]), C.byref(cnt), _stream_handle(stream))
    if st != OK:
        raise GdpError(st, "gdp_scan_noalloc")
    return cnt.value
