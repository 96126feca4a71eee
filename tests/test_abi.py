"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gdp.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gdp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gdp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("gdp_mesh_create", "gdp_mesh_refine", "gdp_mesh_export", "gdp_mesh_destroy",
              "gdp_batch_refine", "gdp_status_str"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2007_00324_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    lib.gdp_status_str.restype = ctypes.c_char_p
    assert lib.gdp_status_str(0) == b"ok"


def test_binding_names_match_header():
    from paper_2007_00324_gb300 import gdp
    assert sorted(gdp.SYMBOLS) == declared_symbols()


def test_no_device_means_an_error_not_a_fallback():
    """Without a GPU every create call must fail with GDP_ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        return
    import numpy as np
    from paper_2007_00324_gb300 import gdp
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    seg = np.array([[0, 1], [1, 2], [2, 3], [3, 0]], np.int32)
    try:
        gdp.Mesh(xy, seg)
    except gdp.GdpError as e:
        assert e.status == gdp.ERR_CUDA
    else:
        raise AssertionError("mesh creation succeeded without a GPU")


def test_server_without_device_is_an_error():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2007_00324_gb300 import gdp
    try:
        gdp.Server(1 << 16, 1 << 16, 1024, 8)
    except gdp.GdpError as e:
        assert e.status == gdp.ERR_CUDA
    else:
        raise AssertionError("server created without a device")
