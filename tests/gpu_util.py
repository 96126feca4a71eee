"""Shared helpers for the GPU parity tests."""
import math

import numpy as np
import pytest

SQ2 = math.sqrt(2.0)
HARD = ("bad_orient", "bad_adjacency", "open_not_sub", "sub_not_edge", "seg_not_covered",
        "not_locally_cd", "euler_defect", "inputs_missing")


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_00324_gb300 import gdp
    gdp.load()
    return gdp


def assert_valid(rep, refined=True, brute=False):
    keys = HARD + (("bad_quality", "encroached") if refined else ()) + (("bf_cd_violations",) if brute else ())
    bad = {k: rep[k] for k in keys if rep[k]}
    assert not bad, bad
