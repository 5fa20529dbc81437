"""The C ABI library loads, exports every declared symbol and rejects bad
arguments before touching a GPU (runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

import paper_2604_02586_b300 as tsp
from paper_2604_02586_b300 import build as tbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsplat.h")


@pytest.fixture(scope="module")
def L():
    tbuild.build()
    return tsp.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsp_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "tsp_fit_motion" in names and "tsp_render" in names and len(names) >= 11
    for name in names:
        assert hasattr(L, name), name


def test_version_and_strings(L):
    assert L.tsp_version() == 1
    for s in range(7):
        assert L.tsp_status_string(s)
    assert L.tsp_last_error(None) == b"no context"


def test_default_options_match_paper_thresholds(L):
    o = tsp.Options()
    assert L.tsp_default_options(C.byref(o)) == tsp.TSP.OK
    assert (o.tile_w, o.tile_h) == (16, 16)
    assert abs(o.det_min - 1e-12) < 1e-18 and abs(o.sumw_min_view - 1e-3) < 1e-9
    assert o.min_px_view == 2 and o.min_views == 2 and o.min_px_total == 3
    assert abs(o.sumw_min_total - 1e-3) < 1e-9
    assert L.tsp_default_options(None) == tsp.TSP.ERR_INVALID_ARG


def test_null_context_is_rejected(L):
    assert L.tsp_fit_motion(None, None, None, 0, None, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_render(None, None, None, 0, None, 0, None, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_sync(None, None, 0) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_inspect(None, 0, None, 0, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_destroy(None) == tsp.TSP.OK


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p(1)
    st = L.tsp_create(0, None, C.byref(h))
    assert st == tsp.TSP.ERR_CUDA and not h.value
    assert L.tsp_create(-1, None, C.byref(h)) == tsp.TSP.ERR_INVALID_ARG


def test_struct_layouts_match_header():
    # sizes implied by the header's field lists (no padding surprises)
    assert C.sizeof(tsp.Camera) == 72
    assert C.sizeof(tsp.Gaussians) == 32
    assert C.sizeof(tsp.ViewTracks) == 16
    assert C.sizeof(tsp.Result) == 56
    assert C.sizeof(tsp.Options) == 72
