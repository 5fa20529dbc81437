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


def test_default_reg_options_match_paper(L):
    o = tsp.RegOptions()
    assert L.tsp_default_reg_options(C.byref(o)) == tsp.TSP.OK
    # Sec. 5.1: 8 nearest neighbours; Sec. 4.5.2: > 9 pixels, > 90 % static, >= 2 views
    assert o.k == 8 and o.static_min_views == 2
    assert o.static_min_px == 9.0 and abs(o.static_frac - 0.9) < 1e-7
    assert L.tsp_default_reg_options(None) == tsp.TSP.ERR_INVALID_ARG


def test_null_context_is_rejected(L):
    assert L.tsp_fit_motion(None, None, None, 0, None, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_render(None, None, None, 0, None, 0, None, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_sync(None, None, 0) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_regularize(None, None, None, None, 0, None, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_knn(None, None, None, 0, 8, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_inspect(None, 0, None, 0, None) == tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_destroy(None) == tsp.TSP.OK


def test_cached_autotune_rejects_null_context_before_touching_the_cache(L, tmp_path):
    path = tmp_path / "tune.txt"
    assert L.tsp_autotune_cached(None, None, 1, 3, None, os.fsencode(str(path)), None, None, None) == \
        tsp.TSP.ERR_INVALID_ARG
    assert L.tsp_autotune_cached(None, None, 1, 3, None, None, None, None, None) == tsp.TSP.ERR_INVALID_ARG
    assert not path.exists()


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p(1)
    st = L.tsp_create(0, None, C.byref(h))
    assert st == tsp.TSP.ERR_CUDA and not h.value
    assert L.tsp_create(-1, None, C.byref(h)) == tsp.TSP.ERR_INVALID_ARG


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets that a C
    compiler gives the header's structure (gcc, compiled here)."""
    import subprocess
    pairs = {"tsp_camera": tsp.Camera, "tsp_gaussians": tsp.Gaussians, "tsp_view_tracks": tsp.ViewTracks,
             "tsp_result": tsp.Result, "tsp_frame": tsp.Frame, "tsp_options": tsp.Options,
             "tsp_render_grads": tsp.RenderGrads, "tsp_reg_options": tsp.RegOptions,
             "tsp_reg_result": tsp.RegResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tsplat.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cname, py in pairs.items():
        assert C.sizeof(py) == got[(cname, "size")], cname
        for fname, _ in py._fields_:
            assert getattr(py, fname).offset == got[(cname, fname)], (cname, fname)
