"""The C-ABI library loads on a CPU-only host, exports every entry point that
include/gs.h declares, agrees with the binding on struct layouts, and rejects
bad arguments on the host (none of these calls reaches a GPU)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gs_[a-z0-9_]+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.EXPORTS, f"binding lacks {n}"
    nm = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gs_\w+)", nm))
    assert exported == set(names)


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gs.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    "sizeof(gs_camera), sizeof(gs_view), sizeof(gs_status), sizeof(gs_anchors),"
                    "sizeof(gs_gauss3d), sizeof(gs_gauss3d_grad), sizeof(gs_splats), sizeof(gs_bins),"
                    "sizeof(gs_anchor_grad), offsetof(gs_gauss3d, cap_rows));"
                    'printf("%zu %zu\\n", sizeof(gs_adam_group), offsetof(gs_adam_group, lr));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [64, C.sizeof(L.gs_view), C.sizeof(L.gs_status), C.sizeof(L.gs_anchors),
            C.sizeof(L.gs_gauss3d), C.sizeof(L.gs_gauss3d_grad), C.sizeof(L.gs_splats),
            C.sizeof(L.gs_bins), C.sizeof(L.gs_anchor_grad), L.gs_gauss3d.cap_rows.offset,
            C.sizeof(L.gs_adam_group), L.gs_adam_group.lr.offset]
    assert got == want


def test_size_queries(lib):
    views = (L.gs_view * 3)(L.gs_view(1241, 376), L.gs_view(1024, 384), L.gs_view(1024, 768))
    assert lib.gs_total_tiles(views, 3) == 78 * 24 + 64 * 24 + 64 * 48
    assert lib.gs_total_pixels(views, 3) == 1241 * 376 + 1024 * 384 + 1024 * 768
    assert lib.gs_total_tiles(views, 0) == -1
    # three heads (k, 3k, 7k outputs) of two layers each on F + 4 inputs
    assert lib.gs_mlp_floats(32, 10, 32) == 3 * (32 * 36 + 32) + (10 + 30 + 70) * 33
    assert lib.gs_bin_sort_workspace(views, 3, 1000, 5000) > 0
    for code in (0, -1, -2, -3, -4, -5):
        assert len(lib.gs_status_string(code)) > 0


def test_bad_arguments_rejected_without_a_gpu(lib):
    views = (L.gs_view * 1)(L.gs_view(64, 48))
    a = L.gs_anchors(10, 0, 4, 8, 1)   # F = 0 is invalid
    g = L.gs_gauss3d()
    assert lib.gs_decode(C.byref(a), None, views, 1, 0, C.byref(g), None, 0, None, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_project(None, None, views, 1, None, None, None) == L.GS_ERR_INVALID_ARG
    bad_views = (L.gs_view * 1)(L.gs_view(0, 48))
    sp = L.gs_splats(1, 16, 16)
    bins = L.gs_bins(10, 16, None, 16, 16)
    assert lib.gs_bin_sort(C.byref(sp), 1, C.c_void_p(16), 10, bad_views, 1, C.byref(bins), C.c_void_p(256),
                           1 << 20, C.c_void_p(16), None) == L.GS_ERR_INVALID_ARG
    bg = (C.c_float * 3)(0, 0, 0)
    assert lib.gs_render_fwd(C.byref(sp), C.byref(bins), views, 65, bg, 0, C.c_void_p(256), 1 << 20,
                             C.c_void_p(16), None, None, None, C.c_void_p(16), None) == L.GS_ERR_INVALID_ARG
    # chunk below 256 and an unaligned workspace are rejected
    assert lib.gs_render_fwd(C.byref(sp), C.byref(bins), views, 1, bg, 100, C.c_void_p(256), 1 << 20,
                             C.c_void_p(16), None, None, None, C.c_void_p(16), None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_render_fwd(C.byref(sp), C.byref(bins), views, 1, bg, 0, C.c_void_p(16), 1 << 20,
                             C.c_void_p(16), None, None, None, C.c_void_p(16), None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_render_workspace(views, 1, 100000, 0) > lib.gs_render_workspace(views, 1, 100000, 4096) > 0
    assert lib.gs_l1_loss(None, None, views, 1, None, None, None) == L.GS_ERR_INVALID_ARG


def test_bad_arguments_of_the_next_rows_rejected_without_a_gpu(lib):
    """The entry points after the reverse pass check their host arguments
    before anything reaches a GPU."""
    views = (L.gs_view * 1)(L.gs_view(64, 48))
    p16 = C.c_void_p(256)
    # photometric loss: lambda outside [0, 1], a small or unaligned workspace
    for lam in (-0.5, 1.5):
        assert lib.gs_photometric_loss(p16, p16, views, 1, lam, p16, 1 << 20, p16, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_photometric_loss(p16, p16, views, 1, 0.8, p16, 8, p16, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_photometric_loss(p16, p16, views, 1, 0.8, C.c_void_p(16), 1 << 20, p16, p16,
                                   None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_photometric_workspace(views, 1) > 0
    # Adam: no group, too many groups, step 0, beta outside [0, 1), a null array
    grp = (L.gs_adam_group * 17)(*[L.gs_adam_group(256, 256, 256, 256, 8, 0.1)] * 17)
    assert lib.gs_adam_step(grp, 0, 1, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_adam_step(grp, 17, 1, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_adam_step(grp, 1, 0, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_adam_step(grp, 1, 1, 0.9, 1.0, 1e-8, None) == L.GS_ERR_INVALID_ARG
    bad = (L.gs_adam_group * 1)(L.gs_adam_group(256, None, 256, 256, 8, 0.1))
    assert lib.gs_adam_step(bad, 1, 1, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG
    # densification statistics and masks
    g = L.gs_gauss3d()
    assert lib.gs_densify_stats(C.byref(g), 1, p16, p16, 10, p16, p16, p16, p16, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_densify_masks(-1, 4, p16, p16, p16, p16, 0.1, 0.1, 1, p16, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_densify_masks(0, 4, p16, p16, p16, p16, 0.1, 0.1, 1, p16, p16, None) == L.GS_OK   # nothing to do
    # voxelisation: negative size, eps <= 0, an existing count without keys, a small workspace
    ws = lib.gs_voxelize_workspace(1000)
    assert ws > 0 and lib.gs_voxelize_workspace(-1) == 0
    assert lib.gs_voxelize(p16, -1, 0.1, None, 0, p16, p16, 10, p16, p16, ws, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_voxelize(p16, 1000, 0.0, None, 0, p16, p16, 10, p16, p16, ws, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_voxelize(p16, 1000, 0.1, None, 5, p16, p16, 10, p16, p16, ws, p16, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_voxelize(p16, 1000, 0.1, None, 0, p16, p16, 10, p16, p16, 64, p16, None) == L.GS_ERR_INVALID_ARG
    # loop closure: no keyframe, z_far <= 0
    assert lib.gs_loop_closure(p16, 10, p16, p16, p16, 0, 10.0, None, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_loop_closure(p16, 10, p16, p16, p16, 1, 0.0, None, None) == L.GS_ERR_INVALID_ARG
    # flow triangulation: empty image, negative tau, a small workspace
    fws = lib.gs_flow_workspace(5000)
    assert lib.gs_flow_triangulate(p16, p16, 0, 48, p16, p16, 10, 1.0, None, p16, p16, 10, p16, p16, fws, p16,
                                   None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_flow_triangulate(p16, p16, 64, 48, p16, p16, 10, -1.0, None, p16, p16, 10, p16, p16, fws, p16,
                                   None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_flow_triangulate(p16, p16, 64, 48, p16, p16, 5000, 1.0, None, p16, p16, 10, p16, p16, 8, p16,
                                   None) == L.GS_ERR_INVALID_ARG
