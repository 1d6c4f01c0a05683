"""The C-ABI without a GPU: struct layouts, exported symbols, host-side planning."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vrs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2410_17932_gb300 import _lib as L
    if not os.path.exists(L.LIB_PATH):
        from paper_2410_17932_gb300 import build
        build.build()
    L.load()
    return L


def _declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:vrs_status|const char \*)\s*(vrs_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_entry_point(lib):
    names = _declared_functions()
    assert len(names) >= 8
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (vrs_\w+)", out))
    for n in names:
        assert n in exported, n
    bound = {s[0] for s in lib.SIGNATURES}
    assert set(names) == bound


def _c_layout(tmp_path):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "vrs.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("vrs_scene %zu\nvrs_camera %zu\nvrs_plan_opts %zu\nvrs_plan %zu\nvrs_run_info %zu\n"
         "vrs_cull_opts %zu\nvrs_combine_opts %zu\n", sizeof(vrs_scene), sizeof(vrs_camera),
         sizeof(vrs_plan_opts), sizeof(vrs_plan), sizeof(vrs_run_info), sizeof(vrs_cull_opts),
         sizeof(vrs_combine_opts));
  P(vrs_plan, max_instances) P(vrs_plan, off_status) P(vrs_plan, off_grad2d) P(vrs_plan, sorted_buf)
  P(vrs_plan, scene_n) P(vrs_plan, view_scene) P(vrs_plan, view_rec_base) P(vrs_plan, view_pix_base)
  P(vrs_camera, fx) P(vrs_camera, width) P(vrs_camera, scene) P(vrs_scene, n)
  P(vrs_run_info, instances) P(vrs_run_info, pair_blends) P(vrs_run_info, block_evals)
  P(vrs_plan_opts, max_instances) P(vrs_plan, off_pairs) P(vrs_cull_opts, abs_margin)
  P(vrs_run_info, visible_pairs) P(vrs_run_info, resort_flagged) P(vrs_plan, resort)
  P(vrs_plan, off_raydepth) P(vrs_plan, off_resort_flags) P(vrs_plan_opts, resort)
  P(vrs_scene, baked) P(vrs_scene, sh_half) P(vrs_plan_opts, half_out) P(vrs_plan, half_out)
  P(vrs_plan_opts, key_bits) P(vrs_plan_opts, tiles_per_pull) P(vrs_plan, tiles_per_pull)
  return 0;
}
"""
    c = tmp_path / "layout.c"
    c.write_text(prog)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True).stdout
    return dict(line.rsplit(" ", 1) for line in out.strip().splitlines())


def test_struct_layouts_match_header(lib, tmp_path):
    c = _c_layout(tmp_path)
    L = lib
    for name in ["vrs_scene", "vrs_camera", "vrs_plan_opts", "vrs_plan", "vrs_run_info", "vrs_cull_opts",
                 "vrs_combine_opts"]:
        assert int(c[name]) == ctypes.sizeof(getattr(L, name)), name
    for key, val in c.items():
        if "." in key:
            sname, field = key.split(".")
            assert getattr(getattr(L, sname), field).offset == int(val), key


def _plan(L, views, scenes=((1000, 3),), **opts):
    sc = (L.vrs_scene * len(scenes))()
    for i, (n, d) in enumerate(scenes):
        sc[i].n, sc[i].sh_degree = n, d
    vs = (L.vrs_camera * len(views))()
    for i, (w, h, s) in enumerate(views):
        vs[i].width, vs[i].height, vs[i].scene, vs[i].fx, vs[i].fy = w, h, s, 100.0, 100.0
    o = L.vrs_plan_opts(opts.get("tile", 0), opts.get("persistent", 0), opts.get("backward", 0), 0,
                        opts.get("max_instances", 0))
    p = L.vrs_plan()
    code = L.vrs_plan_batch(sc, len(scenes), vs, len(views), o, p)
    return code, p


def test_plan_sizes_and_layout_on_host(lib):
    L = lib
    code, p = _plan(L, [(2016, 2240, 0), (2016, 2240, 0)], backward=1)
    assert code == L.VRS_OK
    assert p.n_records == 2000 and p.n_pixels == 2 * 2016 * 2240
    assert p.n_tiles == 2 * 126 * 140
    assert p.key_bits == 32 + 16 and p.sort_passes == 6 and p.sorted_buf == 0
    assert p.view_rec_base[1] == 1000 and p.view_tile_base[1] == 126 * 140
    offs = [p.off_status, p.off_records, p.off_keys[0], p.off_keys[1], p.off_vals[0], p.off_vals[1],
            p.off_hist, p.off_ranges, p.off_ncontrib, p.off_order, p.off_grad2d, p.off_tilesort,
            p.off_pairs]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs) and p.workspace_bytes > offs[-1]
    assert p.off_keys[1] - p.off_keys[0] >= 8 * p.max_instances
    assert p.off_ncontrib - p.off_ranges >= 8 * p.n_tiles
    assert p.off_order - p.off_ncontrib >= 4 * p.n_pixels
    # backward plans: the forward's per-warp work estimates (tile^2 / 64 per tile) take the
    # workspace's last 256-byte-rounded region, after the pair list
    work = (p.n_tiles * (16 * 16 // 64) * 4 + 255) // 256 * 256
    assert p.workspace_bytes - work >= p.off_pairs + 32 * p.n_records
    code, q = _plan(L, [(2016, 2240, 0), (2016, 2240, 0)], backward=0)
    assert code == L.VRS_OK and q.workspace_bytes <= p.workspace_bytes - work


@pytest.mark.parametrize("bad", [
    dict(views=[(0, 10, 0)]), dict(views=[(10, 10, 1)]), dict(views=[(10, 20000, 0)]),
    dict(views=[(10, 10, 0)], tile=12), dict(views=[(10, 10, 0)], scenes=((10, 4),)),
    dict(views=[(10, 10, 0)], scenes=((-1, 0),)), dict(views=[(10, 10, 0)], max_instances=-5),
    dict(views=[(10, 10, 0)], persistent=3), dict(views=[(10, 10, 0)], persistent=-1),
])
def test_plan_rejects_invalid_arguments(lib, bad):
    L = lib
    views = bad.pop("views")
    code, _ = _plan(L, views, **bad)
    assert code == L.VRS_ERR_INVALID


def test_status_strings(lib):
    for code, name in enumerate(lib.STATUS_NAMES):
        assert lib.vrs_status_string(code) == name
    assert lib.vrs_status_string(99) == "VRS_ERR_UNKNOWN"


def test_library_missing_fails_loudly(tmp_path):
    from paper_2410_17932_gb300 import _lib as L
    saved = L._lib
    try:
        L._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            L.load(str(tmp_path / "nope.so"))
    finally:
        L._lib = saved


def test_cull_points_rejects_bad_arguments_on_host(lib):
    """Argument errors return before any CUDA call (so this runs without a GPU)."""
    L = lib
    cam = L.vrs_camera()
    cam.width, cam.height, cam.fx, cam.fy = 16, 16, 10.0, 10.0
    buf = ctypes.create_string_buffer(64)
    ptr = ctypes.addressof(buf)
    ptr = ptr + (-ptr % 16)
    good = dict(points=ptr, n=4, cam=cam, depth=ptr, T=ptr, w=16, h=16, opts=None, mask=ptr, kept=None,
                n_kept=ptr)

    def call(**kw):
        a = dict(good, **kw)
        return L.vrs_cull_points(a["points"], a["n"], a["cam"], 0, 0, a["depth"], a["T"], a["w"], a["h"],
                                 a["opts"], a["mask"], a["kept"], a["n_kept"], None)

    assert call(n=-1) == L.VRS_ERR_INVALID
    assert call(n=1 << 32) == L.VRS_ERR_INVALID
    assert call(cam=None) == L.VRS_ERR_INVALID
    assert call(n_kept=None) == L.VRS_ERR_INVALID
    assert call(points=None) == L.VRS_ERR_INVALID
    assert call(mask=None) == L.VRS_ERR_INVALID
    assert call(points=ptr + 2) == L.VRS_ERR_INVALID
    assert call(w=0) == L.VRS_ERR_INVALID
    bad = L.vrs_camera()
    assert call(cam=bad) == L.VRS_ERR_INVALID
    assert call(opts=L.vrs_cull_opts(0.5, 0.02, 0.05, 1)) == L.VRS_ERR_INVALID


def test_foveal_combine_rejects_bad_arguments_on_host(lib):
    """Argument errors return before any CUDA call (so this runs without a GPU)."""
    L = lib
    buf = ctypes.create_string_buffer(4096)
    base = ctypes.addressof(buf)
    P, F, out = base, base + 1024, base + 2048

    def call(**kw):
        a = dict(P=P, pw=16, ph=16, F=F, w=4, h=4, x0=2, y0=3, opts=None, out=out)
        a.update(kw)
        return L.vrs_foveal_combine(a["P"], a["pw"], a["ph"], a["F"], a["w"], a["h"], a["x0"], a["y0"], 8.0,
                                    8.0, a["opts"], a["out"], None, None)

    assert call(P=None) == L.VRS_ERR_INVALID
    assert call(w=0) == L.VRS_ERR_INVALID
    assert call(x0=13) == L.VRS_ERR_INVALID          # window not inside P
    assert call(y0=-1) == L.VRS_ERR_INVALID
    assert call(out=F + 8) == L.VRS_ERR_INVALID      # out overlaps F
    assert call(opts=L.vrs_combine_opts(0.0, 0.75, 0.2, 0)) == L.VRS_ERR_INVALID
    assert call(opts=L.vrs_combine_opts(256.0, 1.0, 0.2, 0)) == L.VRS_ERR_INVALID
    assert call(opts=L.vrs_combine_opts(256.0, 0.75, 0.2, 3)) == L.VRS_ERR_INVALID
