"""ctypes binding of libvrs (include/vrs.h): argument marshalling only.

Every function here has the C-ABI's name and forwards to it; no step of the
rasterizer runs in Python.  Loading fails loudly when libvrs.so has not been
built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvrs.so")

VRS_MAX_VIEWS = 64
VRS_MAX_SCENES = 16

VRS_OK, VRS_ERR_INVALID, VRS_ERR_CAPACITY, VRS_ERR_CUDA, VRS_ERR_TIMEOUT, VRS_ERR_NONFINITE = range(6)
STATUS_NAMES = ["VRS_OK", "VRS_ERR_INVALID", "VRS_ERR_CAPACITY", "VRS_ERR_CUDA", "VRS_ERR_TIMEOUT",
                "VRS_ERR_NONFINITE"]

_i32, _i64, _u32, _u64, _f32, _vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p)


class vrs_scene(ctypes.Structure):
    _fields_ = [("means", _vp), ("log_scales", _vp), ("quats", _vp), ("opacity_logits", _vp),
                ("sh", _vp), ("n", _i32), ("sh_degree", _i32), ("baked", _vp), ("sh_half", _i32),
                ("reserved", _i32)]


VRS_BAKED_FLOATS = 16


class vrs_camera(ctypes.Structure):
    _fields_ = [("R", _f32 * 9), ("t", _f32 * 3), ("fx", _f32), ("fy", _f32), ("cx", _f32),
                ("cy", _f32), ("znear", _f32), ("tan_fovx", _f32), ("tan_fovy", _f32),
                ("width", _i32), ("height", _i32), ("scene", _i32)]


class vrs_plan_opts(ctypes.Structure):
    _fields_ = [("tile", _i32), ("persistent", _i32), ("backward", _i32), ("sort", _i32),
                ("max_instances", _i64), ("count_pairs", _i32), ("resort", _i32), ("half_out", _i32),
                ("key_bits", _i32), ("tiles_per_pull", _i32), ("reserved", _i32)]


class vrs_plan(ctypes.Structure):
    _fields_ = [("n_views", _i32), ("n_scenes", _i32), ("tile", _i32), ("key_bits", _i32),
                ("sort_passes", _i32), ("persistent", _i32), ("backward", _i32), ("sort_ctas", _i32),
                ("max_instances", _i64), ("n_records", _i64), ("n_tiles", _i64), ("n_pixels", _i64),
                ("workspace_bytes", _i64),
                ("off_status", _i64), ("off_records", _i64), ("off_keys", _i64 * 2),
                ("off_vals", _i64 * 2), ("off_hist", _i64), ("off_ranges", _i64),
                ("off_ncontrib", _i64), ("off_order", _i64), ("off_grad2d", _i64),
                ("off_tilesort", _i64), ("off_pairs", _i64), ("sorted_buf", _i32), ("n_sms", _i32), ("sort_mode", _i32),
                ("count_pairs", _i32),
                ("scene_n", _i32 * VRS_MAX_SCENES), ("scene_deg", _i32 * VRS_MAX_SCENES),
                ("view_scene", _i32 * VRS_MAX_VIEWS), ("view_w", _i32 * VRS_MAX_VIEWS),
                ("view_h", _i32 * VRS_MAX_VIEWS), ("view_gw", _i32 * VRS_MAX_VIEWS),
                ("view_gh", _i32 * VRS_MAX_VIEWS), ("view_rec_base", _i64 * VRS_MAX_VIEWS),
                ("view_tile_base", _i64 * VRS_MAX_VIEWS), ("view_pix_base", _i64 * VRS_MAX_VIEWS),
                ("resort", _i32), ("half_out", _i32), ("tiles_per_pull", _i32), ("reserved", _i32),
                ("off_raydepth", _i64), ("off_resort_flags", _i64)]


class vrs_run_info(ctypes.Structure):
    _fields_ = [("flags", _u32), ("reserved", _u32), ("instances", _u64), ("pair_evals", _u64),
                ("pair_blends", _u64), ("block_evals", _u64), ("visible_pairs", _u64 * VRS_MAX_SCENES),
                ("resort_flagged", _u64)]


class vrs_combine_opts(ctypes.Structure):
    _fields_ = [("d_f", _f32), ("m", _f32), ("gamma", _f32), ("reserved", _i32)]


class vrs_cull_opts(ctypes.Structure):
    _fields_ = [("alpha_min", _f32), ("rel_margin", _f32), ("abs_margin", _f32), ("reserved", _i32)]


# (name, restype, argtypes) of every entry point declared in include/vrs.h
SIGNATURES = [
    ("vrs_plan_batch", _i32, [ctypes.POINTER(vrs_scene), _i32, ctypes.POINTER(vrs_camera), _i32,
                              ctypes.POINTER(vrs_plan_opts), ctypes.POINTER(vrs_plan)]),
    ("vrs_preprocess", _i32, [ctypes.POINTER(vrs_plan), ctypes.POINTER(vrs_scene),
                              ctypes.POINTER(vrs_camera), _vp, _vp]),
    ("vrs_bin_sort", _i32, [ctypes.POINTER(vrs_plan), _vp, _vp]),
    ("vrs_render_fwd", _i32, [ctypes.POINTER(vrs_plan), _vp, _vp, _vp, _vp, _vp]),
    ("vrs_render_bwd", _i32, [ctypes.POINTER(vrs_plan), _vp, ctypes.POINTER(vrs_scene),
                              ctypes.POINTER(vrs_camera), _vp, _vp, _vp, _vp,
                              ctypes.POINTER(vrs_scene), _vp]),
    ("vrs_query_status", _i32, [ctypes.POINTER(vrs_plan), _vp, ctypes.POINTER(vrs_run_info), _vp]),
    ("vrs_reset_status", _i32, [ctypes.POINTER(vrs_plan), _vp, _vp]),
    ("vrs_sort_pairs_noalloc", _i32, [_vp, _vp, _vp, _vp, _i64, _i32, _vp]),
    ("vrs_bake", _i32, [ctypes.POINTER(vrs_scene), _vp, _vp]),
    ("vrs_image_loss_scratch", _i32, [_i32, _i32, _i32, ctypes.POINTER(_i64)]),
    ("vrs_image_loss", _i32, [_vp, _vp, _i32, _i32, _i32, _f32, _vp, _vp, _vp, _i64, _vp]),
    ("vrs_opacity_decay", _i32, [_vp, _i64, _f32, _f32, _vp, _vp, _vp]),
    ("vrs_foveal_combine", _i32, [_vp, _i32, _i32, _vp, _i32, _i32, _i32, _i32, _f32, _f32,
                                  ctypes.POINTER(vrs_combine_opts), _vp, _vp, _vp]),
    ("vrs_foveal_combine_bwd", _i32, [_vp, _i32, _i32, _vp, _i32, _i32, _i32, _i32, _f32, _f32,
                                      ctypes.POINTER(vrs_combine_opts), _vp, _vp, _vp, _vp, _vp]),
    ("vrs_cull_points", _i32, [_vp, _i64, ctypes.POINTER(vrs_camera), _i32, _i32, _vp, _vp, _i32, _i32,
                               ctypes.POINTER(vrs_cull_opts), _vp, _vp, _vp, _vp]),
    ("vrs_status_string", ctypes.c_char_p, [_i32]),
]

VRS_NOALLOC_MAX_PAIRS = 1 << 20

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads libvrs.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libvrs.so is not built ({path}); run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class VrsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


def _check(code: int, where: str) -> int:
    if code != VRS_OK:
        raise VrsError(code, where)
    return code


def status_string(code: int) -> str:
    return load().vrs_status_string(int(code)).decode()


# --- thin wrappers with the C names -------------------------------------------------------

def vrs_plan_batch(scenes, n_scenes, views, n_views, opts, plan) -> int:
    return load().vrs_plan_batch(scenes, n_scenes, views, n_views, ctypes.byref(opts), ctypes.byref(plan))


def vrs_preprocess(plan, scenes, views, workspace: int, stream: int) -> int:
    return load().vrs_preprocess(ctypes.byref(plan), scenes, views, workspace, stream)


def vrs_bin_sort(plan, workspace: int, stream: int) -> int:
    return load().vrs_bin_sort(ctypes.byref(plan), workspace, stream)


def vrs_render_fwd(plan, workspace: int, rgb: int, depth: int, T_final: int, stream: int) -> int:
    return load().vrs_render_fwd(ctypes.byref(plan), workspace, rgb, depth, T_final, stream)


def vrs_render_bwd(plan, workspace: int, scenes, views, T_final: int, dL_drgb: int, dL_ddepth: int,
                   dL_dT, grads, stream: int) -> int:
    return load().vrs_render_bwd(ctypes.byref(plan), workspace, scenes, views, T_final, dL_drgb,
                                 dL_ddepth, dL_dT, grads, stream)


def vrs_query_status(plan, workspace: int, info, stream: int) -> int:
    return load().vrs_query_status(ctypes.byref(plan), workspace, ctypes.byref(info), stream)


def vrs_reset_status(plan, workspace: int, stream: int) -> int:
    return load().vrs_reset_status(ctypes.byref(plan), workspace, stream)


def vrs_status_string(code: int) -> str:
    return status_string(code)


def vrs_sort_pairs_noalloc(keys_in: int, vals_in: int, keys_out: int, vals_out: int, n: int,
                           key_bits: int, stream: int) -> int:
    return load().vrs_sort_pairs_noalloc(keys_in, vals_in, keys_out, vals_out, n, key_bits, stream)


def vrs_cull_points(points: int, n_points: int, fovea, x0: int, y0: int, depth: int, T_final: int,
                    map_w: int, map_h: int, opts, mask: int, kept: Optional[int], n_kept: int,
                    stream: Optional[int]) -> int:
    return load().vrs_cull_points(points, n_points, ctypes.byref(fovea) if fovea is not None else None,
                                  x0, y0, depth, T_final, map_w, map_h,
                                  ctypes.byref(opts) if opts is not None else None, mask, kept, n_kept,
                                  stream)


def vrs_foveal_combine(P: int, pw: int, ph: int, F: int, w: int, h: int, x0: int, y0: int, ex: float,
                       ey: float, opts, out: int, c_out: Optional[int], stream: Optional[int]) -> int:
    return load().vrs_foveal_combine(P, pw, ph, F, w, h, x0, y0, ex, ey,
                                     ctypes.byref(opts) if opts is not None else None, out, c_out, stream)


def vrs_foveal_combine_bwd(P: int, pw: int, ph: int, F: int, w: int, h: int, x0: int, y0: int, ex: float,
                           ey: float, opts, dL_dout: int, dL_dP: int, dL_dF: int, scratch: int,
                           stream: Optional[int]) -> int:
    return load().vrs_foveal_combine_bwd(P, pw, ph, F, w, h, x0, y0, ex, ey,
                                         ctypes.byref(opts) if opts is not None else None, dL_dout, dL_dP,
                                         dL_dF, scratch, stream)


def vrs_bake(scene, baked: int, stream: int) -> int:
    return load().vrs_bake(ctypes.byref(scene), baked, stream)


def vrs_image_loss_scratch(C: int, H: int, W: int) -> int:
    b = _i64(0)
    _check(load().vrs_image_loss_scratch(C, H, W, ctypes.byref(b)), "vrs_image_loss_scratch")
    return int(b.value)


def vrs_image_loss(image: int, target: int, C: int, H: int, W: int, lam: float, loss_out: int,
                   dL_dimage: Optional[int], scratch: int, scratch_bytes: int, stream: int) -> int:
    return load().vrs_image_loss(image, target, C, H, W, lam, loss_out, dL_dimage, scratch, scratch_bytes,
                                 stream)


def vrs_opacity_decay(logits: int, n: int, factor: float, threshold: float, keep: int, n_kept: int,
                      stream: int) -> int:
    return load().vrs_opacity_decay(logits, n, factor, threshold, keep, n_kept, stream)
