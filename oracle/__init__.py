"""CPU oracle for the Gaussian-splatting hot path (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  It never imports the CUDA package: it takes plain
numpy arrays (or the seeded input generator's dataclasses, read by attribute)
and computes, in FP64, what the method defines (Sec. 3.1 projection and
blending of splats, Sec. 3.2 Eq. 1 depth).  The integer decisions (visibility,
radius, tile rectangle, depth key) are taken in FP32, the kernel's precision,
by a fixed sequence of rounded operations in ``vrs_oracle.c``.

Record and tile numbering of a multi-view batch (shared convention with the
library's C-ABI, restated here from its definition):
  record index of (view v, Gaussian g) = sum_{v' < v} N[scene(v')] + g
  global tile id of tile (tx, ty) of view v = sum_{v' < v} gw[v'] gh[v'] + ty gw[v] + tx
  sort key = (global tile id << 32) | float32 bits of the depth key
  sorted order = (key, record index) ascending.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrs_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

ALPHA_WIN = 2e-5     # relative window around 1/255 that marks a knife-edge pixel
T_WIN = 3e-5         # relative window around the 1e-4 transmittance stop


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("tan_fovx", ctypes.c_float),
                ("tan_fovy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class OrcCullOpts(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_float), ("rel_margin", ctypes.c_float),
                ("abs_margin", ctypes.c_float), ("reserved", ctypes.c_int32)]


# Defaults of the occlusion test's reading of Sec. 3.3 (see orc_cull_points).
CULL_ALPHA_MIN = 0.5
CULL_REL_MARGIN = 0.02
CULL_ABS_MARGIN = 0.05


class OrcFlagOpts(ctypes.Structure):
    _fields_ = [("alpha_win", ctypes.c_double), ("t_win", ctypes.c_double)]


PROJ_DTYPE = np.dtype([("ubar", "f8"), ("vbar", "f8"), ("depth", "f8"), ("conic", "f8", 3),
                       ("opacity", "f8"), ("rgb", "f8", 3), ("clamp_rgb", "i4", 3),
                       ("clamp_x", "i4"), ("clamp_y", "i4")], align=True)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            L.orc_exp32.restype = ctypes.c_float
            L.orc_exp32.argtypes = [ctypes.c_float]
            L.orc_log32.restype = ctypes.c_float
            L.orc_log32.argtypes = [ctypes.c_float]
            L.orc_sh_basis_xyz.restype = None
            L.orc_sh_basis_xyz.argtypes = [ctypes.c_double] * 3 + [P]
            L.orc_decide.restype = ctypes.c_int
            L.orc_decide.argtypes = [ctypes.c_int, P, P, P, P, ctypes.POINTER(OrcCamera), ctypes.c_int,
                                     P, P, P, P, P, P, P]
            L.orc_decide64.restype = ctypes.c_int
            L.orc_decide64.argtypes = [ctypes.c_int, P, P, P, P, ctypes.POINTER(OrcCamera), ctypes.c_int,
                                       ctypes.c_int, P]
            L.orc_project.restype = None
            L.orc_project.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                      ctypes.POINTER(OrcCamera), P]
            L.orc_render_brute.restype = None
            L.orc_render_brute.argtypes = [ctypes.c_int, P, P, P, P, ctypes.POINTER(OrcCamera),
                                           ctypes.c_int, ctypes.POINTER(OrcFlagOpts), P, P, P, P, P,
                                           P]
            L.orc_render_bucketed.restype = None
            L.orc_render_bucketed.argtypes = [ctypes.c_int, P, P, P, P, ctypes.POINTER(OrcCamera),
                                              ctypes.c_int, ctypes.POINTER(OrcFlagOpts), P, P, P, P,
                                              P, P, P]
            L.orc_raydepth_setup.restype = None
            L.orc_raydepth_setup.argtypes = [ctypes.c_int, P, P, P, ctypes.POINTER(OrcCamera), P]
            L.orc_render_resort.restype = None
            L.orc_render_resort.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.POINTER(OrcCamera), ctypes.c_int,
                                            ctypes.POINTER(OrcFlagOpts), ctypes.c_double, P, P, P, P, P, P, P]
            L.orc_render_bwd.restype = None
            L.orc_render_bwd.argtypes = [ctypes.c_int, P, P, P, P, ctypes.POINTER(OrcCamera),
                                         ctypes.c_int, P, P, P, P]
            L.orc_param_grads.restype = None
            L.orc_param_grads.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                          ctypes.POINTER(OrcCamera), P, P, P, P, P, P, P]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_combine_bwd.restype = None
            L.orc_combine_bwd.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + [P, P, P]
            L.orc_combine.restype = None
            L.orc_combine.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + [P, P]
            L.orc_cull_points.restype = None
            L.orc_cull_points.argtypes = [ctypes.c_int64, P, ctypes.POINTER(OrcCamera), ctypes.c_int32,
                                          ctypes.c_int32, P, P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(OrcCullOpts), P]
            L.orc_image_loss.restype = None
            L.orc_image_loss.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P]
            L.orc_opacity_decay.restype = None
            L.orc_opacity_decay.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_double, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def camera(cam) -> OrcCamera:
    c = OrcCamera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.znear = float(cam.znear)
    c.tan_fovx = float(np.float32(cam.tan_fovx))
    c.tan_fovy = float(np.float32(cam.tan_fovy))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def num_threads() -> int:
    return int(lib().orc_num_threads())


def exp32(x: float) -> float:
    return float(lib().orc_exp32(float(np.float32(x))))


def log32(x: float) -> float:
    return float(lib().orc_log32(float(np.float32(x))))


def sh_basis(x: float, y: float, z: float) -> np.ndarray:
    out = np.zeros(16, np.float64)
    lib().orc_sh_basis_xyz(float(x), float(y), float(z), _p(out))
    return out


def _nonfinite_rows(scene) -> np.ndarray:
    # a Gaussian with any non-finite parameter is skipped (the C-ABI's NONFINITE rule)
    n = scene.n
    bad = ~np.isfinite(np.asarray(scene.opacity_logits, np.float32))
    if n:
        bad |= ~np.isfinite(np.asarray(scene.sh, np.float32)).reshape(n, -1).all(axis=1)
    return bad


def decide(scene, cam, tile: int = 16, pre: bool = False) -> Dict[str, np.ndarray]:
    """FP32 integer decisions for every Gaussian of `scene` in view `cam`.

    With pre=True also returns `pre` [n, 8]: the FP32 values just before each rounding
    (tz, ubar, vbar, 3 sqrt(lambda), sqrt(thr a), sqrt(thr c), thr, det)."""
    n = scene.n
    means, ls, q = _f32(scene.means), _f32(scene.log_scales), _f32(scene.quats)
    out = dict(visible=np.zeros(n, np.uint8), depth=np.zeros(n, np.float32),
               ubar=np.zeros(n, np.float32), vbar=np.zeros(n, np.float32),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32))
    if pre:
        out["pre"] = np.zeros((n, 8), np.float32)
    c = camera(cam)
    lg = _f32(scene.opacity_logits)
    st = lib().orc_decide(n, _p(means), _p(ls), _p(q), _p(lg), ctypes.byref(c), tile,
                          _p(out["visible"]), _p(out["depth"]), _p(out["ubar"]), _p(out["vbar"]),
                          _p(out["radius"]), _p(out["rect"]), _p(out["pre"]) if pre else None)
    bad = _nonfinite_rows(scene)
    if bad.any():
        out["visible"][bad] = 0
        out["rect"][bad] = 0
        st |= 2
    out["status"] = int(st)
    return out


DEC64_DTYPE = np.dtype([("visible", "i4"), ("vis_amb", "i4"), ("radius", "i4"), ("r_lo", "i4"),
                        ("r_hi", "i4"), ("rect", "i4", 4), ("rect_lo", "i4", 4), ("rect_hi", "i4", 4),
                        ("tz", "f8"), ("e_tz", "f8"), ("ubar", "f8"), ("e_u", "f8"), ("vbar", "f8"),
                        ("e_v", "f8"), ("rho", "f8"), ("e_rho", "f8"), ("hx", "f8"), ("e_hx", "f8"),
                        ("hy", "f8"), ("e_hy", "f8"), ("thr", "f8"), ("e_thr", "f8"), ("det", "f8"),
                        ("e_det", "f8")], align=True)
KNIFE = 2.0      # decision windows are this many times the first-order FP32 error bound


def decide64(scene, cam, tile: int = 16, clip: bool = True) -> np.ndarray:
    """FP64 decisions from the plain definition (DEC64_DTYPE per Gaussian).

    `visible`, `radius`, `rect` are the FP64 decisions; `vis_amb`, `r_lo..r_hi` and
    `rect_lo..rect_hi` say which values an FP32 evaluation may legitimately reach
    (knife edges); the value/bound pairs (tz, e_tz), (ubar, e_u), ... are the
    pre-rounding values and first-order FP32 error bounds.  clip=False gives the
    plain 3-sigma rectangle without the alpha >= 1/255 clip."""
    n = scene.n
    out = np.zeros(n, DEC64_DTYPE)
    c = camera(cam)
    st = lib().orc_decide64(n, _p(_f32(scene.means)), _p(_f32(scene.log_scales)), _p(_f32(scene.quats)),
                            _p(_f32(scene.opacity_logits)), ctypes.byref(c), tile, int(bool(clip)),
                            _p(out))
    bad = _nonfinite_rows(scene)
    if bad.any():
        out["visible"][bad] = 0
        out["vis_amb"][bad] = 0
        out["rect"][bad] = 0
    return out


def dec64_as_decisions(d64: np.ndarray, scene, cam) -> Dict[str, np.ndarray]:
    """The FP64 decisions in the form render()/bin_sort() take (depth key = FP32 of the FP64 z)."""
    vis = d64["visible"].astype(np.uint8)
    return dict(visible=vis, depth=np.where(vis > 0, d64["tz"], 0).astype(np.float32),
                ubar=d64["ubar"].astype(np.float32), vbar=d64["vbar"].astype(np.float32),
                radius=d64["radius"].astype(np.int32), rect=np.ascontiguousarray(d64["rect"], np.int32),
                status=0)


def decision_mismatches(d64: np.ndarray, visible, rect) -> Dict[str, np.ndarray]:
    """Compares another evaluation's visibility and rectangles [n, 4] with the FP64 ones.

    Returns boolean arrays: `differs` (any difference from the FP64 decision) and
    `outside` (a difference that no FP32 rounding of the defined steps can explain)."""
    vis = np.asarray(visible).astype(bool)
    rect = np.asarray(rect).reshape(-1, 4)
    v64 = d64["visible"].astype(bool)
    amb = d64["vis_amb"].astype(bool)
    both = vis & v64
    rdiff = np.zeros(len(vis), bool)
    rout = np.zeros(len(vis), bool)
    rdiff[both] = np.any(rect[both] != d64["rect"][both], axis=1)
    rout[both] = np.any((rect[both] < d64["rect_lo"][both]) | (rect[both] > d64["rect_hi"][both]), axis=1)
    differs = (vis != v64) | rdiff
    outside = ((vis != v64) & ~amb) | rout
    return dict(differs=differs, outside=outside)


def project(scene, cam) -> np.ndarray:
    """FP64 projection record (PROJ_DTYPE) of every Gaussian in view `cam`."""
    n = scene.n
    out = np.zeros(n, PROJ_DTYPE)
    sh = _f32(scene.sh)
    K = sh.shape[1] if n else (scene.sh_degree + 1) ** 2
    c = camera(cam)
    lib().orc_project(n, _p(_f32(scene.means)), _p(_f32(scene.log_scales)), _p(_f32(scene.quats)),
                      _p(_f32(scene.opacity_logits)), _p(sh), K, ctypes.byref(c), _p(out))
    return out


def render(scene, cam, tile: int = 16, mode: str = "bucketed", dec=None, proj=None,
           tile_mask: Optional[np.ndarray] = None, alpha_win: float = ALPHA_WIN,
           t_win: float = T_WIN) -> Dict[str, np.ndarray]:
    """Composited RGB [3,H,W], Eq. 1 depth [H,W], final T [H,W], n_contrib, knife-edge flags."""
    dec = decide(scene, cam, tile) if dec is None else dec
    proj = project(scene, cam) if proj is None else proj
    H, W = cam.height, cam.width
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), T=np.ones((H, W)),
               n_contrib=np.zeros((H, W), np.int32), flags=np.zeros((H, W), np.uint8),
               sig=np.zeros((H, W), np.int32))
    c = camera(cam)
    fo = OrcFlagOpts(alpha_win, t_win)
    args = (scene.n, _p(dec["visible"]), _p(dec["depth"]), _p(dec["rect"]), _p(proj),
            ctypes.byref(c), tile, ctypes.byref(fo))
    if mode == "brute":
        lib().orc_render_brute(*args, _p(out["rgb"]), _p(out["depth"]), _p(out["T"]),
                               _p(out["n_contrib"]), _p(out["flags"]), _p(out["sig"]))
    else:
        tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
        lib().orc_render_bucketed(*args, None if tm is None else _p(tm), _p(out["rgb"]),
                                  _p(out["depth"]), _p(out["T"]), _p(out["n_contrib"]),
                                  _p(out["flags"]), _p(out["sig"]))
    return out


TIE_WIN = 4e-6       # relative window of two per-pixel depths that marks a near tie


RAYDEPTH_DTYPE = np.dtype([("P", "f8", 6), ("Pm", "f8", 3)])


def raydepth(scene, cam) -> np.ndarray:
    """Per Gaussian: the camera-space inverse covariance (xx, xy, xz, yy, yz, zz) and its
    product with the camera-space mean, the terms of the per-pixel depth t*."""
    out = np.zeros(scene.n, RAYDEPTH_DTYPE)
    c = camera(cam)
    lib().orc_raydepth_setup(scene.n, _p(_f32(scene.means)), _p(_f32(scene.log_scales)),
                             _p(_f32(scene.quats)), ctypes.byref(c), _p(out))
    return out


def render_resort(scene, cam, tile: int = 16, dec=None, proj=None, tile_mask: Optional[np.ndarray] = None,
                  alpha_win: float = ALPHA_WIN, t_win: float = T_WIN, tie_win: float = TIE_WIN):
    """Per-pixel depth order (Sec. 3.2 popping fix): RGB [3,H,W], Eq. 1 depth of the per-pixel
    depths [H,W], final T [H,W], knife-edge flags (bit 1 alpha, bit 2 T, bit 4 a run of near-tied
    depths, bit 8 such a run at the stopping candidate), the number of blended splats per pixel
    and `tie_bound` [H,W], the most any order of the near-tied runs can move a colour channel."""
    dec = decide(scene, cam, tile) if dec is None else dec
    proj = project(scene, cam) if proj is None else proj
    rd = raydepth(scene, cam)
    H, W = cam.height, cam.width
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), T=np.ones((H, W)),
               flags=np.zeros((H, W), np.uint8), n_blend=np.zeros((H, W), np.int32),
               tie_bound=np.zeros((H, W)))
    c = camera(cam)
    fo = OrcFlagOpts(alpha_win, t_win)
    tm = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    lib().orc_render_resort(scene.n, _p(dec["visible"]), _p(dec["depth"]), _p(dec["rect"]), _p(proj), _p(rd),
                            ctypes.byref(c), tile, ctypes.byref(fo), float(tie_win),
                            None if tm is None else _p(tm), _p(out["rgb"]), _p(out["depth"]), _p(out["T"]),
                            _p(out["flags"]), _p(out["n_blend"]), _p(out["tie_bound"]))
    return out


def render_bwd(scene, cam, dL_drgb, dL_ddepth, dL_dT=None, tile: int = 16, dec=None, proj=None):
    """Per-Gaussian 2D gradients [N, 10] (d ubar, d vbar, d conic a/b/c, d opacity, d rgb, d depth)."""
    dec = decide(scene, cam, tile) if dec is None else dec
    proj = project(scene, cam) if proj is None else proj
    g2 = np.zeros((scene.n, 10), np.float64)
    gr = np.ascontiguousarray(dL_drgb, np.float64)
    gd = np.ascontiguousarray(dL_ddepth, np.float64)
    gt = None if dL_dT is None else np.ascontiguousarray(dL_dT, np.float64)
    c = camera(cam)
    lib().orc_render_bwd(scene.n, _p(dec["visible"]), _p(dec["depth"]), _p(dec["rect"]), _p(proj),
                         ctypes.byref(c), tile, _p(gr), _p(gd), None if gt is None else _p(gt),
                         _p(g2))
    return g2


def param_grads(scene, cam, g2, dec=None, tile: int = 16, acc=None) -> Dict[str, np.ndarray]:
    """Chain rule from [N,10] 2D gradients to parameter gradients (FP64, accumulated)."""
    dec = decide(scene, cam, tile) if dec is None else dec
    n = scene.n
    K = scene.sh.shape[1]
    if acc is None:
        acc = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                   opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)))
    c = camera(cam)
    g2 = np.ascontiguousarray(g2, np.float64)
    lib().orc_param_grads(n, _p(_f32(scene.means)), _p(_f32(scene.log_scales)),
                          _p(_f32(scene.quats)), _p(_f32(scene.opacity_logits)),
                          _p(_f32(scene.sh)), K, ctypes.byref(c), _p(dec["visible"]), _p(g2),
                          _p(acc["means"]), _p(acc["log_scales"]), _p(acc["quats"]),
                          _p(acc["opacity_logits"]), _p(acc["sh"]))
    return acc


def grads(scene, cam, dL_drgb, dL_ddepth, dL_dT=None, tile: int = 16):
    """Full reverse pass of one view: parameter gradients in FP64."""
    dec = decide(scene, cam, tile)
    proj = project(scene, cam)
    g2 = render_bwd(scene, cam, dL_drgb, dL_ddepth, dL_dT, tile, dec, proj)
    return param_grads(scene, cam, g2, dec, tile)


# ---------------------------------------------------------------------------
# Integer binning and sort of a multi-view batch (Sec. 1: tiling and sorting of
# all primitives), written directly from the key definition.

def grid(cam, tile: int):
    return (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile


def bin_sort(scenes: Sequence, views: Sequence, tile: int = 16, decs: Optional[List] = None):
    """Sorted 64-bit keys, record indices, per-tile [start, end) ranges and per-record counts."""
    rec_base, tile_base = [], []
    r = t = 0
    for v in views:
        rec_base.append(r)
        tile_base.append(t)
        r += scenes[v.scene].n
        gw, gh = grid(v, tile)
        t += gw * gh
    n_tiles = t
    keys, vals = [], []
    counts = np.zeros(r, np.int64)
    if decs is None:
        decs = [decide(scenes[v.scene], v, tile) for v in views]
    for vi, (v, d) in enumerate(zip(views, decs)):
        gw, _ = grid(v, tile)
        vis = np.nonzero(d["visible"])[0]
        rect = d["rect"][vis].astype(np.int64)
        nx = rect[:, 1] - rect[:, 0]
        ny = rect[:, 3] - rect[:, 2]
        cnt = nx * ny
        counts[rec_base[vi] + vis] = cnt
        if cnt.sum() == 0:
            continue
        owner = np.repeat(np.arange(len(vis)), cnt)
        start = np.cumsum(cnt) - cnt
        k = np.arange(cnt.sum()) - np.repeat(start, cnt)
        ox = k % np.repeat(nx, cnt)
        oy = k // np.repeat(nx, cnt)
        tx = rect[owner, 0] + ox
        ty = rect[owner, 2] + oy
        tid = tile_base[vi] + ty * gw + tx
        dbits = d["depth"][vis].view(np.uint32).astype(np.uint64)[owner]
        keys.append((tid.astype(np.uint64) << np.uint64(32)) | dbits)
        vals.append((rec_base[vi] + vis[owner]).astype(np.uint32))
    if keys:
        keys = np.concatenate(keys)
        vals = np.concatenate(vals)
    else:
        keys = np.zeros(0, np.uint64)
        vals = np.zeros(0, np.uint32)
    order = np.lexsort((vals, keys))
    keys, vals = keys[order], vals[order]
    tiles_of = (keys >> np.uint64(32)).astype(np.int64)
    ranges = np.zeros((n_tiles, 2), np.int64)
    if len(keys):
        ids = np.arange(n_tiles)
        ranges[:, 0] = np.searchsorted(tiles_of, ids, side="left")
        ranges[:, 1] = np.searchsorted(tiles_of, ids, side="right")
        ranges[ranges[:, 0] == ranges[:, 1]] = 0      # an empty tile's range is {0, 0}
    return dict(keys=keys, vals=vals, ranges=ranges, counts=counts, rec_base=rec_base,
                tile_base=tile_base)


def cull_points(points, cam, x0: int, y0: int, depth, T_final, alpha_min: float = CULL_ALPHA_MIN,
                rel_margin: float = CULL_REL_MARGIN, abs_margin: float = CULL_ABS_MARGIN) -> np.ndarray:
    """Sec. 3.3 occlusion culling of neural points against the Eq. 1 depth map.

    points [m, 3] world positions; cam the subfrustum (foveal crop) camera whose
    pixel (i, j) is pixel (i + x0, j + y0) of `depth` / `T_final` ([H, W]).
    Returns uint8 [m]: 0 outside the subfrustum, 1 occluded, 2 kept (FP32 decisions)."""
    pts = _f32(points).reshape(-1, 3)
    d = _f32(depth)
    t = _f32(T_final)
    assert d.shape == t.shape and d.ndim == 2
    out = np.zeros(len(pts), np.uint8)
    o = OrcCullOpts(float(np.float32(alpha_min)), float(np.float32(rel_margin)),
                    float(np.float32(abs_margin)), 0)
    c = camera(cam)
    lib().orc_cull_points(len(pts), _p(pts), ctypes.byref(c), int(x0), int(y0), _p(d), _p(t),
                          d.shape[1], d.shape[0], ctypes.byref(o), _p(out))
    return out


# Defaults of Sec. 3.4: fovea radius 256 px, blending interval start m = 0.75, edge weight 0.2.
COMBINE_DF, COMBINE_M, COMBINE_GAMMA = 256.0, 0.75, 0.2


def combine(P, F, x0: int, y0: int, ex: float, ey: float, d_f: float = COMBINE_DF, m: float = COMBINE_M,
            gamma: float = COMBINE_GAMMA):
    """Sec. 3.4 combination of the periphery P [3, H, W] and the foveal crop image F [3, h, w]
    placed at (x0, y0) in P, fixation (ex, ey) in P's pixel frame.  Returns (out [3, h, w], c [h, w])."""
    Pf = _f32(P)
    Ff = _f32(F)
    _, ph, pw = Pf.shape
    _, h, w = Ff.shape
    assert 0 <= x0 and 0 <= y0 and x0 + w <= pw and y0 + h <= ph
    out = np.zeros((3, h, w), np.float64)
    c = np.zeros((h, w), np.float64)
    lib().orc_combine(_p(Pf), pw, ph, _p(Ff), w, h, int(x0), int(y0), float(ex), float(ey), float(d_f),
                      float(m), float(gamma), _p(out), _p(c))
    return out, c


def combine_bwd(P, F, x0: int, y0: int, ex: float, ey: float, g, d_f: float = COMBINE_DF,
                m: float = COMBINE_M, gamma: float = COMBINE_GAMMA):
    """Reverse pass of `combine`: (dL/dP [3, H, W] (nonzero on the window only), dL/dF [3, h, w])
    for the upstream gradient g = dL/dout [3, h, w]."""
    Pf = _f32(P)
    Ff = _f32(F)
    _, ph, pw = Pf.shape
    _, h, w = Ff.shape
    gg = np.ascontiguousarray(g, np.float64)
    dP = np.zeros((3, ph, pw), np.float64)
    dF = np.zeros((3, h, w), np.float64)
    lib().orc_combine_bwd(_p(Pf), pw, ph, _p(Ff), w, h, int(x0), int(y0), float(ex), float(ey), float(d_f),
                          float(m), float(gamma), _p(gg), _p(dP), _p(dF))
    return dP, dF


# Sec. 3.5: the Gaussian branch's loss weights D-SSIM by lambda = 0.2 (as 3DGS).
LOSS_LAMBDA = 0.2


def image_loss(image, target, lam: float = LOSS_LAMBDA, grad: bool = True):
    """L = (1 - lambda) L1 + lambda (1 - SSIM) of image against target ([C, H, W]).
    Returns (L, L1, SSIM, dL/dimage [C, H, W] or None), in FP64."""
    x = _f32(image)
    y = _f32(target)
    assert x.shape == y.shape and x.ndim == 3
    C, H, W = x.shape
    out = np.zeros(3)
    g = np.zeros(x.shape) if grad else None
    lib().orc_image_loss(_p(x), _p(y), C, H, W, float(lam), _p(out), None if g is None else _p(g))
    return float(out[0]), float(out[1]), float(out[2]), g


# Sec. 4 "Training": opacity decay factor and pruning threshold.
DECAY_FACTOR, PRUNE_THRESHOLD = 0.999, 0.005


def opacity_decay(logits, factor: float = DECAY_FACTOR, threshold: float = PRUNE_THRESHOLD):
    """(new logits, new opacities, keep mask) after multiplying every opacity by `factor`."""
    lg = _f32(logits).reshape(-1)
    nl = np.zeros(len(lg))
    no = np.zeros(len(lg))
    keep = np.zeros(len(lg), np.uint8)
    lib().orc_opacity_decay(len(lg), _p(lg), float(factor), float(threshold), _p(nl), _p(no), _p(keep))
    return nl, no, keep
