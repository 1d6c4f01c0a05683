"""PyTorch front end of libvrs: device memory, streams and autograd glue only.

Every step of the rasterizer runs in libvrs's CUDA kernels through the C-ABI
(``_lib``); this module allocates the workspace and outputs with torch, passes
torch's current stream, and splits the packed outputs per view.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@dataclass
class SceneTensors:
    """One scene's Gaussian parameters as contiguous float32 CUDA tensors.

    For inference a scene may carry `baked` attributes (see `baked_scene`), and its
    SH coefficients may be float16 (see `half_sh`)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_degree: int
    baked: Optional[torch.Tensor] = None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda", requires_grad=False) -> "SceneTensors":
        def t(a):
            x = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device)
            return x.requires_grad_(requires_grad) if requires_grad else x
        return SceneTensors(t(scene.means), t(scene.log_scales), t(scene.quats),
                            t(scene.opacity_logits), t(scene.sh), int(scene.sh_degree))

    def tensors(self):
        return [getattr(self, k) for k in PARAM_NAMES]

    def zeros_like(self) -> "SceneTensors":
        return SceneTensors(*[torch.zeros_like(x, requires_grad=False) for x in self.tensors()],
                            self.sh_degree)

    def baked_scene(self, stream=None) -> "SceneTensors":
        """The same scene with its activations baked by vrs_bake (Sec. 4 "Inference"):
        renders bit for bit like this one, without evaluating them per frame."""
        baked = torch.empty((self.n, L.VRS_BAKED_FLOATS), dtype=torch.float32, device=self.means.device)
        L._check(L.vrs_bake(scene_struct(self), baked.data_ptr() if self.n else None, _stream_handle(stream)),
                 "vrs_bake")
        return SceneTensors(self.means, self.log_scales, self.quats, self.opacity_logits, self.sh,
                            self.sh_degree, baked)

    def half_sh(self) -> "SceneTensors":
        """The same scene with its SH coefficients stored in float16 (inference)."""
        return SceneTensors(self.means, self.log_scales, self.quats, self.opacity_logits,
                            self.sh.to(torch.float16).contiguous(), self.sh_degree, self.baked)


def scene_struct(st: SceneTensors) -> L.vrs_scene:
    s = L.vrs_scene()
    for name in PARAM_NAMES:
        x = getattr(st, name)
        ok_dtype = x.dtype == torch.float32 or (name == "sh" and x.dtype == torch.float16)
        if x.numel() and (not x.is_cuda or not ok_dtype or not x.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor (sh may be float16)")
        setattr(s, name, x.data_ptr() if x.numel() else None)
    s.n = st.n
    s.sh_degree = st.sh_degree
    s.sh_half = 1 if st.sh.dtype == torch.float16 else 0
    if st.baked is not None:
        b = st.baked
        if not b.is_cuda or b.dtype != torch.float32 or not b.is_contiguous() or tuple(b.shape) != (st.n, L.VRS_BAKED_FLOATS):
            raise ValueError("baked must be a contiguous float32 CUDA tensor [n, 16]")
        s.baked = b.data_ptr() if st.n else None
    return s


def camera_struct(cam) -> L.vrs_camera:
    c = L.vrs_camera()
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
    c.width, c.height, c.scene = int(cam.width), int(cam.height), int(cam.scene)
    return c


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Rasterizer:
    """A planned batch of views over one or more scenes, with its workspace and outputs."""

    def __init__(self, scenes: Sequence[SceneTensors], views: Sequence, tile: int = 16,
                 persistent: int = 0, backward: bool = False, max_instances: int = 0,
                 sort: int = 0, resort: int = 0, half_out: bool = False, key_bits: int = 0,
                 tiles_per_pull: int = 1, device="cuda"):
        self.scenes = list(scenes)
        self.views = list(views)
        self.device = torch.device(device)
        self.tile = tile
        self.persistent = int(persistent)       # 0 per tile, 1 heaviest first, 2 tile order
        self.backward = bool(backward)
        self.sort = int(sort)
        self.resort = int(resort)    # 0: list order; 4/8/16: per-pixel order through a window of that size
        self.half_out = bool(half_out)   # outputs as float16 (inference)
        self.key_bits = int(key_bits)    # radix key width, 0 = minimal
        self.tiles_per_pull = int(tiles_per_pull)
        self.generation = 0          # forward passes and re-plans; the autograd glue checks it
        self._make_plan(max_instances)

    # -- planning ------------------------------------------------------------------------
    def _make_plan(self, max_instances: int):
        self.generation = getattr(self, "generation", 0) + 1     # a new workspace: old state is gone
        n_s, n_v = len(self.scenes), len(self.views)
        self._scene_arr = (L.vrs_scene * n_s)(*[scene_struct(s) for s in self.scenes])
        self._view_arr = (L.vrs_camera * n_v)(*[camera_struct(v) for v in self.views])
        opts = L.vrs_plan_opts(self.tile, int(self.persistent), int(self.backward), self.sort,
                               int(max_instances), 0, self.resort, int(self.half_out), self.key_bits,
                               self.tiles_per_pull, 0)
        plan = L.vrs_plan()
        L._check(L.vrs_plan_batch(self._scene_arr, n_s, self._view_arr, n_v, opts, plan), "vrs_plan_batch")
        self.plan = plan
        self.workspace = torch.empty(int(plan.workspace_bytes), dtype=torch.uint8, device=self.device)
        P = int(plan.n_pixels)
        dt = torch.float16 if self.half_out else torch.float32
        self.rgb = torch.empty(3 * P, dtype=dt, device=self.device)
        self.depth = torch.empty(P, dtype=dt, device=self.device)
        self.T = torch.empty(P, dtype=dt, device=self.device)

    def set_views(self, views: Sequence):
        """New poses for views of the same sizes (no re-plan)."""
        self.views = list(views)
        self._view_arr = (L.vrs_camera * len(self.views))(*[camera_struct(v) for v in self.views])

    def set_scenes(self, scenes: Sequence[SceneTensors]):
        self.scenes = list(scenes)
        self._scene_arr = (L.vrs_scene * len(self.scenes))(*[scene_struct(s) for s in self.scenes])

    # -- the three steps -----------------------------------------------------------------
    def preprocess(self, stream=None):
        L._check(L.vrs_preprocess(self.plan, self._scene_arr, self._view_arr,
                                  self.workspace.data_ptr(), _stream_handle(stream)), "vrs_preprocess")

    def bin_sort(self, stream=None):
        L._check(L.vrs_bin_sort(self.plan, self.workspace.data_ptr(), _stream_handle(stream)),
                 "vrs_bin_sort")

    def render_fwd(self, rgb=None, depth=None, T=None, stream=None):
        rgb = self.rgb if rgb is None else rgb
        depth = self.depth if depth is None else depth
        T = self.T if T is None else T
        L._check(L.vrs_render_fwd(self.plan, self.workspace.data_ptr(), rgb.data_ptr(),
                                  depth.data_ptr(), T.data_ptr(), _stream_handle(stream)),
                 "vrs_render_fwd")

    def forward_async(self, stream=None):
        """The whole forward path, stream ordered, no host synchronisation."""
        self.generation += 1
        self.preprocess(stream)
        self.bin_sort(stream)
        self.render_fwd(stream=stream)

    def count_pairs(self, stream=None):
        """One counting forward pass (untimed use): Gaussian-pixel pairs evaluated by the
        definition and blended, and (instance, 8x8 block) pairs the blend kernel evaluated."""
        self.preprocess(stream)
        self.bin_sort(stream)
        self.plan.count_pairs = 1
        try:
            self.render_fwd(stream=stream)
        finally:
            self.plan.count_pairs = 0
        info = L.vrs_run_info()
        L._check(L.vrs_query_status(self.plan, self.workspace.data_ptr(), info, _stream_handle(stream)),
                 "count_pairs")
        return int(info.pair_evals), int(info.pair_blends), int(info.block_evals)

    def status(self, stream=None):
        info = L.vrs_run_info()
        code = L.vrs_query_status(self.plan, self.workspace.data_ptr(), info, _stream_handle(stream))
        self.visible_pairs = int(sum(info.visible_pairs[: len(self.scenes)]))
        return code, int(info.flags), int(info.instances)

    def forward(self, stream=None, check: bool = True, grow: bool = True):
        """Forward path; on a capacity overflow re-plans with room for the measured count."""
        self.forward_async(stream)
        if not check:
            return
        code, flags, inst = self.status(stream)
        if code == L.VRS_ERR_CAPACITY and grow:
            self._make_plan(int(inst * 1.25) + 65536)
            self.forward_async(stream)
            code, flags, inst = self.status(stream)
        if code not in (L.VRS_OK, L.VRS_ERR_NONFINITE, L.VRS_ERR_INVALID):
            raise L.VrsError(code, "forward")
        self.last_status = (code, flags, inst)

    def backward_params(self, dL_drgb, dL_ddepth, dL_dT=None, grads: Optional[List[SceneTensors]] = None,
                        stream=None) -> List[SceneTensors]:
        """Accumulates parameter gradients (+=) for upstream gradients of the packed outputs."""
        if grads is None:
            grads = [s.zeros_like() for s in self.scenes]
        garr = (L.vrs_scene * len(grads))(*[scene_struct(g) for g in grads])
        dT = dL_dT.data_ptr() if dL_dT is not None else None
        L._check(L.vrs_render_bwd(self.plan, self.workspace.data_ptr(), self._scene_arr,
                                  self._view_arr, self.T.data_ptr(), dL_drgb.data_ptr(),
                                  dL_ddepth.data_ptr(), dT, garr, _stream_handle(stream)),
                 "vrs_render_bwd")
        return grads

    # -- views of the packed outputs and the workspace ------------------------------------------
    def view_slices(self, v: int):
        p = self.plan
        b = int(p.view_pix_base[v])
        W, H = int(p.view_w[v]), int(p.view_h[v])
        return b, W, H

    def outputs(self, v: int, rgb=None, depth=None, T=None):
        b, W, H = self.view_slices(v)
        rgb = self.rgb if rgb is None else rgb
        depth = self.depth if depth is None else depth
        T = self.T if T is None else T
        return (rgb[3 * b:3 * b + 3 * W * H].view(3, H, W), depth[b:b + W * H].view(H, W),
                T[b:b + W * H].view(H, W))

    def ws_view(self, off: int, count: int, dtype) -> torch.Tensor:
        nbytes = count * torch.tensor([], dtype=dtype).element_size()
        return self.workspace[off:off + nbytes].view(dtype)

    def sorted_lists(self):
        p = self.plan
        _, _, inst = self.status()
        m = min(inst, int(p.max_instances))
        keys = self.ws_view(int(p.off_keys[p.sorted_buf]), m, torch.int64)
        vals = self.ws_view(int(p.off_vals[p.sorted_buf]), m, torch.int32)
        ranges = self.ws_view(int(p.off_ranges), 2 * int(p.n_tiles), torch.int32).view(-1, 2)
        return keys, vals, ranges

    def decisions(self, v: int):
        """The preprocess's integer decisions for view v, read back from the visible-pair
        list (valid after preprocess, until a backward reuses the list): a uint8 visibility
        flag per Gaussian of the view's scene and the tile rectangles [n, 4] as
        (x0, x1, y0, y1), zero where not visible."""
        p = self.plan
        sc = int(p.view_scene[v])
        n = int(p.scene_n[sc])
        base = 0
        for s in range(sc):
            base += int(p.scene_n[s]) * sum(1 for w in range(int(p.n_views)) if int(p.view_scene[w]) == s)
        vlist = [w for w in range(int(p.n_views)) if int(p.view_scene[w]) == sc]
        info = L.vrs_run_info()
        L._check(L.vrs_query_status(self.plan, self.workspace.data_ptr(), info, _stream_handle(None)),
                 "decisions")
        cnt = min(int(info.visible_pairs[sc]), n * len(vlist))
        e = self.ws_view(int(p.off_pairs) + 32 * base, 8 * cnt, torch.int32).view(-1, 8)[:, :4]
        e = e.cpu().numpy().view(np.uint32)
        sel = e[:, 1] == vlist.index(v)
        g = e[sel, 0].astype(np.int64)
        vis = np.zeros(n, np.uint8)
        rect = np.zeros((n, 4), np.int32)
        vis[g] = 1
        rect[g, 0] = e[sel, 2] & 0xffff
        rect[g, 1] = e[sel, 2] >> 16
        rect[g, 2] = e[sel, 3] & 0xffff
        rect[g, 3] = e[sel, 3] >> 16
        return vis, rect

    def records(self) -> torch.Tensor:
        p = self.plan
        return self.ws_view(int(p.off_records), 12 * int(p.n_records), torch.float32).view(-1, 12)

    def resort_flags(self) -> torch.Tensor:
        """Per-pixel order plans: 1 where a pixel's sorting window could not restore its order."""
        p = self.plan
        if not int(p.resort):
            raise ValueError("not a per-pixel order plan")
        return self.ws_view(int(p.off_resort_flags), int(p.n_pixels), torch.uint8)

    def resort_flagged(self, stream=None) -> int:
        info = L.vrs_run_info()
        L._check(L.vrs_query_status(self.plan, self.workspace.data_ptr(), info, _stream_handle(stream)),
                 "resort_flagged")
        return int(info.resort_flagged)

    def n_contrib(self) -> torch.Tensor:
        """Each pixel's last blended list position + 1 (written for backward plans only)."""
        p = self.plan
        return self.ws_view(int(p.off_ncontrib), int(p.n_pixels), torch.int32)


class VrsRenderFunction(torch.autograd.Function):
    """Differentiable forward of a Rasterizer over its scenes' parameter tensors.

    forward(ras, *params) -> (rgb, depth, T) packed over views; params are the
    scenes' [means, log_scales, quats, opacity_logits, sh] in scene order.

    The backward reads the rasterizer's workspace (records, sorted lists, last
    blended positions) and its T, which the next forward overwrites; so one
    forward per backward: a backward whose rasterizer has run another forward
    (or was re-planned) since raises instead of returning wrong gradients.
    """

    @staticmethod
    def forward(ctx, ras: Rasterizer, *params):
        ras.forward()
        ctx.ras = ras
        ctx.generation = ras.generation
        return ras.rgb.clone(), ras.depth.clone(), ras.T.clone()

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_T):
        ras = ctx.ras
        if ras.generation != ctx.generation:
            raise RuntimeError("the Rasterizer ran another forward pass (or was re-planned) after the one "
                               "being differentiated; its workspace no longer holds that pass's state. "
                               "Call backward before the next render(ras), or use one Rasterizer per "
                               "graph")
        g_rgb = torch.zeros_like(ras.rgb) if g_rgb is None else g_rgb.contiguous()
        g_depth = torch.zeros_like(ras.depth) if g_depth is None else g_depth.contiguous()
        g_T = None if g_T is None else g_T.contiguous()
        grads = ras.backward_params(g_rgb, g_depth, g_T)
        out = [None]
        for g in grads:
            out.extend(g.tensors())
        return tuple(out)


def render(ras: Rasterizer):
    """Autograd-aware forward: returns packed (rgb, depth, T)."""
    params = []
    for s in ras.scenes:
        params.extend(s.tensors())
    return VrsRenderFunction.apply(ras, *params)
