"""Foveal neural-point occlusion culling (Sec. 3.3) on the Eq. 1 depth buffer.

Marshalling only: the decision runs in libvrs (vrs_cull_points).  After the
periphery is rendered, the subfrustum camera of the gaze (a crop of the eye,
``Camera.crop``) projects the neural points; points outside it are discarded
and points behind the Gaussians' surface are culled.
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch

from . import _lib as L
from .render import _stream_handle, camera_struct

OUTSIDE, OCCLUDED, KEPT = 0, 1, 2


class PointCuller:
    """Output buffers for culling up to `capacity` points; reusable across frames and
    capturable in a CUDA graph (no allocation, no synchronisation in `cull_async`)."""

    def __init__(self, capacity: int, device: str = "cuda"):
        self.capacity = int(capacity)
        self.mask = torch.empty(self.capacity, dtype=torch.uint8, device=device)
        self.kept = torch.empty(self.capacity, dtype=torch.int32, device=device)   # uint32 bits
        self.n_kept = torch.zeros(1, dtype=torch.int64, device=device)             # uint64 bits

    def cull_async(self, points: torch.Tensor, fovea, x0: int, y0: int, depth: torch.Tensor,
                   T_final: torch.Tensor, alpha_min: float = 0.5, rel_margin: float = 0.02,
                   abs_margin: float = 0.05, stream: Optional[torch.cuda.Stream] = None,
                   write_kept: bool = True) -> None:
        """points [m, 3] float32 CUDA; depth, T_final [H, W] float32 CUDA (the eye's view)."""
        m = int(points.shape[0])
        if m > self.capacity:
            raise ValueError(f"{m} points exceed the culler's capacity {self.capacity}")
        for t in (points, depth, T_final):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("points, depth and T_final must be contiguous float32 CUDA tensors")
        H, W = int(depth.shape[-2]), int(depth.shape[-1])
        self._cam = camera_struct(fovea)
        self._opts = L.vrs_cull_opts(alpha_min, rel_margin, abs_margin, 0)
        L._check(L.vrs_cull_points(points.data_ptr(), m, self._cam, int(x0), int(y0), depth.data_ptr(),
                                   T_final.data_ptr(), W, H, self._opts, self.mask.data_ptr(),
                                   self.kept.data_ptr() if write_kept else None,
                                   self.n_kept.data_ptr(), _stream_handle(stream)), "vrs_cull_points")

    def cull(self, points, fovea, x0, y0, depth, T_final, **kw) -> Tuple[torch.Tensor, torch.Tensor]:
        """Synchronous form: (mask [m] uint8, kept indices [n_kept] int32)."""
        self.cull_async(points, fovea, x0, y0, depth, T_final, **kw)
        n = int(self.n_kept.item())
        return self.mask[: points.shape[0]], self.kept[:n]
