"""Sec. 3.4 combination of the peripheral and foveal images (marshalling only; the math runs in
libvrs, vrs_foveal_combine)."""
from __future__ import annotations

from typing import Optional

import torch

from . import _lib as L
from .render import _stream_handle


def foveal_combine(P: torch.Tensor, F: torch.Tensor, x0: int, y0: int, ex: float, ey: float,
                   d_f: float = 256.0, m: float = 0.75, gamma: float = 0.2,
                   out: Optional[torch.Tensor] = None, c_out: Optional[torch.Tensor] = None,
                   stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """P [3, H, W] periphery, F [3, h, w] foveal image of the crop at (x0, y0), fixation (ex, ey)
    in P's pixel frame; returns the combined crop [3, h, w] (written into `out` when given)."""
    for t in (P, F):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.dim() == 3 and t.shape[0] == 3):
            raise ValueError("P and F must be contiguous float32 CUDA tensors of shape [3, H, W]")
    _, H, W = P.shape
    _, h, w = F.shape
    if out is None:
        out = torch.empty_like(F)
    opts = L.vrs_combine_opts(d_f, m, gamma, 0)
    L._check(L.vrs_foveal_combine(P.data_ptr(), W, H, F.data_ptr(), w, h, int(x0), int(y0), float(ex), float(ey),
                                  opts, out.data_ptr(), c_out.data_ptr() if c_out is not None else None,
                                  _stream_handle(stream)), "vrs_foveal_combine")
    return out
