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


def foveal_combine_bwd(P: torch.Tensor, F: torch.Tensor, x0: int, y0: int, ex: float, ey: float,
                       dL_dout: torch.Tensor, d_f: float = 256.0, m: float = 0.75, gamma: float = 0.2,
                       dL_dP: Optional[torch.Tensor] = None, dL_dF: Optional[torch.Tensor] = None,
                       stream: Optional[torch.cuda.Stream] = None):
    """Gradients of the combination: (dL/dP [3, H, W], dL/dF [3, h, w]), accumulated into the given
    tensors (zeros when not given)."""
    _, H, W = P.shape
    _, h, w = F.shape
    g = dL_dout.contiguous()
    if dL_dP is None:
        dL_dP = torch.zeros_like(P)
    if dL_dF is None:
        dL_dF = torch.zeros_like(F)
    scratch = torch.empty((h, w), dtype=torch.float32, device=F.device)
    opts = L.vrs_combine_opts(d_f, m, gamma, 0)
    L._check(L.vrs_foveal_combine_bwd(P.data_ptr(), W, H, F.data_ptr(), w, h, int(x0), int(y0), float(ex),
                                      float(ey), opts, g.data_ptr(), dL_dP.data_ptr(), dL_dF.data_ptr(),
                                      scratch.data_ptr(), _stream_handle(stream)), "vrs_foveal_combine_bwd")
    return dL_dP, dL_dF


class FovealCombineFunction(torch.autograd.Function):
    """Differentiable Sec. 3.4 combination: out = combine(P, F) over the crop window."""

    @staticmethod
    def forward(ctx, P, F, x0, y0, ex, ey, d_f=256.0, m=0.75, gamma=0.2):
        P = P.contiguous()
        F = F.contiguous()
        ctx.save_for_backward(P, F)
        ctx.args = (x0, y0, ex, ey, d_f, m, gamma)
        return foveal_combine(P, F, x0, y0, ex, ey, d_f=d_f, m=m, gamma=gamma)

    @staticmethod
    def backward(ctx, g):
        P, F = ctx.saved_tensors
        x0, y0, ex, ey, d_f, m, gamma = ctx.args
        dP, dF = foveal_combine_bwd(P, F, x0, y0, ex, ey, g, d_f=d_f, m=m, gamma=gamma)
        return dP, dF, None, None, None, None, None, None, None
