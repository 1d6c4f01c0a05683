"""Training-loop pieces of the Gaussian branch (Sec. 3.5, Sec. 4 "Training"): argument
marshalling for libvrs's loss and opacity-decay kernels, and the autograd glue of the loss.

image_loss(image, target) -> (L, L1, SSIM) as a device tensor [3] and dL/dimage, with
L = (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2.  ImageLossFunction makes L a
differentiable torch scalar, so that render() -> loss -> backward() runs end to end in
libvrs's kernels.  opacity_decay() multiplies opacities by 0.999 in place and returns the
keep mask of the 0.005 pruning threshold.
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch

from . import _lib as L

LOSS_LAMBDA = 0.2
DECAY_FACTOR, PRUNE_THRESHOLD = 0.999, 0.005


def _stream(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_img(x: torch.Tensor, name: str):
    if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous() or x.dim() != 3:
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor [C, H, W]")


def image_loss(image: torch.Tensor, target: torch.Tensor, lam: float = LOSS_LAMBDA, grad: bool = True,
               stream=None) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
    """(loss [3] = (L, L1, SSIM) on the device, dL/dimage or None)."""
    _check_img(image, "image")
    _check_img(target, "target")
    if image.shape != target.shape:
        raise ValueError("image and target differ in shape")
    C, H, W = image.shape
    nbytes = L.vrs_image_loss_scratch(C, H, W)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=image.device)
    out = torch.empty(3, dtype=torch.float32, device=image.device)
    g = torch.empty_like(image) if grad else None
    L._check(L.vrs_image_loss(image.data_ptr(), target.data_ptr(), C, H, W, float(lam), out.data_ptr(),
                              g.data_ptr() if g is not None else None, scratch.data_ptr(), nbytes,
                              _stream(stream)), "vrs_image_loss")
    return out, g


class ImageLossFunction(torch.autograd.Function):
    """L = (1 - lambda) L1 + lambda (1 - SSIM) as a differentiable scalar of the image."""

    @staticmethod
    def forward(ctx, image, target, lam=LOSS_LAMBDA):
        out, g = image_loss(image.detach().contiguous(), target.contiguous(), lam, grad=True)
        ctx.save_for_backward(g)
        return out[0]

    @staticmethod
    def backward(ctx, gL):
        (g,) = ctx.saved_tensors
        return g * gL, None, None


def opacity_decay(logits: torch.Tensor, factor: float = DECAY_FACTOR, threshold: float = PRUNE_THRESHOLD,
                  stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
    """In place on `logits` (float32 CUDA [n]); returns (keep mask uint8 [n], kept count [1])."""
    if not logits.is_cuda or logits.dtype != torch.float32 or not logits.is_contiguous():
        raise ValueError("logits must be a contiguous float32 CUDA tensor")
    n = logits.numel()
    keep = torch.empty(n, dtype=torch.uint8, device=logits.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=logits.device)
    L._check(L.vrs_opacity_decay(logits.data_ptr() if n else None, n, float(factor), float(threshold),
                                 keep.data_ptr() if n else None, cnt.data_ptr(), _stream(stream)),
             "vrs_opacity_decay")
    return keep, cnt
