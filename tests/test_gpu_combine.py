"""GPU parity of the Sec. 3.4 foveal combination with the FP64 oracle.

Bar: every output channel and the factor c within 1e-5 absolute (FP32 arithmetic on values in
[0, 1]; every step of the definition is continuous, so there are no knife edges)."""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _run(P, F, x0, y0, ex, ey, **kw):
    torch = torch_cuda()
    from paper_2410_17932_gb300.combine import foveal_combine
    Pt = torch.as_tensor(P, device="cuda")
    Ft = torch.as_tensor(F, device="cuda")
    c = torch.empty(F.shape[1:], dtype=torch.float32, device="cuda")
    out = foveal_combine(Pt, Ft, x0, y0, ex, ey, c_out=c, **kw)
    return out.cpu().numpy(), c.cpu().numpy()


def _check(P, F, x0, y0, ex, ey, **kw):
    ref, cref = oracle.combine(P, F, x0, y0, ex, ey, **kw)
    out, c = _run(P, F, x0, y0, ex, ey, **kw)
    assert np.abs(out - ref).max() <= TOL and np.abs(c - cref).max() <= TOL
    return cref


def _images(H, W, h, w, seed):
    rng = np.random.default_rng(seed)
    # smooth structure plus texture, so that the edge factor varies
    yy, xx = np.mgrid[0:h, 0:w]
    F = (0.5 + 0.3 * np.sin(xx[None] / (7.0 + np.arange(3)[:, None, None])) * np.cos(yy[None] / 5.0)
         + 0.05 * rng.standard_normal((3, h, w))).astype(np.float32)
    P = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    return P, F


def test_combine_full_size_foveal_crop():
    sc, eye, crop, _ = I.foveal_points_5m(n_points=1)
    x0, y0 = int(round(eye.cx - crop.cx)), int(round(eye.cy - crop.cy))
    P, F = _images(eye.height, eye.width, crop.height, crop.width, 1)
    c = _check(P, F, x0, y0, x0 + 256.0 + 3.3, y0 + 256.0 - 7.9)
    assert c.max() == 1.0 and c.min() == 0.0 and ((c > 0.05) & (c < 0.95)).sum() > 10000


@pytest.mark.parametrize("H,W,h,w,x0,y0", [(40, 50, 40, 50, 0, 0), (300, 400, 1, 1, 17, 33), (300, 400, 5, 1, 0, 295),
                                           (300, 400, 37, 45, 355, 263), (120, 90, 33, 70, 20, 87)])
def test_combine_ragged_windows(H, W, h, w, x0, y0):
    P, F = _images(H, W, h, w, H + w)
    _check(P, F, x0, y0, x0 + w * 0.4, y0 + h * 0.6, d_f=0.5 * max(h, w) + 1.0)


def test_combine_options():
    P, F = _images(200, 260, 150, 170, 9)
    _check(P, F, 40, 30, 120.0, 100.0, d_f=60.0, m=0.5, gamma=1.5)
    _check(P, F, 40, 30, 120.0, 100.0, d_f=300.0, m=-0.5, gamma=0.0)
