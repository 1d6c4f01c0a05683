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


def test_combine_reverse_pass_matches_oracle():
    torch = torch_cuda()
    from paper_2410_17932_gb300.combine import foveal_combine_bwd
    P, F = _images(90, 120, 60, 70, 5)
    x0, y0, ex, ey, d_f, m, gamma = 20, 15, 52.0, 41.0, 40.0, 0.3, 0.6
    rng = np.random.default_rng(6)
    g = rng.standard_normal(F.shape).astype(np.float32)
    dP_ref, dF_ref = oracle.combine_bwd(P, F, x0, y0, ex, ey, g, d_f=d_f, m=m, gamma=gamma)
    Pt, Ft = torch.as_tensor(P, device="cuda"), torch.as_tensor(F, device="cuda")
    dP, dF = foveal_combine_bwd(Pt, Ft, x0, y0, ex, ey, torch.as_tensor(g, device="cuda"), d_f=d_f, m=m,
                                gamma=gamma)
    dP, dF = dP.cpu().numpy(), dF.cpu().numpy()
    for got, ref in ((dP, dP_ref), (dF, dF_ref)):
        assert np.abs(got - ref).max() <= 1e-4 * (1 + np.abs(ref).max())
    assert np.abs(dF_ref).max() > 0.1 and np.abs(dP_ref).max() > 0.1


def test_combine_autograd_function():
    torch = torch_cuda()
    from paper_2410_17932_gb300.combine import FovealCombineFunction
    P, F = _images(50, 60, 30, 34, 8)
    Pt = torch.as_tensor(P, device="cuda").requires_grad_(True)
    Ft = torch.as_tensor(F, device="cuda").requires_grad_(True)
    out = FovealCombineFunction.apply(Pt, Ft, 10, 9, 27.0, 24.0, 20.0, 0.4, 0.5)
    ref, _ = oracle.combine(P, F, 10, 9, 27.0, 24.0, d_f=20.0, m=0.4, gamma=0.5)
    assert np.abs(out.detach().cpu().numpy() - ref).max() <= TOL
    (out * out).sum().backward()
    dP_ref, dF_ref = oracle.combine_bwd(P, F, 10, 9, 27.0, 24.0, 2 * ref, d_f=20.0, m=0.4, gamma=0.5)
    assert np.abs(Pt.grad.cpu().numpy() - dP_ref).max() <= 1e-4 * (1 + np.abs(dP_ref).max())
    assert np.abs(Ft.grad.cpu().numpy() - dF_ref).max() <= 1e-4 * (1 + np.abs(dF_ref).max())
