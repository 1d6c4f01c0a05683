"""Parameter and gradient arrays that start 4 bytes past a 16-byte boundary.

The kernels read quaternions and SH rows, and add SH-gradient rows, as 16-byte
vectors only where the array allows it, element by element otherwise: both forms
give the same images bit for bit and the same gradients (up to the order of the
record-gradient atomics, 1e-6 relative)."""
import numpy as np
import pytest

from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

NAMES = ["means", "log_scales", "quats", "opacity_logits", "sh"]


def _offset_copy(x):
    """x in a buffer one float past its start (4-byte aligned, not 16)."""
    torch = torch_cuda()
    buf = torch.zeros(x.numel() + 1, dtype=x.dtype, device=x.device)
    y = buf[1:].view(x.shape)
    y.copy_(x)
    assert y.data_ptr() % 16 != 0 and y.is_contiguous()
    return y


def _scene():
    scs, _ = I.training_view_1m(n=400, seed=21)
    sc = scs[0]
    rng = np.random.default_rng(5)
    sc.means[:, 0] = rng.uniform(-1.0, 1.0, sc.n)
    sc.means[:, 1] = rng.uniform(-1.0, 1.0, sc.n)
    sc.means[:, 2] = rng.uniform(2.0, 5.0, sc.n)
    sc.log_scales[:] = rng.normal(-2.8, 0.4, sc.log_scales.shape).astype(np.float32)
    cam = I.Camera(np.eye(3), np.zeros(3), 70.0, 70.0, 48.0, 40.0, 96, 80)
    return sc, cam


def test_unaligned_parameters_and_gradients():
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    sc, cam = _scene()
    a = SceneTensors.from_scene(sc)
    b = SceneTensors(*[_offset_copy(x) for x in a.tensors()], a.sh_degree)
    ra = Rasterizer([a], [cam], backward=True)
    rb = Rasterizer([b], [cam], backward=True)
    ra.forward()
    rb.forward()
    torch.cuda.synchronize()
    for x, y in ((ra.rgb, rb.rgb), (ra.depth, rb.depth), (ra.T, rb.T)):
        assert torch.equal(x, y)
    rng = np.random.default_rng(9)
    g_rgb = torch.as_tensor(rng.normal(0, 1, ra.rgb.numel()).astype(np.float32), device="cuda")
    g_d = torch.as_tensor(rng.normal(0, 1, ra.depth.numel()).astype(np.float32), device="cuda")
    ga = ra.backward_params(g_rgb, g_d)[0]
    zb = b.zeros_like()
    gb = SceneTensors(*[_offset_copy(x) for x in zb.tensors()], zb.sh_degree)
    rb.backward_params(g_rgb, g_d, grads=[gb])
    torch.cuda.synchronize()
    for k in NAMES:
        x = getattr(ga, k).cpu().numpy().astype(np.float64).ravel()
        y = getattr(gb, k).cpu().numpy().astype(np.float64).ravel()
        assert np.abs(x).max() > 0, k
        assert np.allclose(x, y, rtol=1e-6, atol=1e-6 * np.abs(x).max()), k


def test_unaligned_half_sh_forward():
    """binary16 SH coefficients 2 bytes past a 16-byte boundary render like aligned ones."""
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    sc, cam = _scene()
    a = SceneTensors.from_scene(sc).half_sh()
    b = SceneTensors(a.means, a.log_scales, a.quats, a.opacity_logits, _offset_copy(a.sh), a.sh_degree)
    ra = Rasterizer([a], [cam])
    rb = Rasterizer([b], [cam])
    ra.forward()
    rb.forward()
    torch.cuda.synchronize()
    for x, y in ((ra.rgb, rb.rgb), (ra.depth, rb.depth), (ra.T, rb.T)):
        assert torch.equal(x, y)
