"""The inference variants of Sec. 4 "Inference": baked attributes and half precision.

Bars:
  - a baked scene (vrs_bake) renders bit for bit the images, sorted lists and
    status of its parameter form: per-tile order, per-pixel order, several
    views and scenes, and with zero-quaternion and non-finite Gaussians;
  - half outputs equal the FP32 outputs rounded to binary16, bit for bit;
  - SH coefficients stored in binary16 render like the oracle fed the same
    (rounded) coefficients, within the FP32 bars plus one binary16 rounding of
    the output (2^-11 relative) when the output is half too;
  - the reverse pass refuses baked or half scenes and half-output plans.
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import DEPTH_ABS, DEPTH_REL, FLAG_FRAC, RGB_TOL, T_TOL, torch_cuda

pytestmark = pytest.mark.gpu

HALF_REL = 2.0 ** -11      # one rounding to binary16


def _sts(scenes):
    from paper_2410_17932_gb300.render import SceneTensors
    return [SceneTensors.from_scene(s) for s in scenes]


def _render(sts, views, **kw):
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer
    ras = Rasterizer(sts, views, **kw)
    ras.forward()
    torch.cuda.synchronize()
    return ras


def _same(a, b):
    torch = torch_cuda()
    for x, y in ((a.rgb, b.rgb), (a.depth, b.depth), (a.T, b.T)):
        assert torch.equal(x, y)
    ka, va, ra = a.sorted_lists()
    kb, vb, rb = b.sorted_lists()
    assert torch.equal(ka, kb) and torch.equal(va, vb) and torch.equal(ra, rb)
    assert a.last_status == b.last_status


@pytest.mark.parametrize("resort", [0, 8])
def test_baked_scene_is_bit_identical(resort):
    scs, cams = I.plain_200()
    sts = _sts(scs)
    _same(_render(sts, cams, resort=resort), _render([s.baked_scene() for s in sts], cams, resort=resort))


def test_baked_bench_frame_and_multiview_bit_identical():
    scenes, views = I.periphery_stereo_05m()
    sts = _sts(scenes)
    _same(_render(sts, views), _render([s.baked_scene() for s in sts], views))
    scenes, views = I.batched_multiview(scale=0.01)
    sts = _sts(scenes)
    _same(_render(sts, views, persistent=True), _render([s.baked_scene() for s in sts], views, persistent=True))


def test_baked_status_rules():
    scs, cams = I.plain_200()
    sc = scs[0].subset(np.arange(400))
    sc.quats[3] = 0.0
    sc.log_scales[7, 1] = np.nan
    sc.means[9, 0] = np.inf
    sc.sh[11, 0, 2] = np.inf
    sts = _sts([sc])
    a = _render(sts, cams)
    b = _render([s.baked_scene() for s in sts], cams)
    assert a.last_status[1] & 1 and a.last_status[1] & 2
    _same(a, b)


def test_half_outputs_are_the_rounded_fp32_outputs():
    torch = torch_cuda()
    scenes, views = I.periphery_stereo_05m()
    sts = _sts(scenes)
    for resort in (0, 8):
        a = _render(sts, views, resort=resort)
        b = _render(sts, views, resort=resort, half_out=True)
        assert b.rgb.dtype == torch.float16
        for x, y in ((a.rgb, b.rgb), (a.depth, b.depth), (a.T, b.T)):
            assert torch.equal(x.half(), y)


@pytest.mark.parametrize("half_out", [False, True])
def test_half_sh_against_oracle(half_out):
    """0.5 M SH-3 Gaussians with binary16 coefficients, both eyes, every pixel."""
    scenes, views = I.periphery_stereo_05m()
    sts = [s.half_sh() for s in _sts(scenes)]
    ras = _render(sts, views, half_out=half_out)
    sc16 = scenes[0].subset(np.arange(scenes[0].n))
    sc16.sh = scenes[0].sh.astype(np.float16).astype(np.float32)
    rel = HALF_REL if half_out else 0.0
    for v, cam in enumerate(views):
        orc = oracle.render(sc16, cam)
        rgb, depth, T = [x.float().cpu().numpy().astype(np.float64) for x in ras.outputs(v)]
        ok = orc["flags"] == 0
        assert (~ok).mean() <= FLAG_FRAC
        e_rgb = np.abs(rgb - orc["rgb"]).max(axis=0)[ok]
        tol_rgb = RGB_TOL + rel * np.abs(orc["rgb"]).max(axis=0)[ok]
        assert np.all(e_rgb <= tol_rgb), e_rgb.max()
        assert np.all(np.abs(T - orc["T"])[ok] <= T_TOL + rel * orc["T"][ok])
        d = np.abs(orc["depth"][ok])
        assert np.all(np.abs(depth - orc["depth"])[ok] <= (DEPTH_REL + rel) * d + DEPTH_ABS)
        print(f"half sh, half out {half_out}, view {v}: worst rgb {e_rgb.max():.2e}")


def test_reverse_pass_refuses_inference_forms():
    torch = torch_cuda()
    from paper_2410_17932_gb300 import _lib as L
    from paper_2410_17932_gb300.render import Rasterizer
    scs, cams = I.plain_200()
    sts = _sts(scs)
    with pytest.raises(L.VrsError):
        Rasterizer(sts, cams, backward=True, half_out=True)
    for inf in (sts[0].baked_scene(), sts[0].half_sh()):
        ras = Rasterizer([inf], cams, backward=True)
        ras.forward()
        g = torch.zeros_like(ras.rgb)
        with pytest.raises(L.VrsError):
            ras.backward_params(g, torch.zeros_like(ras.depth), grads=[sts[0].zeros_like()])
