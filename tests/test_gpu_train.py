"""GPU parity of the training-loop pieces (Sec. 3.5, Sec. 4 "Training") against the oracle.

Bars: the loss L, L1 and SSIM within 1e-5 relative of the FP64 oracle; dL/dimage
element by element within 1e-4 of its largest magnitude (plus 1e-12); a whole
training step (render, loss, reverse pass) against the oracle's chain to the
Gaussian parameters with the backward bars (1e-3 norm-wise, 1e-3 of the largest
magnitude element-wise); the opacity decay's logits within 1e-4 (1 + |logit|),
and its keep mask equal to the oracle's except where the FP64 opacity is within
1e-6 of the threshold.
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

NAMES = ["means", "log_scales", "quats", "opacity_logits", "sh"]


def _target_near(x, seed):
    """A target image near x whose every value differs from x by at least 0.01 (no L1 kink)."""
    rng = np.random.default_rng(seed)
    d = (0.01 + np.abs(rng.normal(0, 0.05, x.shape))) * np.where(rng.uniform(size=x.shape) < 0.5, -1, 1)
    return (x + d).astype(np.float32)


def _loss_check(x, y, label):
    torch = torch_cuda()
    from paper_2410_17932_gb300 import train
    xt = torch.as_tensor(x, device="cuda")
    yt = torch.as_tensor(y, device="cuda")
    out, g = train.image_loss(xt, yt)
    out = out.cpu().numpy().astype(np.float64)
    g = g.cpu().numpy().astype(np.float64)
    L, l1, ssim, gr = oracle.image_loss(x, y)
    for a, b in zip(out, (L, l1, ssim)):
        assert a == pytest.approx(b, rel=1e-5), (label, out, (L, l1, ssim))
    err = np.abs(g - gr).max() / (np.abs(gr).max() + 1e-12)
    print(label, "loss", out, "grad err / max", err)
    assert np.all(np.abs(g - gr) <= 1e-4 * np.abs(gr).max() + 1e-12)


@pytest.mark.parametrize("shape", [(3, 37, 45), (3, 200, 200), (1, 9, 70), (3, 8, 32)])
def test_loss_random_images(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.uniform(0, 1, shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, shape), 0, 1).astype(np.float32)
    _loss_check(x, y, f"random {shape}")


def test_loss_training_view_full_size():
    """The rendered 1264x832 training view against a nearby target."""
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    scs, cams = I.training_view_1m()
    ras = Rasterizer([SceneTensors.from_scene(scs[0])], cams)
    ras.forward()
    torch.cuda.synchronize()
    x = ras.outputs(0)[0].cpu().numpy()
    _loss_check(x, _target_near(x, 5), "training view")


def test_training_step_against_oracle_chain():
    """render -> loss -> backward on the GPU against oracle render -> oracle loss gradient ->
    oracle reverse pass, on the 64x64 / 200-Gaussian subset of the training workload."""
    torch = torch_cuda()
    from paper_2410_17932_gb300 import train
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors, render
    rng = np.random.default_rng(11)
    scs, _ = I.training_view_1m(n=200, seed=311)
    sc = scs[0]
    cam = I.Camera(np.eye(3), np.zeros(3), 60.0, 60.0, 32.0, 32.0, 64, 64)
    sc.means[:, 0] = rng.uniform(-1.2, 1.2, sc.n)
    sc.means[:, 1] = rng.uniform(-1.2, 1.2, sc.n)
    sc.means[:, 2] = rng.uniform(2.0, 5.0, sc.n)
    sc.log_scales[:] = rng.normal(-2.6, 0.4, sc.log_scales.shape).astype(np.float32)
    orc = oracle.render(sc, cam)
    target = _target_near(orc["rgb"].astype(np.float32), 12)
    _, _, _, g_img = oracle.image_loss(orc["rgb"].astype(np.float32), target)
    ref = oracle.grads(sc, cam, g_img, np.zeros((64, 64)), None)
    st = SceneTensors.from_scene(sc, requires_grad=True)
    ras = Rasterizer([st], [cam], backward=True)
    rgb, _, _ = render(ras)
    loss = train.ImageLossFunction.apply(rgb.view(3, 64, 64), torch.as_tensor(target, device="cuda"))
    loss.backward()
    for k in NAMES:
        a = getattr(st, k).grad.cpu().numpy().astype(np.float64).reshape(-1)
        b = np.asarray(ref[k]).reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        el = (np.abs(a - b) / (1e-3 * np.abs(b).max() + 1e-12)).max()
        print("training step", k, rel, el)
        assert rel < 1e-3 and el <= 1.0, k


def test_opacity_decay_against_oracle():
    torch = torch_cuda()
    from paper_2410_17932_gb300 import train
    rng = np.random.default_rng(3)
    logits = np.concatenate([rng.normal(0, 3, 100_000), np.linspace(-5.4, -5.2, 20_001),
                             [-30.0, 30.0, 0.0]]).astype(np.float32)
    t = torch.as_tensor(logits, device="cuda")
    keep, cnt = train.opacity_decay(t)
    nl, no, kp = oracle.opacity_decay(logits)
    got = t.cpu().numpy().astype(np.float64)
    fin = np.isfinite(nl)
    assert np.all(np.abs(got[fin] - nl[fin]) <= 1e-4 * (1 + np.abs(nl[fin])))
    k = keep.cpu().numpy()
    edge = np.abs(no - oracle.PRUNE_THRESHOLD) <= 1e-6
    assert np.array_equal(k[~edge], kp[~edge])
    assert int(cnt.item()) == int(k.sum())
