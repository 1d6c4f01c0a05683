"""Pins of the training-loss and opacity-decay oracle (Sec. 3.5, Sec. 4 "Training").

The loss is (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2, with SSIM as Wang
et al. define it (11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2,
the window zero outside the image).  Pinned by: SSIM(x, x) = 1 with zero
gradient; the closed form for two constant images, whose only ingredient is the
window mass inside the image, computed here from the 1-D Gaussian on its own;
symmetry; the L1 term against numpy; central differences of the loss on
values whose perturbations are exact in FP32; and the decay's closed form.
"""
import math

import numpy as np
import pytest

C1, C2 = 0.01 ** 2, 0.03 ** 2


def _g1():
    g = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    return g / g.sum()


def _mass(n):
    """Window mass inside [0, n) at every position, along one axis."""
    g = _g1()
    return np.array([sum(g[k] for k in range(11) if 0 <= i + k - 5 < n) for i in range(n)])


def test_identical_images(orc):
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (3, 23, 31)).astype(np.float32)
    L, l1, ssim, g = orc.image_loss(x, x)
    assert L == 0.0 and l1 == 0.0 and ssim == pytest.approx(1.0, abs=1e-14)
    assert np.abs(g).max() < 1e-15


@pytest.mark.parametrize("a,b", [(0.3, 0.7), (0.9, 0.1), (0.5, 0.5)])
def test_constant_images_closed_form(orc, a, b):
    """For x = a, y = b: mu = a m, w * x^2 = a^2 m, so s_x^2 = a^2 m (1 - m), s_xy = a b m (1 - m)
    with m the window mass inside the image (m = 1 away from the border)."""
    H, W = 17, 26
    m = np.outer(_mass(H), _mass(W))
    x = np.full((1, H, W), a, np.float32)
    y = np.full((1, H, W), b, np.float32)
    a, b = float(np.float32(a)), float(np.float32(b))
    v = m * (1 - m)
    S = (2 * a * b * m * m + C1) * (2 * a * b * v + C2) / (((a * a + b * b) * m * m + C1) * ((a * a + b * b) * v + C2))
    L, l1, ssim, _ = orc.image_loss(x, y)
    assert ssim == pytest.approx(S.mean(), rel=1e-12)
    assert l1 == pytest.approx(abs(a - b), rel=1e-12, abs=1e-15)
    assert L == pytest.approx(0.8 * abs(a - b) + 0.2 * (1 - S.mean()), rel=1e-12, abs=1e-15)


def test_symmetry_and_l1(orc):
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3, 19, 21)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1).astype(np.float32)
    a = orc.image_loss(x, y, grad=False)
    b = orc.image_loss(y, x, grad=False)
    assert a[2] == pytest.approx(b[2], rel=1e-13)
    assert a[1] == pytest.approx(np.abs(x.astype(np.float64) - y).mean(), rel=1e-13)
    assert 0 < a[2] < 1


@pytest.mark.parametrize("lam", [0.2, 1.0, 0.0])
def test_gradient_against_central_differences(orc, lam):
    rng = np.random.default_rng(2)
    q = 2.0 ** -12
    x = (np.round(rng.uniform(0.1, 0.9, (2, 14, 15)) / q) * q).astype(np.float32)
    y = (np.round(rng.uniform(0.1, 0.9, (2, 14, 15)) / q) * q).astype(np.float32)
    y[np.abs(x - y) < 4 * q] += np.float32(8 * q)       # keep |x - y| away from the L1 kink
    _, _, _, g = orc.image_loss(x, y, lam)
    h = np.float32(q)
    for idx in [(0, 0, 0), (0, 7, 7), (1, 13, 14), (1, 3, 11), (0, 10, 2), (1, 0, 8)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (orc.image_loss(xp, y, lam, grad=False)[0] - orc.image_loss(xm, y, lam, grad=False)[0]) / (2 * float(h))
        assert g[idx] == pytest.approx(fd, rel=2e-5, abs=1e-12), (idx, g[idx], fd)


def test_opacity_decay_closed_form(orc):
    logits = np.array([-8.0, -5.3, -5.29, 0.0, 2.0, 9.0], np.float32)
    nl, no, keep = orc.opacity_decay(logits)
    o = 1.0 / (1.0 + np.exp(-logits.astype(np.float64)))
    np.testing.assert_allclose(no, 0.999 * o, rtol=1e-15)
    np.testing.assert_allclose(1.0 / (1.0 + np.exp(-nl)), 0.999 * o, rtol=1e-13)
    assert list(keep) == [int(v >= 0.005) for v in 0.999 * o]
    assert keep[0] == 0 and keep[3] == 1
    # the threshold lies between logits -5.3 and -5.29 after the decay
    assert keep[1] == 0 and keep[2] == 1
