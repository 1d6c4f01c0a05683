"""Pins of the oracle's Sec. 3.4 combination of the peripheral and foveal images, each against
something other than the oracle's own code: the smootherstep's printed values at hand-worked
radii, the Sobel magnitude of linear ramps (interior and replicated border), identity when both
images agree, convexity, and transpose symmetry."""
import numpy as np

import oracle


def _flat(v, h, w):
    return np.full((3, h, w), v, np.float32)


def test_positional_factor_closed_form(orc):
    """A flat foveal image has no edges: c is 1 inside m * d_f, 0 at d_f and beyond, and on the
    band follows 1 - S2((r - m) / (1 - m)); S2(1/2) = 1/2 and S2(1/4) = 53/512 by hand."""
    H, W, h, w = 64, 80, 64, 80
    P, F = _flat(0.0, H, W), _flat(1.0, h, w)
    d_f, m = 40.0, 0.75
    ex, ey = 40.0, 32.0
    out, c = oracle.combine(P, F, 0, 0, ex, ey, d_f=d_f, m=m, gamma=0.2)
    jj, ii = np.mgrid[0:h, 0:w]
    r = np.hypot(ii + 0.5 - ex, jj + 0.5 - ey) / d_f
    assert np.all(c[r <= m] == 1.0) and np.all(c[r >= 1.0] == 0.0)
    # pixels whose centre lies exactly at the radii where f_p = 1/2 and 1/4
    for fp, s2 in ((0.5, 0.5), (0.25, 53.0 / 512.0)):
        rr = m + fp * (1 - m)
        out1, c1 = oracle.combine(P, F, 0, 0, 0.5 + rr * d_f, 0.5, d_f=d_f, m=m, gamma=0.2)
        assert abs(c1[0, 0] - (1.0 - s2)) < 1e-12
        assert abs(out1[1, 0, 0] - (1.0 - s2)) < 1e-12      # (1 - c) * 0 + c * 1
    assert np.allclose(out[0], c)


def test_sobel_of_linear_ramps(orc):
    """F = a i + b j in every channel: inside, f_e = sqrt(a^2 + b^2); on the left and right
    columns the replicated border halves the x slope.  Checked through c on the band, where
    c = 1 - S2(f_p + gamma f_e) is invertible."""
    h, w = 24, 30
    a, b = 0.03, -0.02
    jj, ii = np.mgrid[0:h, 0:w].astype(np.float64)
    F = np.broadcast_to((a * ii + b * jj)[None], (3, h, w)).astype(np.float32)
    P = np.zeros((3, h, w), np.float32)
    # put every pixel on the band with f_p = 0.1: a huge d_f and a fixation far away
    d_f, m = 1e6, 0.75
    ex = 0.5 + (m + 0.1 * (1 - m)) * d_f
    _, c = oracle.combine(P, F, 0, 0, ex, 0.5, d_f=d_f, m=m, gamma=0.2)
    fp = (np.hypot(ii + 0.5 - ex, jj) / d_f - m) / (1 - m)
    # invert S2 on (0, 1) by bisection
    lo, hi = np.zeros_like(c), np.ones_like(c)
    target = 1.0 - c
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        s = mid ** 3 * (mid * (6 * mid - 15) + 10)
        lo, hi = np.where(s < target, mid, lo), np.where(s < target, hi, mid)
    fe = (0.5 * (lo + hi) - fp) / 0.2
    Fd = F[0].astype(np.float64)
    inner = fe[1:-1, 1:-1]
    assert np.allclose(inner, np.hypot(a, b), atol=2e-6)
    edge_x = np.hypot(a / 2, b)
    assert np.allclose(fe[1:-1, 0], edge_x, atol=2e-6) and np.allclose(fe[1:-1, -1], edge_x, atol=2e-6)
    assert np.allclose(fe[0, 1:-1], np.hypot(a, b / 2), atol=2e-6)
    assert Fd.shape == (h, w)


def test_identity_convexity_and_transpose(orc):
    rng = np.random.default_rng(3)
    H, W, h, w, x0, y0 = 50, 60, 30, 36, 11, 7
    P = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    F = rng.uniform(0, 1, (3, h, w)).astype(np.float32)
    ex, ey, d_f = 30.3, 22.7, 14.0
    # both images agree on the window: the output is that image wherever c is
    Fw = np.ascontiguousarray(P[:, y0:y0 + h, x0:x0 + w])
    out, c = oracle.combine(P, Fw, x0, y0, ex, ey, d_f=d_f)
    assert np.allclose(out, Fw, atol=1e-12) and 0 < c.mean() < 1
    # convex mixture per channel
    out, c = oracle.combine(P, F, x0, y0, ex, ey, d_f=d_f)
    Pw = P[:, y0:y0 + h, x0:x0 + w].astype(np.float64)
    lo = np.minimum(Pw, F) - 1e-12
    hi = np.maximum(Pw, F) + 1e-12
    assert np.all((out >= lo) & (out <= hi)) and np.all((c >= 0) & (c <= 1))
    # transposing both images and swapping the fixation coordinates transposes the result
    outT, cT = oracle.combine(np.ascontiguousarray(P.transpose(0, 2, 1)), np.ascontiguousarray(F.transpose(0, 2, 1)),
                              y0, x0, ey, ex, d_f=d_f)
    assert np.allclose(outT, out.transpose(0, 2, 1), atol=1e-12) and np.allclose(cT, c.T, atol=1e-12)


def test_reverse_pass_matches_central_differences(orc):
    """The oracle's reverse pass against FP64 central differences of its forward, on images
    quantised to 2^-10 so that the +-h perturbations (h = 2^-10) are exact in FP32, with the
    blending band over the whole crop so that the edge-factor path is exercised."""
    rng = np.random.default_rng(21)
    H, W, h, w, x0, y0 = 24, 30, 14, 16, 6, 5
    q = 1.0 / 1024
    P = (np.round(rng.uniform(0.1, 0.9, (3, H, W)) / q) * q).astype(np.float32)
    yy, xx = np.mgrid[0:h, 0:w]
    F = 0.5 + 0.3 * np.sin(xx / 3.0)[None] * np.cos(yy / 2.5)[None] + 0.05 * rng.standard_normal((3, h, w))
    F = (np.round(F / q) * q).astype(np.float32)
    ex, ey, d_f, m, gamma = x0 + 3.3, y0 + 2.2, 14.0, 0.2, 0.8
    g = rng.standard_normal((3, h, w))
    dP, dF = orc.combine_bwd(P, F, x0, y0, ex, ey, g, d_f=d_f, m=m, gamma=gamma)
    _, c = orc.combine(P, F, x0, y0, ex, ey, d_f=d_f, m=m, gamma=gamma)
    assert ((c > 0.02) & (c < 0.98)).mean() > 0.5            # most of the crop is on the band

    def loss(Pv, Fv):
        out, _ = orc.combine(Pv, Fv, x0, y0, ex, ey, d_f=d_f, m=m, gamma=gamma)
        return float((out * g).sum())

    hh = q
    picks_F = [(ch, jy, ix) for ch in range(3) for jy, ix in ((0, 0), (h - 1, w - 1), (0, 7), (5, 0), (6, 9), (9, 4))]
    for ch, jy, ix in picks_F:
        Fp, Fm = F.copy(), F.copy()
        Fp[ch, jy, ix] += hh
        Fm[ch, jy, ix] -= hh
        fd = (loss(P, Fp) - loss(P, Fm)) / (2 * hh)
        assert abs(fd - dF[ch, jy, ix]) <= 2e-4 * (1 + abs(fd)), (ch, jy, ix, fd, dF[ch, jy, ix])
    for ch, jy, ix in ((0, y0, x0), (1, y0 + 7, x0 + 9), (2, y0 + h - 1, x0 + w - 1), (0, 0, 0)):
        Pp, Pm = P.copy(), P.copy()
        Pp[ch, jy, ix] += hh
        Pm[ch, jy, ix] -= hh
        fd = (loss(Pp, F) - loss(Pm, F)) / (2 * hh)
        assert abs(fd - dP[ch, jy, ix]) <= 2e-4 * (1 + abs(fd)), (ch, jy, ix, fd, dP[ch, jy, ix])
