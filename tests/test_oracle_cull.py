"""Pins of the oracle's neural-point occlusion culling (Sec. 3.3 against the
Eq. 1 depth of Sec. 3.2), each against something other than the oracle itself:
closed forms of a planar occluder, the transparency rule, the subfrustum
bounds, a depth map whose every pixel holds a different surface, the crop =
window invariance of the adapted projection, and an FP64 restatement away from
the decision boundaries."""
import numpy as np

import oracle
from paper_2410_17932_gb300 import inputs as I

A_MIN, REL, ABS = oracle.CULL_ALPHA_MIN, oracle.CULL_REL_MARGIN, oracle.CULL_ABS_MARGIN


def _ray_points(cam, ij, z):
    """World points (identity pose) on the rays through pixel centres ij at view depth z."""
    ij = np.asarray(ij, np.float64)
    x = (ij[:, 0] + 0.5 - cam.cx) / cam.fx * z
    y = (ij[:, 1] + 0.5 - cam.cy) / cam.fy * z
    return np.stack([x, y, np.broadcast_to(z, x.shape)], 1).astype(np.float32)


def test_planar_wall_closed_form(orc):
    """An opaque-enough wall at depth Zw (Eq. 1 depth = Zw * alpha, T = 1 - alpha): points
    in front of it or within the margin are kept, points behind it are culled."""
    W, H, Zw, a = 40, 30, 4.0, 0.8
    cam = I.identity_camera(W, H, 30.0)
    depth = np.full((H, W), Zw * a, np.float32)
    T = np.full((H, W), 1.0 - a, np.float32)
    rng = np.random.default_rng(1)
    ij = np.stack([rng.integers(0, W, 600), rng.integers(0, H, 600)], 1)
    lim = Zw * (1 + REL) + ABS
    z = np.concatenate([rng.uniform(0.5, Zw, 200), rng.uniform(Zw, 0.999 * lim, 200),
                        rng.uniform(1.001 * lim, 3 * Zw, 200)])
    m = oracle.cull_points(_ray_points(cam, ij, z), cam, 0, 0, depth, T)
    assert np.all(m[:400] == 2) and np.all(m[400:] == 1)


def test_transparent_pixels_never_occlude(orc):
    W, H = 24, 16
    cam = I.identity_camera(W, H, 20.0)
    for a in (0.0, 0.2, A_MIN * 0.999):
        depth = np.full((H, W), 1.0 * a, np.float32)
        T = np.full((H, W), 1.0 - a, np.float32)
        ij = np.stack(np.meshgrid(np.arange(W), np.arange(H)), -1).reshape(-1, 2)
        m = oracle.cull_points(_ray_points(cam, ij, 50.0), cam, 0, 0, depth, T)
        assert np.all(m == 2), a
    # at exactly alpha_min the pixel occludes
    a = np.float32(A_MIN)
    T = np.full((H, W), np.float32(1.0) - a, np.float32)
    depth = np.full((H, W), np.float32(2.0) * (np.float32(1.0) - T[0, 0]), np.float32)
    m = oracle.cull_points(_ray_points(cam, [[3, 4]], 50.0), cam, 0, 0, depth, T)
    assert m[0] == 1


def test_subfrustum_bounds_and_znear(orc):
    W, H = 32, 20
    cam = I.identity_camera(W, H, 25.0)
    depth = np.zeros((H, W), np.float32)
    T = np.ones((H, W), np.float32)
    z = 3.0
    inside = _ray_points(cam, [[0, 0], [W - 1, H - 1], [5, 7]], z)
    # half a pixel beyond each border, behind the camera, below znear, non-finite
    out = np.concatenate([
        _ray_points(cam, [[-1, 5], [W, 5], [5, -1], [5, H]], z),
        np.array([[0.0, 0.0, -3.0], [0.0, 0.0, 0.5 * cam.znear], [np.nan, 0.0, 3.0],
                  [0.0, np.inf, 3.0], [0.0, 0.0, np.nan]], np.float32)])
    m = oracle.cull_points(np.concatenate([inside, out]), cam, 0, 0, depth, T)
    assert list(m[:3]) == [2, 2, 2] and np.all(m[3:] == 0)


def test_every_pixel_reads_its_own_depth(orc):
    """Each pixel of a crop holds its own opaque surface depth; a point on a pixel's ray just
    behind that pixel's limit is culled and just in front is kept, which fails under any
    transposed, shifted or mis-rounded pixel index."""
    W, H, x0, y0, w, h = 48, 40, 7, 5, 20, 17
    eye = I.identity_camera(W, H, 35.0)
    crop = eye.crop(x0, y0, w, h)
    a = 0.9
    surf = 2.0 + 0.01 * np.arange(W * H, dtype=np.float64).reshape(H, W)
    depth = (surf * a).astype(np.float32)
    T = np.full((H, W), 1.0 - a, np.float32)
    ij = np.stack(np.meshgrid(np.arange(w), np.arange(h)), -1).reshape(-1, 2)
    zsurf = (depth[ij[:, 1] + y0, ij[:, 0] + x0].astype(np.float64) /
             (1.0 - T[ij[:, 1] + y0, ij[:, 0] + x0].astype(np.float64)))
    lim = zsurf * (1 + REL) + ABS
    behind = oracle.cull_points(_ray_points(crop, ij, lim + 0.004), crop, x0, y0, depth, T)
    front = oracle.cull_points(_ray_points(crop, ij, lim - 0.004), crop, x0, y0, depth, T)
    assert np.all(behind == 1) and np.all(front == 2)


def test_crop_equals_window_of_full_view(orc):
    """The subfrustum is the eye camera with a moved principal point: away from pixel edges,
    a point inside the window gets the same decision as in the full view, and a point of
    the full view outside the window is outside the subfrustum."""
    W, H = 96, 80
    eye = I.identity_camera(W, H, 60.0)
    x0, y0, w, h = 30, 22, 40, 36
    crop = eye.crop(x0, y0, w, h)
    depth, T = I.synthetic_depth_map(W, H, 11)
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(-0.8, 0.8, 20000), rng.uniform(-0.7, 0.7, 20000),
                    rng.uniform(0.5, 8.0, 20000)], 1).astype(np.float32)
    u = pts[:, 0].astype(np.float64) / pts[:, 2] * eye.fx + eye.cx
    v = pts[:, 1].astype(np.float64) / pts[:, 2] * eye.fy + eye.cy
    away = (np.abs(u - np.round(u)) > 1e-3) & (np.abs(v - np.round(v)) > 1e-3)
    full = oracle.cull_points(pts, eye, 0, 0, depth, T)
    win = oracle.cull_points(pts, crop, x0, y0, depth, T)
    inwin = (u >= x0) & (u < x0 + w) & (v >= y0) & (v < y0 + h)
    assert np.array_equal(win[away & inwin], full[away & inwin])
    assert np.all(win[away & ~inwin] == 0)
    assert (win == 1).sum() > 100 and (win == 2).sum() > 100


def test_fp64_restatement_away_from_boundaries(orc):
    """The same test written with numpy in FP64 agrees wherever no decision is within a
    relative 1e-4 of its boundary."""
    sc, eye, crop, pts = I.foveal_points_5m(n_points=200_000)
    x0, y0 = int(round(eye.cx - crop.cx)), int(round(eye.cy - crop.cy))
    depth, T = I.synthetic_depth_map(eye.width, eye.height, 5, n_rects=60)
    m = oracle.cull_points(pts, crop, x0, y0, depth, T)
    P = pts.astype(np.float64)
    R = np.asarray(crop.R, np.float64)
    X = P @ R.T + np.asarray(crop.t, np.float64)
    z = X[:, 2]
    ok = z > crop.znear
    u = crop.fx * X[:, 0] / np.where(ok, z, 1.0) + crop.cx
    v = crop.fy * X[:, 1] / np.where(ok, z, 1.0) + crop.cy
    ins = ok & (u >= 0) & (u < crop.width) & (v >= 0) & (v < crop.height)
    i = np.clip(np.floor(u), 0, crop.width - 1).astype(int) + x0
    j = np.clip(np.floor(v), 0, crop.height - 1).astype(int) + y0
    a = 1.0 - T[j, i].astype(np.float64)
    occl = a >= A_MIN
    thr = depth[j, i].astype(np.float64) / np.where(a > 0, a, 1.0) * (1 + REL) + ABS
    ref = np.where(~ins, 0, np.where(occl & (z > thr), 1, 2))
    edge = ((np.abs(z - crop.znear) < 1e-4 * np.abs(z)) |
            (np.abs(u - np.round(u)) < 1e-3) | (np.abs(v - np.round(v)) < 1e-3) |
            (np.abs(z - thr) < 1e-4 * np.abs(thr)) | (np.abs(a - A_MIN) < 1e-6))
    assert np.array_equal(m[~edge], ref[~edge])
    assert (~edge).mean() > 0.99
    assert min((m == 0).sum(), (m == 1).sum(), (m == 2).sum()) > 500
