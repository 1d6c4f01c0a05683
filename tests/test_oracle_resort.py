"""Pins of the per-pixel depth order (the popping fix of Sec. 3.2).

`oracle.render_resort` orders each pixel's splats by t*, the camera-space depth
of the 3D Gaussian's density maximum along the pixel's ray, and accumulates
Eq. 1 with d_i = t*.  Pinned by: the closed form of t* for an isotropic splat
(the projection of the mean onto the ray); two thin slanted splats that cross,
whose order flips across the image exactly where their planes cross (the
plain per-tile order cannot follow that); equality with the plain
compositing where every pixel's order is the list order; input-permutation
invariance over every order of a tiny scene; and the near-tie bound against
the other order of an exact tie.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2410_17932_gb300 import inputs as I


def _scene(means, log_scales, quats, logits, rgb):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = len(means)
    y00 = 0.5 / math.sqrt(math.pi)
    sh = ((np.asarray(rgb, np.float64).reshape(n, 1, 3) - 0.5) / y00).astype(np.float32)
    return I.Scene(means, np.asarray(log_scales, np.float32).reshape(n, 3),
                   np.asarray(quats, np.float32).reshape(n, 4), np.asarray(logits, np.float32).reshape(n), sh, 0)


def test_isotropic_splat_depth_is_the_projection_of_its_mean(orc):
    """For Sigma = s^2 I, t* = (r . mu) / (r . r): the mean projected onto the ray."""
    m = np.array([0.12, -0.07, 2.5], np.float32).astype(np.float64)
    s = _scene(m, [math.log(0.15)] * 3, [1, 0, 0, 0], [2.0], [[0.2, 0.5, 0.8]])
    cam = I.identity_camera(48, 40, 90.0)
    out = orc.render_resort(s, cam)
    plain = orc.render(s, cam)
    jj, ii = np.mgrid[0:40, 0:48]
    rx, ry = (ii + 0.5 - cam.cx) / cam.fx, (jj + 0.5 - cam.cy) / cam.fy
    t = (rx * m[0] + ry * m[1] + m[2]) / (rx * rx + ry * ry + 1.0)
    cov = 1.0 - out["T"]
    hit = cov > 0
    assert hit.sum() > 200
    np.testing.assert_allclose(out["depth"][hit], (t * cov)[hit], rtol=1e-12)
    for k in ("rgb", "T"):
        np.testing.assert_array_equal(out[k], plain[k])      # one splat: order plays no part


def _plane_splat(z0, slope, sign):
    """A thin square splat centred on the optical axis at depth z0, tilted so that its plane
    is z = z0 + sign * slope * x (its normal in the x-z plane), 1000x thinner than wide."""
    ang = math.atan(slope) * sign
    # rotate about the camera y axis by -ang: the local x axis becomes (cos, 0, sin(ang))
    q = [math.cos(-ang / 2), 0.0, math.sin(-ang / 2), 0.0]
    return [0.0, 0.0, z0], [math.log(0.6), math.log(0.6), math.log(0.0006)], q


def test_crossing_thin_splats_swap_order_where_their_planes_cross(orc):
    """Two thin splats through the same centre with planes z = z0 +- k x cross on the line x = 0:
    on pixels left of the principal point the + plane is nearer, right of it the - plane.  For a
    thin splat t* is the ray-plane intersection z0 / (1 -+ k rx) (to its thickness), so the image
    is the two-splat formula with that order and those depths."""
    z0, k = 3.0, 0.8
    m1, ls1, q1 = _plane_splat(z0, k, +1)
    m2, ls2, q2 = _plane_splat(z0, k, -1)
    c1, c2 = [0.9, 0.1, 0.1], [0.1, 0.1, 0.9]
    s = _scene([m1, m2], [ls1, ls2], [q1, q2], [1.5, 1.5], [c1, c2])
    cam = I.identity_camera(64, 32, 60.0)
    cam.cx = 32.25                   # no pixel centre on the crossing line
    out = orc.render_resort(s, cam)
    proj = orc.project(s, cam)
    plain = orc.render(s, cam)
    checked = 0
    for j in range(32):
        for i in range(64):
            px, py = i + 0.5 - cam.cx, j + 0.5 - cam.cy
            rx = px / cam.fx
            al = []
            for g in range(2):
                a, b, c = proj["conic"][g]
                dx, dy = proj["ubar"][g] - px, proj["vbar"][g] - py
                al.append(min(0.99, proj["opacity"][g] * math.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)))
            if min(al) < 1 / 255 + 1e-3:
                continue
            t = [z0 / (1 - k * rx), z0 / (1 + k * rx)]         # ray-plane intersections
            f, bk = (0, 1) if t[0] < t[1] else (1, 0)
            rgb = np.array(proj["rgb"][f]) * al[f] + np.array(proj["rgb"][bk]) * al[bk] * (1 - al[f])
            dep = t[f] * al[f] + t[bk] * al[bk] * (1 - al[f])
            np.testing.assert_allclose(out["rgb"][:, j, i], rgb, rtol=1e-9, atol=1e-12)
            assert out["depth"][j, i] == pytest.approx(dep, rel=2e-6)
            checked += 1
    assert checked > 1000
    # the per-tile order is one order for the whole image: it disagrees on one side
    left = out["rgb"][0, :, :30] > out["rgb"][2, :, :30]        # red in front left of the line
    right = out["rgb"][2, :, 34:] > out["rgb"][0, :, 34:]       # blue in front right of it
    assert left.mean() > 0.9 and right.mean() > 0.9
    assert not np.allclose(plain["rgb"], out["rgb"], atol=1e-3)


def test_list_order_scene_equals_plain_compositing(orc):
    """Small isotropic splats far apart in depth: every pixel's order is the mean-depth order,
    so colour and transmittance equal the plain compositing exactly."""
    rng = np.random.default_rng(4)
    n = 20
    z = 2.0 + 1.0 * np.arange(n)
    # |rx dx + ry dy| < 1 for any two means on any ray of the view: r . mu keeps the z order
    xy = rng.uniform(-0.05, 0.05, (n, 2)) * z[:, None]
    s = _scene(np.column_stack([xy, z]), np.log(0.04 * z)[:, None].repeat(3, 1),
               [[1, 0, 0, 0]] * n, rng.normal(0.5, 1.0, n), rng.uniform(0, 1, (n, 3)))
    cam = I.identity_camera(64, 64, 80.0)
    a = orc.render_resort(s, cam)
    b = orc.render(s, cam)
    assert (a["T"] < 0.5).sum() > 150           # splats overlap: their order decides these pixels
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    np.testing.assert_array_equal(a["T"], b["T"])


def test_permutation_invariance_exhaustive_tiny(orc):
    sc = I.uniform_box_scene(6, 11, xy=(-0.15, 0.15), z=(2, 3), log_scale=(-2.5, 0.3))
    cam = I.identity_camera(48, 48, 150.0)
    base = orc.render_resort(sc, cam)
    assert (base["T"] < 1).sum() > 100
    for perm in itertools.permutations(range(6)):
        out = orc.render_resort(sc.subset(list(perm)), cam)
        for k in ("rgb", "depth", "T"):
            assert np.array_equal(out[k], base[k]), (perm, k)


def test_near_tie_bound_covers_the_other_order(orc):
    """Two splats with the same mean and covariance tie exactly at every pixel (order by index);
    swapping their indices gives the other order, whose colour lies within tie_bound."""
    m = [0.0, 0.0, 2.0]
    ls = [math.log(0.1)] * 3
    s1 = _scene([m, m], [ls, ls], [[1, 0, 0, 0]] * 2, [0.5, 1.5], [[1, 0, 0], [0, 0, 1]])
    s2 = s1.subset([1, 0])
    cam = I.identity_camera(32, 32, 60.0)
    a = orc.render_resort(s1, cam)
    b = orc.render_resort(s2, cam)
    hit = a["tie_bound"] > 0
    assert hit.sum() > 100 and np.all(a["flags"][hit] & 4)
    diff = np.abs(a["rgb"] - b["rgb"]).max(axis=0)
    assert diff[hit].max() > 1e-3                              # the orders really differ
    assert np.all(diff <= a["tie_bound"] + 1e-12)
    np.testing.assert_allclose(a["T"], b["T"], rtol=1e-14)     # T does not depend on the order
