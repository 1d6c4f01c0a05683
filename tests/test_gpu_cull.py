"""GPU parity of the neural-point occlusion culling (Sec. 3.3) with the oracle.

Bars: the three-way decision of every point bit-exact (mask), the kept-index
list equal as a set to the mask's kept points, and its count.  Depth maps are
the oracle's own render or the seeded synthetic generator (never the GPU
renderer's output).
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _gpu_cull(points, crop, x0, y0, depth, T, offset=0, **kw):
    torch = torch_cuda()
    from paper_2410_17932_gb300.cull import PointCuller
    m = len(points)
    flat = torch.zeros(3 * m + 4, dtype=torch.float32, device="cuda")
    flat[offset:offset + 3 * m] = torch.as_tensor(points.reshape(-1))
    pts = flat[offset:offset + 3 * m].view(m, 3)
    c = PointCuller(max(m, 1))
    mask, kept = c.cull(pts, crop, x0, y0, torch.as_tensor(depth, device="cuda"),
                        torch.as_tensor(T, device="cuda"), **kw)
    return mask.cpu().numpy(), kept.cpu().numpy().view(np.uint32)


def _check(points, crop, x0, y0, depth, T, **kw):
    ref = oracle.cull_points(points, crop, x0, y0, depth, T, **kw)
    mask, kept = _gpu_cull(points, crop, x0, y0, depth, T, **kw)
    assert np.array_equal(mask, ref)
    assert len(np.unique(kept)) == len(kept)
    assert np.array_equal(np.sort(kept), np.nonzero(ref == 2)[0])
    return ref


def test_cull_on_oracle_rendered_depth():
    scs, cams = I.plain_200()
    eye = cams[0]
    orc = oracle.render(scs[0], eye)
    depth, T = orc["depth"].astype(np.float32), orc["T"].astype(np.float32)
    x0, y0 = 37, 50
    crop = eye.crop(x0, y0, 100, 90)
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(-1.2, 1.2, 50_000), rng.uniform(-1.2, 1.2, 50_000),
                    rng.uniform(0.1, 7.0, 50_000)], 1).astype(np.float32)
    ref = _check(pts, crop, x0, y0, depth, T)
    assert min(np.bincount(ref, minlength=3)) > 1000


def test_cull_full_size_foveal_points():
    """5 M neural points of the foveal-points workload against a synthetic 2016x2240 map."""
    sc, eye, crop, pts = I.foveal_points_5m()
    x0, y0 = int(round(eye.cx - crop.cx)), int(round(eye.cy - crop.cy))
    depth, T = I.synthetic_depth_map(eye.width, eye.height, 9, n_rects=80)
    ref = _check(pts, crop, x0, y0, depth, T)
    assert (ref == 2).sum() > 1000 and (ref == 1).sum() > 1000


@pytest.mark.parametrize("m,offset", [(0, 0), (1, 0), (1023, 0), (1025, 1), (70_001, 1), (70_001, 0)])
def test_cull_ragged_sizes_and_unaligned_points(m, offset):
    W, H = 120, 96
    eye = I.identity_camera(W, H, 80.0)
    crop = eye.crop(10, 6, 64, 70)
    depth, T = I.synthetic_depth_map(W, H, 3)
    rng = np.random.default_rng(m)
    pts = np.stack([rng.uniform(-1, 1, m), rng.uniform(-1, 1, m), rng.uniform(-1, 9, m)], 1).astype(np.float32)
    if m > 10:
        pts[3] = [np.nan, 0.0, 2.0]
        pts[5] = [0.0, 0.0, np.inf]
    ref = oracle.cull_points(pts, crop, 10, 6, depth, T)
    mask, kept = _gpu_cull(pts, crop, 10, 6, depth, T, offset=offset)
    assert np.array_equal(mask, ref)
    assert np.array_equal(np.sort(kept), np.nonzero(ref == 2)[0])


def test_cull_options_and_graph_capture():
    torch = torch_cuda()
    from paper_2410_17932_gb300.cull import PointCuller
    W, H = 200, 160
    eye = I.identity_camera(W, H, 120.0)
    crop = eye.crop(50, 40, 100, 80)
    depth, T = I.synthetic_depth_map(W, H, 21)
    rng = np.random.default_rng(8)
    pts = np.stack([rng.uniform(-1, 1, 30000), rng.uniform(-1, 1, 30000), rng.uniform(0.5, 8, 30000)],
                   1).astype(np.float32)
    kw = dict(alpha_min=0.25, rel_margin=0.0, abs_margin=0.0)
    _check(pts, crop, 50, 40, depth, T, **kw)
    p = torch.as_tensor(pts, device="cuda")
    d = torch.as_tensor(depth, device="cuda")
    t = torch.as_tensor(T, device="cuda")
    c = PointCuller(len(pts))
    c.cull_async(p, crop, 50, 40, d, t, **kw)
    torch.cuda.synchronize()
    ref_mask = c.mask.clone()
    ref_n = int(c.n_kept.item())
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        c.cull_async(p, crop, 50, 40, d, t, stream=s, **kw)     # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            c.cull_async(p, crop, 50, 40, d, t, stream=s, **kw)
    c.mask.fill_(7)
    c.n_kept.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(c.mask, ref_mask) and int(c.n_kept.item()) == ref_n
