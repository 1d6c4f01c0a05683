"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The whole sorted instance list and every visible record are compared with the
oracle, every pixel of every view is compared with the oracle's compositing,
and the GPU's integer decisions (visibility and tile rectangle of every
Gaussian-view) are compared with the FP64 decisions taken from the plain
definition: every difference must be a counted knife edge, at most 0.01 % of
the Gaussian-views.
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import (DECISION_FRAC, compare_images, decode_records, make_rasterizer,
                            torch_cuda)

pytestmark = pytest.mark.gpu


def _whole_frame_parity(ras, scenes, views, label, tile=16, which=None):
    """Every pixel of each view against the oracle (bucketed traversal, same result as
    the brute force); returns the worst errors and prints the flagged fraction per view."""
    worst = {}
    for v, cam in enumerate(views):
        if which is not None and v not in which:
            continue
        orc = oracle.render(scenes[cam.scene], cam, tile)
        rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(v)]
        w = compare_images((rgb, depth, T), orc, f"{label} view{v}")
        print(f"{label} view{v} {cam.width}x{cam.height}: flagged {w['flagged']:.2e}, worst {w}")
        for k, val in w.items():
            worst[k] = max(worst.get(k, 0.0), val)
    return worst


def _fp64_decisions(ras, scenes, views, label, which=None):
    """GPU visibility and tile rectangles against the FP64 decisions of every Gaussian-view."""
    differs = total = 0
    for v, cam in enumerate(views):
        if which is not None and v not in which:
            continue
        sc = scenes[cam.scene]
        vis, rect = ras.decisions(v)
        d64 = oracle.decide64(sc, cam, ras.tile)
        mm = oracle.decision_mismatches(d64, vis, rect)
        bad = np.nonzero(mm["outside"])[0]
        assert len(bad) == 0, (label, v, bad[:10], rect[bad[:3]], d64[bad[:3]])
        differs += int(mm["differs"].sum())
        total += sc.n
    print(f"{label}: {differs} knife-edge decisions of {total} Gaussian-views differ from FP64")
    assert differs <= DECISION_FRAC * total


def _full_checks(scenes, views, label="full", **kw):
    torch = torch_cuda()
    ras, _ = make_rasterizer(scenes, views, **kw)
    ras.forward()
    torch.cuda.synchronize()
    keys, vals, _ = ras.sorted_lists()
    bs = oracle.bin_sort(scenes, views, ras.tile)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), bs["keys"])
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), bs["vals"])
    _fp64_decisions(ras, scenes, views, label)
    rec = decode_records(ras.records().cpu().numpy())
    for v, cam in enumerate(views):
        sc = scenes[cam.scene]
        d = oracle.decide(sc, cam)
        pr = oracle.project(sc, cam)
        vis = np.nonzero(d["visible"])[0]
        rv = int(ras.plan.view_rec_base[v]) + vis
        assert np.all(rec["depth"][rv] == d["depth"][vis])
        du = np.abs(rec["ubar"][rv] - pr["ubar"][vis])
        assert du.max() < 2e-6 * (1 + np.abs(pr["ubar"][vis]).max()), du.max()
        assert np.abs(rec["rgb"][rv] - pr["rgb"][vis]).max() < 1e-5
    return ras


def test_periphery_stereo_05m_full_size():
    scenes, views = I.periphery_stereo_05m()
    ras = _full_checks(scenes, views, "periphery_stereo_05m")
    worst = _whole_frame_parity(ras, scenes, views, "periphery_stereo_05m")
    print("periphery_stereo_05m worst", worst)


def test_periphery_stereo_05m_tile8_sort():
    # 2 x 252 x 280 tiles: more than 64 Ki, so the tile-count scan takes its
    # two-launch form (block sums, then the scan); tile 16 takes the one-launch form
    torch = torch_cuda()
    scenes, views = I.periphery_stereo_05m()
    ras, _ = make_rasterizer(scenes, views, tile=8)
    ras.forward()
    torch.cuda.synchronize()
    assert int(ras.plan.n_tiles) > 65536
    keys, vals, ranges = ras.sorted_lists()
    bs = oracle.bin_sort(scenes, views, 8)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), bs["keys"])
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), bs["vals"])
    assert np.array_equal(ranges.cpu().numpy().astype(np.int64), bs["ranges"])


def test_periphery_stereo_05m_persistent_identical():
    torch = torch_cuda()
    scenes, views = I.periphery_stereo_05m(n=200_000)
    a, _ = make_rasterizer(scenes, views)
    a.forward()
    for persistent in (1, 2):
        b, _ = make_rasterizer(scenes, views, persistent=persistent)
        b.forward()
        assert torch.equal(a.rgb, b.rgb) and torch.equal(a.depth, b.depth) and torch.equal(a.T, b.T)


@pytest.mark.slow
def test_dense_stereo_3m_with_crops():
    torch = torch_cuda()
    scenes, views = I.dense_stereo_3m()
    ras = _full_checks(scenes, views, "dense_stereo_3m")
    worst = _whole_frame_parity(ras, scenes, views, "dense_stereo_3m")
    print("dense_stereo_3m worst", worst)
    # each aligned foveal crop equals its window of the eye it was cut from
    for c in (2, 3):
        eye = views[c - 2]
        crop = views[c]
        x0 = int(round(eye.cx - crop.cx))
        y0 = int(round(eye.cy - crop.cy))
        f_rgb, f_d, f_T = ras.outputs(c - 2)
        c_rgb, c_d, c_T = ras.outputs(c)
        assert torch.equal(c_rgb, f_rgb[:, y0:y0 + 512, x0:x0 + 512])
        assert torch.equal(c_d, f_d[y0:y0 + 512, x0:x0 + 512])


@pytest.mark.slow
def test_dense_stereo_3m_unaligned_crops():
    """Crops whose origins are not tile-aligned: a different tile grid over the same
    pixels; every pixel against the oracle at the crop's own grid."""
    torch_cuda()
    scenes, views = I.dense_stereo_3m(aligned=False)
    ras, _ = make_rasterizer(scenes, views)
    ras.forward()
    _fp64_decisions(ras, scenes, views, "dense_stereo_3m crops", which=(2, 3))
    _whole_frame_parity(ras, scenes, views, "dense_stereo_3m unaligned", which=(2, 3))
