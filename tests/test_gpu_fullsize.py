"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The whole sorted instance list and every visible record are compared with the
oracle; images are compared on sampled tiles (random ones plus the heaviest),
which the oracle composites one by one.
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import FLAG_FRAC, compare_images, decode_records, make_rasterizer, torch_cuda

pytestmark = pytest.mark.gpu


def _sampled_image_parity(ras, scenes, views, n_random=48, n_heavy=16, seed=0, tile=16):
    rng = np.random.default_rng(seed)
    _, _, ranges = ras.sorted_lists()
    r = ranges.cpu().numpy().astype(np.int64)
    counts = r[:, 1] - r[:, 0]
    worst = {}
    flagged = total = 0
    for v, cam in enumerate(views):
        sc = scenes[cam.scene]
        p = ras.plan
        base = int(p.view_tile_base[v])
        gw, gh = int(p.view_gw[v]), int(p.view_gh[v])
        nt = gw * gh
        c = counts[base:base + nt]
        pick = set(rng.choice(nt, min(n_random, nt), replace=False).tolist())
        pick |= set(np.argsort(-c)[:n_heavy].tolist())
        mask = np.zeros(nt, np.uint8)
        mask[list(pick)] = 1
        orc = oracle.render(sc, cam, tile, tile_mask=mask)
        rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(v)]
        pixmask = np.kron(mask.reshape(gh, gw), np.ones((tile, tile), np.uint8))[:cam.height, :cam.width]
        sel = pixmask.astype(bool)
        sub = dict(rgb=orc["rgb"][:, sel], depth=orc["depth"][sel], T=orc["T"][sel], flags=orc["flags"][sel])
        w = compare_images((rgb[:, sel], depth[sel], T[sel]), sub, f"view{v}")
        flagged += int((sub["flags"] > 0).sum())
        total += int(sel.sum())
        for k, val in w.items():
            worst[k] = max(worst.get(k, 0.0), val)
    assert flagged <= FLAG_FRAC * total
    return worst


def _full_checks(scenes, views, **kw):
    torch = torch_cuda()
    ras, _ = make_rasterizer(scenes, views, **kw)
    ras.forward()
    torch.cuda.synchronize()
    keys, vals, _ = ras.sorted_lists()
    bs = oracle.bin_sort(scenes, views, ras.tile)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), bs["keys"])
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), bs["vals"])
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
    ras = _full_checks(scenes, views)
    worst = _sampled_image_parity(ras, scenes, views)
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
    b, _ = make_rasterizer(scenes, views, persistent=True)
    a.forward()
    b.forward()
    assert torch.equal(a.rgb, b.rgb) and torch.equal(a.depth, b.depth) and torch.equal(a.T, b.T)


@pytest.mark.slow
def test_dense_stereo_3m_with_crops():
    torch = torch_cuda()
    scenes, views = I.dense_stereo_3m()
    ras = _full_checks(scenes, views)
    worst = _sampled_image_parity(ras, scenes, views, n_random=24, n_heavy=8)
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
