"""The CPU-baseline sampler of bench.py: a cropped tile block over the Gaussians that
overlap it composites exactly what the whole-view oracle composites on those tiles,
and a sample that covers the whole view estimates the whole-view time."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2410_17932_gb300 import inputs as I  # noqa: E402


def test_cropped_block_equals_full_view(orc):
    scenes, views = I.plain_200()
    S = bench.OracleFrameSampler(scenes, views, 16)
    cam = views[0]
    gw, gh = oracle.grid(cam, 16)
    dec, proj = S.full[0][0], S.full[0][1]
    for bx, by, bw, bh in ((0, 0, 3, 2), (5, 7, 8, 6), (gw - 2, gh - 3, 2, 3)):
        scn, crop, sdec, sproj = S._block(0, cam, bx, by, bw, bh)
        got = oracle.render(scn, crop, 16, dec=sdec, proj=sproj)
        mask = np.zeros(gw * gh, np.uint8)
        for y in range(by, by + bh):
            mask[y * gw + bx:y * gw + bx + bw] = 1
        full = oracle.render(scenes[0], cam, 16, dec=dec, proj=proj, tile_mask=mask)
        ys = slice(by * 16, min(cam.height, (by + bh) * 16))
        xs = slice(bx * 16, min(cam.width, (bx + bw) * 16))
        assert np.array_equal(got["rgb"], full["rgb"][:, ys, xs])
        assert np.array_equal(got["depth"], full["depth"][ys, xs])
        assert np.array_equal(got["T"], full["T"][ys, xs])


def test_sample_counts_cover_the_view(orc):
    scenes, views = I.plain_200()
    S = bench.OracleFrameSampler(scenes, views, 16)
    ms, g, k = S.sample(5.0, np.random.default_rng(0))
    assert ms > 0 and g == scenes[0].n and k >= 1
