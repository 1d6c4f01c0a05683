"""The batched persistent multi-view path (32 views of uneven size over 4 scenes).

Bars: the batched launch gives exactly the per-view images (bit for bit, same
tile size), a CUDA-graph replay gives exactly the eager result, the autotuner's
choice (tile fixed) gives exactly the default's images, and sampled views match
the oracle; at the full scene sizes (100 k to 2 M Gaussians) every pixel of
the four training views, one crop per scene and two stereo pairs is compared
with the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import compare_images, make_rasterizer, torch_cuda

pytestmark = pytest.mark.gpu


def _multiview(scale=0.02):
    return I.batched_multiview(scale=scale)


def test_batched_equals_per_view():
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    scenes, views = _multiview()
    sts = [SceneTensors.from_scene(s) for s in scenes]
    batched = Rasterizer(sts, views, persistent=True)
    batched.forward()
    for v, cam in enumerate(views):
        single = Rasterizer([sts[cam.scene]], [I.Camera(cam.R, cam.t, cam.fx, cam.fy, cam.cx, cam.cy,
                                                        cam.width, cam.height, cam.znear, 0,
                                                        cam.tan_fovx, cam.tan_fovy)])
        single.forward()
        for x, y in zip(batched.outputs(v), single.outputs(0)):
            assert torch.equal(x, y), v


def test_graph_replay_equals_eager():
    torch = torch_cuda()
    from paper_2410_17932_gb300.autotune import GraphRunner
    scenes, views = _multiview(0.01)
    ras, _ = make_rasterizer(scenes, views, persistent=True)
    ras.forward()
    ref = [x.clone() for x in (ras.rgb, ras.depth, ras.T)]
    for x in (ras.rgb, ras.depth, ras.T):
        x.fill_(-1.0)
    g = GraphRunner(ras)
    for x in (ras.rgb, ras.depth, ras.T):
        x.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    for x, y in zip((ras.rgb, ras.depth, ras.T), ref):
        assert torch.equal(x, y)


def test_autotune_choice_keeps_images(tmp_path, monkeypatch):
    torch = torch_cuda()
    from paper_2410_17932_gb300 import autotune
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "cache.json"))
    scenes, views = _multiview(0.01)
    views = views[:8]
    sts = [SceneTensors.from_scene(s) for s in scenes]
    best = autotune.tune(sts, views, iters=3)
    assert best["tile"] == 16 and best["persistent"] in (0, 1, 2) and best["sort"] in (0, 1)
    assert best["tiles_per_pull"] in (1, 4) and best["key_bits"] in (0, 64)
    assert autotune.tune(sts, views) == best          # served from the cache
    a = Rasterizer(sts, views)
    b = Rasterizer(sts, views, **best)
    a.forward()
    b.forward()
    assert torch.equal(a.rgb, b.rgb) and torch.equal(a.depth, b.depth) and torch.equal(a.T, b.T)


def test_batched_views_match_oracle_on_sampled_tiles():
    scenes, views = _multiview(0.01)
    ras, _ = make_rasterizer(scenes, views, persistent=True)
    ras.forward()
    rng = np.random.default_rng(3)
    for v in (12, 20, 28):       # two foveal crops and a training view
        cam = views[v]
        sc = scenes[cam.scene]
        gw, gh = oracle.grid(cam, 16)
        mask = np.zeros(gw * gh, np.uint8)
        mask[rng.choice(gw * gh, min(40, gw * gh), replace=False)] = 1
        orc = oracle.render(sc, cam, tile_mask=mask)
        pm = np.kron(mask.reshape(gh, gw), np.ones((16, 16), np.uint8))[:cam.height, :cam.width].astype(bool)
        rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(v)]
        sub = dict(rgb=orc["rgb"][:, pm], depth=orc["depth"][pm], T=orc["T"][pm], flags=orc["flags"][pm])
        compare_images((rgb[:, pm], depth[pm], T[pm]), sub, f"view{v}")


def test_batched_full_size_views_match_oracle():
    torch = torch_cuda()
    scenes, views = I.batched_multiview()
    ras, _ = make_rasterizer(scenes, views, persistent=True)
    ras.forward()
    torch.cuda.synchronize()
    # a stereo pair on the 100 k scene and one on the 2 M scene, the first crop of
    # each scene, and the four training views
    for v in (0, 1, 10, 11, 12, 16, 20, 24, 28, 29, 30, 31):
        cam = views[v]
        orc = oracle.render(scenes[cam.scene], cam)
        rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(v)]
        w = compare_images((rgb, depth, T), orc, f"view{v}")
        print(f"batched view{v} {cam.width}x{cam.height} scene {cam.scene}: {w}")


def test_schedule_and_key_width_knobs_keep_images():
    """Tiles per pull of the persistent blend and the radix key width change no image."""
    torch = torch_cuda()
    scenes, views = _multiview(0.01)
    ref, sts = make_rasterizer(scenes, views)
    ref.forward()
    for kw in (dict(persistent=1, tiles_per_pull=4), dict(persistent=1, tiles_per_pull=3),
               dict(persistent=2), dict(persistent=2, tiles_per_pull=4),
               dict(sort=1, key_bits=64), dict(sort=1, key_bits=int(ref.plan.key_bits) + 3)):
        from paper_2410_17932_gb300.render import Rasterizer
        r = Rasterizer(sts, views, **kw)
        r.forward()
        assert torch.equal(r.rgb, ref.rgb) and torch.equal(r.depth, ref.depth) and torch.equal(r.T, ref.T), kw


def test_autotuned_tile_edge_matches_oracle_at_that_tile(tmp_path, monkeypatch):
    """With the tile edge free, the tuner's choice is compared with the oracle at that edge."""
    torch = torch_cuda()
    from paper_2410_17932_gb300 import autotune
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "cache.json"))
    scenes, views = _multiview(0.01)
    views = [views[i] for i in (0, 12, 13, 28)]
    sts = [SceneTensors.from_scene(s) for s in scenes]
    best = autotune.tune(sts, views, allow_tile_change=True, iters=2)
    ras = Rasterizer(sts, views, **best)
    ras.forward()
    torch.cuda.synchronize()
    for v, cam in enumerate(views):
        orc = oracle.render(scenes[cam.scene], cam, best["tile"])
        w = compare_images(tuple(x.cpu().numpy() for x in ras.outputs(v)), orc, f"tile {best['tile']} view{v}")
        print("autotuned", best, "view", v, w)
