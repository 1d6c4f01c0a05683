"""GPU parity of the forward path (preprocess, bin/sort, blend) against the CPU oracle.

Bars: bit-exact instance counts, sorted key lists, record-index lists and tile
ranges; per-pixel images within max abs 2e-4 (RGB, T) and 1e-4 relative
(Eq. 1 depth) outside the knife-edge pixels the oracle flags (alpha within
2e-5 relative of 1/255 or T' within 3e-5 relative of the 1e-4 stop).
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import compare_images, decode_records, make_rasterizer, torch_cuda

pytestmark = pytest.mark.gpu


def _run(scenes, views, **kw):
    torch = torch_cuda()
    ras, sts = make_rasterizer(scenes, views, **kw)
    ras.forward()
    torch.cuda.synchronize()
    return ras


def _check_sort(ras, scenes, views, tile=16):
    keys, vals, ranges = ras.sorted_lists()
    bs = oracle.bin_sort(scenes, views, tile)
    k = keys.cpu().numpy().view(np.uint64)
    v = vals.cpu().numpy().view(np.uint32)
    assert len(k) == len(bs["keys"])
    assert np.array_equal(k, bs["keys"])
    assert np.array_equal(v, bs["vals"])
    r = ranges.cpu().numpy().astype(np.int64)
    assert np.array_equal(r, bs["ranges"])
    return bs


def test_plain_200_records_and_sort():
    scs, cams = I.plain_200()
    ras = _run(scs, cams)
    code, flags, inst = ras.last_status
    assert code == 0 and flags == 0
    bs = _check_sort(ras, scs, cams)
    assert inst == len(bs["keys"]) > 10000
    # preprocess records of the visible Gaussians against the FP64 projection
    rec = decode_records(ras.records().cpu().numpy())
    d = oracle.decide(scs[0], cams[0])
    p = oracle.project(scs[0], cams[0])
    vis = d["visible"].astype(bool)
    assert np.abs(rec["ubar"][vis] - p["ubar"][vis]).max() <= 1e-6 * (1 + np.abs(p["ubar"][vis]).max())
    assert np.abs(rec["vbar"][vis] - p["vbar"][vis]).max() <= 1e-6 * (1 + np.abs(p["vbar"][vis]).max())
    assert np.all(rec["depth"][vis] == d["depth"][vis])
    scale = np.abs(p["conic"][vis]).max(axis=1, keepdims=True)
    assert (np.abs(rec["conic"][vis] - p["conic"][vis]) / scale).max() < 2e-5
    assert np.abs(rec["lo"][vis] - np.log2(p["opacity"][vis])).max() < 2e-6
    assert np.abs(rec["rgb"][vis] - p["rgb"][vis]).max() < 2e-6


@pytest.mark.parametrize("backward", [False, True])
def test_plain_200_image_parity(backward):
    # a forward-only plan skips the last-position plane; a backward plan writes it
    scs, cams = I.plain_200()
    ras = _run(scs, cams, backward=backward)
    rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(0)]
    orc = oracle.render(scs[0], cams[0])
    worst = compare_images((rgb, depth, T), orc, "plain_200")
    if backward:
        nc = ras.n_contrib().cpu().numpy().reshape(200, 200)
        ok = orc["flags"] == 0
        assert np.array_equal(nc[ok], orc["n_contrib"][ok])
    print("plain_200 worst", worst)


def test_plain_200_rendered_colour_reading():
    """The rendered-colour reading of "RGB ~ U[0, 1]", with some channels clamped at 0."""
    from tests.gpu_util import plain_200_c9
    scs, cams = plain_200_c9()
    p = oracle.project(scs[0], cams[0])
    assert p["clamp_rgb"].sum() > 500 and (p["rgb"] < 0.05).mean() > 0.05
    ras = _run(scs, cams, backward=True)
    _check_sort(ras, scs, cams)
    rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(0)]
    print("plain_200 rendered colours", compare_images((rgb, depth, T), oracle.render(scs[0], cams[0]), "c9"))


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tile_sizes_ragged(tile):
    # 203 x 141: not a multiple of any tile size
    scs, _ = I.plain_200()
    cam = I.Camera(np.eye(3), np.zeros(3), 180.0, 190.0, 101.3, 70.6, 203, 141)
    ras = _run(scs, [cam], tile=tile)
    _check_sort(ras, scs, [cam], tile)
    rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(0)]
    orc = oracle.render(scs[0], cam, tile=tile)
    compare_images((rgb, depth, T), orc, f"tile{tile}")


@pytest.mark.parametrize("tile", [16, 32])
def test_one_tile_wide_view(tile):
    # a view one tile wide (gw = 1) and many tiles tall: every tile's column is 0,
    # its row the whole tile index; a ragged width and height too
    scs, _ = I.plain_200()
    cam = I.Camera(np.eye(3), np.zeros(3), 180.0, 190.0, 6.3, 150.2, 13, 301)
    ras = _run(scs, [cam], tile=tile)
    assert int(ras.plan.view_gw[0]) == 1
    _check_sort(ras, scs, [cam], tile)
    rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(0)]
    orc = oracle.render(scs[0], cam, tile=tile)
    compare_images((rgb, depth, T), orc, f"narrow{tile}")


@pytest.mark.parametrize("persistent,tile", [(1, 16), (2, 16), (1, 8), (2, 8), (2, 32)])
def test_persistent_equals_per_tile(persistent, tile):
    torch = torch_cuda()
    scs, cams = I.plain_200()
    a = _run(scs, cams, tile=tile)
    b = _run(scs, cams, persistent=persistent, tile=tile)
    for x, y in zip((a.rgb, a.depth, a.T), (b.rgb, b.depth, b.T)):
        assert torch.equal(x, y)


def test_multiview_multiscene_and_crop_window():
    torch = torch_cuda()
    s0 = I.uniform_box_scene(3000, 41, sh_degree=3)
    s1 = I.uniform_box_scene(2000, 42, sh_degree=1)
    full = I.Camera(I._yaw_pitch(0.05, -0.03), [0.02, -0.01, 0.1], 150.0, 150.0, 96.0, 80.0, 192, 160)
    crop = full.crop(32, 48, 64, 80)
    other = I.Camera(np.eye(3), np.zeros(3), 120.0, 120.0, 50.0, 40.0, 100, 80, scene=1)
    views = [full, other, crop]
    ras = _run([s0, s1], views)
    _check_sort(ras, [s0, s1], views)
    for v, cam in enumerate(views):
        sc = [s0, s1][cam.scene]
        rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(v)]
        compare_images((rgb, depth, T), oracle.render(sc, cam), f"view{v}")
    f_rgb, f_d, f_T = ras.outputs(0)
    c_rgb, c_d, c_T = ras.outputs(2)
    assert torch.equal(c_rgb, f_rgb[:, 48:128, 32:96])
    assert torch.equal(c_d, f_d[48:128, 32:96])
    assert torch.equal(c_T, f_T[48:128, 32:96])


def test_empty_scene_and_all_behind():
    torch = torch_cuda()
    empty = I.uniform_box_scene(0, 1)
    behind = I.uniform_box_scene(500, 2, z=(-6.0, -2.0))
    cam = I.identity_camera(72, 40)
    for sc in (empty, behind):
        ras = _run([sc], [cam])
        assert ras.last_status[2] == 0
        rgb, depth, T = ras.outputs(0)
        assert torch.all(rgb == 0) and torch.all(depth == 0) and torch.all(T == 1)


def test_device_status_zero_quat_and_nonfinite():
    scs, cams = I.plain_200()
    sc = scs[0].subset(np.arange(400))
    sc.quats[3] = 0.0
    sc.means[7, 1] = np.nan
    sc.sh[9, 0, 2] = np.inf
    ras = _run([sc], cams)
    code, flags, _ = ras.last_status
    assert flags & 1 and flags & 2
    keys, vals, _ = ras.sorted_lists()
    v = vals.cpu().numpy()
    assert not np.isin(v, [3, 7, 9]).any()
    bs = oracle.bin_sort([sc], cams)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), bs["keys"])
    assert np.array_equal(v.view(np.uint32), bs["vals"])
    orc = oracle.render(sc.subset(np.setdiff1d(np.arange(400), [3, 7, 9])), cams[0])
    rgb, depth, T = [x.cpu().numpy() for x in ras.outputs(0)]
    compare_images((rgb, depth, T), orc, "skipped")


def test_large_finite_parameters_are_not_flagged():
    # a Gaussian whose parameters are all finite is rendered even when a sum of them
    # would overflow FP32: the check is per value, as the oracle's
    scs, cams = I.plain_200()
    sc = scs[0].subset(np.arange(300))
    sc.quats[5] = [3e38, 3e38, 0.0, 0.0]          # |q|^2 overflows on both sides alike
    sc.sh[11, 0, :] = 1.5e38                      # a colour row whose sum overflows
    ras = _run([sc], cams)
    _, flags, _ = ras.last_status
    assert flags & 2 == 0
    d = oracle.decide(sc, cams[0])
    assert d["status"] & 2 == 0 and d["visible"][11] == 1
    _check_sort(ras, [sc], cams)


def test_capacity_overflow_reported_then_regrown():
    from paper_2410_17932_gb300 import _lib as L
    torch = torch_cuda()
    scs, cams = I.plain_200()
    ras, _ = make_rasterizer(scs, cams, max_instances=1000)
    ras.forward_async()
    code, flags, inst = ras.status()
    assert code == L.VRS_ERR_CAPACITY and flags & 4 and inst > 1000
    ras.forward()          # re-plans with room for the measured count
    assert ras.last_status[0] == 0
    _check_sort(ras, scs, cams)


def test_invalid_arguments_rejected_on_host():
    from paper_2410_17932_gb300 import _lib as L
    torch_cuda()
    scs, cams = I.plain_200()
    ras, _ = make_rasterizer(scs, cams)
    bad = L.vrs_camera.from_buffer_copy(ras._view_arr[0])
    bad.width = 100
    arr = (L.vrs_camera * 1)(bad)
    assert L.vrs_preprocess(ras.plan, ras._scene_arr, arr, ras.workspace.data_ptr(), 0) == L.VRS_ERR_INVALID
    assert L.vrs_preprocess(ras.plan, ras._scene_arr, ras._view_arr, ras.workspace.data_ptr() + 8, 0) \
        == L.VRS_ERR_INVALID


@pytest.mark.parametrize("n", [300, 700, 1100, 3000, 20000])
def test_bucketed_sort_crowded_tiles(n):
    """n splats stacked on four tiles: the warp path and the CTA path of the bucketed sort (runs
    of 128 merged in shared memory for chunks of 512 and 1024, a last chunk of under 256 at
    n = 1100, chunks merged in global memory beyond 1024)."""
    torch = torch_cuda()
    sc = I.uniform_box_scene(n, 90 + n, xy=(-0.01, 0.01), z=(2.0, 6.0), log_scale=(-6.0, 0.2))
    cam = I.identity_camera(64, 64, 200.0)
    a = _run([sc], [cam], sort=0)
    bs = _check_sort(a, [sc], [cam])
    assert (bs["ranges"][:, 1] - bs["ranges"][:, 0]).max() >= n
    b = _run([sc], [cam], sort=1)
    _check_sort(b, [sc], [cam])
    assert torch.equal(a.rgb, b.rgb) and torch.equal(a.depth, b.depth) and torch.equal(a.T, b.T)
    rgb, depth, T = [x.cpu().numpy() for x in a.outputs(0)]
    compare_images((rgb, depth, T), oracle.render(sc, cam), f"crowded{n}")


def test_bucketed_sort_repeated_calls():
    """vrs_bin_sort called again on the same instances, without a new preprocess, gives the same
    lists: the big-tile list and its claim counter start from zero on every call (the last CTA
    of each tile sort clears them)."""
    torch = torch_cuda()
    sc = I.uniform_box_scene(1500, 77, xy=(-0.01, 0.01), z=(2.0, 6.0), log_scale=(-6.0, 0.2))
    cam = I.identity_camera(64, 64, 200.0)
    a = _run([sc], [cam], sort=0)
    bs = _check_sort(a, [sc], [cam])
    assert (bs["ranges"][:, 1] - bs["ranges"][:, 0]).max() > 1024
    for _ in range(3):
        a.bin_sort()
        torch.cuda.synchronize()
        _check_sort(a, [sc], [cam])


@pytest.mark.parametrize("n,mode", [(60, "equal"), (120, "equal"), (200, "equal"), (256, "equal"),
                                    (200, "near"), (250, "near")])
def test_bucketed_sort_depth_ties(n, mode):
    """Tiles of up to 256 instances whose depths tie: "equal" stacks the splats on five depth
    planes (equal keys, ordered by record index), "near" spreads half over 2..6 and puts the
    rest within a few units in the last place of 3.0, so that the warp sort's shifted 32-bit
    keys tie while the depths differ.  Both must take the exact 64-bit order."""
    torch = torch_cuda()
    sc = I.uniform_box_scene(n, 700 + n, xy=(-0.01, 0.01), z=(2.0, 6.0), log_scale=(-6.0, 0.2))
    rng = np.random.default_rng(n)
    if mode == "equal":
        sc.means[:, 2] = np.float32(2.0) + np.float32(0.5) * rng.integers(0, 5, n).astype(np.float32)
    else:
        near = rng.random(n) < 0.5
        ulps = rng.integers(0, 6, int(near.sum())).astype(np.uint32)
        sc.means[near, 2] = (np.float32(3.0).view(np.uint32) + ulps).view(np.float32)
    cam = I.identity_camera(64, 64, 200.0)
    a = _run([sc], [cam], sort=0)
    bs = _check_sort(a, [sc], [cam])
    assert (bs["ranges"][:, 1] - bs["ranges"][:, 0]).max() >= n // 2
    b = _run([sc], [cam], sort=1)
    _check_sort(b, [sc], [cam])


def test_radix_and_bucketed_sorts_agree_multiview():
    torch = torch_cuda()
    s0 = I.uniform_box_scene(4000, 51, sh_degree=2)
    views = [I.identity_camera(120, 96, 110.0), I.Camera(I._yaw_pitch(0.1, 0.0), [0.0, 0.0, 0.2], 90.0, 90.0,
                                                         40.0, 50.0, 88, 104)]
    a = _run([s0], views, sort=0)
    b = _run([s0], views, sort=1)
    ka, va, ra = a.sorted_lists()
    kb, vb, rb = b.sorted_lists()
    assert torch.equal(ka, kb) and torch.equal(va, vb) and torch.equal(ra, rb)
    _check_sort(a, [s0], views)


@pytest.mark.parametrize("tile", [8, 32])
def test_emission_large_rectangles(tile):
    """Splats whose rectangles span most of a 1024x768 view: the warp-cooperative key
    emission's row/column split over rectangles of thousands of tiles, bit-exact."""
    sc = I.uniform_box_scene(96, 77, xy=(-2.0, 2.0), z=(2.0, 4.0), log_scale=(-0.7, 0.4))
    cam = I.identity_camera(1024, 768, 400.0)
    ras = _run([sc], [cam], tile=tile)
    bs = _check_sort(ras, [sc], [cam], tile)
    r = bs["ranges"]
    assert len(bs["keys"]) > 20 * 96 and (r[:, 1] - r[:, 0]).max() > 40


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_sort_mode_2_matches_mode_0(tile):
    """Tiles of one blend batch ordered inside the blend: the same images bit for bit, the same
    sorted lists after the forward (checked against the oracle), persistent too."""
    torch = torch_cuda()
    scenes, views = I.batched_multiview(scale=0.01)
    views = views[:6] + views[12:16] + views[28:]
    a = _run(scenes, views, tile=tile)
    for kw in (dict(sort=2), dict(sort=2, persistent=True)):
        b = _run(scenes, views, tile=tile, **kw)
        assert torch.equal(a.rgb, b.rgb) and torch.equal(a.depth, b.depth) and torch.equal(a.T, b.T), kw
    _check_sort(b, scenes, views, tile)


def test_sort_mode_2_backward_identical():
    # the gradients accumulate with float atomics in no fixed order, so two runs agree to
    # rounding, not bit for bit, in either mode
    torch = torch_cuda()
    scs, cams = I.plain_200()
    g = I.upstream_grads(cams, 3)[0]
    out = []
    for sort in (0, 2):
        ras, sts = make_rasterizer(scs, cams, backward=True, sort=sort)
        ras.forward()
        gr = ras.backward_params(torch.as_tensor(g[0].reshape(-1), device="cuda"),
                                 torch.as_tensor(g[1].reshape(-1), device="cuda"))
        torch.cuda.synchronize()
        out.append([x.clone() for x in gr[0].tensors()])
    for x, y in zip(*out):
        assert torch.allclose(x, y, rtol=1e-5, atol=1e-6 * float(y.abs().max()))
