"""GPU parity of the hand-written backward pass against the CPU oracle's FP64 reverse pass.

The oracle's reverse pass is itself pinned to FP64 central finite differences
(tests/test_oracle_pins.py).  Bars, per parameter array: the GPU gradient is
within 1e-3 relative of the oracle's norm-wise, and element by element
|g_gpu - g_orc| <= 1e-3 max|g_orc| + 1e-6.  Besides the 64x64 / 200-Gaussian
subsets, the full training view (1 M SH-3 Gaussians, 1264x832, upstream
gradients N(0, 1)) is compared whole; the upstream gradient is zeroed on the
pixels the oracle flags as knife edges (an alpha at 1/255 or a T at the stop
threshold, where FP32 and FP64 may blend different sets), on both sides.
"""
import numpy as np
import pytest

import oracle
from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import make_rasterizer, record_grads_wrt_sigma, torch_cuda

pytestmark = pytest.mark.gpu

NAMES = ["means", "log_scales", "quats", "opacity_logits", "sh"]
REL = 1e-3


def _training_subset(seed=0, n=200, W=64, H=64):
    rng = np.random.default_rng(100 + seed)
    scs, _ = I.training_view_1m(n=n, seed=300 + seed)
    sc = scs[0]
    cam = I.Camera(np.eye(3), np.zeros(3), 60.0, 60.0, W / 2, H / 2, W, H)
    sc.means[:, 0] = rng.uniform(-1.2, 1.2, sc.n)
    sc.means[:, 1] = rng.uniform(-1.2, 1.2, sc.n)
    sc.means[:, 2] = rng.uniform(2.0, 5.0, sc.n)
    sc.log_scales[:] = rng.normal(-2.6, 0.4, sc.log_scales.shape).astype(np.float32)
    g = I.upstream_grads([cam], seed + 7)[0]
    gT = rng.standard_normal((H, W)).astype(np.float32)
    return sc, cam, g[0], g[1], gT


def _gpu_grads(scenes, views, gC_list, gD_list, gT_list=None, **kw):
    torch = torch_cuda()
    ras, sts = make_rasterizer(scenes, views, backward=True, **kw)
    ras.forward()
    gC = torch.zeros_like(ras.rgb)
    gD = torch.zeros_like(ras.depth)
    gT = torch.zeros_like(ras.T) if gT_list is not None else None
    for v in range(len(views)):
        b, W, H = ras.view_slices(v)
        gC[3 * b:3 * b + 3 * W * H] = torch.as_tensor(gC_list[v].reshape(-1), device="cuda")
        gD[b:b + W * H] = torch.as_tensor(gD_list[v].reshape(-1), device="cuda")
        if gT is not None:
            gT[b:b + W * H] = torch.as_tensor(gT_list[v].reshape(-1), device="cuda")
    grads = ras.backward_params(gC, gD, gT)
    torch.cuda.synchronize()
    return ras, [{k: getattr(g, k).cpu().numpy().astype(np.float64) for k in NAMES} for g in grads]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


ELEM_REL, ELEM_ABS = 1e-3, 1e-6


def _elem(a, b):
    """Largest element error in units of the element-wise bar (<= 1 passes)."""
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    if b.size == 0:
        return 0.0
    return float((np.abs(a - b) / (ELEM_REL * np.abs(b).max() + ELEM_ABS)).max())


def _check(got, ref, label):
    errs = {k: (_rel(got[k], ref[k]), _elem(got[k], ref[k])) for k in NAMES}
    print(label, "norm-wise / element-wise errors", errs)
    for k in NAMES:
        assert errs[k][0] < REL and errs[k][1] <= 1.0, (label, k, errs[k])


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_oracle_reverse(seed):
    sc, cam, gC, gD, gT = _training_subset(seed)
    ras, g = _gpu_grads([sc], [cam], [gC], [gD], [gT])
    ref = oracle.grads(sc, cam, gC, gD, gT)
    _check(g[0], ref, f"subset seed {seed}")


def test_backward_record_gradients():
    torch = torch_cuda()
    sc, cam, gC, gD, gT = _training_subset(2)
    ras, _ = _gpu_grads([sc], [cam], [gC], [gD], [gT])
    p = ras.plan
    g2 = ras.ws_view(int(p.off_grad2d), 10 * int(p.n_records), torch.float32).view(-1, 10).cpu().numpy()
    ref = record_grads_wrt_sigma(oracle.render_bwd(sc, cam, gC, gD, gT), oracle.project(sc, cam)["conic"])
    for c in range(10):
        assert _rel(g2[:, c].astype(np.float64), ref[:, c]) < REL, c
        assert _elem(g2[:, c], ref[:, c]) <= 1.0, c


def test_backward_accumulates_over_views_and_no_upstream_T():
    sc, cam, gC, gD, _ = _training_subset(3)
    cam2 = I.Camera(I._yaw_pitch(0.04, 0.02), [0.05, 0.0, 0.1], 55.0, 55.0, 30.0, 34.0, 60, 68)
    g2 = I.upstream_grads([cam2], 5)[0]
    ras, g = _gpu_grads([sc], [cam, cam2], [gC, g2[0]], [gD, g2[1]])
    r1 = oracle.grads(sc, cam, gC, gD, None)
    r2 = oracle.grads(sc, cam2, g2[0], g2[1], None)
    _check(g[0], {k: r1[k] + r2[k] for k in NAMES}, "two views")


def test_backward_tile_sizes_agree():
    sc, cam, gC, gD, gT = _training_subset(4)
    ref = oracle.grads(sc, cam, gC, gD, gT, tile=8)
    _, g8 = _gpu_grads([sc], [cam], [gC], [gD], [gT], tile=8)
    _check(g8[0], ref, "tile 8")


@pytest.mark.parametrize("two_views", [False, True])
def test_backward_twice_after_one_forward(two_views):
    """A second reverse pass after the same forward gives the same gradients: the 2D-gradient
    rows start at zero each time (one view: cleared by the preprocess and by the chain rule
    after reading them; several views: cleared before the reverse pass)."""
    torch = torch_cuda()
    sc, cam, gC, gD, _ = _training_subset(8)
    views, gCs, gDs = [cam], [gC], [gD]
    if two_views:
        cam2 = I.Camera(I._yaw_pitch(0.03, 0.01), [0.02, 0.0, 0.05], 57.0, 57.0, 31.0, 30.0, 62, 60)
        g2 = I.upstream_grads([cam2], 11)[0]
        views, gCs, gDs = [cam, cam2], [gC, g2[0]], [gD, g2[1]]
    ras, sts = make_rasterizer([sc], views, backward=True)
    ras.forward()
    gCt = torch.zeros_like(ras.rgb)
    gDt = torch.zeros_like(ras.depth)
    for v in range(len(views)):
        b, W, H = ras.view_slices(v)
        gCt[3 * b:3 * b + 3 * W * H] = torch.as_tensor(gCs[v].reshape(-1), device="cuda")
        gDt[b:b + W * H] = torch.as_tensor(gDs[v].reshape(-1), device="cuda")
    runs = []
    for _ in range(2):
        gr = ras.backward_params(gCt, gDt, None)
        torch.cuda.synchronize()
        runs.append({k: getattr(gr[0], k).cpu().numpy().astype(np.float64) for k in NAMES})
    for k in NAMES:
        a, b = runs
        assert np.abs(a[k]).max() > 0, k
        assert np.allclose(a[k], b[k], rtol=1e-4, atol=1e-6 * np.abs(a[k]).max()), k


def _order_bucket(c):
    """Four buckets per octave of a work estimate, 0 for none (the work order's buckets)."""
    if c == 0:
        return 0
    lz = c.bit_length() - 1
    sub = (c >> (lz - 2)) & 3 if lz >= 2 else ((c & 1) << 1 if lz == 1 else 0)
    return 1 + 4 * lz + sub


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_tile_order_heaviest_first(tile):
    """The reverse pass takes its tiles heaviest first: the forward records, per tile and 8x8
    block, the block's largest last blended position; the order is a permutation of the tiles
    whose estimates (the largest of the tile's blocks) never rise by a bucket along it."""
    sc, cam, gC, gD, _ = _training_subset(6)
    cam2 = I.Camera(I._yaw_pitch(0.05, -0.03), [0.02, 0.01, 0.05], 58.0, 58.0, 37.0, 29.0, 75, 57)
    g2 = I.upstream_grads([cam2], 9)[0]
    ras, _ = _gpu_grads([sc], [cam, cam2], [gC, g2[0]], [gD, g2[1]], tile=tile)
    P = ras.plan
    ws = ras.workspace.cpu().numpy()
    n_tiles, wpt, wgx = int(P.n_tiles), tile * tile // 64, tile // 8
    order = ws[P.off_order:P.off_order + 4 * n_tiles].view(np.uint32)
    assert np.array_equal(np.sort(order), np.arange(n_tiles, dtype=np.uint32))
    nb = n_tiles * wpt * 4
    off_work = int(P.workspace_bytes) - (nb + 255) // 256 * 256
    work = ws[off_work:off_work + nb].view(np.uint32).reshape(n_tiles, wpt)
    last = ws[P.off_ncontrib:P.off_ncontrib + 4 * int(P.n_pixels)].view(np.uint32)
    expect = np.zeros_like(work)
    for v in range(2):
        W, H, gw, gh = P.view_w[v], P.view_h[v], P.view_gw[v], P.view_gh[v]
        plane = np.zeros((gh * tile, gw * tile), np.uint32)
        b = P.view_pix_base[v]
        plane[:H, :W] = last[b:b + W * H].reshape(H, W)
        blocks = plane.reshape(gh * tile // 8, 8, gw * tile // 8, 8).max(axis=(1, 3))
        for lt in range(gw * gh):
            ty, tx = divmod(lt, gw)
            for w in range(wpt):
                expect[P.view_tile_base[v] + lt, w] = blocks[ty * wgx + w // wgx, tx * wgx + w % wgx]
    assert np.array_equal(work, expect)
    assert last.max() > 0
    est = work.max(axis=1)
    b = np.array([_order_bucket(int(est[t])) for t in order])
    assert np.all(np.diff(b) <= 0)


def test_autograd_function():
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors, render
    sc, cam, gC, gD, _ = _training_subset(5)
    st = SceneTensors.from_scene(sc, requires_grad=True)
    ras = Rasterizer([st], [cam], backward=True)
    rgb, depth, T = render(ras)
    loss = (rgb * torch.as_tensor(gC.reshape(-1), device="cuda")).sum() + \
        (depth * torch.as_tensor(gD.reshape(-1), device="cuda")).sum()
    loss.backward()
    ref = oracle.grads(sc, cam, gC, gD, None)
    _check({k: getattr(st, k).grad.cpu().numpy() for k in NAMES}, ref, "autograd")


def test_training_view_1m_full_size():
    """The whole 1264x832 training view of 1 M SH-3 Gaussians, in the bench's launch
    configuration, against the oracle's FP64 reverse pass and chain rule."""
    scs, cams = I.training_view_1m()
    sc, cam = scs[0], cams[0]
    gC, gD = I.upstream_grads([cam], 41)[0]
    orc = oracle.render(sc, cam)
    knife = orc["flags"] > 0
    assert knife.mean() <= 5e-4
    gC = np.where(knife[None], 0.0, gC).astype(np.float32)
    gD = np.where(knife, 0.0, gD).astype(np.float32)
    ras, g = _gpu_grads([sc], [cam], [gC], [gD])
    ref = oracle.grads(sc, cam, gC, gD, None)
    _check(g[0], ref, "training_view_1m")


def test_autograd_rejects_a_stale_rasterizer():
    """A second forward through the same Rasterizer before the first graph's backward
    overwrites the state that backward reads: it must raise, not return wrong grads."""
    torch = torch_cuda()
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors, render
    sc, cam, gC, gD, _ = _training_subset(6)
    st = SceneTensors.from_scene(sc, requires_grad=True)
    ras = Rasterizer([st], [cam], backward=True)
    rgb1, _, _ = render(ras)
    rgb2, _, _ = render(ras)
    with pytest.raises(RuntimeError, match="another forward"):
        rgb1.sum().backward()
    rgb2.sum().backward()                      # the latest pass is still differentiable
    assert st.means.grad is not None


def test_backward_with_clamped_colours():
    """The colour clamp passes no gradient: a 64x64 window of the rendered-colour scene, where
    some channels are clamped at 0, against the oracle's chain rule."""
    from tests.gpu_util import plain_200_c9
    scs, _ = plain_200_c9()
    sc = scs[0].subset(np.arange(300))
    cam = I.Camera(np.eye(3), np.zeros(3), 100.0, 100.0, 32.0, 32.0, 64, 64)
    g = I.upstream_grads([cam], 21)[0]
    ref = oracle.grads(sc, cam, g[0], g[1], None)
    p = oracle.project(sc, cam)
    d = oracle.decide(sc, cam)
    assert (p["clamp_rgb"][d["visible"] > 0]).sum() > 10
    _, got = _gpu_grads([sc], [cam], [g[0]], [g[1]])
    _check(got[0], ref, "clamped colours")
