"""Helpers shared by the GPU parity tests (compare libvrs with the CPU oracle)."""
import math

import numpy as np

KCHOL2 = math.log2(math.e) / 2.0          # conic = L^T L / KCHOL2

RGB_TOL = 2e-4          # max abs per channel (stated tolerance for the FP32 images)
T_TOL = 2e-4            # max abs of the final transmittance
DEPTH_REL = 1e-4        # relative tolerance of the Eq. 1 depth
DEPTH_ABS = 1e-6        # absolute floor for uncovered pixels
FLAG_FRAC = 5e-4        # at most 0.05 % knife-edge pixels excluded
DECISION_FRAC = 1e-4    # at most 0.01 % of Gaussian-views whose decisions differ from FP64 (knife edges)


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def make_rasterizer(scenes, views, **kw):
    from paper_2410_17932_gb300.render import Rasterizer, SceneTensors
    sts = [SceneTensors.from_scene(s) for s in scenes]
    return Rasterizer(sts, views, **kw), sts


def decode_records(rec: np.ndarray):
    """[R,12] records -> dict of ubar, vbar (double-float summed), conic a/b/c, log2 opacity, rgb, depth."""
    r = rec.astype(np.float64)
    l0, l1, l2 = r[:, 4], r[:, 5], r[:, 6]
    return dict(ubar=r[:, 0] + r[:, 2], vbar=r[:, 1] + r[:, 3],
                conic=np.stack([l0 * l0, l0 * l1, l1 * l1 + l2 * l2], 1) / KCHOL2,
                lo=r[:, 7], rgb=r[:, 8:11], depth=rec[:, 11])


def compare_images(gpu, orc, label=""):
    """Asserts the stated per-channel tolerances outside knife-edge pixels."""
    rgb, depth, T = gpu
    flags = orc["flags"] > 0
    frac = flags.mean()
    assert frac <= FLAG_FRAC, f"{label}: {frac:.2e} knife-edge pixels"
    ok = ~flags
    e_rgb = np.abs(rgb.astype(np.float64) - orc["rgb"]).max(axis=0)[ok]
    e_T = np.abs(T.astype(np.float64) - orc["T"])[ok]
    e_d = np.abs(depth.astype(np.float64) - orc["depth"])[ok]
    tol_d = DEPTH_REL * np.abs(orc["depth"][ok]) + DEPTH_ABS
    worst = dict(rgb=float(e_rgb.max(initial=0)), T=float(e_T.max(initial=0)),
                 depth_rel=float((e_d / np.maximum(np.abs(orc["depth"][ok]), 1e-12)).max(initial=0)),
                 flagged=float(frac))
    assert e_rgb.max(initial=0) <= RGB_TOL, (label, worst)
    assert e_T.max(initial=0) <= T_TOL, (label, worst)
    assert np.all(e_d <= tol_d), (label, worst)
    return worst


def record_grads_wrt_sigma(g2: np.ndarray, conic: np.ndarray) -> np.ndarray:
    """The oracle's 2D gradients [n, 10] with columns 2..4 taken from the conic (a, b, c)
    to the 2D covariance Sigma' = [[A, B], [B, C]] (B one variable), the form the GPU
    records hold: dL/dSigma' = -C G C with C the conic and G = [[g_a, g_b/2], [g_b/2, g_c]]
    (in FP64)."""
    out = np.array(g2, np.float64, copy=True)
    a, b, c = conic[:, 0], conic[:, 1], conic[:, 2]
    ga, gb, gc = g2[:, 2], 0.5 * g2[:, 3], g2[:, 4]
    # H = -C G C, C = [[a, b], [b, c]]
    cg00, cg01 = a * ga + b * gb, a * gb + b * gc
    cg10, cg11 = b * ga + c * gb, b * gb + c * gc
    h00 = -(cg00 * a + cg01 * b)
    h01 = -(cg00 * b + cg01 * c)
    h11 = -(cg10 * b + cg11 * c)
    out[:, 2], out[:, 3], out[:, 4] = h00, 2.0 * h01, h11
    return out


def plain_200_c9(seed: int = 91, dark_frac: float = 0.15):
    """The 200x200 workload with the colour reading where "RGB ~ U[0, 1]" is the rendered colour:
    the DC coefficient is (rgb - 0.5) / Y_00, so a splat renders exactly rgb.  A fraction of the
    splats get channels below 0 before the max(0, .) clamp (rgb drawn from [-0.3, 0)), so the
    clamp and dark colours are exercised."""
    from paper_2410_17932_gb300 import inputs as I
    scs, cams = I.plain_200()
    sc = scs[0]
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(0.0, 1.0, (sc.n, 3))
    dark = rng.uniform(size=(sc.n, 3)) < dark_frac
    rgb[dark] = rng.uniform(-0.3, 0.0, dark.sum())
    y00 = 0.5 / math.sqrt(math.pi)
    sc.sh[:, 0, :] = ((rgb - 0.5) / y00).astype(np.float32)
    return [sc], cams
