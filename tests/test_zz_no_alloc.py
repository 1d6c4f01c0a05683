"""vrs_sort_pairs_noalloc: the radix sort for callers that cannot allocate device memory.

Code inside a CUDA stream capture cannot call cudaMalloc, a real-time frame
loop must not risk the synchronisation an allocation can cause, and a plug-in
may live inside a host application's fixed memory budget; this entry point
sorts with a static device array instead.  The test compares it with the
library's regular sort (vrs_bin_sort) on the same instance lists, for two
calls in a row of different sizes, bit for bit as every sort test here does.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2410_17932_gb300 import inputs as I
from tests.gpu_util import make_rasterizer, torch_cuda

pytestmark = pytest.mark.gpu


def _unsorted_and_sorted(scenes, views):
    """Instance list of vrs_preprocess (unsorted copy) and vrs_bin_sort's sorted list."""
    torch = torch_cuda()
    ras, _ = make_rasterizer(scenes, views)
    ras.forward()                      # sizes the instance list
    ras.preprocess()
    _, _, inst = ras.status()
    p = ras.plan
    keys0 = ras.ws_view(int(p.off_keys[0]), inst, torch.int64).clone()
    vals0 = ras.ws_view(int(p.off_vals[0]), inst, torch.int32).clone()
    ras.bin_sort()
    keys, vals, _ = ras.sorted_lists()
    torch.cuda.synchronize()
    return ras, keys0, vals0, keys.clone(), vals.clone()


def _canonical(keys: np.ndarray, vals: np.ndarray):
    """Orders every run of equal keys by value (vrs_bin_sort's tie rule)."""
    order = np.lexsort((vals, keys))
    return keys[order], vals[order]


def test_noalloc_sort_matches_bin_sort_two_calls():
    from paper_2410_17932_gb300 import _lib as L
    torch = torch_cuda()
    cases = [I.plain_200(),
             ([I.clustered_room_scene(60_000, 77)], I.stereo_eyes(78, width=640, height=720))]
    stream = torch.cuda.current_stream().cuda_stream
    for scenes, views in cases:
        ras, k_in, v_in, k_ref, v_ref = _unsorted_and_sorted(scenes, views)
        n = k_in.numel()
        assert 0 < n <= L.VRS_NOALLOC_MAX_PAIRS
        k_out = torch.full_like(k_in, -1)
        v_out = torch.full_like(v_in, -1)
        code = L.vrs_sort_pairs_noalloc(k_in.data_ptr(), v_in.data_ptr(), k_out.data_ptr(),
                                        v_out.data_ptr(), n, int(ras.plan.key_bits), stream)
        assert code == L.VRS_OK, L.status_string(code)
        torch.cuda.synchronize()
        ko = k_out.cpu().numpy().view(np.uint64)
        vo = v_out.cpu().numpy().view(np.uint32)
        kr = k_ref.cpu().numpy().view(np.uint64)
        vr = v_ref.cpu().numpy().view(np.uint32)
        assert np.array_equal(ko, kr)
        assert np.array_equal(*[_canonical(ko, vo)[1], vr])
        # stable: within a run of equal keys the input order is kept
        ki = k_in.cpu().numpy().view(np.uint64)
        vi = v_in.cpu().numpy().view(np.uint32)
        stable = np.argsort(ki, kind="stable")
        assert np.array_equal(vo, vi[stable])


def test_noalloc_rejects_oversize_and_bad_arguments():
    from paper_2410_17932_gb300 import _lib as L
    torch = torch_cuda()
    k = torch.zeros(4, dtype=torch.int64, device="cuda")
    v = torch.zeros(4, dtype=torch.int32, device="cuda")
    k2, v2 = torch.zeros_like(k), torch.zeros_like(v)
    s = torch.cuda.current_stream().cuda_stream
    big = L.VRS_NOALLOC_MAX_PAIRS + 1
    assert L.vrs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k2.data_ptr(), v2.data_ptr(), big, 40, s) \
        == L.VRS_ERR_CAPACITY
    assert L.vrs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k2.data_ptr(), v2.data_ptr(), 4, 0, s) \
        == L.VRS_ERR_INVALID
    assert L.vrs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k.data_ptr(), v2.data_ptr(), 4, 40, s) \
        == L.VRS_ERR_INVALID
    assert L.vrs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k2.data_ptr(), v2.data_ptr(), 0, 40, s) \
        == L.VRS_OK
