"""vrs_sort_pairs_noalloc: the radix sort for callers that cannot allocate device memory.

A real-time frame loop must not risk the device-wide synchronisation an
allocation can cause, and a plug-in may live inside a host application's fixed
memory budget; this entry point sorts with a static device array instead.  The
test compares it with the library's regular sort (vrs_bin_sort) on the same
instance lists, for two calls in a row of different sizes, bit for bit as every
sort test here does; then with a stable host sort at exactly the size limit and
with a key width that ends inside a byte while the bits above it are nonzero.
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


def _noalloc_vs_stable_host_sort(n, key_bits, seed):
    from paper_2410_17932_gb300 import _lib as L
    torch = torch_cuda()
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, np.iinfo(np.int64).max, n, dtype=np.int64)     # high bits set too
    keys[: n // 4] = keys[n // 4: n // 2]                                  # runs of equal sort bits
    vals = rng.integers(0, 2**31 - 1, n, dtype=np.int64).astype(np.int32)
    k_in = torch.as_tensor(keys, device="cuda")
    v_in = torch.as_tensor(vals, device="cuda")
    k_out = torch.full_like(k_in, -1)
    v_out = torch.full_like(v_in, -1)
    stream = torch.cuda.current_stream().cuda_stream
    code = L.vrs_sort_pairs_noalloc(k_in.data_ptr(), v_in.data_ptr(), k_out.data_ptr(), v_out.data_ptr(), n,
                                    key_bits, stream)
    assert code == L.VRS_OK, L.status_string(code)
    torch.cuda.synchronize()
    ku = keys.view(np.uint64)
    sort_bits = ku & np.uint64((1 << key_bits) - 1) if key_bits < 64 else ku
    order = np.argsort(sort_bits, kind="stable")
    assert np.array_equal(k_out.cpu().numpy(), keys[order])
    assert np.array_equal(v_out.cpu().numpy(), vals[order])


def test_noalloc_key_width_inside_a_byte():
    """key_bits = 12: the second pass sorts 4 bits; bits 12..63 are nonzero and must not
    reorder pairs whose low 12 bits are equal."""
    _noalloc_vs_stable_host_sort(200_000, 12, 5)
    _noalloc_vs_stable_host_sort(70_001, 37, 6)


def test_noalloc_at_the_size_limit():
    from paper_2410_17932_gb300 import _lib as L
    _noalloc_vs_stable_host_sort(L.VRS_NOALLOC_MAX_PAIRS, 40, 7)
