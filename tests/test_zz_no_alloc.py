"""The allocation-free tree-order entry point (lm_tree_order_noalloc) against
the tree order lm_build_tree produces, through the C ABI, on two calls in a
row.  It serves callers that cannot allocate device memory (start-up-only
allocation, allocator callbacks, memory owned by another framework's pool).

Collected last on purpose (file name), so a run that stops at the first
failure has run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _noalloc(lm, xd, yd, d, depth, cap):
    import torch

    n = xd.numel()
    perm = torch.empty(n, dtype=torch.int64, device=xd.device)
    ls = torch.empty(cap, dtype=torch.int64, device=xd.device)
    x0 = ctypes.c_double()
    R = ctypes.c_int()
    st = lm._lib.lm_tree_order_noalloc(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), n, d,
                                       depth, ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(ls.data_ptr()),
                                       cap, ctypes.byref(x0), ctypes.byref(R),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, perm.cpu().numpy(), ls.cpu().numpy(), x0.value, R.value


def test_tree_order_noalloc_matches_build_tree():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    import paper_1902_08250_gb300 as lm

    large = (workloads.wide_uniform(200_000, 1)[:2], workloads.MEDIUM_B, 5)
    small = (workloads.small_uniform(1000)[:2], workloads.MEDIUM_A, 3)
    # calls in a row: large, small, large.  The small call reuses counters that the
    # large call left in the shared array, and the second large call reuses
    # counters beyond the small call's range, so a missing clear fails a comparison.
    for (x, y), med, depth in (large, small, large):
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y).cuda()
        t = lm.build_tree(lm.create_medium(*med, p=4, depth=depth), xd, yd)
        perm, ls = t.export()
        nleaf = t.info["nleaf"]
        st, perm2, ls2, x0, R = _noalloc(lm, xd, yd, med[3], depth, nleaf + 1)
        assert st == 0, lm._lib.lm_last_error()
        assert R == t.info["R"] and x0 == t.info["x_origin"]
        assert np.array_equal(perm2, perm)
        assert np.array_equal(ls2[:nleaf + 1], ls)
    # sizes beyond the fixed scratch are rejected with a clear error
    x, y = workloads.small_uniform(16)[:2]
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    st, *_ = _noalloc(lm, xd, yd, 1.0, 3, 8)      # leaf_start too short
    assert st == 1 and b"entries" in lm._lib.lm_last_error()
    st, *_ = _noalloc(lm, xd, yd, 1.0, 10, 1 << 22)  # too many leaves
    assert st == 1 and b"scratch limit" in lm._lib.lm_last_error()
    st, *_ = _noalloc(lm, xd, yd, float("inf"), 3, 1 << 10)  # non-finite thickness
    assert st == 1 and b"finite" in lm._lib.lm_last_error()
    # an x spread of 3e9 thicknesses: the leaf count is rejected, not wrapped to a negative int
    xw = x.copy()
    xw[-1] = 3e9
    st, *_ = _noalloc(lm, torch.from_numpy(xw).cuda(), yd, 1.0, 0, 1 << 10)
    assert st == 1 and b"scratch limit" in lm._lib.lm_last_error()
    # the same spread through lm_build_tree: more than 2^30 roots is an invalid argument
    with pytest.raises(lm.LMError) as e:
        lm.build_tree(lm.create_medium(*workloads.MEDIUM_A, p=4, depth=0), torch.from_numpy(xw).cuda(), yd)
    assert e.value.status == 1 and "roots" in str(e.value)
