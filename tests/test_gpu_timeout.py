"""Failure path of the bounded device waits (no GPU fault is provoked): with the
tensor-core M2L's first operand wait limited to zero polls (lm_set_poll_limit),
every CTA gives up at once, lets its copies in flight land, frees its tensor
memory and returns; lm_sync_status reports LM_ETIMEOUT.  The next apply on the
same tree, with the library's limit, is correct again."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

LM_ETIMEOUT = 4


def test_tensor_core_wait_timeout_is_reported_and_recovers():
    import torch

    import paper_1902_08250_gb300 as lm

    x, y, q = workloads.wide_uniform(60_000, 16, seed=4)
    xd, yd, qd = (torch.from_numpy(a).cuda() for a in (x, y, q))
    m = lm.create_medium(*workloads.MEDIUM_B, p=14, depth=3, precision="mixed")
    t = lm.build_tree(m, xd, yd)
    ref = lm.apply(t, qd)
    lm.sync_status(t)
    lm.set_poll_limit(t, 0)
    lm.apply(t, qd)
    with pytest.raises(lm.LMError) as e:
        lm.sync_status(t)
    assert e.value.status == LM_ETIMEOUT
    # the limit applied to one apply; the flag was cleared by sync_status
    u = lm.apply(t, qd)
    lm.sync_status(t)
    assert torch.equal(u, ref)
    # and the result meets the mixed bar against the FP64 apply of the same points
    uf = lm.apply(lm.build_tree(lm.create_medium(*workloads.MEDIUM_B, p=20), xd, yd), qd)
    err = float(torch.linalg.norm(u - uf) / torch.linalg.norm(uf))
    assert err < 1e-6, err
