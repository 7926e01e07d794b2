"""The adaptive tree's host half (lm_adaptive_plan, no GPU) against the oracle's
adaptive tree and lists (Algorithm 1, step 1): bit-exact boxes, point order,
per-box point ranges, V and U lists; and its input checks."""
import numpy as np
import pytest

import workloads


@pytest.fixture(scope="module")
def lm():
    import paper_1902_08250_gb300 as lm

    return lm


@pytest.mark.parametrize("s,Lmax,seed,n", [(16, 8, 5, 3000), (40, 5, 6, 3000), (5000, 3, 7, 1200), (1, 2, 8, 600),
                                           (8, 10, 9, 2000)])
def test_plan_matches_oracle(lm, oracle, s, Lmax, seed, n):
    x, y, _ = workloads.clustered(n, 1, seed=seed)
    x = x * 0.4  # four roots
    d = workloads.MEDIUM_A[3]
    (x0, R), boxes, perm, pstart, V, U = lm.adaptive_plan(x, y, d, s, Lmax)
    (ox0, oR), oboxes, operm, opstart = oracle.adaptive_tree(x, y, d, s, Lmax)
    assert (x0, R) == (ox0, oR)
    assert np.array_equal(boxes, oboxes)
    assert np.array_equal(perm, operm) and np.array_equal(pstart, opstart)
    assert np.array_equal(V, oracle.adaptive_lists(x, y, d, s, Lmax, 0))
    assert np.array_equal(U, oracle.adaptive_lists(x, y, d, s, Lmax, 1))


def test_plan_edge_cases(lm):
    # one point: one root, one leaf; its reflected self terms are U entries, tb/bt are V at the root
    (x0, R), boxes, perm, pstart, V, U = lm.adaptive_plan(np.array([0.3]), np.array([-0.5]), 1.0, 16, -1)
    assert R == 1 and boxes.tolist() == [[0, 0, 0, 1]] and perm.tolist() == [0] and pstart.tolist() == [0, 1]
    assert U.tolist() == [[0, 0, 0], [0, 1, 0], [0, 2, 0]] and V.tolist() == [[0, 3, 0], [0, 4, 0]]
    # duplicate points refine to the depth limit and stay together in one leaf
    x, y = np.full(40, 0.25), np.full(40, -0.25)
    _, boxes, perm, pstart, _, _ = lm.adaptive_plan(x, y, 1.0, 4, 3)
    assert boxes[:, 0].max() == 3 and np.array_equal(perm, np.arange(40))
    assert np.diff(pstart).max() == 40
    for bad in ((np.array([0.1]), np.array([0.0])), (np.array([np.nan]), np.array([-0.5])),
                (np.array([0.1]), np.array([-1.0]))):
        with pytest.raises(lm.LMError):
            lm.adaptive_plan(*bad, 1.0, 16, -1)
    with pytest.raises(lm.LMError):
        lm.adaptive_plan(np.array([0.1]), np.array([-0.5]), 1.0, 0, -1)
