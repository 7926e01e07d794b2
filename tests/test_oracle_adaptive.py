"""Pins of the oracle's adaptive tree and its dual-traversal lists (Algorithm 1
step 1): on a tree refined uniformly they are the uniform V and U lists; on
clustered points every (target leaf, source leaf, term) is covered exactly once
-- by a U entry or by one V entry of an ancestor pair -- and every V entry is
well separated."""
import numpy as np
import pytest

import workloads


def _map_to_levels(boxes, rows):
    """global box ids -> (level, id within level) with the level's ids = row * ncol + col"""
    lev_start = {}
    for i, (l, c, r, leaf) in enumerate(boxes):
        lev_start.setdefault(int(l), i)
    return lev_start


def test_uniform_refinement_gives_the_uniform_lists(oracle):
    x, y, _ = workloads.small_uniform(300, 1, seed=2)
    d, L = 1.0, 3
    (x0, R), boxes, perm, pstart = oracle.adaptive_tree(x, y, d, -1, L)   # s = -1: split every box
    assert len(boxes) == sum(R * 4 ** l for l in range(L + 1))
    V = oracle.adaptive_lists(x, y, d, -1, L, 0)
    U = oracle.adaptive_lists(x, y, d, -1, L, 1)
    ls = _map_to_levels(boxes, V)
    lev = boxes[:, 0]
    for l in range(L + 1):
        sel = lev[V[:, 0]] == l
        got = V[sel].copy()
        got[:, 0] -= ls[l]
        assert np.all(lev[V[sel][:, 2]] == l)
        got[:, 2] -= ls[l]
        ref = oracle.vlist(R, l)
        assert np.array_equal(got, ref), l
    got = U.copy()
    got[:, 0] -= ls[L]
    got[:, 2] -= ls[L]
    assert np.array_equal(got, oracle.ulist(R, L))
    # the uniform tree's point order
    _, _, perm_u, start_u = oracle.tree_build(x, y, d, L)
    assert np.array_equal(perm, perm_u)
    assert np.array_equal(pstart[ls[L]:], start_u) and not pstart[:ls[L] + 1].any()


def _descendant_leaves(boxes):
    """leaf ids under every box (boxes numbered level by level, row * ncol + col)"""
    index = {(int(l), int(c), int(r)): i for i, (l, c, r, _) in enumerate(boxes)}
    out = {}
    for i in range(len(boxes) - 1, -1, -1):
        l, c, r, leaf = (int(v) for v in boxes[i])
        if leaf:
            out[i] = {i}
        else:
            s = set()
            for k in range(4):
                s |= out[index[(l + 1, 2 * c + (k & 1), 2 * r + (k >> 1))]]
            out[i] = s
    return out


def test_clustered_lists_cover_every_leaf_pair_once(oracle):
    x, y, _ = workloads.clustered(1500, 1, seed=5)
    x = x * 0.3   # three roots
    d, s, L = 1.0, 20, 8
    (x0, R), boxes, perm, pstart = oracle.adaptive_tree(x, y, d, s, L)
    leaves = [i for i in range(len(boxes)) if boxes[i, 3]]
    assert pstart[-1] == x.size
    counts = np.diff(pstart)
    assert np.all(counts[boxes[:, 3] == 0] == 0)
    assert max(int(boxes[:, 0].max()), 1) > 2          # refined near y = 0
    assert np.all(counts[[i for i in leaves if boxes[i, 0] < L]] <= s)
    V = oracle.adaptive_lists(x, y, d, s, L, 0)
    U = oracle.adaptive_lists(x, y, d, s, L, 1)
    under = _descendant_leaves(boxes)
    pos = {b: k for k, b in enumerate(leaves)}
    for m in range(5):
        cover = np.zeros((len(leaves), len(leaves)), np.int64)
        for t, term, sb in U[U[:, 1] == m]:
            cover[pos[t], pos[sb]] += 1
        for t, term, sb in V[V[:, 1] == m]:
            for a in under[t]:
                for b in under[sb]:
                    cover[pos[a], pos[b]] += 1
        assert np.all(cover == 1), (m, int(cover.min()), int(cover.max()))


def test_clustered_v_entries_are_separated(oracle):
    x, y, _ = workloads.clustered(1500, 1, seed=5)
    d, s, L = 1.0, 20, 8
    (x0, R), boxes, perm, pstart = oracle.adaptive_tree(x, y, d, s, L)
    V = oracle.adaptive_lists(x, y, d, s, L, 0)

    def centre(b, m):
        l, c, r, _ = (int(v) for v in boxes[b])
        w = d / 2 ** l
        yc = -(r + 0.5) * w
        yi = [yc, -yc, -2 * d - yc, yc + 2 * d, yc - 2 * d][m]   # image centre
        return x0 + (c + 0.5) * w, yi, w

    for t, m, sb in V[:: max(1, len(V) // 4000)]:
        xt, yt, wt = centre(t, 0)
        xs, ys, ws = centre(sb, m)
        assert max(abs(xt - xs), abs(yt - ys)) >= (wt + ws) * (1 - 1e-12)
