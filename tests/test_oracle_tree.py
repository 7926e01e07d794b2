"""Pins for the oracle's tree and interaction lists (no GPU): brute-force
checks of the FMM partition property on the image lattices."""
import numpy as np


def _img_row(term, r, nrow):
    return [r, -1 - r, 2 * nrow - 1 - r, r - 2 * nrow, r + 2 * nrow][term]


def test_tree_sorts_points_into_their_leaves(oracle):
    rng = np.random.default_rng(0)
    n, d, L = 500, 1.0, 3
    x = rng.uniform(0.3, 3.7, n)
    y = rng.uniform(-0.95, -0.05, n)
    x0, R, perm, ls = oracle.tree_build(x, y, d, L)
    assert x0 == 0.0 and R == 4
    assert np.array_equal(np.sort(perm), np.arange(n))
    w = d / 2 ** L
    ncol = R << L
    for leaf in range(len(ls) - 1):
        idx = perm[ls[leaf]:ls[leaf + 1]]
        assert np.all(np.diff(idx) > 0)          # ties broken by input index
        r, c = divmod(leaf, ncol)
        assert np.all((x[idx] >= x0 + c * w) & (x[idx] < x0 + (c + 1) * w))
        assert np.all((-y[idx] >= r * w) & (-y[idx] < (r + 1) * w))


def test_lists_partition_every_leaf_pair(oracle):
    # For every term and every (target leaf, source leaf) pair, exactly one of:
    # the ancestors at exactly one level are in a V list, or the leaves are in U.
    R, L = 3, 3
    seen = {}
    for l in range(L + 1):
        for t, term, s in oracle.vlist(R, l):
            seen.setdefault(("V", l), set()).add((int(t), int(term), int(s)))
    U = {(int(t), int(term), int(s)) for t, term, s in oracle.ulist(R, L)}
    ncolL, nrowL = R << L, 1 << L
    for term in range(5):
        for tl in range(ncolL * nrowL):
            for sl in range(ncolL * nrowL):
                hits = int((tl, term, sl) in U)
                for l in range(L + 1):
                    sh = L - l
                    ncol = R << l
                    ta = (tl // ncolL >> sh) * ncol + ((tl % ncolL) >> sh)
                    sa = (sl // ncolL >> sh) * ncol + ((sl % ncolL) >> sh)
                    hits += int((ta, term, sa) in seen.get(("V", l), set()))
                assert hits == 1, (term, tl, sl, hits)


def test_list_geometry(oracle):
    R, L = 4, 3
    for l in range(1, L + 1):
        V = oracle.vlist(R, l)
        ncol, nrow = R << l, 1 << l
        free = V[V[:, 1] == 0]
        counts = np.bincount(free[:, 0], minlength=ncol * nrow)
        assert counts.max() <= 27
        for t, term, s in V:
            rt, ct = divmod(t, ncol)
            rs, cs = divmod(s, ncol)
            ri = _img_row(term, rs, nrow)
            assert max(abs(ct - cs), abs(rt - ri)) >= 2
            assert abs(ct - cs) <= 3 and abs(rt - ri) <= 3
        # tb / bt images are never near: they only appear at level 0
        assert not np.any(V[:, 1] >= 3)
        # image terms only touch the two rows next to an interface
        tt = V[V[:, 1] == 1]
        assert np.all(tt[:, 0] // ncol <= 1) and np.all(tt[:, 2] // ncol <= 1)
    V0 = oracle.vlist(R, 0)
    assert np.sum(V0[:, 1] == 3) == R * R and np.sum(V0[:, 1] == 4) == R * R
    U = oracle.ulist(R, L)
    assert not np.any(U[:, 1] >= 3)
