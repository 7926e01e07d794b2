"""GPU parity of the adaptive tree (Algorithm 1, step 1): boxes, tree order and
interaction lists bit-exact against the oracle's adaptive tree, the uniform
tree reproduced when every box is refined, and the FMM (apply, adjoint, target
gradient, dG/dd; FP64 and mixed) against the oracle's direct sums on clustered
points."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
MED_A = workloads.MEDIUM_A


@pytest.fixture(scope="module")
def lm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    import paper_1902_08250_gb300 as lm

    return lm


def _dev(*arrs):
    import torch

    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _tree(lm, x, y, **opt):
    m = lm.create_medium(*MED_A, adaptive=True, **opt)
    return lm.build_tree(m, *_dev(x, y))


@pytest.mark.parametrize("s,Lmax", [(16, 8), (40, 5), (5000, 3), (1, 2)])
def test_tree_and_lists_bit_exact(lm, oracle, s, Lmax):
    """Clustered points (half within 0.01 of y = 0): boxes, perm, per-box point
    ranges, V and U lists equal the oracle's.  s = 5000 leaves the roots unsplit;
    s = 1 refines every occupied box to the depth limit."""
    x, y, _ = workloads.clustered(3000, 1, seed=5)
    d = MED_A[3]
    t = _tree(lm, x, y, p=6, depth=Lmax, leaf_target=s)
    (x0, R), boxes, perm, pstart = oracle.adaptive_tree(x, y, d, s, Lmax)
    info = t.info
    assert info["adaptive"] == 1 and info["R"] == R and info["x_origin"] == x0
    assert info["nbox"] == boxes.shape[0] and info["nleaf"] == int(boxes[:, 3].sum())
    assert info["depth"] == int(boxes[:, 0].max())
    assert np.array_equal(t.boxes(), boxes)
    p2, ls2 = t.export()
    assert np.array_equal(p2, perm) and np.array_equal(ls2, pstart)
    for which in (0, 1):
        assert np.array_equal(t.list_export(which), oracle.adaptive_lists(x, y, d, s, Lmax, which)), which


def test_uniform_refinement_equivalence(lm):
    """When every box below the depth limit holds more than s points, the adaptive
    tree is the uniform tree: same boxes, the uniform V lists of every level and
    the U list (box ids offset by the boxes of the coarser levels), and the same
    FMM result."""
    import torch

    rng = np.random.default_rng(7)
    n, L = 20000, 3
    x = rng.uniform(0.0, 2.0, n)
    y = rng.uniform(-0.999, -0.001, n)
    q = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    ta = _tree(lm, x, y, p=16, depth=L, leaf_target=16)
    mu = lm.create_medium(*MED_A, p=16, depth=L)
    tu = lm.build_tree(mu, *_dev(x, y))
    assert ta.info["nbox"] == tu.info["nbox"] and ta.info["depth"] == L
    assert np.array_equal(ta.boxes(), tu.boxes())
    R = tu.info["R"]
    off = np.cumsum([0] + [R * 4 ** l for l in range(L + 1)])
    vu = []
    for l in range(L + 1):
        rows = tu.list_export(0, l).copy()
        rows[:, 0] += off[l]
        rows[:, 2] += off[l]
        vu.append(rows)
    vu = np.concatenate(vu)
    vu = vu[np.lexsort((vu[:, 2], vu[:, 1], vu[:, 0]))]
    assert np.array_equal(ta.list_export(0), vu)
    uu = tu.list_export(1).copy()
    uu[:, 0] += off[L]
    uu[:, 2] += off[L]
    assert np.array_equal(ta.list_export(1), uu)
    qd = torch.from_numpy(q).cuda()
    ua = lm.apply(ta, qd).cpu().numpy()
    ub = lm.apply(tu, qd).cpu().numpy()
    assert np.linalg.norm(ua - ub) <= 1e-14 * np.linalg.norm(ub)


def _sample(n, y, rng, k):
    near = np.nonzero(y > -0.01)[0]
    far = np.nonzero(y <= -0.01)[0]
    return np.sort(np.concatenate([rng.choice(near, k, replace=False), rng.choice(far, k, replace=False)]))


def test_clustered_fmm_apply_and_adjoint(lm, oracle):
    """n = 6000 clustered points, automatic depth limit, s = 24, p = 20: u = G q and
    w = G^H v = conj(G conj v) against the oracle's direct sum on 32 targets."""
    import torch

    x, y, q = workloads.clustered(6000, 2, seed=3)
    t = _tree(lm, x, y, p=20, leaf_target=24)
    info = t.info  # refined near the interface only
    assert info["depth"] >= 5 and info["nleaf"] < info["R"] * 4 ** info["depth"] // 8
    sub = _sample(x.size, y, np.random.default_rng(4), 16)
    qd = torch.from_numpy(q).cuda()
    u = lm.apply(t, qd).cpu().numpy()[:, sub]
    ref = oracle.direct_apply(MED_A, x, y, q, targets=sub)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    w = lm.apply_adjoint(t, qd).cpu().numpy()[:, sub]
    refw = np.conj(oracle.direct_apply(MED_A, x, y, np.conj(q), targets=sub))
    assert np.linalg.norm(w - refw) <= 1e-10 * np.linalg.norm(refw)


def test_clustered_gradient_and_dg_dd(lm, oracle):
    """Target gradient (lm_apply_grad) and the dG/dd kernel on an adaptive tree
    against the oracle's differentiated direct sums; p = 22 as for the uniform
    tree's gradients (differentiating the local expansion costs about one order)."""
    import torch

    x, y, q = workloads.clustered(3000, 1, seed=8)
    sub = _sample(x.size, y, np.random.default_rng(9), 8)
    qd = torch.from_numpy(q).cuda()
    t = _tree(lm, x, y, p=22, leaf_target=24)
    u, ux, uy = lm.apply_grad(t, qd)
    for got, der in ((ux, oracle.DX), (uy, oracle.DY)):
        ref = oracle.direct_apply_deriv(MED_A, x, y, q, der, targets=sub)
        g = got.cpu().numpy()[:, sub]
        err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        print(f"adaptive gradient d{'xy'[der - 1]}: rel-l2 {err:.3e}")
        assert err <= 1e-9, der
    ref = oracle.direct_apply(MED_A, x, y, q, targets=sub)
    assert np.linalg.norm(u.cpu().numpy()[:, sub] - ref) <= 1e-10 * np.linalg.norm(ref)
    td = _tree(lm, x, y, p=22, leaf_target=24, kernel=lm.KERNEL_DG_DD)
    ud = lm.apply(td, qd).cpu().numpy()[:, sub]
    ref = oracle.direct_apply_deriv(MED_A, x, y, q, oracle.DD, targets=sub)
    assert np.linalg.norm(ud - ref) <= 1e-9 * np.linalg.norm(ref)


def test_single_point_and_unrefined(lm, oracle):
    """n = 1 (one root, one box: only the reflected self-interaction) and a tree whose
    roots are all leaves (s >= n): the FMM against the direct sum."""
    import torch

    x, y = np.array([0.3]), np.array([-0.02])
    q = np.array([[1.0 - 2.0j]])
    t = _tree(lm, x, y, p=12)
    assert t.info["nbox"] == 1 and t.info["nleaf"] == 1
    u = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()
    ref = oracle.direct_apply(MED_A, x, y, q)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)  # one pair: the near-field quadrature alone
    x, y, q = workloads.clustered(400, 1, seed=2)
    t = _tree(lm, x, y, p=20, leaf_target=1000)
    assert t.info["depth"] == 0
    u = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()
    ref = oracle.direct_apply(MED_A, x, y, q)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("nvec", [2, 16])
def test_adaptive_mixed_matches_oracle(lm, oracle, nvec):
    """The mixed form on the adaptive tree: cross-level M2L on the staged CUDA-core
    contraction, the leaf, S2M, M2M, L2L and segment kernels over the box lists.
    Clustered points (half within 0.01 of y = 0), p = 14, apply and adjoint against the
    oracle's direct sum at 1e-6; 2 vectors run the 4-slot kernels, 16 the full width."""
    import torch

    x, y, q = workloads.clustered(6000, nvec, seed=5)
    t = _tree(lm, x, y, p=14, leaf_target=24, precision="mixed")
    assert t.info["adaptive"] == 1 and t.info["depth"] >= 5
    sub = _sample(x.size, y, np.random.default_rng(6), 16)
    qd = torch.from_numpy(q).cuda()
    u = lm.apply(t, qd).cpu().numpy()[:, sub]
    ref = oracle.direct_apply(MED_A, x, y, q, targets=sub)
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    w = lm.apply_adjoint(t, qd).cpu().numpy()[:, sub]
    refw = np.conj(oracle.direct_apply(MED_A, x, y, np.conj(q), targets=sub))
    errw = np.linalg.norm(w - refw) / np.linalg.norm(refw)
    print(f"adaptive mixed nvec={nvec}: apply rel-l2 {err:.3e}, adjoint {errw:.3e}")
    assert err < 1e-6 and errw < 1e-6
    # complex64 buffers give the same result rounded
    u64 = lm.apply(t, qd.to(torch.complex64)).cpu().numpy()[:, sub]
    assert np.linalg.norm(u64 - ref) <= 1e-6 * np.linalg.norm(ref)


def test_adaptive_mixed_near_walls(lm, oracle):
    """Mixed adaptive tree refined next to two impedance walls (reflected tails and the
    factorised segment over the box lists), 16 vectors, against the oracle at 1e-6."""
    import torch

    rng = np.random.default_rng(33)
    n = 4000
    x = rng.uniform(0.0, 3.0, n)
    y = np.concatenate([-0.01 * (1.0 - rng.uniform(0.0, 1.0, n // 4)),
                        -1.0 + 0.01 * (1.0 - rng.uniform(0.0, 1.0, n // 4)),
                        rng.uniform(-0.9, -0.1, n - n // 2)])
    q = rng.standard_normal((16, n)) + 1j * rng.standard_normal((16, n))
    med = (1.0, 1.5, 2.0, 1.0)
    m = lm.create_medium(*med, p=14, adaptive=True, leaf_target=16, precision="mixed", top_bc="impedance",
                         top_alpha=0.7, bottom_bc="impedance", bottom_alpha=-0.3)
    t = lm.build_tree(m, *_dev(x, y))
    sub = np.sort(np.concatenate([rng.choice(n // 4, 12, replace=False), n // 4 + rng.choice(n // 4, 12, replace=False),
                                  n // 2 + rng.choice(n - n // 2, 8, replace=False)]))
    u = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()[:, sub]
    try:
        oracle.set_boundaries("impedance", 0.7, "impedance", -0.3)
        ref = oracle.direct_apply(med, x, y, q, targets=sub)
    finally:
        oracle.set_boundaries()
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    print(f"adaptive mixed impedance walls: rel-l2 {err:.3e}")
    assert err < 1e-6


@pytest.mark.parametrize("media", [(("impedance", 0.7), ("impedance", -0.3)), (("neumann", 0.0), ("dirichlet", 0.0))])
def test_adaptive_media_near_both_walls(lm, oracle, media):
    """Walls in place of the interfaces (Sec. 3, Examples 2 and 3) on an adaptive tree
    refined near both of them: points within 0.01 of y = 0 and of y = -d, the FMM
    against the oracle's direct sum on 32 targets."""
    import torch

    (tb, ta), (bb, ba) = media
    rng = np.random.default_rng(31)
    n = 4000
    x = rng.uniform(0.0, 3.0, n)
    y = np.concatenate([-0.01 * (1.0 - rng.uniform(0.0, 1.0, n // 4)),
                        -1.0 + 0.01 * (1.0 - rng.uniform(0.0, 1.0, n // 4)),
                        rng.uniform(-0.9, -0.1, n - n // 2)])
    q = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    med = (1.0, 1.5, 2.0, 1.0)
    m = lm.create_medium(*med, p=22, adaptive=True, leaf_target=16, top_bc=tb, top_alpha=ta, bottom_bc=bb,
                         bottom_alpha=ba)
    t = lm.build_tree(m, *_dev(x, y))
    sub = np.sort(np.concatenate([rng.choice(n // 4, 12, replace=False), n // 4 + rng.choice(n // 4, 12, replace=False),
                                  n // 2 + rng.choice(n - n // 2, 8, replace=False)]))
    u = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()[:, sub]
    try:
        oracle.set_boundaries(tb, ta, bb, ba)
        ref = oracle.direct_apply(med, x, y, q, targets=sub)
    finally:
        oracle.set_boundaries()
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    print(f"adaptive {tb}/{bb}: rel-l2 {err:.3e}")
    assert err <= 1e-10


def test_adaptive_vector_chunks(lm):
    """18 vectors on an adaptive tree go as 16 + 2: each chunk equals the same
    vectors applied alone (the 2-vector chunk bit for bit; the 16-vector chunk to
    the double-float rounding, its M2L tables being read in the other layout)."""
    import torch

    x, y, q = workloads.clustered(5000, 18, seed=12)
    t = _tree(lm, x, y, p=18, leaf_target=16)
    qd = torch.from_numpy(q).cuda()
    u = lm.apply(t, qd).cpu().numpy()
    assert np.array_equal(u[16:], lm.apply(t, qd[16:].contiguous()).cpu().numpy())
    u4 = lm.apply(t, qd[4:8].contiguous()).cpu().numpy()
    assert np.array_equal(u[4:8], u4)
    u1 = lm.apply(t, qd[5:6].contiguous()).cpu().numpy()
    assert np.linalg.norm(u1[0] - u[5]) <= 1e-12 * np.linalg.norm(u[5])
