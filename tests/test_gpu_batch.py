"""Batched form: complex64 buffers on mixed-precision trees, the M2L tile
autotuner, and many independent instances (own medium, size) in one captured
graph, each checked against the oracle on sampled targets."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    import paper_1902_08250_gb300 as lm

    return lm


def test_complex64_buffers_match_complex128(lm):
    """The mixed path computes in FP32 either way: complex64 output is the complex128
    output rounded, bit for bit; the same for the adjoint."""
    import torch

    x, y, q = workloads.uniform_strip(30_000, 0.0, 6.0, -0.9, -0.1, nvec=5, seed=3)
    q = q.astype(np.complex64)
    m = lm.create_medium(*workloads.MEDIUM_A, p=12, precision="mixed")
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    q64 = torch.from_numpy(q).cuda()
    q128 = q64.to(torch.complex128)
    for fn in (lm.apply, lm.apply_adjoint):
        u64 = fn(t, q64)
        u128 = fn(t, q128)
        assert u64.dtype == torch.complex64
        assert torch.equal(u64, u128.to(torch.complex64))
    m64 = lm.create_medium(*workloads.MEDIUM_A, p=12)
    t64 = lm.build_tree(m64, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    with pytest.raises(lm.LMError):
        lm.apply(t64, q64)   # complex64 buffers need a mixed-precision tree


def test_autotune_choices_and_accuracy(lm):
    import torch

    x, y, q = workloads.wide_uniform(400_000, 16, seed=5)
    m = lm.create_medium(*workloads.MEDIUM_B, p=14, precision="mixed")
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    qd = torch.from_numpy(q).cuda()
    u0 = lm.apply(t, qd).cpu().numpy()
    tune = t.autotune()
    print("autotune (choice, ms) per level:", tune)
    assert tune[0][0] == -1
    assert all(c in (0, 2, 4, 8) and ms > 0 for c, ms in tune[1:])
    u1 = lm.apply(t, qd).cpu().numpy()
    # different M2L kernels round differently; both are FP32-accurate
    assert np.linalg.norm(u1 - u0) <= 5e-7 * np.linalg.norm(u0)


def test_batched_instances_match_oracle(lm, oracle):
    """Instances shaped like the batched workload (random media, log-uniform N,
    4 complex64 vectors), autotuned, captured in one graph; per instance the
    density sits on 600 random sources so the oracle's exact values at 16 other
    targets are short sums; bar 1e-6 relative per instance."""
    import torch

    inst = workloads.batched_instances(count=6, n_lo=10_000, n_hi=120_000, nvec=4, seed=11)
    rng = np.random.default_rng(12)
    trees, qs, us, refs, tgs = [], [], [], [], []
    for med, x, y, q in inst:
        n = x.size
        perm = rng.permutation(n)
        src, tg = np.sort(perm[:600]), np.sort(perm[600:616])
        qq = np.zeros_like(q)
        qq[:, src] = q[:, src]
        m = lm.create_medium(*med, p=14, precision="mixed", autotune=1)
        t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
        xs, ys = np.concatenate([x[src], x[tg]]), np.concatenate([y[src], y[tg]])
        qo = np.concatenate([qq[:, src], np.zeros((4, tg.size))], axis=1).astype(np.complex128)
        refs.append(oracle.direct_apply(med, xs, ys, qo, targets=np.arange(src.size, src.size + tg.size)))
        trees.append(t)
        qs.append(torch.from_numpy(qq).cuda())
        us.append(torch.zeros_like(qs[-1]))
        tgs.append(tg)
    b = lm.Batch(trees, qs, us)
    b.launch()
    torch.cuda.synchronize()
    for (med, *_), u, ref, tg in zip(inst, us, refs, tgs):
        got = u.cpu().numpy()[:, tg].astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"instance k={np.round(med[:3], 2)} d={med[3]:.2f}: rel-l2 {err:.2e}")
        assert err < 1e-6


def test_few_vectors_match_full_width(lm):
    """Applies of up to 4 vectors take the 4-vector forms of every contraction (S2M,
    M2M, L2L, rest-list and tensor-core M2L: 32 boxes x 4 vectors per tile; the leaf
    kernel); they agree with the same vectors computed inside a 16-vector apply.  The
    16-vector apply runs the tile-form M2L of all levels, which orders its sums
    differently (and splits the tables from FP64), so the two agree to the mixed
    path's rounding, not bit for bit; both meet the mixed bar against the FP64 apply."""
    import torch

    x, y, q = workloads.uniform_strip(60_000, 0.0, 8.0, -0.95, -0.05, nvec=16, seed=9)
    m = lm.create_medium(*workloads.MEDIUM_B, p=14, precision="mixed")
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    qd = torch.from_numpy(q).cuda()
    full = lm.apply(t, qd).cpu().numpy()
    ref = lm.apply(lm.build_tree(lm.create_medium(*workloads.MEDIUM_B, p=20), t._x, t._y), qd[:3].contiguous())
    ref = ref.cpu().numpy()
    assert np.linalg.norm(full[:3] - ref) <= 1e-6 * np.linalg.norm(ref)
    for nv in (3, 1):
        few = lm.apply(t, qd[:nv].contiguous()).cpu().numpy()
        assert np.linalg.norm(few - full[:nv]) <= 1e-6 * np.linalg.norm(full[:nv]), nv
        assert np.linalg.norm(few - ref[:nv]) <= 1e-6 * np.linalg.norm(ref[:nv]), nv


@pytest.mark.parametrize("nvec", [4, 16])
def test_joint_tile_batch_matches_separate_applies(lm, nvec):
    """A batch whose mixed trees all run the tile-form M2L with one expansion order
    takes one persistent M2L launch over the concatenated work lists of every tree.
    Each tile sums the same entries in the same order as in a separate apply, so the
    batch reproduces the separate applies bit for bit, complex64 and complex128
    buffers alike; a batch mixing 4- and 16-vector entries falls back to per-tree
    applies and matches too."""
    import torch

    inst = workloads.batched_instances(count=5, n_lo=8_000, n_hi=90_000, nvec=nvec, seed=21)
    trees, qs = [], []
    for i, (med, x, y, q) in enumerate(inst):
        m = lm.create_medium(*med, p=14, precision="mixed")
        trees.append(lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()))
        qd = torch.from_numpy(q).cuda()
        qs.append(qd if i % 2 else qd.to(torch.complex128))
    sep = [lm.apply(t, q) for t, q in zip(trees, qs)]
    us = [torch.zeros_like(q) for q in qs]
    b = lm.Batch(trees, qs, us)
    kernels, joint = b.info()
    assert joint and kernels > len(trees)
    for _ in range(2):
        b.launch()
        torch.cuda.synchronize()
        for i, (u, s) in enumerate(zip(us, sep)):
            assert torch.equal(u, s), i
    mix_q = [q if i % 2 else q[:2].contiguous() for i, q in enumerate(qs)]
    mix_u = [torch.zeros_like(q) for q in mix_q]
    mix_sep = [lm.apply(t, q) for t, q in zip(trees, mix_q)]
    bm = lm.Batch(trees, mix_q, mix_u)
    assert bm.info()[1] == (nvec == 4)
    bm.launch()
    torch.cuda.synchronize()
    for i, (u, s) in enumerate(zip(mix_u, mix_sep)):
        assert torch.equal(u, s), i
