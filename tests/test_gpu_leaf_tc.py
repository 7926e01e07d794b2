"""Tensor-core leaf step (L2T and direct S2T of 16-vector mixed applies on
uniform trees): against the CUDA-core leaf kernel of the same tree and against
the FP64 apply, on the short-series case (k2 w <= 0.7), the general case with
the far form of H0 and leaves of more than 64 points, and points crowding an
interface (reflected tails in the U lists)."""
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


def _case(name):
    if name == "strip_series":   # 80k points, depth 4: k2 w = 0.5, degree-6 series
        x, y, q = workloads.uniform_strip(80_000, 0.0, 4.0, -0.95, -0.05, nvec=16, seed=31)
        return x, y, q, workloads.MEDIUM_B, 14, 4
    if name == "strip_far":      # depth 3: k2 w = 1, far form; ~310 points per leaf (5 passes)
        x, y, q = workloads.uniform_strip(60_000, 0.0, 3.0, -0.95, -0.05, nvec=16, seed=32)
        return x, y, q, workloads.MEDIUM_B, 14, 3
    if name == "interface":      # half the points within 0.01 of y = 0 on a uniform tree
        x, y, _ = workloads.clustered(40_000, 1, seed=33)
        q = workloads.densities(np.random.default_rng(34), 16, x.size)
        return x, y, q, workloads.MEDIUM_A, 10, 4
    raise KeyError(name)


@pytest.mark.parametrize("name", ["strip_series", "strip_far", "interface"])
def test_tensor_leaf_matches_cuda_core_leaf(lm, name):
    import torch

    x, y, q, med, p, depth = _case(name)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    qd = torch.from_numpy(q).cuda()
    tc = lm.build_tree(lm.create_medium(*med, p=p, depth=depth, precision="mixed"), xd, yd)
    cc = lm.build_tree(lm.create_medium(*med, p=p, depth=depth, precision="mixed", tensor_leaf=0), xd, yd)
    ref = lm.build_tree(lm.create_medium(*med, p=20, depth=depth), xd, yd)
    u_tc = lm.apply(tc, qd).cpu().numpy()
    u_cc = lm.apply(cc, qd).cpu().numpy()
    u_64 = lm.apply(ref, qd).cpu().numpy()
    lm.sync_status(tc)
    e_cc = np.linalg.norm(u_tc - u_cc) / np.linalg.norm(u_cc)
    e_tc = np.linalg.norm(u_tc - u_64) / np.linalg.norm(u_64)
    e_ref = np.linalg.norm(u_cc - u_64) / np.linalg.norm(u_64)
    print(f"{name}: tensor-core leaf vs CUDA-core leaf {e_cc:.2e}; vs FP64 {e_tc:.2e} (CUDA-core leaf {e_ref:.2e})")
    # the leaf step alone: same tree, same expansions, same truncation
    assert e_cc < 1e-6
    per = np.linalg.norm(u_tc - u_cc, axis=1) / np.linalg.norm(u_cc, axis=1)
    assert per.max() < 1e-6
    # the whole apply against FP64, at the mixed bar (the FMM truncation included)
    assert e_tc < max(1e-6, 1.2 * e_ref)


def test_tensor_leaf_few_vectors_and_off(lm):
    """Applies of at most 4 vectors keep the CUDA-core leaf kernel, and tensor_leaf = 0
    gives the CUDA-core result bit for bit."""
    import torch

    x, y, q, med, p, depth = _case("strip_series")
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    tc = lm.build_tree(lm.create_medium(*med, p=p, depth=depth, precision="mixed"), xd, yd)
    cc = lm.build_tree(lm.create_medium(*med, p=p, depth=depth, precision="mixed", tensor_leaf=0), xd, yd)
    q3 = torch.from_numpy(q[:3]).cuda()
    assert torch.equal(lm.apply(tc, q3), lm.apply(cc, q3))


@pytest.mark.parametrize("e", [24, -24])
def test_power_of_two_scaling_is_exact(lm, e):
    """The FP16 operands of the tensor-core leaf step and of the tile-form M2L take
    power-of-two scales from the apply's largest density, multipole and local-expansion
    components; every other step is linear FP32 arithmetic, which a power of two passes
    through exactly.  So the apply of 2^e q is 2^e times the apply of q, bit for bit, with
    densities far outside FP16's range (2^24 above its largest value, or 2^-24 below 1)."""
    import torch

    x, y, q, med, p, depth = _case("strip_series")
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    t = lm.build_tree(lm.create_medium(*med, p=p, depth=depth, precision="mixed"), xd, yd)
    assert t.info["tensor_leaf"]
    qd = torch.from_numpy(q).cuda()
    u1 = lm.apply(t, qd)
    u2 = lm.apply(t, qd * 2.0**e)
    lm.sync_status(t)
    assert torch.isfinite(u1.real).all() and torch.isfinite(u1.imag).all()
    assert torch.equal(u2, u1 * 2.0**e)
