"""Cross-layer operator (Sec. 3, Example 4 as printed): layer-1 sources to
middle-layer targets through g_2^t + g_2^b, by the two-wave-number FMM,
against the oracle's direct sum on sampled targets."""
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


def _case(ns, nt, x_hi, band_s, band_t, d, seed):
    rng = np.random.default_rng(seed)
    xs = rng.uniform(0.0, x_hi, ns)
    ys = rng.uniform(band_s[0], band_s[1], ns) * d
    xt = rng.uniform(0.0, x_hi, nt)
    yt = -rng.uniform(band_t[0], band_t[1], nt) * d
    q = rng.standard_normal((2, ns)) + 1j * rng.standard_normal((2, ns))
    return xs, ys, xt, yt, q


CASES = {
    # name: (medium, p, depth, tol, (ns, nt, x_hi, source band, target band))
    "uniform": (workloads.MEDIUM_A, 22, 2, 1e-10, (1000, 1200, 3.0, (0.05, 0.95), (0.05, 0.95))),
    "thin_interface": (workloads.MEDIUM_A, 22, 3, 1e-10, (1000, 1200, 3.0, (0.001, 0.02), (0.001, 0.02))),
    "k2_8": (workloads.MEDIUM_B, 30, 3, 1e-9, (1000, 1200, 3.0, (0.05, 0.95), (0.05, 0.95))),
}


@pytest.mark.parametrize("name", list(CASES))
def test_cross_fmm_matches_oracle(lm, oracle, name):
    import torch

    med, p, depth, tol, shape = CASES[name]
    xs, ys, xt, yt, q = _case(*shape, d=med[3], seed=31)
    m = lm.create_medium(*med, p=p, depth=depth)
    c = lm.build_cross(m, *(torch.from_numpy(a).cuda() for a in (xs, ys, xt, yt)))
    u = c.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    sub = np.sort(np.random.default_rng(32).choice(xt.size, 48, replace=False))
    ref = oracle.cross_direct(med, xs, ys, xt, yt, q, targets=sub)
    err = np.linalg.norm(u[:, sub] - ref) / np.linalg.norm(ref)
    print(f"cross {name} p={p} depth={c.info['depth']}: rel-l2 {err:.2e}")
    assert err < tol


def test_cross_rejects_points_on_the_wrong_side(lm):
    import torch

    xs = torch.tensor([0.5, 1.0], dtype=torch.float64, device="cuda")
    ys = torch.tensor([0.2, -0.1], dtype=torch.float64, device="cuda")   # one source below y = 0
    xt = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    yt = torch.tensor([-0.3], dtype=torch.float64, device="cuda")
    m = lm.create_medium(*workloads.MEDIUM_A, p=10)
    with pytest.raises(lm.LMError):
        lm.build_cross(m, xs, ys, xt, yt)
    mw = lm.create_medium(*workloads.MEDIUM_A, p=10, top_bc="dirichlet")
    with pytest.raises(lm.LMError):
        lm.build_cross(mw, xs, torch.abs(ys), xt, yt)   # the cross operator needs transmission interfaces


MIXED = {
    # name: (medium, p, depth, (ns, nt, x_hi, source band, target band))
    "uniform": (workloads.MEDIUM_A, 14, 2, (1000, 1200, 3.0, (0.05, 0.95), (0.05, 0.95))),
    "thin_interface": (workloads.MEDIUM_A, 14, 3, (1000, 1200, 3.0, (0.001, 0.02), (0.001, 0.02))),
    "k2_8": (workloads.MEDIUM_B, 18, 3, (1000, 1200, 3.0, (0.05, 0.95), (0.05, 0.95))),
}


@pytest.mark.parametrize("name", list(MIXED))
def test_cross_mixed_matches_oracle(lm, oracle, name):
    """The mixed form of the cross operator (FP32 expansions, translations and
    multiply-adds): 1e-6 against the oracle's direct sum, and close to the FP64 form."""
    import torch

    med, p, depth, shape = MIXED[name]
    xs, ys, xt, yt, q = _case(*shape, d=med[3], seed=41)
    pts = [torch.from_numpy(a).cuda() for a in (xs, ys, xt, yt)]
    c = lm.build_cross(lm.create_medium(*med, p=p, depth=depth, precision="mixed"), *pts)
    c64 = lm.build_cross(lm.create_medium(*med, p=p, depth=depth), *pts)
    qd = torch.from_numpy(q).cuda()
    u = c.apply(qd).cpu().numpy()
    u64 = c64.apply(qd).cpu().numpy()
    sub = np.sort(np.random.default_rng(42).choice(xt.size, 48, replace=False))
    ref = oracle.cross_direct(med, xs, ys, xt, yt, q, targets=sub)
    err = np.linalg.norm(u[:, sub] - ref) / np.linalg.norm(ref)
    e64 = np.linalg.norm(u - u64) / np.linalg.norm(u64)
    print(f"cross mixed {name} p={p}: rel-l2 {err:.2e} against the oracle, {e64:.2e} against the FP64 form")
    assert err < 1e-6 and e64 < 1e-6
