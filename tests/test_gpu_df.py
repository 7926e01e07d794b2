"""The FP64 form's double-float M2L, M2M and L2L (pairs of FP32 numbers on the
FP32 pipes; M2L tables row-major, or transposed for applies of 1-2 vectors)
against the IEEE FP64 contractions, on uniform and adaptive trees, and its
exponent scaling over the whole FP64 range of density magnitudes."""
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


def _apply(lm, x, y, q, **opt):
    import torch

    m = lm.create_medium(*MED_A, **opt)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    return lm.apply(t, torch.from_numpy(np.ascontiguousarray(q)).cuda()).cpu().numpy()


@pytest.mark.parametrize("case", ["uniform", "uniform1", "adaptive", "adaptive1", "dg_dd"])
def test_df_m2l_matches_fp64_m2l(lm, case):
    """Same tree, same everything but the M2L arithmetic: the two results agree to
    the double-float rounding -- each of the ~1300 additions per output rounds the
    low word at 2^-48 of the partial sum, sqrt(1300) 2^-48 ~ 1.3e-13 -- far inside
    the 1e-10 bar against the oracle."""
    nvec = 1 if case.endswith("1") else 5
    if case.startswith("adaptive"):
        x, y, q = workloads.clustered(6000, nvec, seed=3)
        opt = dict(p=20, adaptive=True, leaf_target=16)
    else:
        x, y, q = workloads.uniform_strip(20000, 0.0, 4.0, -0.9, -0.1, nvec=nvec, seed=2)
        opt = dict(p=20, depth=3)
        if case == "dg_dd":
            opt["kernel"] = lm.KERNEL_DG_DD
    a = _apply(lm, x, y, q, **opt)
    b = _apply(lm, x, y, q, m2l_fp64=True, **opt)
    err = np.linalg.norm(a - b) / np.linalg.norm(b)
    print(f"{case}: double-float vs FP64 M2L rel-l2 {err:.3e}")
    assert err <= 1e-12


def test_df_m2l_density_scale(lm):
    """u(s q) = s u(q) for s from 1e-200 to 1e200: the multipoles are rescaled by a
    power of two per apply, so FP32's exponent range never binds; zero densities
    give exactly zero."""
    x, y, q = workloads.uniform_strip(5000, 0.0, 2.0, -0.9, -0.1, nvec=4, seed=4)
    opt = dict(p=16, depth=3)
    u1 = _apply(lm, x, y, q, **opt)
    for s in (1e-200, 1e-30, 1e30, 1e200):
        us = _apply(lm, x, y, q * s, **opt) / s
        assert np.linalg.norm(us - u1) <= 1e-12 * np.linalg.norm(u1), s
    assert not np.any(_apply(lm, x, y, np.zeros_like(q), **opt))
