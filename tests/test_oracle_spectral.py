"""Pins for the oracle's densities, branch and quadrature rule (no GPU).

Each check compares against something other than the oracle's own formula:
the paper's 4x4 system solved numerically, a direct solve of the interface
conditions, exact polynomial integration, and closed-form limits.
"""
import numpy as np
import pytest


def test_gk15_integrates_polynomials_exactly(oracle):
    # The Kronrod 15-point rule is exact to degree 3*7+1 = 22 on any interval.
    for n in range(0, 23):
        val, _ = oracle.gk15_pow(n, -0.5, 2.0)
        exact = (2.0 ** (n + 1) - (-0.5) ** (n + 1)) / (n + 1)
        assert abs(val - exact) <= 1e-13 * max(1.0, abs(exact)), n
    # ...and its embedded 7-point Gauss rule is exact to degree 13: error estimate ~ 0
    _, err = oracle.gk15_pow(13, 0.0, 1.0)
    assert err < 1e-15
    _, err = oracle.gk15_pow(20, 0.0, 1.0)
    assert err > 1e-10


def test_branch_sheet(oracle):
    rng = np.random.default_rng(1)
    k = 1.7
    for _ in range(200):
        lam = complex(rng.normal() * 4, rng.normal() * 2)
        s = oracle.sroot(lam, k)
        assert s.real >= 0.0
        assert abs(s * s - (lam * lam - k * k)) < 1e-12 * (1 + abs(lam) ** 2)
    # propagating interval: s = -i sqrt(k^2 - lam^2)  (outgoing wave e^{-s|y|})
    for lam in (0.0, 0.5, -1.2):
        assert abs(oracle.sroot(lam, k) - (-1j) * np.sqrt(k * k - lam * lam)) < 1e-14
    # evanescent: s = +sqrt(lam^2 - k^2)
    for lam in (2.0, -5.0):
        assert abs(oracle.sroot(lam, k) - np.sqrt(lam * lam - k * k)) < 1e-14
    # independent of the sign of a zero imaginary part on the real axis
    assert oracle.sroot(complex(3.0, 0.0), k) == oracle.sroot(complex(3.0, -0.0), k)
    # continuous along the contour lambda(t) = t - 0.5 i sin(pi t / c)
    c = 4.0
    t = np.linspace(0, c, 2001)
    s = np.array([oracle.sroot(complex(tt, -0.5 * np.sin(np.pi * tt / c)), k) for tt in t])
    assert np.max(np.abs(np.diff(s))) < 0.05


@pytest.mark.parametrize("lam", [1.3 + 0.2j, -0.4 + 0.7j, 2.5 - 0.3j, 0.9 - 0.05j, 4.0 + 1.0j])
def test_paper_4x4_system_vs_printed_closed_forms(oracle, lam):
    k1, k2, k3, d = 1.0, 1.5, 2.0, 0.8
    solved = oracle.sigma_paper_solve(lam, k1, k2, k3, d)
    closed = oracle.sigma_paper_closed(lam, k1, k2, k3, d)
    s2 = oracle.sroot(lam, k2)
    s3 = oracle.sroot(lam, k3)
    # sigma_1 and sigma_2^t agree as printed
    assert abs(solved[0] - closed[0]) < 1e-12 * abs(closed[0])
    assert abs(solved[1] - closed[1]) < 1e-12 * abs(closed[1])
    # sigma_2^b and sigma_3: the printed closed forms carry the normalisation
    # e^{d s2} and e^{d s3} of the closed-form exponents (reading G5)
    assert abs(solved[2] - closed[2] * np.exp(-d * s2)) < 1e-12 * abs(solved[2])
    assert abs(solved[3] - closed[3] * np.exp(-d * s3)) < 1e-12 * abs(solved[3])
    safe = oracle.sigma2t_safe(lam, k1, k2, k3, d)
    assert abs(safe - closed[1]) < 1e-12 * abs(closed[1])


def test_paper_densities_homogeneous_limit(oracle):
    # k1 = k2 = k3: no interfaces, the top-layer source transmits unchanged
    for lam in (0.3 + 0.1j, 2.0 - 0.4j, 5.0 + 0.0j):
        s = oracle.sigma_paper_closed(lam, 1.5, 1.5, 1.5, 1.0)
        assert abs(s[0]) < 1e-13 and abs(s[2]) < 1e-13
        assert abs(s[1] - 1) < 1e-13 and abs(s[3] - 1) < 1e-13
        t = oracle.sigma_layer2(lam, 1.5, 1.5, 1.5, 1.0)
        assert np.all(t == 0)


@pytest.mark.parametrize("seed", range(6))
def test_middle_layer_spectral_field_vs_interface_solve(oracle, seed):
    rng = np.random.default_rng(seed)
    k1, k2, k3 = rng.uniform(0.5, 4.0, 3)
    d = rng.uniform(0.5, 2.0)
    lam = complex(rng.uniform(-6, 6), rng.uniform(-0.6, 0.6))
    y, y0 = -d * rng.uniform(0.02, 0.98, 2)
    a = oracle.spectral_refl(lam, k1, k2, k3, d, y, y0)
    b = oracle.spectral_refl_solve(lam, k1, k2, k3, d, y, y0)
    assert abs(a - b) <= 1e-11 * abs(b)


def test_densities_tend_to_constants(oracle):
    # sigma -> constant as lambda -> inf (Sec. 3 remark after Example 4);
    # for a middle-layer source the constants are 0 with R ~ (k1^2-k2^2)/(4 lam^2)
    k1, k2, k3, d = 1.0, 1.5, 2.0, 1.0
    for lam in (1e3, 1e4):
        tt, bb, tb = oracle.sigma_layer2(lam, k1, k2, k3, d)
        assert abs(tt * 4 * lam * lam - (k1 * k1 - k2 * k2)) < 1e-5
        assert abs(bb * 4 * lam * lam - (k3 * k3 - k2 * k2)) < 1e-5
        assert abs(tb * 16 * lam ** 4 - (k1 * k1 - k2 * k2) * (k3 * k3 - k2 * k2)) < 1e-4
    a = oracle.sigma2t_safe(1e4, k1, k2, k3, d)
    b = oracle.sigma2t_safe(2e4, k1, k2, k3, d)
    assert abs(a - b) < 1e-8
