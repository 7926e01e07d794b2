"""Pins for the oracle's Sommerfeld integrals (no GPU): closed forms,
homogeneous limits, north/east agreement, reciprocity and an independent
contour integration with scipy."""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import hankel1

MED0 = (1.0, 1.5, 2.0, 1.0)      # three-layer medium of the small configuration
MED2 = (1.0, 8.0, 2.0, 1.0)      # k2 = 8: guided-mode poles on the real axis in (2, 8)


@pytest.mark.parametrize("k,X,Y", [(1.5, 0.3, 0.2), (1.5, 1.0, 0.01), (8.0, 0.05, 0.3),
                                   (2.0, 3.0, 0.0), (1.0, 0.0, 0.5), (4.0, 0.7, 0.7)])
def test_sommerfeld_identity(oracle, k, X, Y):
    # Example 1: (1/4pi) Int e^{i lam X} e^{-s|Y|}/s d lam = (i/4) H0^(1)(k r)
    exact = 0.25j * hankel1(0, k * np.hypot(X, Y))
    for tail in (oracle.NORTH, oracle.EAST):
        if (tail == oracle.EAST and X == 0) or (tail == oracle.NORTH and Y == 0):
            continue
        v = oracle.sommerfeld_free(k, X, Y, tail)
        assert abs(v - exact) <= 1e-12 * abs(exact)


def test_dirichlet_image(oracle):
    # Example 2: sigma = -1 gives the image charge at (x0, -y0)
    k = 1.3
    for (x, y, x0, y0) in [(0.2, 0.5, -0.1, 0.3), (2.0, 0.05, 0.0, 0.02), (0.0, 1.0, 0.0, 0.1)]:
        exact = -0.25j * hankel1(0, k * np.hypot(x - x0, y + y0))
        for tail in (oracle.NORTH, oracle.EAST):
            if tail == oracle.EAST and x == x0:
                continue
            v = oracle.dirichlet(k, x, y, x0, y0, tail)
            assert abs(v - exact) <= 1e-12 * abs(exact)


def test_paper_g2t_homogeneous_limit_is_free_space(oracle):
    # Example 4 with k1 = k2 = k3: sigma_2^t = 1 and g_2^t is the free-space kernel
    k = 1.7
    for (x, y, x0, y0) in [(0.3, -0.2, 0.0, 0.4), (1.5, -0.05, 0.0, 0.01)]:
        exact = 0.25j * hankel1(0, k * np.hypot(x - x0, y - y0))
        for tail in (oracle.NORTH, oracle.EAST):
            v = oracle.g2t_paper(k, k, k, 1.0, x, y, x0, y0, tail)
            assert abs(v - exact) <= 1e-12 * abs(exact)


def test_middle_layer_homogeneous_limit(oracle):
    v = oracle.green_refl(1.5, 1.5, 1.5, 1.0, 0.3, -0.2, 0.1, -0.6)
    assert v == 0


@pytest.mark.parametrize("med", [MED0, MED2])
@pytest.mark.parametrize("pair", [(0.3, -0.2, 0.1, -0.7), (0.5, -0.02, 0.0, -0.01),
                                  (0.02, -0.9, 0.0, -0.95), (1.7, -0.4, 0.0, -0.5),
                                  (0.0, -0.3, 0.0, -0.6)])
def test_north_equals_east_and_reciprocity(oracle, med, pair):
    x, y, x0, y0 = pair
    for term in range(4):
        mask = 1 << term
        auto = oracle.green_refl(*med, x, y, x0, y0, mask)
        swap = oracle.green_refl(*med, x0, y0, x, y, 1 << [0, 1, 3, 2][term])
        assert abs(auto - swap) <= 1e-12 * abs(auto)
        if x != x0:
            n = oracle.green_refl(*med, x, y, x0, y0, mask, oracle.NORTH)
            e = oracle.green_refl(*med, x, y, x0, y0, mask, oracle.EAST)
            assert abs(n - e) <= 2e-11 * abs(auto), (term, n, e)
    full = oracle.green_refl(*med, x, y, x0, y0)
    assert abs(full - oracle.green_refl(*med, x0, y0, x, y)) <= 1e-12 * abs(full)


def _scipy_contour(oracle, med, x, y, x0, y0):
    """Independent integration of the reflected field: scipy's QUADPACK along a
    polygonal contour 0 -> c/2 - 0.35i -> c (folded) plus an east tail rotated
    at 45 degrees, using the pinned spectral function."""
    k1, k2, k3, d = med
    X = abs(x - x0)
    c = 1.2 * max(med[:3]) + 2.0

    def F(lam):
        return oracle.spectral_refl(lam, k1, k2, k3, d, y, y0)

    def seg(z0, z1):
        dz = z1 - z0
        f = lambda t: 2 * np.cos((z0 + t * dz) * X) * F(z0 + t * dz) * dz
        re = quad(lambda t: f(t).real, 0, 1, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
        im = quad(lambda t: f(t).imag, 0, 1, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
        return re + 1j * im

    total = seg(0.0, c / 2 - 0.35j) + seg(c / 2 - 0.35j, c)
    # tail: rays c + t e^{+i pi/4} for e^{i lam X} and c + t e^{-i pi/4} for e^{-i lam X}
    w = np.exp(1j * np.pi / 4)

    def tail(t):
        lp, lm = c + t * w, c + t * np.conj(w)
        return np.exp(1j * lp * X) * F(lp) * w + np.exp(-1j * lm * X) * F(lm) * np.conj(w)

    re = quad(lambda t: tail(t).real, 0, np.inf, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    im = quad(lambda t: tail(t).imag, 0, np.inf, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    return (total + re + 1j * im) / (4 * np.pi)


@pytest.mark.parametrize("med,pair", [(MED0, (0.4, -0.3, 0.0, -0.5)), (MED2, (0.3, -0.2, 0.0, -0.4))])
def test_reflected_field_vs_independent_contour(oracle, med, pair):
    v = oracle.green_refl(*med, *pair)
    ref = _scipy_contour(oracle, med, *pair)
    assert abs(v - ref) <= 1e-10 * abs(ref)
