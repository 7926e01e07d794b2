"""Pins of the oracle's other media (Sec. 3, Examples 2 and 3): walls with a
one-sided condition in place of either interface.  Checked against the method
of images (a Dirichlet or Neumann wall over a homogeneous half-space is one
image point) and against the boundary conditions themselves, evaluated from
the oracle's value and y-derivative kernels at the wall."""
import numpy as np
import pytest

K = 1.5
D = 1.0


@pytest.fixture(autouse=True)
def reset(oracle):
    yield
    oracle.set_boundaries()


PAIRS = [(0.7, -0.3, 0.1, -0.2), (2.5, -0.05, 0.0, -0.1), (0.0, -0.6, 0.0, -0.4), (0.2, -0.9, 1.4, -0.8)]


@pytest.mark.parametrize("kind,sign", [("dirichlet", -1.0), ("neumann", 1.0)])
def test_wall_over_half_space_is_one_image(oracle, kind, sign):
    oracle.set_boundaries(top=kind)
    for x, y, x0, y0 in PAIRS:
        g = oracle.green_refl(1.0, K, K, D, x, y, x0, y0)          # k3 = k2: nothing below
        ref = sign * oracle.green_free(K, np.hypot(x - x0, y + y0))  # image at (x0, -y0)
        assert abs(g - ref) <= 1e-12 * abs(ref)


def test_bottom_dirichlet_is_image_about_minus_d(oracle):
    oracle.set_boundaries(bottom="dirichlet")
    for x, y, x0, y0 in PAIRS:
        g = oracle.green_refl(K, K, 3.0, D, x, y, x0, y0)          # k1 = k2: nothing above
        ref = -oracle.green_free(K, np.hypot(x - x0, y + y0 + 2 * D))
        assert abs(g - ref) <= 1e-12 * abs(ref)


def _total(oracle, x, y, x0, y0, k1=1.0, k3=2.0):
    u = oracle.green_free(K, np.hypot(x - x0, y - y0)) + oracle.green_refl(k1, K, k3, D, x, y, x0, y0)
    _, gy = oracle.green_free_grad(K, x - x0, y - y0)
    uy = gy + oracle.green_refl_deriv(k1, K, k3, D, x, y, x0, y0, oracle.DY)
    return u, uy


@pytest.mark.parametrize("alpha", [0.7, -0.4, 2.0])
def test_impedance_conditions_hold_at_both_walls(oracle, alpha):
    """du/dn - i k alpha u = 0 at y = 0 (n = +y) and y = -d (n = -y) with two impedance walls."""
    ab = 0.5
    oracle.set_boundaries(top="impedance", top_alpha=alpha, bottom="impedance", bottom_alpha=ab)
    for x, _, x0, y0 in PAIRS:
        u, uy = _total(oracle, x, 0.0, x0, y0)
        assert abs(uy - 1j * K * alpha * u) <= 1e-10 * (abs(uy) + abs(u))
        u, uy = _total(oracle, x, -D, x0, y0)
        assert abs(-uy - 1j * K * ab * u) <= 1e-10 * (abs(uy) + abs(u))


def test_dirichlet_waveguide_vanishes_on_both_walls(oracle):
    oracle.set_boundaries(top="dirichlet", bottom="dirichlet")
    for x, _, x0, y0 in PAIRS:
        for yw in (0.0, -D):
            u, uy = _total(oracle, x, yw, x0, y0)
            assert abs(u) <= 1e-10 * abs(uy)


def test_impedance_limits_and_reciprocity(oracle):
    x, y, x0, y0 = PAIRS[0]
    oracle.set_boundaries(top="neumann")
    gn = oracle.green_refl(1.0, K, K, D, x, y, x0, y0)
    oracle.set_boundaries(top="impedance", top_alpha=0.0)
    assert abs(oracle.green_refl(1.0, K, K, D, x, y, x0, y0) - gn) <= 1e-13 * abs(gn)
    oracle.set_boundaries(top="impedance", top_alpha=0.7, bottom="impedance", bottom_alpha=-0.3)
    for x, y, x0, y0 in PAIRS:
        a = oracle.green_refl(1.0, K, 2.0, D, x, y, x0, y0)
        b = oracle.green_refl(1.0, K, 2.0, D, x0, y0, x, y)
        assert abs(a - b) <= 1e-12 * abs(a)
