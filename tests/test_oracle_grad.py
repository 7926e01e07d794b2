"""Pins of the oracle's derivative kernels (used by the gradient tests):
d/dx, d/dy (target) and d/dd of the reflected Green's function against
fourth-order central differences of the oracle's own value kernel; the
free-space gradient against differences of (i/4) H0; and the assembled
gradient identity (reciprocity) against differences of the whole direct sum."""
import numpy as np
import pytest

MED = (1.0, 1.5, 2.0, 1.0)
MED_B = (1.0, 8.0, 2.0, 1.0)


def fd4(f, h):
    return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)


PAIRS = [
    (0.3, -0.05, 0.0, -0.02),   # both near y = 0, X >> h: east tails
    (2.0, -0.5, 0.1, -0.3),     # interior
    (0.05, -0.95, 0.0, -0.9),   # near y = -d
    (5.0, -0.1, 0.0, -0.2),     # far in x
    (0.0, -0.4, 0.0, -0.6),     # X = 0
]


@pytest.mark.parametrize("med", [MED, MED_B])
@pytest.mark.parametrize("pair", PAIRS)
def test_refl_derivatives_vs_differences(oracle, med, pair):
    k1, k2, k3, d = med
    x, y, x0, y0 = pair
    h = 2e-4  # d/dd is steep at k2 = 8 (guided modes): h = 1e-3 leaves 1e-7 truncation
    fx = fd4(lambda e: oracle.green_refl(k1, k2, k3, d, x + e, y, x0, y0), h)
    fy = fd4(lambda e: oracle.green_refl(k1, k2, k3, d, x, y + e, x0, y0), h)
    fdd = fd4(lambda e: oracle.green_refl(k1, k2, k3, d + e, x, y, x0, y0), h)
    gx = oracle.green_refl_deriv(k1, k2, k3, d, x, y, x0, y0, oracle.DX)
    gy = oracle.green_refl_deriv(k1, k2, k3, d, x, y, x0, y0, oracle.DY)
    gd = oracle.green_refl_deriv(k1, k2, k3, d, x, y, x0, y0, oracle.DD)
    scale = abs(fy) + abs(fdd) + abs(fx)
    for a, b in ((gx, fx), (gy, fy), (gd, fdd)):
        assert abs(a - b) <= 1e-8 * scale, (a, b)
    if x == x0:
        assert gx == 0.0  # even in x - x0


def test_refl_derivatives_vanish_in_homogeneous_medium(oracle):
    for deriv in (oracle.DX, oracle.DY, oracle.DD):
        assert oracle.green_refl_deriv(1.5, 1.5, 1.5, 1.0, 0.4, -0.3, 0.0, -0.6, deriv) == 0.0


def test_free_gradient_vs_differences(oracle):
    k = 1.5
    for dx, dy in ((0.3, 0.1), (-0.02, 0.05), (1.7, -2.2)):
        gx, gy = oracle.green_free_grad(k, dx, dy)
        fx = fd4(lambda e: oracle.green_free(k, np.hypot(dx + e, dy)), 1e-4)
        fy = fd4(lambda e: oracle.green_free(k, np.hypot(dx, dy + e)), 1e-4)
        assert abs(gx - fx) <= 1e-9 * abs(fx) + 1e-12
        assert abs(gy - fy) <= 1e-9 * abs(fy) + 1e-12


def test_gradient_identity_vs_differences_of_direct_sum(oracle):
    """S(x, y, d) = sum_i conj(w_i) u_i with u = G q moving all points together:
    dS/dx_j = conj(w_j) Dx(q)_j + q_j Dx(conj w)_j (reciprocity), dS/dd = sum_i conj(w_i) Dd(q)_i."""
    rng = np.random.default_rng(5)
    n = 6
    x = rng.uniform(0.0, 1.5, n)
    y = rng.uniform(-0.9, -0.1, n)
    q = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)

    def S(xx, yy, med=MED):
        return np.vdot(w, oracle.direct_apply(med, xx, yy, q))

    V = np.stack([q, np.conj(w)])
    Dx = oracle.direct_apply_deriv(MED, x, y, V, oracle.DX)
    Dy = oracle.direct_apply_deriv(MED, x, y, V, oracle.DY)
    Dd = oracle.direct_apply_deriv(MED, x, y, q, oracle.DD)
    h = 1e-4
    for j in range(n):
        def mv(e, axis):
            xx, yy = x.copy(), y.copy()
            (xx if axis == 0 else yy)[j] += e
            return S(xx, yy)
        fx = fd4(lambda e: mv(e, 0), h)
        fy = fd4(lambda e: mv(e, 1), h)
        ax = np.conj(w[j]) * Dx[0, j] + q[j] * Dx[1, j]
        ay = np.conj(w[j]) * Dy[0, j] + q[j] * Dy[1, j]
        assert abs(ax - fx) <= 1e-7 * abs(fx), (j, ax, fx)
        assert abs(ay - fy) <= 1e-7 * abs(fy), (j, ay, fy)
    k1, k2, k3, d = MED
    fdd = fd4(lambda e: S(x, y, (k1, k2, k3, d + e)), h)
    assert abs(np.vdot(w, Dd) - fdd) <= 1e-7 * abs(fdd)
