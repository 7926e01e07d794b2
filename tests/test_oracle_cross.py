"""Pins of the oracle's cross-layer fields (Sec. 3, Example 4 as printed: a
source in layer 1, y0 > 0): the homogeneous limit (g_2^t + g_2^b is the free
field, g_2^b vanishes), agreement with the oracle's earlier literal g_2^t, and
the transmission conditions at y = 0 -- the layer-1 total field (free field
plus g_1^s) and the layer-2 field g_2^t + g_2^b have equal values and
y-derivatives there."""
import numpy as np
import pytest

MED = (1.0, 1.5, 2.0, 1.0)
PTS = [(0.3, -0.2, 0.0, 0.1), (1.7, -0.6, 0.2, 0.4), (0.0, -0.05, 0.0, 0.03), (4.0, -0.9, 0.5, 0.7)]


def test_homogeneous_limit_is_free_space(oracle):
    k = 1.5
    for x, y, x0, y0 in PTS:
        g = oracle.cross_field((k, k, k, 1.0), x, y, x0, y0)
        assert abs(g - oracle.green_free(k, np.hypot(x - x0, y - y0))) <= 1e-11 * abs(g)
        assert abs(oracle.cross_field((k, k, k, 1.0), x, y, x0, y0, oracle.G2B)) <= 1e-14


def test_g2t_matches_literal_form(oracle):
    for x, y, x0, y0 in PTS:
        a = oracle.cross_field(MED, x, y, x0, y0, oracle.G2T)
        tail = oracle.NORTH if y0 - y >= abs(x - x0) else oracle.EAST
        b = oracle.g2t_paper(*MED, x, y, x0, y0, tail)
        assert abs(a - b) <= 1e-10 * abs(b)


@pytest.mark.parametrize("med", [MED, (3.0, 1.0, 0.5, 0.6)])
def test_transmission_conditions_at_y0(oracle, med):
    k1 = med[0]
    for x, _, x0, y0 in PTS:
        dx = x - x0
        u1 = oracle.green_free(k1, np.hypot(dx, y0)) + oracle.cross_field(med, x, 0.0, x0, y0, oracle.G1)
        _, fy = oracle.green_free_grad(k1, dx, -y0)
        du1 = fy + oracle.cross_field(med, x, 0.0, x0, y0, oracle.G1, dy=True)
        u2 = oracle.cross_field(med, x, 0.0, x0, y0)
        du2 = oracle.cross_field(med, x, 0.0, x0, y0, dy=True)
        assert abs(u1 - u2) <= 1e-10 * abs(u1)
        assert abs(du1 - du2) <= 1e-9 * abs(du1)
