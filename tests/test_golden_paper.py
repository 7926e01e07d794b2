"""Numbers the paper prints, reproduced by the oracle (no GPU)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _read(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_three_layer_local_expansion_ratio(oracle):
    # Sec. 5, Fig. order3layer: |J_{p+1} Psi_{p+1}| / |J_p Psi_p| -> r/rho ~= 0.416
    g = _read("e4_three_layer_ratio.txt")
    med = (g["k1"], g["k2"], g["k3"], 1.0)
    r = g["r"]
    ps = [40, 80, 120, 150]
    ratios = []
    for p in ps:
        a = oracle.psi_e4(med, p, g["X"], g["Y"])
        b = oracle.psi_e4(med, p + 1, g["X"], g["Y"])
        ratios.append(abs(b * oracle.besj(p + 1, g["k2"] * r)) / abs(a * oracle.besj(p, g["k2"] * r)))
    assert np.all(np.diff(ratios) > 0)                     # approaches from below
    assert abs(ratios[-1] - g["ratio"]) < 0.01 * g["ratio"]
    # the O(1/p) approach extrapolates to the printed limit
    a1, a2 = ratios[-2], ratios[-1]
    lim = (a2 * ps[-1] - a1 * ps[-2]) / (ps[-1] - ps[-2])
    assert abs(lim - g["ratio"]) < 0.003
    assert abs(lim - r / np.hypot(g["X"], g["Y"])) < 0.003
