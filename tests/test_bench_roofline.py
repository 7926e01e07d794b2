"""The bench's roofline arithmetic (host logic): the ALU peak derived from unit
counts and clocks, and the leaf phase's algorithmic work over its time, with a
stand-in library and tree (no GPU)."""
import os
import sys
import types

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_alu_peak_from_unit_counts_and_clocks():
    import bench

    peak, src = bench.alu_peak("mixed", 152, 2070.0)
    assert peak == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)   # 80.5 TFLOP/s
    assert "152 SMs" in src and "2070 MHz" in src
    assert bench.alu_peak("mixed", 152, None)[0] == pytest.approx(peak)   # no sample: the maximum
    assert bench.alu_peak("mixed", 152, 1035.0)[0] == pytest.approx(peak / 2)
    assert bench.alu_peak("fp64", 152, 2070.0)[0] == pytest.approx(1.25)


def test_leaf_phase_roofline(monkeypatch):
    import bench

    # two leaves of 3 and 2 points; U list: (0,0), (0,1), (1,0), (1,1), term 0, and a
    # reflected (tt) entry (0,0)
    ls = np.array([0, 3, 5])
    U = np.array([[0, 0, 0], [0, 0, 1], [1, 0, 0], [1, 0, 1], [0, 1, 0]])
    med = types.SimpleNamespace(options={"precision": 1, "tail_order": 0})
    tree = types.SimpleNamespace(info={"depth": 1}, n=5, export=lambda: (np.arange(5), ls),
                                 list_export=lambda which, level=0: U, medium=med)
    monkeypatch.setattr(bench, "_probe", lambda lm, kind, dev: 76.0)
    monkeypatch.setattr(bench, "recorded_traffic", lambda phase: None)
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        get_device_properties=lambda dev: types.SimpleNamespace(multi_processor_count=152)))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    r = bench.roofline(None, tree, "l2t_s2t", 1.0, 29, "mixed", "cuda:0", None, 2070.0)
    free = (3 + 2) ** 2 - 5                        # free pairs of the U list, self pairs out
    refl = 3 * 3                                   # the tt entry of leaf 0 with itself
    # per unit: H0 (60 flop) + 16 complex MACs per free pair; 24 tail nodes x 35 flop + 16 MACs per
    # reflected pair; 29 orders x (20 flop recurrence + 16 MACs) per target
    flops = free * (60 + 128) + refl * (24 * 35 + 128) + 5 * 29 * (20 + 128)
    mac = 128.0 * (free + refl) + 128.0 * 29 * 5
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / 1e-3 / 1e12)
    assert r["achieved_mac_only"] == pytest.approx(mac / 1e-3 / 1e12)
    assert r["peak"] == pytest.approx(80.5, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["peak_probe"] == 76.0
