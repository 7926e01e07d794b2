"""Seeded synthetic inputs shaped like the paper's experiments.

Shared by the tests, the benchmark and the oracle-side golden scripts; it
holds no arithmetic of the method -- only random draws (numpy default_rng),
in a fixed order per workload: x, y, then the real and imaginary parts of the
densities.
"""
from __future__ import annotations

import numpy as np

# (k1, k2, k3, d): interfaces at y = 0 and y = -d
MEDIUM_A = (1.0, 1.5, 2.0, 1.0)   # the three-layer medium of the small and clustered cases
MEDIUM_B = (1.0, 8.0, 2.0, 1.0)   # k2 raised to 8 (guided-mode poles on the real axis)


def densities(rng, nvec, n, dtype=np.complex128):
    q = rng.standard_normal((nvec, n)) + 1j * rng.standard_normal((nvec, n))
    return q.astype(dtype)


def uniform_strip(n, x_lo, x_hi, y_lo, y_hi, nvec=1, seed=0):
    """n points uniform in [x_lo, x_hi) x [y_lo, y_hi) and nvec N(0,1) complex densities."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(x_lo, x_hi, n)
    y = rng.uniform(y_lo, y_hi, n)
    return x, y, densities(rng, nvec, n)


def small_uniform(n=1000, nvec=1, seed=0):
    """N = 1000 sources = targets uniform in x in [0,4], y in [-0.9,-0.1] (medium A)."""
    return uniform_strip(n, 0.0, 4.0, -0.9, -0.1, nvec, seed)


def clustered(n=100_000, nvec=1, seed=0):
    """Half the points uniform in the middle layer, half within 0.01 of y = 0 (x spread 10)."""
    rng = np.random.default_rng(seed)
    h = n // 2
    x = np.concatenate([rng.uniform(0.0, 10.0, h), rng.uniform(0.0, 10.0, n - h)])
    y = np.concatenate([rng.uniform(-0.9, -0.1, h), -0.01 * (1.0 - rng.uniform(0.0, 1.0, n - h))])
    return x, y, densities(rng, nvec, n)


def wide_uniform(n=1_000_000, nvec=16, seed=0):
    """N uniform in x in [0,20], y in [-0.95,-0.05] (medium B), nvec densities."""
    return uniform_strip(n, 0.0, 20.0, -0.95, -0.05, nvec, seed)


def batched_instances(count=48, n_lo=10_000, n_hi=500_000, nvec=4, seed=0, dtype=np.complex64):
    """Independent instances: per instance N log-uniform in [n_lo, n_hi], wave numbers
    k1, k2, k3 ~ U[0.5, 4], thickness d ~ U[0.5, 2], points x ~ U[0, 10], y ~ U[-0.9 d, -0.1 d],
    nvec N(0,1) complex densities.  Returns a list of (medium, x, y, q); drawn in order
    (N, k1, k2, k3, d, x, y, q) per instance from one generator."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        k1, k2, k3 = rng.uniform(0.5, 4.0, 3)
        d = rng.uniform(0.5, 2.0)
        x = rng.uniform(0.0, 10.0, n)
        y = rng.uniform(-0.9 * d, -0.1 * d, n)
        out.append(((float(k1), float(k2), float(k3), float(d)), x, y, densities(rng, nvec, n, dtype)))
    return out
