"""The oracle FMM (Algorithm 1) against the oracle direct sum (no GPU): the
error falls geometrically with the expansion order, as Theorem 1 predicts."""
import numpy as np

MED0 = (1.0, 1.5, 2.0, 1.0)


def test_fmm_converges_to_direct_sum(oracle):
    rng = np.random.default_rng(0)
    n = 90
    x = rng.uniform(0, 2, n)
    y = rng.uniform(-0.9, -0.1, n)
    q = rng.normal(size=n) + 1j * rng.normal(size=n)
    ref = oracle.direct_apply(MED0, x, y, q)
    errs = []
    for P in (4, 8, 12):
        u = oracle.fmm_apply(MED0, x, y, q, 2, P)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[0] > 5 * errs[1] > 25 * errs[2]
    assert errs[2] < 1e-7


def test_fmm_two_vectors_and_linearity(oracle):
    rng = np.random.default_rng(1)
    n = 40
    x = rng.uniform(0, 1.5, n)
    y = rng.uniform(-0.9, -0.1, n)
    q = rng.normal(size=(2, n)) + 1j * rng.normal(size=(2, n))
    u = oracle.fmm_apply(MED0, x, y, q, 1, 6)
    u0 = oracle.fmm_apply(MED0, x, y, q[0], 1, 6)
    u1 = oracle.fmm_apply(MED0, x, y, q[0] + 2 * q[1], 1, 6)
    assert np.allclose(u[0], u0, rtol=1e-14, atol=0)
    assert np.allclose(u1, u[0] + 2 * u[1], rtol=1e-12, atol=1e-14)
