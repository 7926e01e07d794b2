"""Pins for the oracle's expansions and translations (no GPU): each composite
(S2M -> translation -> L2T) is compared with direct evaluation of the kernel it
compresses, which the Sommerfeld/closed-form tests pin independently."""
import numpy as np
import pytest
from scipy.special import hankel1

MED0 = (1.0, 1.5, 2.0, 1.0)


def _cluster(rng, centre, half, n):
    return (centre[0] + rng.uniform(-half, half, n), centre[1] + rng.uniform(-half, half, n))


def test_free_m2l_matches_hankel_sum(oracle):
    # S2M (Eq. multipole_coef) -> free-space M2L -> L2T (Eq. local) vs (i/4)H0 sums
    rng = np.random.default_rng(3)
    k, w, P = 1.5, 0.25, 18
    cs, ct = (0.125, -0.125), (0.125 + 2 * w, -0.125 - w)
    xs, ys = _cluster(rng, cs, w / 2, 12)
    xt, yt = _cluster(rng, ct, w / 2, 9)
    q = rng.normal(size=12) + 1j * rng.normal(size=12)
    M = oracle.s2m(xs, ys, q, cs, k, P)
    T = oracle.m2l_free_table(k, ct[0] - cs[0], ct[1] - cs[1], P)
    u = oracle.l2t(xt, yt, T @ M, ct, k, P)
    ref = np.array([np.sum(q * 0.25j * hankel1(0, k * np.hypot(a - xs, b - ys))) for a, b in zip(xt, yt)])
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


def test_m2m_and_l2l_shift_consistency(oracle):
    rng = np.random.default_rng(4)
    k, P = 2.0, 20
    parent = (0.0, -0.5)
    child = (0.125, -0.375)      # child centre; child width 0.25
    xs, ys = _cluster(rng, child, 0.125, 10)
    q = rng.normal(size=10) + 1j * rng.normal(size=10)
    # M2M (Lemma M2M with reading G3): shift = child - parent
    Mc = oracle.s2m(xs, ys, q, child, k, P)
    Mp = oracle.shift(Mc, child[0] - parent[0], child[1] - parent[1], k, P)
    Mp_direct = oracle.s2m(xs, ys, q, parent, k, P)
    inner = slice(P - 8, P + 9)
    assert np.max(np.abs(Mp[inner] - Mp_direct[inner])) <= 1e-12 * np.max(np.abs(Mp_direct))
    # the exact shifted expansion reproduces a far field: compare via M2L + L2T
    ct = (1.0, -0.5)
    T = oracle.m2l_free_table(k, ct[0] - parent[0], ct[1] - parent[1], P)
    xt, yt = _cluster(rng, ct, 0.2, 6)
    a = oracle.l2t(xt, yt, T @ Mp, ct, k, P)
    b = oracle.l2t(xt, yt, T @ Mp_direct, ct, k, P)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)
    # L2L (Lemma L2L with reading G3): shift = parent - child
    Lp = rng.normal(size=2 * P + 1) * 0.5 ** np.abs(np.arange(-P, P + 1)) + 0j
    xt, yt = _cluster(rng, child, 0.125, 8)
    Lc = oracle.shift(Lp, parent[0] - child[0], parent[1] - child[1], k, P)
    a = oracle.l2t(xt, yt, Lc, child, k, P)
    b = oracle.l2t(xt, yt, Lp, parent, k, P)
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("term", [1, 2, 3, 4])
def test_layered_m2l_matches_image_term(oracle, term):
    # S2M -> layered M2L (Lemma M2L, reading G2) -> L2T vs the direct image term G_m
    rng = np.random.default_rng(10 + term)
    k1, k2, k3, d = MED0
    P, w = 14, 0.125
    ycs = {1: -w / 2, 2: -d + w / 2, 3: -d + w / 2, 4: -w / 2}[term]
    yct = {1: -w / 2 - w, 2: -d + w / 2 + w, 3: -w / 2, 4: -d + w / 2}[term]
    cs, ct = (0.0, ycs), (2 * w, yct)
    xs, ys = _cluster(rng, cs, w / 2, 8)
    xt, yt = _cluster(rng, ct, w / 2, 6)
    q = rng.normal(size=8) + 1j * rng.normal(size=8)
    tau, vs, cm = {1: (-1, -1, 0), 2: (1, 1, 2 * d), 3: (-1, 1, 2 * d), 4: (1, -1, 2 * d)}[term]
    h = tau * ct[1] + vs * cs[1] + cm
    A = oracle.m2l_image_table(MED0, term, ct[0] - cs[0], h, P)
    u = oracle.l2t(xt, yt, A @ oracle.s2m(xs, ys, q, cs, k2, P), ct, k2, P)
    ref = np.array([sum(qj * oracle.green_term(k1, k2, k3, d, term, a, b, xj, yj)
                        for qj, xj, yj in zip(q, xs, ys)) for a, b in zip(xt, yt)])
    assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)
