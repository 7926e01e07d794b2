"""Other media (Sec. 3, Examples 2 and 3): Dirichlet, Neumann and impedance
walls in place of the interfaces, through the same FMM, against the oracle's
direct sums (FP64 path 1e-10, mixed path 1e-6) on sampled targets."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

MEDIA = {
    # name: ((k1, k2, k3, d), top, top_alpha, bottom, bottom_alpha)
    "dirichlet_half_space": ((1.0, 1.5, 1.5, 1.0), "dirichlet", 0.0, "transmission", 0.0),
    "neumann_over_dirichlet": ((1.0, 1.5, 2.0, 1.0), "neumann", 0.0, "dirichlet", 0.0),
    "impedance_walls": ((1.0, 1.5, 2.0, 1.0), "impedance", 0.7, "impedance", -0.3),
    "impedance_over_layer": ((1.0, 1.5, 2.0, 1.0), "impedance", 1.0, "transmission", 0.0),
}


@pytest.fixture(scope="module")
def lm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    import paper_1902_08250_gb300 as lm

    return lm


@pytest.fixture
def case(oracle):
    x, y, q = workloads.uniform_strip(1500, 0.0, 3.0, -0.95, -0.05, nvec=2, seed=21)
    sub = np.sort(np.random.default_rng(22).choice(x.size, 64, replace=False))
    yield x, y, q, sub
    oracle.set_boundaries()


def _widen(q, nvec, seed):
    """q with further N(0,1) vectors up to nvec (16-vector applies take the tile-form
    tensor-core M2L and the tensor-core leaf step; 1-4 vectors the 4-slot kernels)."""
    rng = np.random.default_rng(seed)
    extra = rng.standard_normal((nvec - q.shape[0], q.shape[1])) + 1j * rng.standard_normal((nvec - q.shape[0],
                                                                                              q.shape[1]))
    return np.concatenate([q, extra])


def _ref(oracle, spec, x, y, q, sub, deriv=None):
    med, tb, ta, bb, ba = spec
    oracle.set_boundaries(tb, ta, bb, ba)
    if deriv is None:
        return oracle.direct_apply(med, x, y, q, targets=sub)
    return oracle.direct_apply_deriv(med, x, y, q, deriv, targets=sub)


@pytest.mark.parametrize("name", list(MEDIA))
@pytest.mark.parametrize("prec,p,tol", [("fp64", 24, 1e-10), ("mixed", 14, 1e-6), ("mixed16", 14, 1e-6)])
def test_media_fmm_matches_oracle(lm, oracle, case, name, prec, p, tol):
    import torch

    x, y, q, sub = case
    if prec == "mixed16":
        q = _widen(q, 16, 23)
    med, tb, ta, bb, ba = MEDIA[name]
    m = lm.create_medium(*med, p=p, depth=2, precision=prec[:5], top_bc=tb, top_alpha=ta, bottom_bc=bb,
                         bottom_alpha=ba)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    u = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()[:, sub]
    ref = _ref(oracle, MEDIA[name], x, y, q, sub)
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    print(f"{name} {prec} p={p}: rel-l2 {err:.2e}")
    assert err < tol


def test_impedance_target_gradient_matches_oracle(lm, oracle, case):
    import torch

    x, y, q, sub = case
    spec = MEDIA["impedance_walls"]
    med, tb, ta, bb, ba = spec
    m = lm.create_medium(*med, p=24, depth=2, top_bc=tb, top_alpha=ta, bottom_bc=bb, bottom_alpha=ba)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    _, ux, uy = (None if a is None else a.cpu().numpy()[:, sub]
                 for a in lm.apply_grad(t, torch.from_numpy(q).cuda(), want_u=False))
    for got, deriv in ((ux, oracle.DX), (uy, oracle.DY)):
        ref = _ref(oracle, spec, x, y, q, sub, deriv)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"impedance gradient {deriv}: rel-l2 {err:.2e}")
        assert err < 1e-9


def test_invalid_boundary_rejected(lm):
    with pytest.raises(ValueError):
        lm.create_medium(1.0, 1.5, 2.0, 1.0, top_bc="absorbing")
    with pytest.raises(lm.LMError):
        lm.create_medium(1.0, 1.5, 2.0, 1.0, top_bc="impedance", top_alpha=float("nan"))


def _near_walls(n, seed):
    """Points within 0.01 of both walls and in the bulk (the image sources of a wall
    make the reflected near field log-singular as pairs approach it)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 3.0, n)
    y = np.concatenate([-0.01 * (1.0 - rng.uniform(0.0, 1.0, n // 4)),
                        -1.0 + 0.01 * (1.0 - rng.uniform(0.0, 1.0, n // 4)),
                        rng.uniform(-0.9, -0.1, n - n // 2)])
    q = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    sub = np.sort(np.concatenate([rng.choice(n // 4, 16, replace=False),
                                  n // 4 + rng.choice(n // 4, 16, replace=False)]))
    return x, y, q, sub


@pytest.mark.parametrize("name", list(MEDIA))
@pytest.mark.parametrize("prec,p,tol", [("fp64", 22, 1e-10), ("mixed", 14, 1e-6), ("mixed16", 14, 1e-6)])
def test_media_near_the_walls(lm, oracle, name, prec, p, tol):
    """Pairs within 0.02 of a wall: the quadratures integrate sigma - R_inf and each
    pair adds R_inf (i/4) H0 of its image point in closed form (uniform tree of
    automatic depth).  The 16-vector case runs the reflected tails inside the
    tensor-core leaf step."""
    import torch

    x, y, q, sub = _near_walls(3000, 41)
    if prec == "mixed16":
        q = _widen(q, 16, 42)
    med, tb, ta, bb, ba = MEDIA[name]
    m = lm.create_medium(*med, p=p, precision=prec[:5], top_bc=tb, top_alpha=ta, bottom_bc=bb, bottom_alpha=ba)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    u = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()[:, sub]
    try:
        ref = _ref(oracle, MEDIA[name], x, y, q, sub)
    finally:
        oracle.set_boundaries()
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    print(f"near walls {name} {prec} p={p}: rel-l2 {err:.2e}")
    assert err < tol


@pytest.mark.parametrize("name", ["impedance_walls", "impedance_over_layer", "neumann_over_dirichlet"])
def test_media_gradient_near_the_walls(lm, oracle, name):
    """The target gradient near the walls, with the closed-form image term's H1.
    Beside an impedance wall the y-derivative of the single reflection integrates
    (R - 1) s2 ~ 2 i beta, which does not decay beyond e^{-lambda h}; the kernels take
    2 i beta / s2 out of that integrand and add -2 i beta (i/4) H0(k2 rho) instead."""
    import torch

    x, y, q, sub = _near_walls(3000, 43)
    med, tb, ta, bb, ba = MEDIA[name]
    m = lm.create_medium(*med, p=22, top_bc=tb, top_alpha=ta, bottom_bc=bb, bottom_alpha=ba)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    _, ux, uy = lm.apply_grad(t, torch.from_numpy(q).cuda())
    try:
        for got, der in ((ux, oracle.DX), (uy, oracle.DY)):
            ref = _ref(oracle, MEDIA[name], x, y, q, sub, deriv=der)
            g = got.cpu().numpy()[:, sub]
            err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
            print(f"near walls {name} gradient {der}: rel-l2 {err:.2e}")
            assert err < 1e-9
    finally:
        oracle.set_boundaries()
