"""Gradients of J = sum_i |u_i - u_obs_i|^2, u = G(x, y, d) q through the FMM:
with respect to the complex densities (adjoint apply), the point coordinates
(target-gradient apply + reciprocity) and the layer thickness d (the dG/dd
tree).  Checked against the oracle's gradients -- built from oracle-only
residuals -- and against central differences of J (h = 1e-6)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

MED = workloads.MEDIUM_A
P, DEPTH = 22, 3


@pytest.fixture(scope="module")
def lm():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    import paper_1902_08250_gb300 as lm

    return lm


def _setup(n, seed_q=0, seed_ref=1):
    x, y, q = workloads.uniform_strip(n, 0.0, 4.0, -0.9, -0.1, nvec=1, seed=seed_q)
    _, _, qref = workloads.uniform_strip(n, 0.0, 4.0, -0.9, -0.1, nvec=1, seed=seed_ref)
    return x, y, q[0], qref[0]


def test_apply_grad_matches_oracle(lm, oracle):
    import torch

    n = 2000
    x, y, q, qref = _setup(n)
    V = np.stack([q, qref])
    m = lm.create_medium(*MED, p=P, depth=DEPTH)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    u, ux, uy = (a.cpu().numpy() for a in lm.apply_grad(t, torch.from_numpy(V).cuda()))
    u0 = lm.apply(t, torch.from_numpy(V).cuda()).cpu().numpy()
    assert np.linalg.norm(u - u0) <= 1e-13 * np.linalg.norm(u0)
    sub = np.sort(np.random.default_rng(3).choice(n, 64, replace=False))
    rx = oracle.direct_apply_deriv(MED, x, y, V, oracle.DX, targets=sub)
    ry = oracle.direct_apply_deriv(MED, x, y, V, oracle.DY, targets=sub)
    for a, r in ((ux[:, sub], rx), (uy[:, sub], ry)):
        assert np.linalg.norm(a - r) <= 1e-9 * np.linalg.norm(r), np.linalg.norm(a - r) / np.linalg.norm(r)


@pytest.mark.parametrize("prec,p,tol", [("fp64", 22, 1e-9), ("mixed", 14, 1e-6)])
def test_dG_dd_tree_matches_oracle(lm, oracle, prec, p, tol):
    import torch

    n = 2000
    x, y, q, _ = _setup(n)
    m = lm.create_medium(*MED, p=p, depth=DEPTH, precision=prec, kernel=lm.KERNEL_DG_DD)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    du = lm.apply(t, torch.from_numpy(q).cuda()).cpu().numpy()
    sub = np.sort(np.random.default_rng(4).choice(n, 64, replace=False))
    ref = oracle.direct_apply_deriv(MED, x, y, q, oracle.DD, targets=sub)
    assert np.linalg.norm(du[sub] - ref) <= tol * np.linalg.norm(ref), np.linalg.norm(du[sub] - ref) / np.linalg.norm(ref)


def _grads(lm, t, x, y, q, uobs, d):
    import torch

    qd = torch.from_numpy(q).cuda().requires_grad_(True)
    xd = t._x.clone().requires_grad_(True)
    yd = t._y.clone().requires_grad_(True)
    dd = torch.tensor(d, dtype=torch.float64, requires_grad=True)
    u = lm.green_apply(t, qd, xd, yd, dd)
    J = torch.sum(torch.abs(u - uobs) ** 2)
    gq, gx, gy, gd = torch.autograd.grad(J, (qd, xd, yd, dd))
    return gq.cpu().numpy(), gx.cpu().numpy(), gy.cpu().numpy(), float(gd)


def test_gradients_match_oracle_2k(lm, oracle):
    """Densities and coordinates at N = 2000 against the oracle: r from the
    oracle's own FMM (p = 22), gradients by oracle direct sums on 64 points."""
    import torch

    n = 2000
    x, y, q, qref = _setup(n)
    m = lm.create_medium(*MED, p=P, depth=DEPTH)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    uobs = lm.apply(t, torch.from_numpy(qref).cuda())
    gq, gx, gy, _ = _grads(lm, t, x, y, q, uobs, MED[3])
    # oracle: g = dJ/du = 2 r, r = G q - G qref (oracle FMM at the same p and depth)
    r = oracle.fmm_apply(MED, x, y, np.stack([q, qref]), DEPTH, P)
    r = r[0] - r[1]
    g = 2.0 * r
    sub = np.sort(np.random.default_rng(2).choice(n, 64, replace=False))
    gq_ref = np.conj(oracle.direct_apply(MED, x, y, np.conj(g), targets=sub))
    assert np.linalg.norm(gq[sub] - gq_ref) <= 1e-9 * np.linalg.norm(gq_ref)
    V = np.stack([q, np.conj(g)])
    Dx = oracle.direct_apply_deriv(MED, x, y, V, oracle.DX, targets=sub)
    Dy = oracle.direct_apply_deriv(MED, x, y, V, oracle.DY, targets=sub)
    gx_ref = np.real(np.conj(g[sub]) * Dx[0] + q[sub] * Dx[1])
    gy_ref = np.real(np.conj(g[sub]) * Dy[0] + q[sub] * Dy[1])
    assert np.linalg.norm(gx[sub] - gx_ref) <= 1e-9 * np.linalg.norm(gx_ref)
    assert np.linalg.norm(gy[sub] - gy_ref) <= 1e-9 * np.linalg.norm(gy_ref)


def test_thickness_gradient_matches_oracle_500(lm, oracle):
    """dJ/dd needs dG/dd q at every target: oracle direct sums at N = 500."""
    import torch

    n = 500
    x, y, q, qref = _setup(n, 7, 8)
    m = lm.create_medium(*MED, p=P, depth=2)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    uobs = lm.apply(t, torch.from_numpy(qref).cuda())
    _, _, _, gd = _grads(lm, t, x, y, q, uobs, MED[3])
    u = oracle.direct_apply(MED, x, y, np.stack([q, qref]))
    g = 2.0 * (u[0] - u[1])
    dq = oracle.direct_apply_deriv(MED, x, y, q, oracle.DD)
    gd_ref = float(np.real(np.vdot(g, dq)))
    assert abs(gd - gd_ref) <= 1e-9 * abs(gd_ref), (gd, gd_ref)


def test_gradients_match_central_differences(lm):
    """Central differences (h = 1e-6) of J at N = 2000 for x_j, y_j and d.  The
    difference J+ - J- is formed as sum Re[(u+ - u-) conj(r+ + r-)], which
    keeps the rounding of J itself out of it."""
    import torch

    n = 2000
    x, y, q, qref = _setup(n)
    m = lm.create_medium(*MED, p=P, depth=DEPTH)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    uobs = lm.apply(t, torch.from_numpy(qref).cuda())
    gq, gx, gy, gd = _grads(lm, t, x, y, q, uobs, MED[3])
    qd = torch.from_numpy(q).cuda()
    uo = uobs.cpu().numpy()

    def u_at(xx, yy, d):
        mm = lm.create_medium(MED[0], MED[1], MED[2], d, p=P, depth=DEPTH)
        tt = lm.build_tree(mm, torch.from_numpy(xx).cuda(), torch.from_numpy(yy).cuda())
        return lm.apply(tt, qd).cpu().numpy()

    def dJ(up, um, h):
        return float(np.sum(np.real((up - um) * np.conj(up + um - 2 * uo)))) / (2 * h)

    h = 1e-6
    for j in (3, 777, 1999):
        for arr, an in ((0, gx[j]), (1, gy[j])):
            xp, yp, xm, ym = x.copy(), y.copy(), x.copy(), y.copy()
            (xp if arr == 0 else yp)[j] += h
            (xm if arr == 0 else ym)[j] -= h
            fd = dJ(u_at(xp, yp, MED[3]), u_at(xm, ym, MED[3]), h)
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-2 * np.max(np.abs(gx))), (j, arr, fd, an)
    fd = dJ(u_at(x, y, MED[3] + h), u_at(x, y, MED[3] - h), h)
    assert abs(fd - gd) <= 1e-5 * abs(gd), (fd, gd)
    # densities: J is quadratic in q, so the difference is exact up to rounding
    for j in (5, 1500):
        e = np.zeros(n, complex)
        e[j] = h
        up = lm.apply(t, torch.from_numpy(q + e).cuda()).cpu().numpy()
        um = lm.apply(t, torch.from_numpy(q - e).cuda()).cpu().numpy()
        assert abs(dJ(up, um, h) - gq[j].real) <= 1e-5 * (abs(gq[j].real) + 1e-3)


def test_gradients_at_200k_match_central_differences(lm):
    """The gradient workload at full size (N = 200k): autograd coordinate and
    thickness gradients against central differences (h = 1e-6) of J.  Both use
    the IEEE FP64 M2L: central differences divide the apply's rounding by 2h,
    and the double-float M2L's (2e-13, from rounding at 2^-48 rather than 2^-53)
    changes with the moved point and would dominate the difference."""
    import torch

    n = 200_000
    x, y, q = workloads.uniform_strip(n, 0.0, 40.0, -0.9, -0.1, nvec=1, seed=0)
    _, _, qref = workloads.uniform_strip(n, 0.0, 40.0, -0.9, -0.1, nvec=1, seed=1)
    q, qref = q[0], qref[0]
    p = 20
    m = lm.create_medium(*MED, p=p, m2l_fp64=True)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    uobs = lm.apply(t, torch.from_numpy(qref).cuda())
    _, gx, gy, gd = _grads(lm, t, x, y, q, uobs, MED[3])
    qd = torch.from_numpy(q).cuda()
    uo = uobs.cpu().numpy()

    def u_at(xx, yy, d):
        mm = lm.create_medium(MED[0], MED[1], MED[2], d, p=p, depth=t.info["depth"], m2l_fp64=True)
        tt = lm.build_tree(mm, torch.from_numpy(xx).cuda(), torch.from_numpy(yy).cuda())
        return lm.apply(tt, qd).cpu().numpy()

    def dJ(up, um, h):
        return float(np.sum(np.real((up - um) * np.conj(up + um - 2 * uo)))) / (2 * h)

    h = 1e-6
    for j in (11, 123_456):
        for arr, an in ((0, gx[j]), (1, gy[j])):
            xp, yp, xm, ym = x.copy(), y.copy(), x.copy(), y.copy()
            (xp if arr == 0 else yp)[j] += h
            (xm if arr == 0 else ym)[j] -= h
            fd = dJ(u_at(xp, yp, MED[3]), u_at(xm, ym, MED[3]), h)
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-2 * np.max(np.abs(gx))), (j, arr, fd, an)
    fd = dJ(u_at(x, y, MED[3] + h), u_at(x, y, MED[3] - h), h)
    assert abs(fd - gd) <= 1e-5 * abs(gd), (fd, gd)


def test_misfit_grad_entry_point(lm):
    """lm_misfit_grad through the C ABI: the same gradients as the autograd path (which calls
    it), a NULL output skips that gradient, and bad arguments are rejected before any work."""
    import ctypes

    import torch

    x, y, q = workloads.uniform_strip(3000, 0.0, 3.0, -0.9, -0.1, nvec=2, seed=31)
    _, _, gg = workloads.uniform_strip(3000, 0.0, 3.0, -0.9, -0.1, nvec=2, seed=32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    t = lm.build_tree(lm.create_medium(*workloads.MEDIUM_A, p=20), xd, yd)
    dt = t.d_tree()
    qd, gd_in = torch.from_numpy(q).cuda(), torch.from_numpy(gg).cuda()
    b = ctypes.c_size_t()
    assert lm._lib.lm_misfit_grad_workspace(t._h, 2, ctypes.byref(b)) == 0
    ws = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    gq = torch.empty_like(qd)
    gx = torch.empty(t.n, dtype=torch.float64, device="cuda")
    gy = torch.empty_like(gx)
    gdd = torch.empty((), dtype=torch.float64, device="cuda")
    P = lambda a: None if a is None else ctypes.c_void_p(a.data_ptr())  # noqa: E731
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lm._lib.lm_misfit_grad(t._h, dt._h, P(qd), P(gd_in), 2, P(gq), P(gx), P(gy), P(gdd), P(ws), b.value,
                                  st) == 0, lm._lib.lm_last_error()
    # the same quantities from the separate applies, combined here in float64 as the check
    ref_q = lm.apply_adjoint(t, gd_in)
    _, ux, uy = lm.apply_grad(t, torch.cat([qd, torch.conj(gd_in)]).contiguous(), want_u=False)
    ref_x = torch.real(torch.conj(gd_in) * ux[:2] + qd * ux[2:]).sum(0)
    ref_y = torch.real(torch.conj(gd_in) * uy[:2] + qd * uy[2:]).sum(0)
    ref_d = torch.real(torch.sum(torch.conj(gd_in) * lm.apply(dt, qd)))
    assert torch.equal(gq, ref_q)
    for got, ref in ((gx, ref_x), (gy, ref_y)):
        assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) < 1e-13
    assert abs(float(gdd) - float(ref_d)) <= 1e-12 * abs(float(ref_d))
    # outputs left NULL are not computed; the d-gradient alone needs no coordinate work
    gd2 = torch.empty((), dtype=torch.float64, device="cuda")
    assert lm._lib.lm_misfit_grad(t._h, dt._h, P(qd), P(gd_in), 2, None, None, None, P(gd2), P(ws), b.value,
                                  st) == 0
    assert float(gd2) == float(gdd)
    # a short workspace, a missing dG/dd tree and a mixed tree's coordinate gradient are rejected
    assert lm._lib.lm_misfit_grad(t._h, dt._h, P(qd), P(gd_in), 2, None, P(gx), None, None, P(ws), b.value - 8,
                                  st) == 1
    assert lm._lib.lm_misfit_grad(t._h, None, P(qd), P(gd_in), 2, None, None, None, P(gdd), P(ws), b.value,
                                  st) == 1
    tm = lm.build_tree(lm.create_medium(*workloads.MEDIUM_A, p=12, precision="mixed"), xd, yd)
    assert lm._lib.lm_misfit_grad(tm._h, None, P(qd), P(gd_in), 2, None, P(gx), None, None, P(ws), b.value,
                                  st) == 5
