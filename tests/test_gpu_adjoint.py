"""Gradients of J = sum_i |u_i - u_obs_i|^2 with respect to the complex
densities, u = G q through the FMM: autograd (adjoint apply) against central
finite differences and against the oracle's gradient 2 G^H (u - u_obs)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_density_gradient_matches_fd_and_oracle(oracle):
    import torch

    import paper_1902_08250_gb300 as lm

    med = workloads.MEDIUM_A
    n = 2000
    x, y, q = workloads.uniform_strip(n, 0.0, 4.0, -0.9, -0.1, nvec=1, seed=0)
    _, _, qref = workloads.uniform_strip(n, 0.0, 4.0, -0.9, -0.1, nvec=1, seed=1)
    m = lm.create_medium(*med, p=22, depth=3)
    t = lm.build_tree(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    uobs = lm.apply(t, torch.from_numpy(qref[0]).cuda())
    qd = torch.from_numpy(q[0]).cuda().requires_grad_(True)
    u = lm.green_apply(t, qd)
    J = torch.sum(torch.abs(u - uobs) ** 2)
    (g,) = torch.autograd.grad(J, qd)
    g = g.detach().cpu().numpy()
    # oracle gradient: 2 G^H r = 2 conj(G conj(r)), r = u - u_obs, on a 64-point target subset
    r = (u - uobs).detach().cpu().numpy()
    sub = np.sort(np.random.default_rng(2).choice(n, 64, replace=False))
    gref = 2 * np.conj(oracle.direct_apply(med, x, y, np.conj(r), targets=sub))
    assert np.linalg.norm(g[sub] - gref) <= 1e-9 * np.linalg.norm(gref)
    # central differences (h = 1e-6) of J in Re q_j and Im q_j for a few j
    def J_of(qv):
        uu = lm.apply(t, torch.from_numpy(qv).cuda())
        return float(torch.sum(torch.abs(uu - uobs) ** 2))

    h = 1e-6
    for j in (3, 777, 1999):
        for part, unit in ((0, 1.0), (1, 1j)):
            qp = q[0].copy()
            qm = q[0].copy()
            qp[j] += h * unit
            qm[j] -= h * unit
            fd = (J_of(qp) - J_of(qm)) / (2 * h)
            an = g[j].real if part == 0 else g[j].imag
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-3), (j, part, fd, an)
