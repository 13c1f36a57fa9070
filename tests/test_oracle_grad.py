"""Pins of the oracle adjoint gradient against finite differences."""
import numpy as np

from oracle import fem, grad
from paper_1201_5991_gb300 import meshgen


def test_compliance_gradient_vs_fd_identity_and_naive_fd():
    p = meshgen.elasticity3d(4, 2, seed=5, nrhs=2)
    u = fem.direct_solve(p)
    g, lam = grad.adjoint_gradient(p, u, p.f)
    np.testing.assert_allclose(lam, u, rtol=1e-10, atol=1e-14)      # compliance: lambda = u
    Khat = fem.element_matrices(p) / p.coef[:, None, None]
    for e in [0, 17, 40, 63]:
        fd = grad.compliance_fd(p, e, 1e-6, Khat[e])
        assert abs(g[e] - fd) <= 1e-6 * abs(fd)
        nfd = grad.compliance_naive_fd(p, e, 1e-3 * p.coef[e])
        assert abs(g[e] - nfd) <= 1e-4 * abs(nfd)


def test_general_adjoint_vs_naive_fd():
    p = meshgen.elasticity3d(4, 2, seed=6)
    w = np.random.default_rng(7).standard_normal((p.n_free, 1))
    u = fem.direct_solve(p)
    g, lam = grad.adjoint_gradient(p, u, w)
    for e in [3, 30]:
        h = 1e-4 * p.coef[e]
        J = []
        for sgn in (1, -1):
            c = p.coef.copy()
            p.coef[e] += sgn * h
            J.append(float(np.sum(w * fem.direct_solve(p))))
            p.coef = c
        fd = (J[0] - J[1]) / (2 * h)
        assert abs(g[e] - fd) <= 1e-6 * max(abs(fd), 1e-300) + 1e-12
    # dJ/df = lambda: J = w^T K^{-1} f is linear in f
    k = 11
    p2 = meshgen.elasticity3d(4, 2, seed=6)
    fp = p2.f_full.copy()
    free_idx = np.nonzero(p2.free)[0]
    p2.f_full[free_idx[k]] += 1.0
    du = fem.direct_solve(p2) - u
    np.testing.assert_allclose(float(np.sum(w * du)), lam[k, 0], rtol=1e-9)
