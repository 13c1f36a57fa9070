"""Oracle adjoint gradient (not in the paper; the differentiable solve around it).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For u_k = K(theta)^{-1} f_k and a scalar objective with dJ/du_k = w_k:
  * adjoint solve K lambda_k = w_k (K symmetric);
  * dJ/df_k = lambda_k;
  * dJ/dtheta_e = - sum_k lambda_k,e^T (dK_e/dtheta_e) u_k,e.
K_e is linear in the element coefficient (Young's modulus / conductivity), so
dK_e/dtheta_e = K_e / theta_e = the unit-coefficient element matrix.  Prescribed DOFs carry
zero displacement and zero adjoint, so they drop out of the element contraction.

For the compliance J = sum_k f_k^T u_k one has lambda_k = u_k.  A central difference of J in
theta_e can be written without cancellation: with u_k,+/- solved at theta_e +/- h,
(J(+) - J(-)) / (2h) = - sum_k u_k,+^T (K_e / theta_e) u_k,-  (exact for K linear in theta_e).

Parity: pinned in ``tests/test_oracle_grad.py`` by the finite-difference identity above
and by naive central differences on a small mesh.
"""
from __future__ import annotations

import numpy as np

from . import fem


def element_vectors(prob, v_free: np.ndarray) -> np.ndarray:
    """Gather a free-DOF vector [n_free, nrhs] into element vectors [n_elems, ne, nrhs]."""
    nrhs = v_free.shape[1]
    full = np.zeros((prob.n_nodes * prob.dofs_per_node, nrhs))
    full[prob.free] = v_free
    return full[fem.element_dofs(prob)]


def adjoint_gradient(prob, u: np.ndarray, w: np.ndarray, Khat=None):
    """(dJ/dtheta [n_elems], dJ/df [n_free, nrhs]) for dJ/du = w."""
    u = u.reshape(u.shape[0], -1)
    w = w.reshape(w.shape[0], -1)
    Kff, _ = fem.free_system(prob)
    import scipy.sparse.linalg as spla
    lam = spla.splu(Kff.tocsc()).solve(w)
    if Khat is None:
        Khat = fem.element_matrices(prob) / prob.coef[:, None, None]
    ue = element_vectors(prob, u)
    le = element_vectors(prob, lam)
    g = -np.einsum("eak,eab,ebk->e", le, Khat, ue)
    return g, lam


def compliance_fd(prob, e: int, h: float, Khat_e: np.ndarray):
    """Cancellation-free central difference of J = sum_k f_k^T u_k in theta_e."""
    cp = prob.coef.copy()
    out = []
    for sgn in (+1.0, -1.0):
        prob.coef = cp.copy()
        prob.coef[e] += sgn * h
        out.append(fem.direct_solve(prob))
    prob.coef = cp
    up = element_vectors(prob, out[0])[e]
    um = element_vectors(prob, out[1])[e]
    return -float(np.einsum("ak,ab,bk->", up, Khat_e, um))


def compliance_naive_fd(prob, e: int, h: float):
    """Plain (J(theta_e + h) - J(theta_e - h)) / (2h) for comparison."""
    cp = prob.coef.copy()
    J = []
    for sgn in (+1.0, -1.0):
        prob.coef = cp.copy()
        prob.coef[e] += sgn * h
        u = fem.direct_solve(prob)
        J.append(float(np.sum(prob.f * u)))
    prob.coef = cp
    return (J[0] - J[1]) / (2 * h)
