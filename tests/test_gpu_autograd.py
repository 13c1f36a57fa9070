"""The differentiable solve (torch.autograd.Function around bddc_solve / bddc_grad) and the adjoint
gradient at a size with many load cases, against the oracle's adjoint gradient (sparse direct
solves) and against central differences in cancellation-free form.

For J = sum_k w_k^T u_k with u_k = K(E)^{-1} f_k and K linear in E_e (dK/dE_e = K_e / E_e):
    J(E_e + h) - J(E_e - h) = - sum_k lambda_k,+^T (2h K_e / E_e) u_k,-,
with lambda_+ = K(E_e + h)^{-1} w and u_- = K(E_e - h)^{-1} f: an exact identity, so the central
difference is evaluated from solves at E_e +/- h without subtracting two nearly equal J values
(Sec. 2 is silent on gradients; this is the reading the gradient checks take).  Tolerances:
gradients within 1e-5 relative, lambda within 1e-8 (solves to 1e-12)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem
from oracle import grad as og
from paper_1201_5991_gb300 import meshgen
from paper_1201_5991_gb300.solver import BddcSolver, bddc_solve

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("coef_device", ["cpu", "cuda"])
def test_autograd_function_matches_oracle_and_central_differences(coef_device):
    p = meshgen.elasticity3d(6, 2, seed=7, nrhs=2)
    s = BddcSolver(p, precision="mixed")
    F = torch.tensor(np.ascontiguousarray(p.f.T), dtype=torch.float64, device="cuda", requires_grad=True)
    coef = torch.tensor(p.coef, dtype=torch.float64, device=coef_device, requires_grad=True)
    w = torch.tensor(np.random.default_rng(8).standard_normal((2, p.n_free)), dtype=torch.float64, device="cuda")
    u = bddc_solve(F, coef, s, tol=1e-12)
    J = (w * u).sum()
    gF, gc = torch.autograd.grad(J, [F, coef])
    assert gc.device == coef.device and gF.device == F.device
    u_ref = fem.direct_solve(p)
    g_ref, lam_ref = og.adjoint_gradient(p, u_ref, w.cpu().numpy().T)
    assert _rel(u.detach().cpu().numpy().T, u_ref) < 1e-8
    assert _rel(gc.cpu().numpy(), g_ref) < 1e-5
    assert _rel(gF.cpu().numpy().T, lam_ref) < 1e-8
    # central differences through the Function's forward: every call with changed coefficients
    # re-runs the numerical set-up (bddc_update_coef) before solving
    Khat = fem.element_matrices(p) / p.coef[:, None, None]
    for e in np.random.default_rng(9).choice(p.n_elems, 4, replace=False):
        h = 1e-6 * p.coef[e]
        cp, cm = coef.detach().clone(), coef.detach().clone()
        cp[e] += h
        cm[e] -= h
        with torch.no_grad():
            lam_p = bddc_solve(w, cp, s, tol=1e-13).cpu().numpy().T     # K symmetric: adjoint = solve
            u_m = bddc_solve(F.detach(), cm, s, tol=1e-13).cpu().numpy().T
        le = og.element_vectors(p, lam_p)[e]
        ue = og.element_vectors(p, u_m)[e]
        fd = -float(np.einsum("ak,ab,bk->", le, Khat[e], ue))
        assert abs(fd - float(gc[e])) <= 1e-5 * abs(fd), (e, fd, float(gc[e]))
    # back at the original coefficients the Function re-factors and reproduces the first solve
    u2 = bddc_solve(F.detach(), coef.detach(), s, tol=1e-12)
    assert _rel(u2.cpu().numpy(), u.detach().cpu().numpy()) < 1e-10


def test_adjoint_gradient_24_16_load_cases_matches_oracle():
    # the largest size the oracle's sparse direct solve handles in seconds, with 16 load cases
    # and a general objective (lambda != u)
    p = meshgen.elasticity3d(24, 4, seed=5, nrhs=16)
    u_ref = fem.direct_solve(p)
    w = np.random.default_rng(11).standard_normal(u_ref.shape)
    g_ref, lam_ref = og.adjoint_gradient(p, u_ref, w)
    s = BddcSolver(p, precision="mixed")
    U = s.solve(torch.tensor(np.ascontiguousarray(p.f.T), dtype=torch.float64, device="cuda"), tol=1e-12)
    assert _rel(U.cpu().numpy().T, u_ref) < 1e-8
    W = torch.tensor(np.ascontiguousarray(w.T), dtype=torch.float64, device="cuda")
    gc, gr = s.grad(W, U, tol=1e-12)
    assert _rel(gc.cpu().numpy(), g_ref) < 1e-5
    assert _rel(gr.cpu().numpy().T, lam_ref) < 1e-8
