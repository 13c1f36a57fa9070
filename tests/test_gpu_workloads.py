"""GPU checks at the full sizes of the paper-shaped workloads, through the C ABI.

Where the oracle cannot solve the whole problem in seconds, the checks use properties that
hold at any size: the FP64 residual of the assembled system (the oracle's sparse assembly, or
its matrix-free product for the cavity) against the stopping test and the library's reported
true residual; for the 16-load-case gradient, the closed form of the compliance gradient on
32 sampled elements and a cancellation-free central difference on all 32 of them over all 16
load cases.  The per-subdomain coarse matrices are compared with the oracle's in
tests/test_gpu_coarse.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, grad as ograd
from oracle import maps as om
from oracle.bddc import setup_level
from paper_1201_5991_gb300 import meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _residual_norm(p, u):
    """||K u - f|| of the assembled FP64 system (oracle assembly)."""
    Kff, f = fem.free_system(p)
    return np.linalg.norm(Kff @ u - f[:, 0])


def _check_true_residual(p, s, u, tol):
    # u_I is recovered exactly from u_G, so K u - f vanishes on interior DOFs and equals
    # g - S u_G on the interface: the oracle's FP64 residual must match the true interface
    # residual the library reports, and satisfy the stopping test ||g - S u|| <= tol ||g||.
    st = s.last_stats
    r = _residual_norm(p, u)
    assert st.converged == 1
    assert r <= tol * st.rhs_norm * 1.0001
    assert abs(r - st.rel_residual * st.rhs_norm) <= 0.02 * r + 1e-13 * st.rhs_norm


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_elasticity48_full_size(prec):
    # the bench workload (345,744 DOFs, 64 subdomains, the launch configuration bench.py times)
    p = meshgen.config("elasticity3d_48")
    s = BddcSolver(p, precision=prec)
    u = s.solve(_dev(p.f[:, 0]), tol=1e-8).cpu().numpy()
    _check_true_residual(p, s, u, 1e-8)
    assert s.last_stats.lambda_min >= 1 - 1e-6


def test_kmeans_three_levels():
    # irregular k-means partition (24^3 elements, 40 subdomains in 5 groups), three levels
    p = meshgen.elasticity3d_kmeans(24, 40, 5, seed=3, seed2=33)
    ref = fem.direct_solve(p)[:, 0]
    for prec in ("mixed", "fp64"):
        s = BddcSolver(p, precision=prec)
        u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
        assert s.last_stats.n_levels == 3
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-8


@pytest.mark.slow
def test_kmeans_96_three_levels_full_size():
    # the 96^3 k-means workload (512 subdomains, 8 level-2 subdomains): FP64 residual property
    p = meshgen.config("elasticity3d_96_kmeans")
    s = BddcSolver(p, precision="mixed")
    u = s.solve(_dev(p.f[:, 0]), tol=1e-8).cpu().numpy()
    _check_true_residual(p, s, u, 1e-8)


def _gradient_64_16_load_cases():
    # 64^3 elasticity, 512 subdomains, 16 seeded load cases; compliance J = sum_k f_k^T u_k,
    # so lambda_k = u_k and dJ/dE_e = -sum_k u_k,e^T (K_e / E_e) u_k,e: closed form on the 32
    # elements drawn by default_rng(5).choice(n_elems, 32)
    p = meshgen.elasticity3d(64, 8, seed=5, nrhs=16)
    s = BddcSolver(p, precision="mixed")
    F = _dev(p.f.T)
    U = s.solve(F, tol=1e-12)
    gc, gr = s.grad(F, U, tol=1e-12)
    u = U.cpu().numpy().T
    g = gc.cpu().numpy()
    sample = np.random.default_rng(5).choice(p.n_elems, 32, replace=False)
    Khat = fem.element_matrices(p)[sample] / p.coef[sample, None, None]
    ue = ograd.element_vectors(p, u)[sample]
    closed = -np.einsum("eak,eab,ebk->e", ue, Khat, ue)
    np.testing.assert_allclose(g[sample], closed, rtol=1e-5)
    np.testing.assert_allclose(gr.cpu().numpy(), U.cpu().numpy(), rtol=0, atol=1e-8 * np.abs(u).max())
    return p, s, F, g, sample, Khat


def test_adjoint_gradient_64_16_load_cases():
    _gradient_64_16_load_cases()


@pytest.mark.slow
def test_adjoint_gradient_64_central_differences_all_32_elements():
    # central difference (h = 1e-6 E_e) of the compliance on all 32 sampled elements over all 16
    # load cases, in cancellation-free form: (J(E+h) - J(E-h)) / 2h = -sum_k u_k,+^T K^_e u_k,-
    # with u_+/- solved at E_e +/- h (tol 1e-13); the gradient must agree within 1e-5
    p, s, F, g, sample, Khat = _gradient_64_16_load_cases()
    for q, e in enumerate(sample):
        h = 1e-6 * p.coef[e]
        sols = []
        for sgn in (+1, -1):
            c = p.coef.copy()
            c[e] += sgn * h
            s.update_coef(c)
            sols.append(s.solve(F, tol=1e-13).cpu().numpy().T)
        up = ograd.element_vectors(p, sols[0])[e]
        um = ograd.element_vectors(p, sols[1])[e]
        fd = -float(np.einsum("ak,ab,bk->", up, Khat[q], um))
        assert abs(fd - g[e]) <= 1e-5 * abs(g[e]), (int(e), fd, float(g[e]))
    s.update_coef(p.coef)


def _stokes_residual(p, u):
    """f_f - K_ff u_f - K_fd u_d over the free DOFs, by the oracle's matrix-free product."""
    full = np.array(p.dir_values, dtype=np.float64)
    full[p.free] = u
    return (p.f_full[:, 0] - fem.apply_K(p, full))[p.free]


@pytest.mark.parametrize("name", ["stokes_cavity_32", "stokes_cavity_32_3lev", "stokes_cavity_32_4lev"])
def test_stokes_cavity32_full_size(name):
    # 32^3 Taylor-Hood cavity, 512 subdomains of 4^3, 2 / 3 / 4 levels, mixed precision
    # (FGMRES outer iteration): the oracle's FP64 residual of the full system must meet the
    # stopping test and match the library's true interface residual
    p = meshgen.config(name)
    s = BddcSolver(p, precision="mixed")
    u = s.solve(_dev(p.f[:, 0]), tol=1e-8).cpu().numpy()
    st = s.last_stats
    assert st.converged == 1 and st.n_levels == p.n_levels
    r = np.linalg.norm(_stokes_residual(p, u))
    assert r <= 1e-8 * st.rhs_norm * 1.0001
    assert abs(r - st.rel_residual * st.rhs_norm) <= 0.02 * r + 1e-13 * st.rhs_norm
    # the lid drives a circulation: the velocity field is not trivial
    assert np.abs(u).max() > 0.1
