"""Pins of the oracle BDDC against definitions that do not share its code path."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, maps
from oracle.bddc import Bddc, bicgstab, fgmres, lanczos_extremes, pcg
from paper_1201_5991_gb300 import meshgen

SMALL = {
    "poisson": lambda: meshgen.poisson2d(16, 4),
    "elast": lambda: meshgen.elasticity3d(6, 2, seed=1),
    "elast_corners": lambda: meshgen.elasticity3d(6, 2, seed=1, constraints=meshgen.CORNERS),
    "tet": lambda: meshgen.elasticity3d_tet(5, 6, seed=1),
    "tri": lambda: meshgen.poisson2d_tri(16, 6, seed=2),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_pcg_matches_direct_solve(name):
    p = SMALL[name]()
    u_ref = fem.direct_solve(p)[:, 0]
    b = Bddc(p)
    u, info = b.solve(p.f[:, 0], tol=1e-12)
    assert info[0].converged
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-10


def _global_schur(p, iface):
    """Schur complement of the global K_ff onto the interface DOFs (global elimination)."""
    Kff, f = fem.free_system(p)
    Kff = Kff.tocsr()
    n = Kff.shape[0]
    mask = np.zeros(n, bool)
    mask[iface] = True
    I = np.nonzero(~mask)[0]
    G = iface
    KII = Kff[I][:, I].tocsc()
    lu = spla.splu(KII)
    KIG = Kff[I][:, G].toarray()
    S = Kff[G][:, G].toarray() - Kff[G][:, I] @ lu.solve(KIG)
    g = f[G, 0] - Kff[G][:, I] @ lu.solve(f[I, 0])
    return S, g


@pytest.mark.parametrize("name", ["poisson", "elast"])
def test_schur_and_condensed_rhs_vs_global_elimination(name):
    p = SMALL[name]()
    b = Bddc(p)
    iface = b.l1.maps.iface_dofs
    S_ref, g_ref = _global_schur(p, iface)
    S = np.stack([b.schur(e) for e in np.eye(iface.size)], axis=1)
    np.testing.assert_allclose(S, S_ref, atol=1e-11 * np.abs(S_ref).max())
    np.testing.assert_allclose(b.condensed_rhs(p.f[:, 0]), g_ref, atol=1e-12 * np.abs(g_ref).max())


def test_promoted_corners_solve():
    # a floating subdomain with corners only: three promoted corners make A_i nonsingular
    p = meshgen.elasticity3d(4, 1, seed=0, constraints=meshgen.CORNERS)
    cent = p.coords[p.conn].mean(axis=1)
    p.parts = [(cent[:, 0] > 0.5).astype(np.int32)]
    p.n_parts = [2]
    b = Bddc(p)
    assert b.l1.maps.n_promoted == 3
    u, info = b.solve(p.f[:, 0], tol=1e-12)
    u_ref = fem.direct_solve(p)[:, 0]
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-10


def test_one_subdomain_is_exact():
    p = meshgen.elasticity3d(4, 1, seed=3)
    b = Bddc(p)
    assert b.n_iface == 0
    u, info = b.solve(p.f[:, 0])
    assert info[0].iterations == 0
    u_ref = fem.direct_solve(p)[:, 0]
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-13


@pytest.mark.parametrize("name", ["poisson", "elast"])
def test_all_interface_corners_is_exact(name):
    # coarse space = whole interface => M^{-1} = S^{-1}, PCG converges in one step
    p = SMALL[name]()
    b = Bddc(p, constraints=meshgen.CORNERS, all_corners_levels=(1,))
    r = np.random.default_rng(0).standard_normal(b.n_iface)
    np.testing.assert_allclose(b.schur(b.precond(r)), r, rtol=0, atol=1e-10 * np.abs(r).max())
    _, info = b.solve(p.f[:, 0], tol=1e-10)
    assert info[0].iterations == 1


@pytest.mark.parametrize("name", list(SMALL))
def test_coarse_basis_identities(name):
    p = SMALL[name]()
    b = Bddc(p)
    d = b.l1
    for s in range(len(d.K)):
        C, Psi, K = d.maps.sub_C[s], d.Psi[s], d.K[s]
        np.testing.assert_allclose(C @ Psi, np.eye(C.shape[0]), atol=1e-12)
        KC = Psi.T @ K @ Psi
        np.testing.assert_allclose(d.KC[s], KC, atol=1e-10 * np.abs(KC).max())
        np.testing.assert_allclose(d.KC[s], -d.Lam[s], atol=0)


@pytest.mark.parametrize("name", list(SMALL))
def test_lambda_min_at_least_one(name):
    # BDDC theory: the eigenvalues of M^{-1} S are >= 1 (dense eigensolve on a tiny mesh)
    p = SMALL[name]()
    b = Bddc(p)
    E = np.eye(b.n_iface)
    S = np.stack([b.schur(e) for e in E], axis=1)
    M = np.stack([b.precond(e) for e in E], axis=1)
    ev = np.sort(np.linalg.eigvals(M @ S).real)
    assert ev[0] >= 1 - 1e-10
    _, info = b.solve(p.f[:, 0], tol=1e-12)
    lmin, lmax = info[0].lanczos()
    assert lmin >= 1 - 1e-8
    assert lmax <= ev[-1] * (1 + 1e-8)


def test_lanczos_of_cg_recovers_spectrum():
    # plain CG on a diagonal matrix: the Lanczos tridiagonal's extremes match the spectrum
    d = np.linspace(1.0, 50.0, 40)
    x, info = pcg(lambda v: d * v, lambda v: v, np.ones(40), 1e-14, 200)
    lmin, lmax = lanczos_extremes(info.alphas, info.betas)
    assert abs(lmin - 1.0) < 1e-8 and abs(lmax - 50.0) < 1e-8


def test_three_level_with_exact_level_two_equals_two_level():
    # static condensation reading of the interior pre-/post-correction: with every level-2
    # interface pseudo-node a corner the level-2 step is an exact solve with K_C, so the
    # three-level preconditioner equals the two-level one.
    p = meshgen.elasticity3d(8, 4, seed=4, group=2)
    b2 = Bddc(p, n_levels=2)
    b3 = Bddc(p, n_levels=3, all_corners_levels=(2,))
    r = np.random.default_rng(1).standard_normal(b2.n_iface)
    z2, z3 = b2.precond(r), b3.precond(r)
    np.testing.assert_allclose(z3, z2, atol=1e-9 * np.abs(z2).max())


def test_three_level_converges_and_kappa_grows():
    p = meshgen.elasticity3d(8, 4, seed=4, group=2)
    u_ref = fem.direct_solve(p)[:, 0]
    u2, i2 = Bddc(p, n_levels=2).solve(p.f[:, 0], tol=1e-12)
    u3, i3 = Bddc(p, n_levels=3).solve(p.f[:, 0], tol=1e-12)
    for u in (u2, u3):
        assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-9
    k2 = np.divide(*reversed(i2[0].lanczos()))
    k3 = np.divide(*reversed(i3[0].lanczos()))
    assert i3[0].lanczos()[0] >= 1 - 1e-8
    assert k3 >= k2 * 0.999         # Sec. 2 bound: each level can only worsen kappa


def test_multiplicity_weights_also_converge():
    p = SMALL["elast"]()
    u_ref = fem.direct_solve(p)[:, 0]
    u, info = Bddc(p, weights="multiplicity").solve(p.f[:, 0], tol=1e-12)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-10


def test_planted_dropped_coarse_term_is_caught():
    # a dropped term (no coarse correction: z_C = 0) must violate lambda_min(M^{-1} S) >= 1;
    # guards the eigenvalue pin above against vacuity.
    p = SMALL["elast"]()
    b = Bddc(p)
    n = b.KC.shape[0]
    b.KC_chol = (np.eye(n) * 1e30, np.arange(n))
    E = np.eye(b.n_iface)
    S = np.stack([b.schur(e) for e in E], axis=1)
    M = np.stack([b.precond(e) for e in E], axis=1)
    ev = np.sort(np.linalg.eigvals(M @ S).real)
    assert ev[0] < 0.5


# ---------------------------------------------------------------- Stokes (indefinite, Sec. 4)
def test_bicgstab_solves_a_nonsymmetric_system():
    # right-preconditioned BiCGstab against a dense LAPACK solve, with a diagonal preconditioner
    rng = np.random.default_rng(5)
    n = 60
    A = np.eye(n) * 4.0 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    d = np.diag(A).copy()
    x, info = bicgstab(lambda v: A @ v, lambda v: v / d, b, 1e-13, 200)
    assert info.converged
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-11)


def test_fgmres_with_a_changing_preconditioner():
    # a preconditioner that differs on every call (a few Jacobi sweeps with a call-dependent
    # count) is allowed in flexible GMRES; the answer must still be LAPACK's
    rng = np.random.default_rng(6)
    n = 80
    A = np.eye(n) * 3.0 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    d = np.diag(A).copy()
    calls = [0]

    def M(v):
        calls[0] += 1
        z = v / d
        for _ in range(calls[0] % 3):
            z = z + (v - A @ z) / d
        return z

    x, info = fgmres(lambda v: A @ v, M, b, 1e-12, 300, restart=10)
    assert info.converged and calls[0] > 10       # restarted at least once
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10)


def test_stokes_fgmres_matches_direct_solve():
    p = meshgen.stokes_cavity(4, 2)
    _, feff = fem.free_system(p)
    u_ref = fem.direct_solve(p)[:, 0]
    u, info = Bddc(p).solve(feff[:, 0], tol=1e-13, maxit=200, krylov="fgmres")
    assert info[0].converged
    assert np.abs(u - u_ref).max() < 1e-8 * np.abs(u_ref).max()


STOKES = {
    "two_level": lambda: meshgen.stokes_cavity(4, 2),
    "two_level_27": lambda: meshgen.stokes_cavity(6, 3),
    "three_level": lambda: meshgen.stokes_cavity(8, 4, (2,)),
}


@pytest.mark.parametrize("name", list(STOKES))
def test_stokes_bicgstab_matches_direct_solve(name):
    # the lid-driven cavity: prescribed lid velocities are lifted to the right-hand side
    p = STOKES[name]()
    _, feff = fem.free_system(p)
    u_ref = fem.direct_solve(p)[:, 0]
    u, info = Bddc(p).solve(feff[:, 0], tol=1e-13, maxit=200)
    assert info[0].converged
    assert np.abs(u - u_ref).max() < 1e-8 * np.abs(u_ref).max()
    # the discrete velocity is divergence free: the pressure rows of K_ff u = f hold
    Kff, _ = fem.free_system(p)
    full = np.nonzero(p.free)[0]
    isp = (full % p.dofs_per_node) == 3
    res = (Kff @ u - feff[:, 0])[isp]
    assert np.abs(res).max() < 1e-9 * np.abs(feff).max()


def test_stokes_weights_are_a_partition_of_unity():
    # pressure interface DOFs have a zero diagonal: their weights fall back to multiplicity
    p = STOKES["two_level_27"]()
    b = Bddc(p)
    m = b.l1.maps
    acc = np.zeros(m.iface_dofs.size)
    for s in range(len(m.sub_dofs)):
        np.add.at(acc, m.sub_iface[s], b.l1.w[s])
    np.testing.assert_allclose(acc, 1.0, rtol=0, atol=1e-14)
