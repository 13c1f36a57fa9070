"""Pins of the oracle's finite elements against closed forms and patch tests."""
import numpy as np
import pytest

from oracle import fem
from paper_1201_5991_gb300 import meshgen


def test_q1_laplace_rectangle_closed_form():
    # Bilinear element on [0,a]x[0,b], lexicographic nodes (0,0),(a,0),(0,b),(a,b).
    # Textbook closed form: K = (b/a)/6 * Kx + (a/b)/6 * Ky with
    # Kx = [[2,-2,1,-1],[-2,2,-1,1],[1,-1,2,-2],[-1,1,-2,2]] (x-derivative part) and
    # Ky = [[2,1,-2,-1],[1,2,-1,-2],[-2,-1,2,1],[-1,-2,1,2]] (y-derivative part).
    a, b = 0.5, 2.0
    X = np.array([[0, 0], [a, 0], [0, b], [a, b]], dtype=float)
    Kx = np.array([[2, -2, 1, -1], [-2, 2, -1, 1], [1, -1, 2, -2], [-1, 1, -2, 2]], float)
    Ky = np.array([[2, 1, -2, -1], [1, 2, -1, -2], [-2, -1, 2, 1], [-1, -2, 1, 2]], float)
    ref = (b / a) / 6.0 * Kx + (a / b) / 6.0 * Ky
    np.testing.assert_allclose(fem.element_laplace(X), ref, rtol=0, atol=1e-14)
    # the unit square reduces to (1/6)[[4,-1,-1,-2],...]
    K1 = fem.element_laplace(np.array([[0, 0], [1, 0], [0, 1], [1, 1]], float))
    np.testing.assert_allclose(K1[0], np.array([4, -1, -1, -2]) / 6.0, atol=1e-15)


def _hex(a=1.0, b=1.0, c=1.0):
    return np.array([[(i & 1) * a, ((i >> 1) & 1) * b, ((i >> 2) & 1) * c] for i in range(8)], float)


def test_q1_elasticity_rigid_null_space():
    X = _hex(0.5, 1.0, 2.0)
    K = fem.element_elasticity(X, 3.0, 0.3)
    assert np.allclose(K, K.T, atol=1e-13)
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6
    assert ev.min() > -1e-12 * ev.max()
    # explicit rigid motions: translations and infinitesimal rotations omega x x
    for t in np.eye(3):
        u = np.tile(t, 8)
        assert np.linalg.norm(K @ u) < 1e-12
    for w in np.eye(3):
        u = np.cross(w, X).ravel()
        assert np.linalg.norm(K @ u) < 1e-12


@pytest.mark.parametrize("case", ["uniaxial", "shear"])
def test_q1_elasticity_constant_strain_energy(case):
    # u = G x gives a constant strain; energy = vol * 0.5 * eps:sigma exactly (trilinear
    # interpolation is exact for linear fields, 2x2x2 Gauss exact for constants).
    E, nu = 1.0, 0.3
    lam = 0.3 / (1.3 * 0.4)          # E nu / ((1+nu)(1-2nu)) with E=1, nu=0.3
    mu = 1.0 / 2.6                   # E / (2(1+nu))
    dims = (0.5, 1.0, 2.0)
    X = _hex(*dims)
    vol = np.prod(dims)
    G = np.zeros((3, 3))
    if case == "uniaxial":
        G[0, 0] = 1.0                # eps_xx = 1 -> density (lam + 2 mu)/2
        dens = 0.5 * (lam + 2 * mu)
    else:
        G[0, 1] = 1.0                # u_x = y -> gamma_xy = 1 -> density mu/2
        dens = 0.5 * mu
    u = (X @ G.T).ravel()
    K = fem.element_elasticity(X, E, nu)
    np.testing.assert_allclose(0.5 * u @ K @ u, dens * vol, rtol=1e-13)


def test_poisson_patch_bilinear_exact():
    # u = 1 + 2x + 3y + 4xy is bilinear and harmonic; with Dirichlet data u and f = 0 the
    # Q1 solution equals u at every node.
    p = meshgen.poisson2d(8, 2)
    x, y = p.coords[:, 0], p.coords[:, 1]
    uex = 1 + 2 * x + 3 * y + 4 * x * y
    p.f_full = np.zeros_like(p.f_full)
    p.dir_values = uex.copy()
    u = fem.direct_solve(p)[:, 0]
    np.testing.assert_allclose(u, uex[p.free], atol=1e-12)


def test_elasticity_patch_linear_exact():
    # Homogeneous material, f = 0, u = a + B x prescribed on the whole boundary: the
    # interior nodes reproduce the linear field exactly (patch test).
    p = meshgen.elasticity3d(4, 2, seed=0)
    p.coef = np.full(p.n_elems, 2.5)
    p.dirichlet = meshgen.mask_boundary(p.coords, 3)
    rng = np.random.default_rng(1)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    uex = (a[None, :] + p.coords @ B.T).ravel()
    p.f_full = np.zeros_like(p.f_full)
    p.dir_values = uex
    u = fem.direct_solve(p)[:, 0]
    np.testing.assert_allclose(u, uex[p.free], atol=1e-12)


def test_body_load_sums_to_total_force():
    p = meshgen.elasticity3d(6, 2, seed=0)
    tot = p.f_full[:, 0].reshape(-1, 3).sum(axis=0)
    np.testing.assert_allclose(tot, [0, 0, -1.0], atol=1e-14)   # unit cube, b = (0,0,-1)


# ---------------------------------------------------------------- Taylor-Hood Q2-Q1 (Stokes)
def _q2_hex(a=1.0, b=1.0, c=1.0):
    # 27 nodes, local a = ix + 3 iy + 9 iz at (ix a/2, iy b/2, iz c/2)
    return np.array([[ix * a / 2, iy * b / 2, iz * c / 2]
                     for iz in range(3) for iy in range(3) for ix in range(3)], float)


def _vel(X, fn):
    """Velocity slots (4a + c, c < 3) filled with fn(x) = (u, v, w); pressure slots 0."""
    u = np.zeros(108)
    for a in range(27):
        u[4 * a:4 * a + 3] = fn(X[a])
    return u


def test_q2q1_stokes_structure_and_null_spaces():
    X = _q2_hex(0.5, 1.0, 2.0)
    K = fem.element_stokes(X, 1.0)
    assert np.allclose(K, K.T, atol=1e-14)
    vert = [0, 2, 6, 8, 18, 20, 24, 26]
    pres = [4 * a + 3 for a in range(27)]
    nonvert = [4 * a + 3 for a in range(27) if a not in vert]
    assert np.all(K[nonvert] == 0.0) and np.all(K[:, nonvert] == 0.0)
    assert np.all(K[np.ix_(pres, pres)] == 0.0)           # no pressure-pressure block
    # constant velocities lie in the null space of the viscous block and are divergence free
    for t in np.eye(3):
        assert np.abs(K @ _vel(X, lambda x: t)).max() < 1e-13
    # a constant pressure only sees the boundary: B^T 1 = -int grad phi_b, whose sum over the
    # (partition-of-unity) velocity basis vanishes
    p1 = np.zeros(108)
    p1[[4 * a + 3 for a in vert]] = 1.0
    f = K @ p1
    for j in range(3):
        assert abs(f[j::4][:27].sum()) < 1e-13


def test_q2q1_stokes_closed_forms_on_a_box():
    a, b, c = 0.5, 1.0, 2.0
    X = _q2_hex(a, b, c)
    K = fem.element_stokes(X, 1.0)
    vol = a * b * c
    vert = [0, 2, 6, 8, 18, 20, 24, 26]
    # viscous energy of u = (y, 0, 0): int |grad u|^2 = vol
    u = _vel(X, lambda x: (x[1], 0.0, 0.0))
    assert abs(u @ K @ u - vol) < 1e-13
    # u = (x^2, 0, 0) is exact in Q2: int |grad u|^2 = int 4 x^2 = 4 a^3 b c / 3
    u = _vel(X, lambda x: (x[0] ** 2, 0.0, 0.0))
    assert abs(u @ K @ u - 4.0 * a ** 3 * b * c / 3.0) < 1e-13
    # divergence rows: (B u)_p = -int psi_p div u.  div (x, 0, 0) = 1: -vol / 8 at every vertex
    Bu = (K @ _vel(X, lambda x: (x[0], 0.0, 0.0)))[[4 * v + 3 for v in vert]]
    np.testing.assert_allclose(Bu, -vol / 8.0, rtol=0, atol=1e-14)
    # div (0, 0, z^2) = 2z: -int psi_p 2 z = -(a/2)(b/2) 2 int_0^c z l(z) dz with l = 1 - z/c or z/c
    Bu = (K @ _vel(X, lambda x: (0.0, 0.0, x[2] ** 2)))[[4 * v + 3 for v in vert]]
    lo = -(a / 2) * (b / 2) * 2 * (c ** 2 / 6.0)
    hi = -(a / 2) * (b / 2) * 2 * (c ** 2 / 3.0)
    np.testing.assert_allclose(Bu, [lo] * 4 + [hi] * 4, rtol=0, atol=1e-14)


def test_q2q1_stokes_inf_sup_on_two_elements():
    # the assembled pressure Schur complement B A^{-1} B^T of a small Dirichlet cavity is
    # positive definite on the pressures once one pressure is pinned (Taylor-Hood is stable)
    prob = meshgen.stokes_cavity(2, 1)
    Kff, _ = fem.free_system(prob)
    Kff = Kff.toarray()
    ndof = prob.dofs_per_node
    full = np.nonzero(prob.free)[0]
    isp = (full % ndof) == 3
    A = Kff[np.ix_(~isp, ~isp)]
    B = Kff[np.ix_(isp, ~isp)]
    assert np.linalg.eigvalsh(A).min() > 0
    ev = np.linalg.eigvalsh(B @ np.linalg.solve(A, B.T))
    assert ev.min() > 1e-6 * ev.max()


@pytest.mark.parametrize("mk", [lambda: meshgen.stokes_cavity(3, 1), lambda: meshgen.elasticity3d(4, 2, seed=3),
                                lambda: meshgen.poisson2d(8, 2)])
def test_matrix_free_apply_equals_assembled_product(mk):
    p = mk()
    u = np.random.default_rng(2).standard_normal(p.n_nodes * p.dofs_per_node)
    np.testing.assert_allclose(fem.apply_K(p, u, chunk=7), fem.assemble(p) @ u, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- linear simplices (Sec. 4's tetrahedra)
def test_p1_laplace_reference_simplices_closed_form():
    # Textbook element matrices of the reference triangle and tetrahedron: the gradients are
    # (-1,-1), (1,0), (0,1) (resp. the 3D analogues) times the area 1/2 (volume 1/6).
    K2 = fem.element_laplace_p1(np.array([[0, 0], [1, 0], [0, 1]], float))
    np.testing.assert_allclose(K2, np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]]) / 2.0, atol=1e-15)
    K3 = fem.element_laplace_p1(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float), 3.0)
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    np.testing.assert_allclose(K3, 3.0 * ref, atol=1e-15)
    # an equilateral triangle of side s has K_ab = (2 delta_ab - 1 + delta_ab) / (2 sqrt 3)
    # (cotangent formula: off-diagonal -cot(60)/2 = -1/(2 sqrt 3), diagonal 2 / (2 sqrt 3))
    s = 1.7
    T = np.array([[0, 0], [s, 0], [s / 2, s * np.sqrt(3) / 2]])
    Ke = fem.element_laplace_p1(T)
    np.testing.assert_allclose(Ke, (3 * np.eye(3) - 1) / (2 * np.sqrt(3)), atol=1e-14)
    # node order and orientation do not matter
    perm = [2, 0, 1]
    np.testing.assert_allclose(fem.element_laplace_p1(T[perm]), Ke[np.ix_(perm, perm)], atol=1e-14)


def _tet(rng):
    X = rng.standard_normal((4, 3))
    return X if np.linalg.det(X[1:] - X[0]) != 0 else _tet(rng)


def test_p1_elasticity_rigid_null_space_and_rank():
    X = _tet(np.random.default_rng(7))
    K = fem.element_elasticity_p1(X, 2.0, 0.3)
    np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6      # 12 DOFs - 6 constant strains
    assert ev.min() > -1e-10 * ev.max()
    for t in np.eye(3):
        assert np.linalg.norm(K @ np.tile(t, 4)) < 1e-10 * np.abs(K).max()
    for w in np.eye(3):
        assert np.linalg.norm(K @ np.cross(w, X).ravel()) < 1e-10 * np.abs(K).max()


def test_p1_elasticity_constant_strain_energy():
    # u = G x: strain eps = sym(G) is exact on a linear element, so
    # 0.5 u^T K u = vol * (lam/2 tr(eps)^2 + mu eps:eps)
    rng = np.random.default_rng(9)
    X = _tet(rng)
    vol = abs(np.linalg.det(X[1:] - X[0])) / 6.0
    E, nu = 3.0, 0.25
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    G = rng.standard_normal((3, 3))
    eps = 0.5 * (G + G.T)
    u = (X @ G.T).ravel()
    dens = 0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps)
    K = fem.element_elasticity_p1(X, E, nu)
    np.testing.assert_allclose(0.5 * u @ K @ u, vol * dens, rtol=1e-12)


def test_simplex_meshes_are_conforming_and_fill_the_box():
    for dim, n in ((2, 5), (3, 3)):
        coords, conn = meshgen.simplex_mesh(dim, n, jitter=0.2, seed=4)
        E = coords[conn[:, 1:]] - coords[conn[:, :1]]
        vol = np.linalg.det(E) / (2.0 if dim == 2 else 6.0)
        assert np.all(vol > 0)                                 # positively oriented
        np.testing.assert_allclose(vol.sum(), 1.0, atol=1e-13)
        ea, eb = meshgen.simplex_face_pairs(conn)
        n_bnd = (dim + 1) * conn.shape[0] - 2 * ea.size        # facets with one owner
        assert n_bnd == (2 * dim * n ** (dim - 1) * (2 if dim == 3 else 1))


@pytest.mark.parametrize("dim", [2, 3])
def test_p1_patch_tests_on_jittered_meshes(dim):
    # homogeneous material, f = 0 and a linear field prescribed on the whole boundary: a
    # linear-element solution on any valid mesh reproduces it exactly at the interior nodes
    rng = np.random.default_rng(5)
    if dim == 2:
        p = meshgen.poisson2d_tri(6, 4, seed=3)
        uex = 1.0 + p.coords @ rng.standard_normal(2)
    else:
        p = meshgen.elasticity3d_tet(3, 2, seed=3)
        p.coef = np.full(p.n_elems, 2.5)            # homogeneous: the linear field is in equilibrium
        p.dirichlet = meshgen.mask_boundary(p.coords, 3)
        uex = (rng.standard_normal(3)[None, :] + p.coords @ rng.standard_normal((3, 3)).T).ravel()
    p.f_full = np.zeros_like(p.f_full)
    p.dir_values = uex.copy()
    u = fem.direct_solve(p)[:, 0]
    np.testing.assert_allclose(u, uex[p.free], atol=1e-11)


def test_simplex_body_load_and_partition():
    p = meshgen.elasticity3d_tet(4, 6, seed=2)
    np.testing.assert_allclose(p.f_full[:, 0].reshape(-1, 3).sum(axis=0), [0, 0, -1.0], atol=1e-13)
    # every subdomain face-connected (a facet-sharing chain joins its elements rigidly)
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    ea, eb = meshgen.simplex_face_pairs(p.conn)
    part = p.parts[0]
    for s in range(p.n_parts[0]):
        els = np.nonzero(part == s)[0]
        loc = -np.ones(p.n_elems, dtype=np.int64)
        loc[els] = np.arange(els.size)
        keep = (part[ea] == s) & (part[eb] == s)
        g = sp.coo_matrix((np.ones(int(keep.sum())), (loc[ea[keep]], loc[eb[keep]])), shape=(els.size,) * 2)
        assert connected_components(g, directed=False)[0] == 1
