"""Finite elements for the oracle: element matrices, global assembly, direct solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's starting point is the assembled system K u = f of a finite-element
discretisation; the local subdomain matrix K_i is obtained "by sub-assembling element
matrices" (Sec. 2, Eq. psi_def context).  Element types (Sec. 4): linear elasticity and, as
the scalar model problem of the first workload, the Laplace operator.

Element conventions
  * Linear simplices (triangles, tetrahedra; Sec. 4's geocomposite mesh is made of linear
    tetrahedra): constant gradients from the inverse of the vertex matrix, exact one-term
    integration.
  * Q1 element on 2**dim nodes, local node a has reference position xi_a[d] = 2*bit_d(a) - 1
    (lexicographic order, x fastest); 2-point Gauss rule per direction.
  * Elasticity DOF order inside an element is (node a, component c) -> 3a + c; strains use
    Voigt order [xx, yy, zz, yz, xz, xy] with engineering shears; isotropic D with
    lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)).

Parity: pinned (closed-form 2D Laplace element, closed-form reference-tetrahedron Laplace
element, rigid-body null spaces, constant-strain energies, Poisson and elasticity patch tests on
boxes and on jittered tetrahedral meshes) in ``tests/test_oracle_fem.py``.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

GAUSS2 = np.array([-1.0, 1.0]) / np.sqrt(3.0)


def q1_ref_nodes(dim: int) -> np.ndarray:
    """Reference positions of the 2**dim lexicographically numbered Q1 nodes."""
    return np.array([[2.0 * ((a >> d) & 1) - 1.0 for d in range(dim)] for a in range(2 ** dim)])


def q1_grad_ref(dim: int, xi: np.ndarray) -> np.ndarray:
    """dN_a/dxi_d at reference point xi, shape [2**dim, dim]; N_a = prod_d (1 + xi_a,d xi_d)/2."""
    nodes = q1_ref_nodes(dim)
    g = np.empty((2 ** dim, dim))
    for a in range(2 ** dim):
        for d in range(dim):
            v = nodes[a, d] / 2.0
            for e in range(dim):
                if e != d:
                    v *= (1.0 + nodes[a, e] * xi[e]) / 2.0
            g[a, d] = v
    return g


def gauss_points(dim: int):
    for pt in itertools.product(GAUSS2, repeat=dim):
        yield np.array(pt), 1.0


def element_laplace(X: np.ndarray, coef: float = 1.0) -> np.ndarray:
    """K_e[a, b] = coef * int grad N_a . grad N_b over a Q1 element with node coordinates X."""
    dim = X.shape[1]
    K = np.zeros((2 ** dim, 2 ** dim))
    for xi, w in gauss_points(dim):
        G = q1_grad_ref(dim, xi)          # [nn, dim] in reference coords
        J = X.T @ G                       # dx/dxi, [dim, dim]
        detJ = np.linalg.det(J)
        Gx = G @ np.linalg.inv(J)         # physical gradients [nn, dim]
        K += coef * w * detJ * (Gx @ Gx.T)
    return K


def elasticity_D(E: float, nu: float) -> np.ndarray:
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[[0, 1, 2], [0, 1, 2]] += 2.0 * mu
    D[[3, 4, 5], [3, 4, 5]] = mu
    return D


def elasticity_B(Gx: np.ndarray) -> np.ndarray:
    """Strain-displacement matrix, Voigt [xx, yy, zz, yz, xz, xy], DOF order 3a + c."""
    nn = Gx.shape[0]
    B = np.zeros((6, 3 * nn))
    for a in range(nn):
        dx, dy, dz = Gx[a]
        B[0, 3 * a + 0] = dx
        B[1, 3 * a + 1] = dy
        B[2, 3 * a + 2] = dz
        B[3, 3 * a + 1] = dz
        B[3, 3 * a + 2] = dy
        B[4, 3 * a + 0] = dz
        B[4, 3 * a + 2] = dx
        B[5, 3 * a + 0] = dy
        B[5, 3 * a + 1] = dx
    return B


def element_elasticity(X: np.ndarray, E: float, nu: float) -> np.ndarray:
    """K_e = int B^T D B dV over a trilinear hex, 2x2x2 Gauss."""
    D = elasticity_D(E, nu)
    K = np.zeros((24, 24))
    for xi, w in gauss_points(3):
        G = q1_grad_ref(3, xi)
        J = X.T @ G
        detJ = np.linalg.det(J)
        Gx = G @ np.linalg.inv(J)
        B = elasticity_B(Gx)
        K += w * detJ * (B.T @ D @ B)
    return K


def p1_gradients(X: np.ndarray):
    """Linear simplex (triangle / tetrahedron) with vertices X [dim+1, dim]: the shape functions
    N_a(x) = c_a + g_a . x are fixed by N_a(x_b) = delta_ab, i.e. the coefficient columns are the
    inverse of the vertex matrix M = [1 x_b^T] (rows b).  Returns (g [dim+1, dim], volume), the
    volume being |det M| / dim!."""
    dim = X.shape[1]
    M = np.hstack([np.ones((dim + 1, 1)), X])
    Cinv = np.linalg.inv(M)               # column a holds (c_a, g_a)
    vol = abs(np.linalg.det(M)) / float(np.prod(np.arange(1, dim + 1)))
    return Cinv[1:, :].T.copy(), vol


def element_laplace_p1(X: np.ndarray, coef: float = 1.0) -> np.ndarray:
    """K_e[a, b] = coef * vol * g_a . g_b on a linear simplex (the gradients are constant)."""
    g, vol = p1_gradients(X)
    return coef * vol * (g @ g.T)


def element_elasticity_p1(X: np.ndarray, E: float, nu: float) -> np.ndarray:
    """K_e = vol B^T D B on a linear tetrahedron (constant strain), DOF order 3a + c."""
    g, vol = p1_gradients(X)
    B = elasticity_B(g)
    return vol * (B.T @ elasticity_D(E, nu) @ B)


GAUSS3 = (np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)]), np.array([5.0, 8.0, 5.0]) / 9.0)


def q2_1d(x: float):
    """Quadratic Lagrange functions on nodes -1, 0, 1 and their derivatives."""
    return (np.array([0.5 * x * (x - 1.0), 1.0 - x * x, 0.5 * x * (x + 1.0)]),
            np.array([x - 0.5, -2.0 * x, x + 0.5]))


def element_stokes(X: np.ndarray, nu: float = 1.0) -> np.ndarray:
    """Taylor-Hood Q2-Q1 hex, DOF slots (node a of 27, component c of 4) -> 4a + c.

    Velocity (c = 0, 1, 2) on all 27 nodes, pressure (c = 3) on the 8 vertex nodes; the
    pressure slots of the other 19 nodes carry zero rows and columns.  Blocks:
    A[(a,i),(b,j)] = nu delta_ij int grad phi_a . grad phi_b  (vector Laplacian form),
    B[(p,3),(b,j)] = -int psi_p d phi_b / dx_j  and its transpose; 3x3x3 Gauss rule,
    isoparametric Q2 geometry.  Local node a = ix + 3 iy + 9 iz.
    """
    K = np.zeros((108, 108))
    vert = [ix + 3 * iy + 9 * iz for iz in (0, 2) for iy in (0, 2) for ix in (0, 2)]
    pts, wts = GAUSS3
    for gz, wz in zip(pts, wts):
        for gy, wy in zip(pts, wts):
            for gx, wx in zip(pts, wts):
                fx, dx = q2_1d(gx)
                fy, dy = q2_1d(gy)
                fz, dz = q2_1d(gz)
                G = np.zeros((27, 3))
                for a in range(27):
                    ix, iy, iz = a % 3, (a // 3) % 3, a // 9
                    G[a] = [dx[ix] * fy[iy] * fz[iz], fx[ix] * dy[iy] * fz[iz], fx[ix] * fy[iy] * dz[iz]]
                J = X.T @ G
                detJ = np.linalg.det(J)
                Gx = G @ np.linalg.inv(J)
                w = wx * wy * wz * detJ
                Lap = nu * w * (Gx @ Gx.T)
                for i in range(3):
                    K[i:108:4, i:108:4][:27, :27] += Lap
                xi = np.array([gx, gy, gz])
                for k, a in enumerate(vert):
                    c = np.array([-1.0 if (k >> d) & 1 == 0 else 1.0 for d in range(3)])
                    psi = np.prod((1.0 + c * xi) / 2.0)
                    for b in range(27):
                        for j in range(3):
                            v = -w * psi * Gx[b, j]
                            K[4 * a + 3, 4 * b + j] += v
                            K[4 * b + j, 4 * a + 3] += v
    return K


def unit_element(prob, X: np.ndarray) -> np.ndarray:
    """Element matrix with unit coefficient for the Problem's element type: Q1 boxes (2**dim
    nodes), linear simplices (dim + 1 nodes) or the Q2-Q1 hexahedron (Stokes)."""
    simplex = prob.nodes_per_elem == prob.dim + 1
    if prob.physics == 0:
        return element_laplace_p1(X, 1.0) if simplex else element_laplace(X, 1.0)
    if prob.physics == 1:
        return element_elasticity_p1(X, 1.0, prob.nu) if simplex else element_elasticity(X, 1.0, prob.nu)
    if prob.physics == 2:
        return element_stokes(X, 1.0)
    raise NotImplementedError("physics")


def element_matrices(prob) -> np.ndarray:
    """All element matrices of a Problem, [n_elems, ne, ne], each scaled by its coefficient.

    Structured box meshes have congruent elements, so elements with identical geometry
    reuse one unit-coefficient matrix (scaled by coef_e); this is exact, not an approximation.
    """
    X = prob.coords[prob.conn]                        # [nel, nn, dim]
    shape_key = np.round(X - X[:, :1, :], 14).reshape(X.shape[0], -1)
    uniq, inv = np.unique(shape_key, axis=0, return_inverse=True)
    inv = inv.ravel()
    unit = np.stack([unit_element(prob, X[int(np.nonzero(inv == u)[0][0])]) for u in range(uniq.shape[0])])
    return unit[inv] * prob.coef[:, None, None]


def apply_K(prob, u_full: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """K u over all DOFs without forming K: sum_e P_e^T (coef_e K_e^unit) P_e u, elements with
    identical geometry sharing one unit matrix (as in element_matrices).  For meshes too large
    for the assembled matrix; u_full is [n_nodes * ndof] or [n_nodes * ndof, k]."""
    X = prob.coords[prob.conn]
    shape_key = np.round(X - X[:, :1, :], 14).reshape(X.shape[0], -1)
    uniq, inv = np.unique(shape_key, axis=0, return_inverse=True)
    inv = inv.ravel()
    ed = element_dofs(prob)
    U = u_full if u_full.ndim == 2 else u_full[:, None]
    out = np.zeros_like(U)
    for u in range(uniq.shape[0]):
        els = np.nonzero(inv == u)[0]
        K1 = unit_element(prob, X[int(els[0])])
        for c0 in range(0, els.size, chunk):
            ec = els[c0:c0 + chunk]
            ue = U[ed[ec]]                                   # [ne_chunk, ne, k]
            ye = np.einsum("ab,ebk->eak", K1, ue) * prob.coef[ec][:, None, None]
            for k in range(U.shape[1]):
                out[:, k] += np.bincount(ed[ec].ravel(), weights=ye[:, :, k].ravel(), minlength=U.shape[0])
    return out if u_full.ndim == 2 else out[:, 0]


def element_dofs(prob) -> np.ndarray:
    """Global DOF ids (node * ndof + comp) of every element, [n_elems, nn * ndof]."""
    nd = prob.dofs_per_node
    return (prob.conn[:, :, None].astype(np.int64) * nd + np.arange(nd)[None, None, :]).reshape(
        prob.n_elems, -1)


def assemble(prob, Ke=None):
    """Global stiffness over all DOFs (CSR).  K = sum_e P_e^T K_e P_e."""
    if Ke is None:
        Ke = element_matrices(prob)
    ed = element_dofs(prob)
    n = prob.n_nodes * prob.dofs_per_node
    rows = np.repeat(ed, ed.shape[1], axis=1).ravel()
    cols = np.tile(ed, (1, ed.shape[1])).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    K.sum_duplicates()
    return K


def free_system(prob, K=None):
    """K_ff, f_f with Dirichlet DOFs eliminated (zero or prescribed values lifted to the RHS)."""
    if K is None:
        K = assemble(prob)
    free = prob.free
    Kff = K[free][:, free].tocsc()
    f = prob.f_full[free].copy()
    if prob.dir_values is not None:
        ud = prob.dir_values[~free]
        f -= (K[free][:, ~free] @ ud)[:, None]
    return Kff, f


def direct_solve(prob, K=None):
    """u = K_ff^{-1} f over the free DOFs (SuperLU), [n_free, nrhs]."""
    Kff, f = free_system(prob, K)
    lu = spla.splu(Kff)
    return lu.solve(f)
