"""Seeded synthetic inputs: structured meshes, coefficients, boundary masks, loads, partitions.

This module is shared by the tests, the oracle-side checks and the benchmark.  It holds
none of the solver's arithmetic: no element integrals, no assembly, no interface analysis.
It only lays out the problem data that the paper's workloads are made of (Sec. 4):

* ``box_mesh``         -- structured Q1 meshes of the unit square / cube.  Node ids are
                          lexicographic with x fastest; element ids likewise; the local node
                          order inside an element is lexicographic too (a = ix + 2 iy + 4 iz).
* ``box_mesh_q2``      -- the 27-node Q2 hex mesh used by the Taylor--Hood cavity problem.
* ``simplex_mesh``     -- linear triangles / tetrahedra (Kuhn's split of the box lattice) with
                          seeded interior-node jitter: the element type of the paper's
                          geocomposite problem on an irregular, non-congruent mesh.
* ``loguniform_coef``  -- per-element Young's modulus E = 10**(3 U), U ~ U[0,1) (seeded).
* masks                -- clamped face x = 0, or the whole boundary.
* ``box_body_load``    -- nodal load of a constant body force on axis-aligned box elements
                          (each node of a box element receives vol / 2**dim of the force).
* partitions           -- cubic blocks, seeded Lloyd k-means, and block groupings for the
                          higher levels (Sec. 3, Algorithm 1: the division into subdomains
                          is an input of the solver).

All random numbers come from ``numpy.random.default_rng(seed)`` (PCG64) and are drawn on
the host once; both the CUDA path and the oracle receive the same arrays.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

POISSON = 0
ELASTICITY = 1
STOKES = 2

CORNERS = 1
EDGES = 2
FACES = 4


@dataclasses.dataclass
class Problem:
    """One synthetic workload, in the layout of the C ABI's ``bddc_mesh``/``bddc_partition``."""
    name: str
    dim: int
    nodes_per_elem: int
    dofs_per_node: int
    physics: int
    coords: np.ndarray          # [n_nodes, dim] float64
    conn: np.ndarray            # [n_elems, nodes_per_elem] int32
    coef: np.ndarray            # [n_elems] float64
    nu: float
    dirichlet: np.ndarray       # [n_nodes * dofs_per_node] uint8, 1 = prescribed
    f_full: np.ndarray          # [n_nodes * dofs_per_node, nrhs] float64 nodal loads
    parts: List[np.ndarray]     # parts[0]: elem -> level-1 sub; parts[l]: level-l sub -> level-(l+1) sub
    n_parts: List[int]
    n_levels: int
    constraints: int
    dir_values: Optional[np.ndarray] = None

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def n_elems(self) -> int:
        return self.conn.shape[0]

    @property
    def free(self) -> np.ndarray:
        return self.dirichlet == 0

    @property
    def n_free(self) -> int:
        return int(self.free.sum())

    @property
    def f(self) -> np.ndarray:
        """Loads restricted to the free DOFs (ascending global DOF order), [n_free, nrhs]."""
        return np.ascontiguousarray(self.f_full[self.free])


# ----------------------------------------------------------------------------- meshes
def box_mesh(dim: int, n: int, length: float = 1.0):
    """Structured Q1 mesh of [0, length]^dim with n elements per side."""
    h = length / n
    m = n + 1
    if dim == 2:
        iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        coords = np.stack([ix.ravel() * h, iy.ravel() * h], axis=1)
        ey, ex = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        base = (ey * m + ex).ravel()
        offs = np.array([0, 1, m, m + 1])
    elif dim == 3:
        iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
        coords = np.stack([ix.ravel() * h, iy.ravel() * h, iz.ravel() * h], axis=1)
        ez, ey, ex = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        base = ((ez * m + ey) * m + ex).ravel()
        offs = np.array([0, 1, m, m + 1, m * m, m * m + 1, m * m + m, m * m + m + 1])
    else:
        raise ValueError("dim must be 2 or 3")
    conn = (base[:, None] + offs[None, :]).astype(np.int32)
    return coords.astype(np.float64), conn


def box_mesh_q2(n: int, length: float = 1.0):
    """Structured 27-node Q2 hex mesh of [0, length]^3 with n elements per side.

    Nodes form the (2n+1)^3 lattice, lexicographic with x fastest; local node order is
    lexicographic a = ix + 3 iy + 9 iz with ix, iy, iz in {0, 1, 2}.  The Q1 pressure
    nodes of the Taylor--Hood pair are the lattice points with all-even indices.
    """
    m = 2 * n + 1
    h = length / (2 * n)
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([ix.ravel() * h, iy.ravel() * h, iz.ravel() * h], axis=1)
    ez, ey, ex = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = ((2 * ez * m + 2 * ey) * m + 2 * ex).ravel()
    offs = np.array([(kz * m + ky) * m + kx for kz in range(3) for ky in range(3) for kx in range(3)])
    conn = (base[:, None] + offs[None, :]).astype(np.int32)
    return coords.astype(np.float64), conn


# Kuhn's split of the unit cube into six tetrahedra along the diagonal from corner 0 to corner 7
# (corner a at bits (x, y, z) of a): tetrahedron pi runs 0 -> e_pi0 -> e_pi0 + e_pi1 -> 7 for a
# permutation pi of the axes.  Every cube of a lattice split the same way gives a conforming mesh
# (each square face is cut along the diagonal through its lowest corner in both cubes).
_KUHN = [(0, 1 << p0, (1 << p0) | (1 << p1), 7)
         for p0, p1 in ((0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1))]


def simplex_mesh(dim: int, n: int, jitter: float = 0.0, seed: int = 0, length: float = 1.0):
    """Linear simplices on [0, length]^dim: the n^dim box lattice with every square cut into two
    triangles along the diagonal from its corner 0 (2D) or every cube into Kuhn's six tetrahedra
    (3D); interior nodes moved by U(-jitter, jitter) h per coordinate from default_rng(seed)
    (boundary nodes stay on the boundary planes).  Every element is numbered with positive
    orientation.  jitter < 0.25 keeps every element valid (checked)."""
    coords, hexes = box_mesh(dim, n, length)
    h = length / n
    if jitter > 0.0:
        inner = np.all((coords > 0.0) & (coords < length), axis=1)
        d = np.random.default_rng(seed).uniform(-jitter, jitter, size=coords.shape) * h
        coords = coords + d * inner[:, None]
    split = _KUHN if dim == 3 else [(0, 1, 3), (0, 3, 2)]
    conn = np.concatenate([hexes[:, list(t)] for t in split], axis=0)
    order = np.argsort(np.tile(np.arange(hexes.shape[0]), len(split)), kind="stable")
    conn = conn[order]                                    # the simplices of box e are 6e.. (3D)
    E = coords[conn[:, 1:]] - coords[conn[:, :1]]
    det = np.linalg.det(E)
    flip = det < 0.0
    conn[flip, 1], conn[flip, 2] = conn[flip, 2].copy(), conn[flip, 1].copy()
    det = np.abs(det)
    if not np.all(det > 1e-3 * h ** dim):
        raise ValueError("jitter produced a degenerate simplex")
    return coords, conn.astype(np.int32)


def simplex_body_load(coords: np.ndarray, conn: np.ndarray, ndof: int, b) -> np.ndarray:
    """Nodal load of a constant body force b on linear simplices: each of the dim + 1 vertices
    receives vol / (dim + 1) of the element's force."""
    dim = coords.shape[1]
    b = np.asarray(b, dtype=np.float64).reshape(ndof)
    vol = np.abs(np.linalg.det(coords[conn[:, 1:]] - coords[conn[:, :1]])) / math.factorial(dim)
    f = np.zeros(coords.shape[0] * ndof)
    w = np.repeat(vol / (dim + 1), conn.shape[1])
    for c in range(ndof):
        np.add.at(f, conn.ravel() * ndof + c, w * b[c])
    return f


def simplex_face_pairs(conn: np.ndarray):
    """Pairs (ea, eb), ea < eb, of simplices sharing a facet (dim of their dim + 1 nodes)."""
    nn = conn.shape[1]
    facets = np.concatenate([np.sort(np.delete(conn, k, axis=1), axis=1) for k in range(nn)], axis=0)
    owner = np.tile(np.arange(conn.shape[0]), nn)
    _, inv = np.unique(facets, axis=0, return_inverse=True)
    inv = inv.ravel()
    order = np.argsort(inv, kind="stable")
    si, so = inv[order], owner[order]
    twin = np.nonzero(si[1:] == si[:-1])[0]               # interior facets appear twice
    a, b = so[twin], so[twin + 1]
    return np.minimum(a, b), np.maximum(a, b)


def loguniform_coef(n_elems: int, seed: int, decades: float = 3.0) -> np.ndarray:
    """E_e = 10**(decades * U_e), U_e ~ U[0, 1) from default_rng(seed)."""
    u = np.random.default_rng(seed).random(n_elems)
    return 10.0 ** (decades * u)


def mask_face_x0(coords: np.ndarray, ndof: int) -> np.ndarray:
    on = coords[:, 0] == 0.0
    return np.repeat(on, ndof).astype(np.uint8)


def mask_boundary(coords: np.ndarray, ndof: int, length: float = 1.0) -> np.ndarray:
    on = np.any((coords == 0.0) | (coords == length), axis=1)
    return np.repeat(on, ndof).astype(np.uint8)


def box_body_load(coords: np.ndarray, conn: np.ndarray, ndof: int, b) -> np.ndarray:
    """Nodal load of a constant body force b on axis-aligned box elements.

    The node count of a box element is 2**dim; each node receives vol/2**dim * b.
    """
    dim = coords.shape[1]
    b = np.asarray(b, dtype=np.float64).reshape(ndof)
    lo = coords[conn[:, 0]]
    hi = coords[conn[:, -1]]
    vol = np.prod(hi - lo, axis=1)
    share = vol / (2 ** dim)
    f = np.zeros(coords.shape[0] * ndof)
    nodes = conn.ravel()
    w = np.repeat(share, conn.shape[1])
    for c in range(ndof):
        np.add.at(f, nodes * ndof + c, w * b[c])
    return f


# ----------------------------------------------------------------------------- partitions
def cubic_partition(dim: int, n: int, nsub: int) -> np.ndarray:
    """Element -> subdomain for nsub^dim cubic blocks of (n/nsub)^dim elements.

    Subdomain ids are lexicographic in the block grid, x fastest.
    """
    if n % nsub:
        raise ValueError("n must be a multiple of nsub")
    s = n // nsub
    idx = np.arange(n)
    if dim == 2:
        ey, ex = np.meshgrid(idx, idx, indexing="ij")
        p = (ey // s) * nsub + ex // s
    else:
        ez, ey, ex = np.meshgrid(idx, idx, idx, indexing="ij")
        p = ((ez // s) * nsub + ey // s) * nsub + ex // s
    return p.ravel().astype(np.int32)


def block_grouping(dim: int, nsub: int, group: int) -> np.ndarray:
    """Level-l subdomain (lexicographic in an nsub^dim grid) -> level-(l+1) block of group^dim."""
    ng = nsub // group
    idx = np.arange(nsub)
    if dim == 2:
        sy, sx = np.meshgrid(idx, idx, indexing="ij")
        p = (sy // group) * ng + sx // group
    else:
        sz, sy, sx = np.meshgrid(idx, idx, idx, indexing="ij")
        p = ((sz // group) * ng + sy // group) * ng + sx // group
    return p.ravel().astype(np.int32)


def kmeans(points: np.ndarray, k: int, seed: int, iters: int = 5) -> np.ndarray:
    """Lloyd's k-means: default_rng(seed) uniform initial centres inside the points' bounding
    box, exactly ``iters`` update steps (empty clusters keep their centre), nearest centre by
    |c|^2 - 2 p.c with ties to the lower index."""
    rng = np.random.default_rng(seed)
    lo, hi = points.min(axis=0), points.max(axis=0)
    centres = lo + (hi - lo) * rng.random((k, points.shape[1]))
    lab = _nearest(points, centres)
    for _ in range(iters):
        cnt = np.bincount(lab, minlength=k)
        sums = np.stack([np.bincount(lab, weights=points[:, d], minlength=k) for d in range(points.shape[1])], axis=1)
        keep = cnt > 0
        centres[keep] = sums[keep] / cnt[keep, None]
        lab = _nearest(points, centres)
    return lab.astype(np.int32)


def _nearest(points, centres, chunk=131072):
    out = np.empty(points.shape[0], dtype=np.int64)
    cc = (centres * centres).sum(axis=1)
    for s in range(0, points.shape[0], chunk):
        p = points[s:s + chunk]
        d = cc[None, :] - 2.0 * (p @ centres.T)
        out[s:s + chunk] = np.argmin(d, axis=1)
    return out


def face_connected_fix(conn: np.ndarray, part: np.ndarray, dim: int, pairs=None) -> np.ndarray:
    """Make every subdomain face-connected: each face-connected component other than the
    largest (ties: the one holding the smallest element id) moves to the face-adjacent
    subdomain with the smallest id.  Repeats until stable; empty labels are then compacted.
    ``pairs`` = (ea, eb) lists the face-adjacent element pairs; by default the elements are
    taken as lexicographic in an n^dim box grid (as built by box_mesh)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    part = part.astype(np.int64).copy()
    nel = conn.shape[0]
    if pairs is None:
        n = int(round(nel ** (1.0 / dim)))
        idx = np.arange(nel).reshape((n,) * dim)
        ea = np.concatenate([np.take(idx, np.arange(n - 1), axis=ax).ravel() for ax in range(dim)])
        eb = np.concatenate([np.take(idx, np.arange(1, n), axis=ax).ravel() for ax in range(dim)])
    else:
        ea, eb = (np.asarray(x, dtype=np.int64) for x in pairs)
    for _ in range(100):
        same = part[ea] == part[eb]
        g = sp.coo_matrix((np.ones(int(same.sum())), (ea[same], eb[same])), shape=(nel, nel))
        ncomp, comp = connected_components(g, directed=False)
        # component sizes and first element; the kept component per part is the largest
        size = np.bincount(comp, minlength=ncomp)
        first = np.full(ncomp, nel, dtype=np.int64)
        np.minimum.at(first, comp, np.arange(nel))
        cpart = part[first]
        order = np.lexsort((first, -size, cpart))          # by part, then size desc, then first
        keep = np.zeros(ncomp, dtype=bool)
        _, start = np.unique(cpart[order], return_index=True)
        keep[order[start]] = True
        if keep.all():
            break
        # move each dropped component to its smallest face-adjacent other part
        diff = ~same
        cand = np.full(ncomp, np.iinfo(np.int64).max)
        for x, y in ((ea[diff], eb[diff]), (eb[diff], ea[diff])):
            np.minimum.at(cand, comp[x], part[y])
        move = (~keep) & (cand < np.iinfo(np.int64).max)
        if not move.any():
            break
        sel = move[comp]
        part[sel] = cand[comp[sel]]
    _, part = np.unique(part, return_inverse=True)
    return part.astype(np.int32)


# ----------------------------------------------------------------------------- configurations
def poisson2d(n: int = 32, nsub: int = 4) -> Problem:
    """-Laplace u = 1 on the unit square, Q1, homogeneous Dirichlet, nsub^2 square subdomains,
    corner constraints only, two levels."""
    coords, conn = box_mesh(2, n)
    dirichlet = mask_boundary(coords, 1)
    f = box_body_load(coords, conn, 1, [1.0])[:, None]
    return Problem(
        name=f"poisson2d_{n}_{nsub}x{nsub}", dim=2, nodes_per_elem=4, dofs_per_node=1,
        physics=POISSON, coords=coords, conn=conn, coef=np.ones(conn.shape[0]), nu=0.0,
        dirichlet=dirichlet, f_full=f, parts=[cubic_partition(2, n, nsub)], n_parts=[nsub * nsub],
        n_levels=2, constraints=CORNERS)


def elasticity3d(n: int, nsub: int, seed: int, nrhs: int = 1, group: int = 0,
                 constraints: int = CORNERS | EDGES | FACES, nu: float = 0.3) -> Problem:
    """Linear elasticity on the unit cube, Q1 hexes n^3, clamped at x = 0, gravity (0,0,-1),
    E_e log-uniform in [1, 1e3] from default_rng(seed), nsub^3 cubic subdomains.

    ``group`` > 0 adds a level grouping group^3 level-1 subdomains per level-2 subdomain.
    Load cases beyond the first add N(0,1)/sqrt(n_free) noise on the free DOFs drawn from
    default_rng(seed + k) for load case k (k = 0 is also perturbed when nrhs > 1).
    """
    coords, conn = box_mesh(3, n)
    coef = loguniform_coef(conn.shape[0], seed)
    dirichlet = mask_face_x0(coords, 3)
    g = box_body_load(coords, conn, 3, [0.0, 0.0, -1.0])
    f = np.repeat(g[:, None], nrhs, axis=1)
    if nrhs > 1:
        free = dirichlet == 0
        nf = int(free.sum())
        for k in range(nrhs):
            noise = np.random.default_rng(seed + k).standard_normal(nf) / math.sqrt(nf)
            f[free, k] += noise
    parts = [cubic_partition(3, n, nsub)]
    n_parts = [nsub ** 3]
    levels = 2
    if group:
        parts.append(block_grouping(3, nsub, group))
        n_parts.append((nsub // group) ** 3)
        levels = 3
    return Problem(
        name=f"elasticity3d_{n}_{nsub}", dim=3, nodes_per_elem=8, dofs_per_node=3,
        physics=ELASTICITY, coords=coords, conn=conn, coef=coef, nu=nu, dirichlet=dirichlet,
        f_full=f, parts=parts, n_parts=n_parts, n_levels=levels, constraints=constraints)


def elasticity3d_kmeans(n: int, nsub: int, ngroup: int, seed: int, seed2: int, kmeans_iters: int = 5) -> Problem:
    """Elasticity as ``elasticity3d`` with a seeded k-means split of element centroids into
    nsub subdomains (made face-connected), grouped by k-means of subdomain centroids into
    ngroup level-2 subdomains; three levels."""
    coords, conn = box_mesh(3, n)
    coef = loguniform_coef(conn.shape[0], seed)
    dirichlet = mask_face_x0(coords, 3)
    g = box_body_load(coords, conn, 3, [0.0, 0.0, -1.0])
    cent = coords[conn].mean(axis=1)
    p1 = kmeans(cent, nsub, seed, iters=kmeans_iters)
    p1 = face_connected_fix(conn, p1, 3)
    ns = int(p1.max()) + 1
    scent = np.stack([np.bincount(p1, weights=cent[:, d], minlength=ns) for d in range(3)], axis=1)
    scent /= np.bincount(p1, minlength=ns)[:, None]
    p2 = kmeans(scent, ngroup, seed2)
    _, p2 = np.unique(p2, return_inverse=True)
    return Problem(
        name=f"elasticity3d_kmeans_{n}_{ns}_{ngroup}", dim=3, nodes_per_elem=8, dofs_per_node=3,
        physics=ELASTICITY, coords=coords, conn=conn, coef=coef, nu=0.3, dirichlet=dirichlet,
        f_full=g[:, None], parts=[p1, p2.astype(np.int32)], n_parts=[ns, int(p2.max()) + 1],
        n_levels=3, constraints=CORNERS | EDGES | FACES)


def elasticity3d_tet(n: int, nsub: int, seed: int, jitter: float = 0.2, ngroup: int = 0,
                     nrhs: int = 1, kmeans_iters: int = 10) -> Problem:
    """Elasticity on linear tetrahedra (the element of Sec. 4's geocomposite problem): Kuhn's
    six tetrahedra per cube of the n^3 lattice, interior nodes jittered by U(-jitter, jitter) h
    (default_rng(seed)), E_e log-uniform in [1, 1e3] (default_rng(seed + 1)), clamped at x = 0,
    gravity (0, 0, -1); subdomains by seeded k-means of element centroids (made face-connected),
    optionally grouped by k-means of subdomain centroids into ngroup level-2 subdomains (three
    levels); corners + edge and face averages.  Load cases beyond the first add noise as in
    ``elasticity3d``."""
    coords, conn = simplex_mesh(3, n, jitter, seed)
    coef = loguniform_coef(conn.shape[0], seed + 1)
    dirichlet = mask_face_x0(coords, 3)
    g = simplex_body_load(coords, conn, 3, [0.0, 0.0, -1.0])
    f = np.repeat(g[:, None], nrhs, axis=1)
    if nrhs > 1:
        free = dirichlet == 0
        nf = int(free.sum())
        for k in range(nrhs):
            f[free, k] += np.random.default_rng(seed + k).standard_normal(nf) / math.sqrt(nf)
    cent = coords[conn].mean(axis=1)
    p1 = kmeans(cent, nsub, seed, iters=kmeans_iters)
    p1 = face_connected_fix(conn, p1, 3, simplex_face_pairs(conn))
    ns = int(p1.max()) + 1
    parts, n_parts = [p1], [ns]
    if ngroup:
        scent = np.stack([np.bincount(p1, weights=cent[:, d], minlength=ns) for d in range(3)], axis=1)
        scent /= np.bincount(p1, minlength=ns)[:, None]
        _, p2 = np.unique(kmeans(scent, ngroup, seed + 2), return_inverse=True)
        parts.append(p2.astype(np.int32))
        n_parts.append(int(p2.max()) + 1)
    return Problem(
        name=f"elasticity3d_tet_{n}_{ns}", dim=3, nodes_per_elem=4, dofs_per_node=3,
        physics=ELASTICITY, coords=coords, conn=conn, coef=coef, nu=0.3, dirichlet=dirichlet,
        f_full=f, parts=parts, n_parts=n_parts, n_levels=len(parts) + 1,
        constraints=CORNERS | EDGES | FACES)


def poisson2d_tri(n: int, nsub: int, seed: int, jitter: float = 0.2) -> Problem:
    """-Laplace u = 1 on the unit square with linear triangles (two per square of the n^2
    lattice, interior nodes jittered), homogeneous Dirichlet, nsub k-means subdomains (made
    edge-connected), corners only, two levels."""
    coords, conn = simplex_mesh(2, n, jitter, seed)
    cent = coords[conn].mean(axis=1)
    p1 = face_connected_fix(conn, kmeans(cent, nsub, seed, iters=10), 2, simplex_face_pairs(conn))
    ns = int(p1.max()) + 1
    return Problem(
        name=f"poisson2d_tri_{n}_{ns}", dim=2, nodes_per_elem=3, dofs_per_node=1, physics=POISSON,
        coords=coords, conn=conn, coef=np.ones(conn.shape[0]), nu=0.0,
        dirichlet=mask_boundary(coords, 1), f_full=simplex_body_load(coords, conn, 1, [1.0])[:, None],
        parts=[p1], n_parts=[ns], n_levels=2, constraints=CORNERS)


def stokes_cavity(n: int, nsub: int, groups=(), lid=(1.0 / math.sqrt(3.0), math.sqrt(2.0 / 3.0), 0.0)) -> Problem:
    """3D lid-driven cavity (Sec. 4): Taylor-Hood Q2-Q1 hexes n^3 on the unit cube, viscosity 1,
    zero velocity on every face except z = 1, where the lid velocity is prescribed on all its
    nodes (its edges included), no body force; nsub^3 cubic subdomains.

    Every lattice node has 4 DOF slots (u, v, w, p); the pressure slots of nodes that are not
    element vertices do not exist and are masked as prescribed (value 0); the pressure at node 0
    is pinned to 0 to remove the constant.  ``groups`` lists the level groupings (g -> g^3
    subdomains of the previous level per subdomain of the next).
    """
    coords, conn = box_mesh_q2(n)
    m = 2 * n + 1
    nn = coords.shape[0]
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    vertex = (ix % 2 == 0) & (iy % 2 == 0) & (iz % 2 == 0)
    bnd = (ix == 0) | (ix == m - 1) | (iy == 0) | (iy == m - 1) | (iz == 0) | (iz == m - 1)
    top = iz == m - 1
    dirichlet = np.zeros(nn * 4, dtype=np.uint8)
    values = np.zeros(nn * 4)
    for c in range(3):
        dirichlet[np.nonzero(bnd)[0] * 4 + c] = 1
        values[np.nonzero(top)[0] * 4 + c] = lid[c]
    dirichlet[np.nonzero(~vertex)[0] * 4 + 3] = 1
    dirichlet[3] = 1
    parts = [cubic_partition(3, n, nsub)]
    n_parts = [nsub ** 3]
    cur = nsub
    for g in groups:
        parts.append(block_grouping(3, cur, g))
        cur //= g
        n_parts.append(cur ** 3)
    return Problem(
        name=f"stokes_cavity_{n}_{nsub}", dim=3, nodes_per_elem=27, dofs_per_node=4, physics=STOKES,
        coords=coords, conn=conn, coef=np.ones(conn.shape[0]), nu=1.0, dirichlet=dirichlet,
        f_full=np.zeros((nn * 4, 1)), parts=parts, n_parts=n_parts, n_levels=len(parts) + 1,
        constraints=CORNERS | EDGES | FACES, dir_values=values)


def config(name: str) -> Problem:
    """The named workloads: the paper's problem classes (Sec. 4) at synthetic sizes."""
    if name == "poisson2d_32":
        return poisson2d(32, 4)
    if name == "elasticity3d_48":
        return elasticity3d(48, 4, seed=2)
    if name == "elasticity3d_24":            # same 12^3 subdomains, 2^3 of them (profiling case)
        return elasticity3d(24, 2, seed=2)
    if name == "elasticity3d_96_kmeans":
        return elasticity3d_kmeans(96, 512, 8, seed=3, seed2=33, kmeans_iters=20)
    if name == "elasticity3d_64_16rhs":
        return elasticity3d(64, 8, seed=5, nrhs=16)
    if name == "elasticity3d_tet_48":          # cfg2's node lattice as 663,552 jittered tetrahedra, 64 k-means subdomains
        return elasticity3d_tet(48, 64, seed=2)
    if name == "stokes_cavity_32":             # 512 subdomains of 4^3, two levels
        return stokes_cavity(32, 8)
    if name == "stokes_cavity_32_3lev":        # 512 / 64 / 1
        return stokes_cavity(32, 8, groups=(2,))
    if name == "stokes_cavity_32_4lev":        # 512 / 64 / 8 / 1
        return stokes_cavity(32, 8, groups=(2, 2))
    raise KeyError(name)
