"""Oracle index analysis of one BDDC level (Sec. 2-3, Algorithm 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1 asks, per level, to divide the (pseudo-)mesh into subdomains, classify the
interface into faces, edges and vertices, select corners, and -- for levels above the
first -- build a pseudo-mesh whose "elements" are the subdomains and whose "nodes" are the
corners, edges and faces.  The constraint matrices C_i hold one row per constraint: corner
values and arithmetic averages over edges and faces (Sec. 2 after Eq. psi_def; Sec. 4).
The coarse restriction R_Ci maps global coarse DOFs to the local ones (Sec. 2).

The paper gives no rule for the classification or for the cited face-based corner
selection; this oracle takes the following readings (the CUDA library takes the same):

  * interface node: a node contained in >= 2 subdomains.
  * glob: a maximal set of interface nodes with identical sharing sets, split into
    components connected through shared (pseudo-)elements; globs are ordered by their
    smallest node id.
  * type: sharing set of size 2 -> face (3D) / edge (2D); size >= 3 -> vertex when the glob
    is a single node, edge otherwise.
  * corners are the vertex globs.  Per subdomain with interface nodes a rigid-body
    sufficiency test counts as
    points the centroids of globs constrained in every component and the nodes whose DOFs
    are all prescribed; scalar problems need one point, 2D elasticity two distinct points,
    3D elasticity three non-collinear points.  A failing subdomain (ascending order)
    promotes one of its interface nodes with all DOFs free to an extra corner: the smallest
    id when it has no point, else the node farthest from the first point (one point) or
    from the line through the first point and the point farthest from it; ties go to the
    smaller id.  Promoted corners are appended after the regular globs.
  * constraint rows: for every constrained glob and component with a free DOF on the glob,
    one coarse DOF; its row averages (weight 1/count) that component over the glob's free
    DOFs.  Coarse DOFs are numbered by (glob order, component).
  * local DOF order of a subdomain: interior DOFs ascending by global id, then interface
    DOFs ascending; for Stokes the pressure DOFs follow the velocity DOFs inside each of the
    two groups.  The global interface numbers the interface DOFs ascending.
  * rigid-body test for Stokes: the floating modes are the constant velocities, so one point
    constrained in the three velocity components suffices.
  * multiplicity weight of an interface DOF: 1 / |sharing set of its node|.
  * pseudo-mesh of the next level: one pseudo-node per glob carrying coarse DOFs (in glob
    order) with coordinates at the centroid of the glob's nodes that carry a free DOF; one
    pseudo-element per subdomain whose DOFs are its coarse DOFs in ascending order.

Parity: pinned by hand-counted structured sizes (interface and coarse counts) and by the
partition-of-unity identity sum_i R_i^T D_i R_i = I in ``tests/test_oracle_maps.py``.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Tuple

import numpy as np

VERTEX, EDGE, FACE = 0, 1, 2
CORNERS, EDGES, FACES = 1, 2, 4


@dataclasses.dataclass
class LevelMesh:
    """A (pseudo-)mesh: nodes with component DOFs, elements as node lists, a partition."""
    dim: int
    ncomp: int
    coords: np.ndarray                 # [n_nodes, dim]
    node_dofs: List[np.ndarray]        # per node: array of (comp, dof) pairs, dof = -1 prescribed
    elem_nodes: List[np.ndarray]       # per element: node ids (ascending not required)
    elem_dofs: List[np.ndarray]        # per element: its matrix's DOF ids (-1 = prescribed)
    part: np.ndarray                   # [n_elems] -> subdomain
    n_sub: int
    n_dof: int                         # number of free DOFs of this level
    rigid_comps: Tuple[int, ...] = ()  # components carrying the floating (rigid) modes
    rigid_points: int = 1              # constrained points needed: 1, 2 (2D elast.) or 3 (3D elast.)
    last_comp: int = -1                # component ordered after the others in local orders (-1: none)


@dataclasses.dataclass
class Glob:
    nodes: np.ndarray
    subs: Tuple[int, ...]
    kind: int
    promoted: bool = False


@dataclasses.dataclass
class LevelMaps:
    mesh: LevelMesh
    node_subs: List[Tuple[int, ...]]
    globs: List[Glob]
    coarse_glob: np.ndarray            # [n_coarse] glob index of every coarse DOF
    coarse_comp: np.ndarray            # [n_coarse] component of every coarse DOF
    iface_dofs: np.ndarray             # global interface: free DOF ids ascending
    sub_elems: List[np.ndarray]
    sub_dofs: List[np.ndarray]         # local order: interior then interface (global DOF ids)
    sub_nI: List[int]
    sub_iface: List[np.ndarray]        # positions of the local interface DOFs in iface_dofs
    sub_coarse: List[np.ndarray]       # R_Ci: global coarse ids, ascending
    sub_C: List[np.ndarray]            # dense C_i [n_c, n_local]
    sub_wmult: List[np.ndarray]        # multiplicity weights of the local interface DOFs
    n_promoted: int

    @property
    def n_coarse(self) -> int:
        return int(self.coarse_glob.shape[0])


def mesh_level1(prob) -> LevelMesh:
    """Level-1 mesh from a Problem: DOF node*ndof+comp, free DOFs numbered ascending."""
    nd = prob.dofs_per_node
    free = prob.dirichlet == 0
    dof_id = np.full(prob.n_nodes * nd, -1, dtype=np.int64)
    dof_id[free] = np.arange(int(free.sum()))
    node_dofs = [np.array([(c, dof_id[p * nd + c]) for c in range(nd)], dtype=np.int64)
                 for p in range(prob.n_nodes)]
    elem_nodes = [np.asarray(r, dtype=np.int64) for r in prob.conn]
    elem_dofs = [dof_id[(r[:, None].astype(np.int64) * nd + np.arange(nd)).ravel()] for r in prob.conn]
    if prob.physics == 2:          # Stokes: constant velocities float; pressures ordered last
        rc, rp, last = (0, 1, 2), 1, 3
    elif prob.physics == 1:
        rc, rp, last = tuple(range(nd)), (3 if prob.dim == 3 else 2), -1
    else:
        rc, rp, last = (0,), 1, -1
    return LevelMesh(prob.dim, nd, prob.coords, node_dofs, elem_nodes, elem_dofs,
                     np.asarray(prob.parts[0]), int(prob.n_parts[0]), int(free.sum()), rc, rp, last)


def _seqmean(X: np.ndarray) -> np.ndarray:
    """Mean of the rows of X summed one after another in row order."""
    return np.cumsum(X, axis=0)[-1] / X.shape[0]


def _find(parent, x):
    while parent[x] != x:
        parent[x] = parent[parent[x]]
        x = parent[x]
    return x


def analyze(mesh: LevelMesh, constraints: int, all_corners: bool = False) -> LevelMaps:
    """Interface classification, corner selection and coarse numbering of one level.

    ``all_corners`` makes every interface node a glob of its own (a corner); the coarse
    space then spans the whole interface, the special case in which BDDC is exact.
    """
    n_nodes = mesh.coords.shape[0]
    nsub = mesh.n_sub
    sub_elems = [[] for _ in range(nsub)]
    for e, s in enumerate(mesh.part):
        sub_elems[int(s)].append(e)
    sub_elems = [np.array(v, dtype=np.int64) for v in sub_elems]

    # sharing sets
    subsets = [set() for _ in range(n_nodes)]
    for e, s in enumerate(mesh.part):
        for p in mesh.elem_nodes[e]:
            subsets[int(p)].add(int(s))
    node_subs = [tuple(sorted(x)) for x in subsets]
    iface = np.array([len(x) >= 2 for x in node_subs])

    # globs: equal sharing sets, connected through elements
    parent = np.arange(n_nodes)
    for e in range(len(mesh.elem_nodes)):
        by_set: Dict[Tuple[int, ...], int] = {}
        for p in mesh.elem_nodes[e]:
            p = int(p)
            if not iface[p]:
                continue
            q = by_set.setdefault(node_subs[p], p)
            if q != p:
                a, b = _find(parent, p), _find(parent, q)
                if a != b:
                    parent[max(a, b)] = min(a, b)
    comp: Dict[int, List[int]] = {}
    for p in np.nonzero(iface)[0]:
        comp.setdefault(int(p) if all_corners else _find(parent, int(p)), []).append(int(p))
    globs = []
    for root in sorted(comp, key=lambda r: min(comp[r])):
        nodes = np.array(sorted(comp[root]), dtype=np.int64)
        subs = node_subs[int(nodes[0])]
        if all_corners:
            kind = VERTEX
        elif len(subs) == 2:
            kind = FACE if mesh.dim == 3 else EDGE
        else:
            kind = VERTEX if nodes.size == 1 else EDGE
        globs.append(Glob(nodes, subs, kind))

    def glob_is_constrained(g: Glob) -> bool:
        if g.promoted:
            return True
        return bool(constraints & {VERTEX: CORNERS, EDGE: EDGES, FACE: FACES}[g.kind])

    def glob_free_comps(g: Glob):
        comps = []
        for c in range(mesh.ncomp):
            if any(int(d) >= 0 for p in g.nodes for cc, d in mesh.node_dofs[int(p)] if cc == c):
                comps.append(c)
        return comps

    def glob_centroid(g: Glob):
        pts = [p for p in g.nodes if any(int(d) >= 0 for _, d in mesh.node_dofs[int(p)])]
        if not pts:
            pts = list(g.nodes)
        return _seqmean(mesh.coords[np.array(pts)])

    # corner selection with the rigid-body sufficiency test
    sub_nodes = []
    for s in range(nsub):
        ns = set()
        for e in sub_elems[s]:
            ns.update(int(p) for p in mesh.elem_nodes[e])
        sub_nodes.append(np.array(sorted(ns), dtype=np.int64))
    n_promoted = 0
    corner_nodes = set()
    for g in globs:
        if g.kind == VERTEX and glob_is_constrained(g):
            corner_nodes.add(int(g.nodes[0]))
    diam = np.linalg.norm(mesh.coords.max(axis=0) - mesh.coords.min(axis=0))
    tol = 1e-12 * diam * diam

    rigid = set(mesh.rigid_comps)

    def node_rigid_state(p):
        """(all rigid-mode DOFs prescribed, all rigid-mode DOFs present and free)"""
        nd = [(int(c), int(d)) for c, d in mesh.node_dofs[int(p)] if int(c) in rigid]
        present = {c for c, _ in nd}
        return (len(nd) > 0 and all(d < 0 for _, d in nd),
                present == rigid and all(d >= 0 for _, d in nd))

    def points_of(s):
        pts = []
        for g in globs:
            if s in g.subs and glob_is_constrained(g):
                if rigid.issubset(glob_free_comps(g)):
                    pts.append(glob_centroid(g))
        for p in sub_nodes[s]:
            if node_rigid_state(p)[0]:
                pts.append(mesh.coords[int(p)])
        return np.array(pts).reshape(-1, mesh.dim)

    def sufficient(pts):
        if mesh.rigid_points == 1:
            return pts.shape[0] >= 1
        if pts.shape[0] == 0:
            return False
        d0 = np.linalg.norm(pts - pts[0], axis=1)
        j = int(np.argmax(d0))
        if mesh.rigid_points == 2:
            return d0[j] * d0[j] > tol
        if d0[j] * d0[j] <= tol:
            return False
        u = pts[j] - pts[0]
        cr = np.linalg.norm(np.cross(pts - pts[0], u), axis=1)
        return cr.max() > tol

    for s in range(nsub):
        if not any(iface[p] for p in sub_nodes[s]):
            continue          # a subdomain without interface is the whole (connected) problem
        for _ in range(16):
            pts = points_of(s)
            if sufficient(pts):
                break
            cand = [int(p) for p in sub_nodes[s] if iface[p] and int(p) not in corner_nodes
                    and node_rigid_state(p)[1]]
            if not cand:
                raise ValueError(f"subdomain {s}: no candidate corner")
            cand = np.array(cand, dtype=np.int64)
            X = mesh.coords[cand]
            if pts.shape[0] == 0:
                pick = int(cand[0])
            else:
                d0 = np.linalg.norm(pts - pts[0], axis=1)
                j = int(np.argmax(d0))
                if d0[j] * d0[j] <= tol or mesh.rigid_points <= 2:
                    dist = np.linalg.norm(X - pts[0], axis=1)
                else:
                    u = (pts[j] - pts[0]) / d0[j]
                    dist = np.linalg.norm(np.cross(X - pts[0], u), axis=1)
                pick = int(cand[int(np.argmax(dist))])   # argmax returns the first maximum
            globs.append(Glob(np.array([pick], dtype=np.int64), node_subs[pick], VERTEX, True))
            corner_nodes.add(pick)
            n_promoted += 1
        else:
            raise ValueError(f"subdomain {s}: corner selection did not terminate")

    # coarse DOFs
    cg, cc = [], []
    for gi, g in enumerate(globs):
        if glob_is_constrained(g):
            for c in glob_free_comps(g):
                cg.append(gi)
                cc.append(c)
    coarse_glob = np.array(cg, dtype=np.int64)
    coarse_comp = np.array(cc, dtype=np.int64)

    # global interface numbering
    iface_dofs = sorted(int(d) for p in np.nonzero(iface)[0] for _, d in mesh.node_dofs[int(p)] if d >= 0)
    iface_dofs = np.array(iface_dofs, dtype=np.int64)
    iface_pos = {d: k for k, d in enumerate(iface_dofs)}

    sub_dofs, sub_nI, sub_iface, sub_coarse, sub_C, sub_w = [], [], [], [], [], []
    for s in range(nsub):
        interior, inter = [], []
        for p in sub_nodes[s]:
            for c, d in mesh.node_dofs[int(p)]:
                if d >= 0:
                    key = (1 if int(c) == mesh.last_comp else 0, int(d))
                    (inter if iface[p] else interior).append(key)
        interior = [d for _, d in sorted(interior)]
        inter = [d for _, d in sorted(inter)]
        dofs = np.array(interior + inter, dtype=np.int64)
        loc = {d: k for k, d in enumerate(dofs)}
        sub_dofs.append(dofs)
        sub_nI.append(len(interior))
        sub_iface.append(np.array([iface_pos[d] for d in inter], dtype=np.int64))
        mult = {}
        for p in sub_nodes[s]:
            if iface[p]:
                for _, d in mesh.node_dofs[int(p)]:
                    if d >= 0:
                        mult[int(d)] = 1.0 / len(node_subs[int(p)])
        sub_w.append(np.array([mult[d] for d in inter]))
        rows = [k for k in range(coarse_glob.shape[0]) if s in globs[coarse_glob[k]].subs]
        sub_coarse.append(np.array(rows, dtype=np.int64))
        C = np.zeros((len(rows), dofs.size))
        for r, k in enumerate(rows):
            g = globs[coarse_glob[k]]
            c = coarse_comp[k]
            ds = [int(d) for p in g.nodes for cc2, d in mesh.node_dofs[int(p)] if cc2 == c and d >= 0]
            for d in ds:
                C[r, loc[d]] = 1.0 / len(ds)
        sub_C.append(C)

    return LevelMaps(mesh, node_subs, globs, coarse_glob, coarse_comp, iface_dofs, sub_elems,
                     sub_dofs, sub_nI, sub_iface, sub_coarse, sub_C, sub_w, n_promoted)


def next_level_mesh(maps: LevelMaps, part_next: np.ndarray, n_sub_next: int) -> LevelMesh:
    """Pseudo-mesh of level l+1 (Algorithm 1): subdomains -> 'elements', globs -> 'nodes'."""
    mesh = maps.mesh
    carrying = sorted(set(int(g) for g in maps.coarse_glob))
    node_of_glob = {g: q for q, g in enumerate(carrying)}
    coords = []
    node_dofs = []
    for g in carrying:
        glob = maps.globs[g]
        pts = [p for p in glob.nodes if any(int(d) >= 0 for _, d in mesh.node_dofs[int(p)])]
        coords.append(_seqmean(mesh.coords[np.array(pts)]))
        ks = np.nonzero(maps.coarse_glob == g)[0]
        node_dofs.append(np.array([(int(maps.coarse_comp[k]), int(k)) for k in ks], dtype=np.int64))
    elem_nodes, elem_dofs = [], []
    for s in range(mesh.n_sub):
        gl = sorted(set(int(maps.coarse_glob[k]) for k in maps.sub_coarse[s]))
        elem_nodes.append(np.array([node_of_glob[g] for g in gl], dtype=np.int64))
        elem_dofs.append(maps.sub_coarse[s].copy())
    return LevelMesh(mesh.dim, mesh.ncomp, np.array(coords), node_dofs, elem_nodes, elem_dofs,
                     np.asarray(part_next), int(n_sub_next), maps.n_coarse, mesh.rigid_comps,
                     mesh.rigid_points, mesh.last_comp)
