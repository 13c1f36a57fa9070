"""C ABI on CPU: the library loads, exports every declared symbol, and its index analysis
(bddc_analyze, no GPU call) matches the oracle's maps bit for bit on every level."""
import os
import re

import numpy as np
import pytest

from oracle import maps as om
from paper_1201_5991_gb300 import capi, meshgen, solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "bddc.h")).read()
    declared = set(re.findall(r"\b(bddc_[a-z_]+)\s*\(", hdr))
    L = capi.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(capi.EXPORTED)


def _oracle_levels(p, n_levels, all_corners=()):
    mesh = om.mesh_level1(p)
    out = []
    for lev in range(1, n_levels):
        if lev > 1:
            mesh = om.next_level_mesh(out[-1], p.parts[lev - 1], p.n_parts[lev - 1])
        out.append(om.analyze(mesh, p.constraints, lev in all_corners))
    return out


def _compare(lib, orc):
    assert lib["n_dof"] == orc.mesh.n_dof
    assert lib["n_sub"] == orc.mesh.n_sub
    np.testing.assert_array_equal(lib["iface_dofs"], orc.iface_dofs)
    assert lib["n_coarse"] == orc.n_coarse
    assert lib["n_promoted"] == orc.n_promoted
    np.testing.assert_array_equal(lib["coarse_glob"], orc.coarse_glob)
    np.testing.assert_array_equal(lib["coarse_comp"], orc.coarse_comp)
    assert lib["n_globs"] == len(orc.globs)
    for g, G in enumerate(orc.globs):
        np.testing.assert_array_equal(lib["glob_nodes"][lib["glob_ptr"][g]:lib["glob_ptr"][g + 1]], G.nodes)
        assert lib["glob_kind"][g] == G.kind
        assert bool(lib["glob_promoted"][g]) == G.promoted
    sp = lib["sub_dof_ptr"]
    cp = lib["sub_coarse_ptr"]
    for s in range(orc.mesh.n_sub):
        dofs = lib["sub_dofs"][sp[s]:sp[s + 1]]
        np.testing.assert_array_equal(dofs, orc.sub_dofs[s])
        nI = lib["sub_nI"][s]
        assert nI == orc.sub_nI[s]
        np.testing.assert_array_equal(lib["sub_iface"][sp[s] + nI:sp[s + 1]], orc.sub_iface[s])
        assert np.all(lib["sub_iface"][sp[s]:sp[s] + nI] == -1)
        np.testing.assert_array_equal(lib["sub_wmult"][sp[s] + nI:sp[s + 1]], orc.sub_wmult[s])   # bit-exact
        np.testing.assert_array_equal(lib["sub_coarse"][cp[s]:cp[s + 1]], orc.sub_coarse[s])
        C = np.zeros((cp[s + 1] - cp[s], dofs.size))
        for r in range(cp[s], cp[s + 1]):
            for t in range(lib["c_ptr"][r], lib["c_ptr"][r + 1]):
                C[r - cp[s], lib["c_col"][t]] = lib["c_val"][t]
        np.testing.assert_array_equal(C, orc.sub_C[s])                                            # bit-exact


def _floating_half(constraints=meshgen.CORNERS):
    # 4^3 cube cut at x = 0.5, corners only: the right half floats (no Dirichlet node, no
    # vertex glob), so the rigid-body test must promote three interface nodes to corners.
    p = meshgen.elasticity3d(4, 1, seed=0, constraints=constraints)
    cent = p.coords[p.conn].mean(axis=1)
    p.parts = [(cent[:, 0] > 0.5).astype(np.int32)]
    p.n_parts = [2]
    return p


CASES = {
    "promoted_corners": (_floating_half, 2),
    "poisson32": (lambda: meshgen.poisson2d(32, 4), 2),
    "elast12": (lambda: meshgen.elasticity3d(12, 2, seed=0), 2),
    "elast8_3lev": (lambda: meshgen.elasticity3d(8, 4, seed=0, group=2), 3),
    "elast6_corners": (lambda: meshgen.elasticity3d(6, 2, seed=1, constraints=meshgen.CORNERS), 2),
    "kmeans_small": (lambda: meshgen.elasticity3d_kmeans(12, 24, 3, seed=3, seed2=33), 3),
    "tri_kmeans": (lambda: meshgen.poisson2d_tri(16, 6, seed=2), 2),   # linear triangles
    "tet_kmeans": (lambda: meshgen.elasticity3d_tet(6, 10, seed=1), 2),   # jittered linear tetrahedra
    "tet_3lev": (lambda: meshgen.elasticity3d_tet(8, 24, seed=3, ngroup=3), 3),
    "stokes6": (lambda: meshgen.stokes_cavity(6, 3), 2),              # velocities before pressures
    "stokes8_3lev": (lambda: meshgen.stokes_cavity(8, 4, (2,)), 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_maps_bit_exact_vs_oracle(name):
    mk, L = CASES[name]
    p = mk()
    lib = solver.analyze(p, n_levels=L)
    orc = _oracle_levels(p, L)
    assert len(lib) == len(orc) == L - 1
    if name == "promoted_corners":
        assert lib[0]["n_promoted"] == 3
    for a, b in zip(lib, orc):
        _compare(a, b)


def test_all_corners_maps_bit_exact():
    p = meshgen.poisson2d(16, 4)
    lib = solver.analyze(p, all_corners=1)
    orc = _oracle_levels(p, 2, all_corners=(1,))
    _compare(lib[0], orc[0])
    assert lib[0]["n_coarse"] == lib[0]["n_iface"]


def test_promoted_corners_maps_bit_exact():
    # corners only on slab partitions along x: the inner slabs float with too few corners, so
    # corners are promoted subdomain after subdomain, and a promotion on one slab adds a
    # constrained point to its neighbour (the order of the promotions matters)
    p = meshgen.elasticity3d(12, 3, seed=2, constraints=meshgen.CORNERS)
    cent = p.coords[p.conn].mean(axis=1)
    p.parts = [np.minimum((cent[:, 0] * 4).astype(np.int32), 3)]
    p.n_parts = [4]
    lib = solver.analyze(p, n_levels=2)
    orc = _oracle_levels(p, 2)
    assert lib[0]["n_promoted"] == 7
    _compare(lib[0], orc[0])


@pytest.mark.slow
def test_maps_bit_exact_elasticity_48():
    p = meshgen.config("elasticity3d_48")
    lib = solver.analyze(p)
    orc = _oracle_levels(p, 2)
    _compare(lib[0], orc[0])


def test_invalid_partition_is_rejected():
    p = meshgen.poisson2d(8, 2)
    p.parts[0] = p.parts[0].copy()
    p.parts[0][3] = 99                      # subdomain id out of range
    with pytest.raises(capi.BddcError) as ei:
        solver.analyze(p)
    assert ei.value.code == capi.ERR_INVALID
    p = meshgen.poisson2d(8, 2)
    p.n_parts = [5]                          # subdomain 4 is empty
    with pytest.raises(capi.BddcError) as ei:
        solver.analyze(p)
    assert ei.value.code == capi.ERR_INVALID
    p = meshgen.poisson2d(8, 2)
    p.n_parts = [65536]                      # more subdomains than a launch grid's y extent
    with pytest.raises(capi.BddcError) as ei:
        solver.analyze(p)
    assert ei.value.code == capi.ERR_INVALID
    assert "65,535" in capi.lib().bddc_last_error().decode()


def test_stokes_local_order_puts_pressures_last():
    p = meshgen.stokes_cavity(6, 3)
    lib = solver.analyze(p)[0]
    full = np.nonzero(p.free)[0]
    comp = full % 4
    sp = lib["sub_dof_ptr"]
    for s in range(lib["n_sub"]):
        nI = lib["sub_nI"][s]
        dofs = lib["sub_dofs"][sp[s]:sp[s + 1]]
        for seg in (dofs[:nI], dofs[nI:]):
            c = comp[seg]
            k = np.argmax(c == 3) if np.any(c == 3) else c.size
            assert np.all(c[:k] < 3) and np.all(c[k:] == 3)


def test_stokes_mesh_validation():
    p = meshgen.stokes_cavity(2, 1)
    p.nodes_per_elem = 8
    p.conn = p.conn[:, :8]
    with pytest.raises(capi.BddcError) as ei:
        solver.analyze(p)
    assert ei.value.code == capi.ERR_INVALID


def test_degenerate_simplex_is_rejected():
    p = meshgen.elasticity3d_tet(2, 2, seed=0)
    p.conn = p.conn.copy()
    p.conn[5, 3] = p.conn[5, 2]              # two equal vertices: a flat tetrahedron
    with pytest.raises(capi.BddcError) as ei:
        solver.analyze(p)
    assert ei.value.code == capi.ERR_INVALID
    assert "element 5" in capi.lib().bddc_last_error().decode()
    p = meshgen.elasticity3d_tet(2, 2, seed=0)
    p.nodes_per_elem = 5                     # neither a box nor a simplex
    p.conn = np.hstack([p.conn, p.conn[:, :1]])
    with pytest.raises(capi.BddcError) as ei:
        solver.analyze(p)
    assert ei.value.code == capi.ERR_INVALID
