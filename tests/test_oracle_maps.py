"""Pins of the oracle's interface analysis: hand-counted sizes and partition of unity."""
import numpy as np
import pytest

from oracle import maps
from paper_1201_5991_gb300 import meshgen


def _analyze(p, **kw):
    return maps.analyze(maps.mesh_level1(p), p.constraints, **kw)


def test_poisson_32_sizes():
    # 4x4 subdomains of 8x8: 3 vertical + 3 horizontal interface lines of 31 free nodes,
    # 9 cross points counted twice -> 177 interface DOFs; 9 interior cross points = corners.
    m = _analyze(meshgen.poisson2d(32, 4))
    assert m.iface_dofs.size == 177
    assert m.n_coarse == 9
    assert sorted({g.kind for g in m.globs}) == [maps.VERTEX, maps.EDGE]
    assert m.n_promoted == 0


def test_elasticity_small_sizes():
    # 12^3 elements, 2^3 subdomains: planes x,y,z = 6 with 13x13 nodes; 3 lines of 13 nodes
    # counted twice; the centre counted three times -> 3*169 - 3*13 + 1 = 469 nodes, minus
    # the 25 Dirichlet ones on x = 0 (two planes of 13, their common node once) = 444 nodes.
    # Globs: 1 vertex, 6 edges (4 of them touch x = 0 only at a Dirichlet end), 12 faces.
    m = _analyze(meshgen.elasticity3d(12, 2, seed=0))
    assert m.iface_dofs.size == 444 * 3
    kinds = [g.kind for g in m.globs]
    assert kinds.count(maps.VERTEX) == 1
    assert kinds.count(maps.EDGE) == 6
    assert kinds.count(maps.FACE) == 12
    assert m.n_coarse == 3 * 19


@pytest.mark.slow
def test_elasticity_48_sizes():
    # 48^3, 4^3 subdomains (the 345,744-DOF workload): hand count 20,028 free interface
    # nodes; 27 vertices + 108 edges + 144 faces = 279 globs -> 837 coarse DOFs.
    p = meshgen.config("elasticity3d_48")
    assert p.n_free == 345744
    m = _analyze(p)
    assert m.iface_dofs.size == 60084
    assert m.n_coarse == 837
    nI = np.array(m.sub_nI)
    n = np.array([d.size for d in m.sub_dofs])
    assert nI.min() == 3993 and nI.max() == 5184
    assert n.min() == 6084 and n.max() == 6591


@pytest.mark.parametrize("mk", [lambda: meshgen.poisson2d(16, 4), lambda: meshgen.elasticity3d(6, 2, seed=1)])
def test_partition_of_unity_and_constraint_rows(mk):
    p = mk()
    m = _analyze(p)
    acc = np.zeros(m.iface_dofs.size)
    for s in range(m.mesh.n_sub):
        np.add.at(acc, m.sub_iface[s], m.sub_wmult[s])
        C = m.sub_C[s]
        np.testing.assert_allclose(C.sum(axis=1), 1.0, atol=1e-15)   # averages
        assert np.linalg.matrix_rank(C) == C.shape[0]
        nI = m.sub_nI[s]
        assert np.all(C[:, :nI] == 0)                                  # interface-only rows
    np.testing.assert_allclose(acc, 1.0, atol=1e-15)


def test_all_corners_mode():
    p = meshgen.poisson2d(16, 4)
    m = _analyze(p, all_corners=True)
    assert m.n_coarse == m.iface_dofs.size


def test_next_level_pseudo_mesh():
    # 8^3 elements, 4^3 subdomains grouped 2^3 -> level 2 has 8 subdomains over the globs
    p = meshgen.elasticity3d(8, 4, seed=0, group=2)
    m1 = _analyze(p)
    mesh2 = maps.next_level_mesh(m1, p.parts[1], p.n_parts[1])
    assert mesh2.n_dof == m1.n_coarse
    assert len(mesh2.elem_nodes) == 64
    m2 = maps.analyze(mesh2, p.constraints)
    # the level-2 interface of a 2x2x2 block grouping: every level-2 glob lies on the three
    # mid-planes; the centre vertex is shared by all 8 level-2 subdomains
    assert any(len(g.subs) == 8 for g in m2.globs)
    assert m2.n_coarse > 0
