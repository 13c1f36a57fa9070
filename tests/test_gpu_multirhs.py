"""Blocks of right-hand sides: the PCG columns run in lockstep and every factor-streaming kernel
(sweeps, factor products) reads each tile once for up to eight columns (four in FP64).  Each
column's arithmetic is the single-column arithmetic, so a block must reproduce the columns solved
one at a time (to round-off of the restart points; both solved to 1e-12) and the direct solve
within 1e-8; block operator applications must equal column-by-column ones to round-off.
Five columns exercise the grouping 4 + 1 of the kernels; nine the blocks 8 + 1 of the solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem
from paper_1201_5991_gb300 import meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("nrhs,group", [(5, 0), (9, 2)])
def test_block_solve_matches_single_column_solves(prec, nrhs, group):
    p = meshgen.elasticity3d(8, 4, seed=4, nrhs=nrhs, group=group)   # group 2: three levels
    ref = fem.direct_solve(p)
    s = BddcSolver(p, precision=prec)
    F = _dev(p.f.T)
    U = s.solve(F, tol=1e-12).cpu().numpy()
    assert s.last_stats.converged == 1
    for k in range(nrhs):
        uk = s.solve(F[k].contiguous(), tol=1e-12).cpu().numpy()
        assert _rel(U[k], uk) < 1e-9, k
        assert _rel(U[k], ref[:, k]) < 1e-8, k


def test_block_operators_match_column_applications():
    p = meshgen.elasticity3d(8, 4, seed=4, group=2)
    rng = np.random.default_rng(12)
    for prec in ("mixed", "fp64"):
        s = BddcSolver(p, precision=prec)
        R = _dev(rng.standard_normal((6, s.n_iface)))
        Z = s.apply_precond(R).cpu().numpy()
        Y = s.apply_schur(R).cpu().numpy()
        for k in range(6):
            np.testing.assert_allclose(Z[k], s.apply_precond(R[k].contiguous()).cpu().numpy(), rtol=1e-13, atol=0)
            np.testing.assert_allclose(Y[k], s.apply_schur(R[k].contiguous()).cpu().numpy(), rtol=1e-13, atol=0)


def test_block_graph_replay_matches_eager():
    p = meshgen.elasticity3d(8, 4, seed=4, nrhs=4)
    F = _dev(p.f.T)
    a = BddcSolver(p, precision="mixed", use_graph=1).solve(F, tol=1e-10).cpu().numpy()
    b = BddcSolver(p, precision="mixed", use_graph=0).solve(F, tol=1e-10).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_block_stokes_and_lifted_columns():
    # BiCGstab / FGMRES solve columns one at a time; the lifted right-hand sides of a block
    p = meshgen.stokes_cavity(4, 2)
    ref = fem.direct_solve(p)[:, 0]
    s = BddcSolver(p, precision="fp64")
    F = _dev(np.stack([p.f[:, 0], p.f[:, 0]]))
    U = s.solve(F, tol=1e-12).cpu().numpy()
    for k in range(2):
        assert np.abs(U[k] - ref).max() < 1e-7 * np.abs(ref).max()
    q = meshgen.elasticity3d(6, 2, seed=1, nrhs=3)
    q.dir_values = np.where(q.dirichlet == 1, np.random.default_rng(4).standard_normal(q.dirichlet.size), 0.0)
    refq = fem.direct_solve(q)
    U = BddcSolver(q, precision="mixed").solve(_dev(q.f.T), tol=1e-12).cpu().numpy()
    for k in range(3):
        assert _rel(U[k], refq[:, k]) < 1e-8
