"""Linear simplices on irregular inputs: the geocomposite problem of Sec. 4 is meshed by linear
tetrahedra and divided by METIS.  Its stand-in here is Kuhn's tetrahedral split of the box
lattice with seeded interior-node jitter (no two elements congruent), seeded k-means subdomains
made face-connected (ragged interfaces, globs of every shape) and log-uniform E; the 2D
counterpart is jittered linear triangles with the Poisson operator.

Tolerances as in the box-mesh parity tests: solutions within 1e-8 of the oracle's direct solve
(both precisions solved to 1e-12), FP64 operators within 1e-11 / 1e-10, the FP32 preconditioner
within 1e-3, FP64 coarse matrices within 1e-10, PCG iteration counts within one of the oracle's.
The tetrahedral subdomains hold 340-1,130 unknowns, more than one 256-wide panel, so the mixed
form's factor runs its trailing updates on tcgen05; the triangles' 140-200 stay on CUDA cores."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem
from oracle.bddc import Bddc
from paper_1201_5991_gb300 import meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = {
    "tet": lambda: meshgen.elasticity3d_tet(12, 8, seed=1),
    "tet_3lev": lambda: meshgen.elasticity3d_tet(12, 24, seed=3, ngroup=3),
    "tri": lambda: meshgen.poisson2d_tri(40, 10, seed=2),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_solution_matches_direct_solve(name, prec):
    p = CASES[name]()
    ref = fem.direct_solve(p)[:, 0]
    s = BddcSolver(p, precision=prec)
    u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    assert s.last_stats.converged == 1
    assert s.last_stats.n_levels == p.n_levels
    assert _rel(u, ref) < 1e-8


@pytest.mark.parametrize("name", ["tet", "tri"])
def test_operators_and_coarse_matrices_match_oracle(name):
    p = CASES[name]()
    o = Bddc(p)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(o.n_iface)
    r = rng.standard_normal(o.n_iface)
    y_ref, z_ref = o.schur(x), o.precond(r)
    s64 = BddcSolver(p, precision="fp64")
    assert _rel(s64.apply_schur(_dev(x)).cpu().numpy(), y_ref) < 1e-11
    assert _rel(s64.apply_precond(_dev(r)).cpu().numpy(), z_ref) < 1e-10
    kc = s64.coarse_matrices(1)
    KC = o.levels[0].KC
    assert len(kc) == len(KC)
    assert max(_rel(a, b) for a, b in zip(kc, KC)) < 1e-10
    s32 = BddcSolver(p, precision="mixed")
    assert _rel(s32.apply_schur(_dev(x)).cpu().numpy(), y_ref) < 1e-11
    assert _rel(s32.apply_precond(_dev(r)).cpu().numpy(), z_ref) < 1e-3


def test_iterations_and_spectrum_match_oracle():
    p = CASES["tet"]()
    _, info = Bddc(p).solve(p.f[:, 0], tol=1e-10)
    s = BddcSolver(p, precision="fp64")
    s.solve(_dev(p.f[:, 0]), tol=1e-10)
    assert abs(s.last_stats.iterations - info[0].iterations) <= 1
    _, lmax = info[0].lanczos()
    assert s.last_stats.lambda_min >= 1 - 1e-6
    assert abs(s.last_stats.lambda_max - lmax) <= 1e-3 * lmax


def test_gradient_matches_oracle():
    from oracle import grad as og
    p = meshgen.elasticity3d_tet(6, 6, seed=7, nrhs=2)
    u_ref = fem.direct_solve(p)
    w = np.random.default_rng(8).standard_normal(u_ref.shape)
    g_ref, lam_ref = og.adjoint_gradient(p, u_ref, w)
    s = BddcSolver(p, precision="mixed")
    u = s.solve(_dev(p.f.T), tol=1e-12)
    gc, gr = s.grad(_dev(w.T), u, tol=1e-12)
    assert _rel(gc.cpu().numpy(), g_ref) < 1e-5
    assert _rel(gr.cpu().numpy().T, lam_ref) < 1e-8
