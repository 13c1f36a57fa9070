"""The mixed factorisation's panel solves on the tensor cores (tensor_cores = 1): per 256-wide
sub-panel the 256 x 256 diagonal block D is factored (L_D S_D L_D^T) and inverted on CUDA cores,
and the rows below it are solved as L(i, D) = A(i, D) X^T S_D with X = L_D^{-1}, through the
tcgen05 update kernel (two scaled FP16 parts per operand, three products), against the same
factorisation with the panel solved tile by tile on CUDA cores (tensor_cores = 2) and entirely
on CUDA cores (tensor_cores = 0).

Error model: the substitution through an explicit inverse carries kappa(L_D) u instead of u per
solve (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 14.3), and the split products
about 2^-22 relative instead of 2^-24.  On these subdomains the three FP32 preconditioners differ
from the FP64 one by the factor's FP32 error amplified by kappa(A_i); the tensor-core forms may
exceed the CUDA-core error by a small factor (bound 4x, as for the trailing update alone), while a
misplaced tile, a wrong sign, a row of the diagonal block solved twice or a dropped row below it
gives O(1).  Cases: uniform 12^3-element subdomains (one ragged last sub-panel per subdomain),
irregular k-means tetrahedral subdomains (every subdomain's block count differs, so the last
diagonal block holds 1 to 4 tiles and constraint rows start inside a sub-panel), three levels,
and the Stokes cavity (indefinite levels: pivot signs folded into the inverse's rows)."""
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


CASES = {
    "elast24": lambda: meshgen.elasticity3d(24, 2, seed=2),
    "tet12": lambda: meshgen.elasticity3d_tet(12, 8, seed=1),
    "elast16_3lev": lambda: meshgen.elasticity3d(16, 4, seed=3, group=2),
    "cavity8": lambda: meshgen.stokes_cavity(8, 2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_panel_solves_on_tensor_cores(name):
    p = CASES[name]()
    s = {tc: BddcSolver(p, precision="mixed", tensor_cores=tc) for tc in (1, 2, 0)}
    s64 = BddcSolver(p, precision="fp64")
    r = _dev(np.random.default_rng(6).standard_normal(s64.n_iface))
    z = {tc: sv.apply_precond(r).cpu().numpy() for tc, sv in s.items()}
    z64 = s64.apply_precond(r).cpu().numpy()
    e = {tc: _rel(z[tc], z64) for tc in z}
    print(f"{name}: FP32 preconditioner error vs FP64: panels on tensor cores {e[1]:.3e}, "
          f"updates only {e[2]:.3e}, CUDA cores {e[0]:.3e}")
    assert e[1] < 4.0 * e[0] + 1e-7
    assert e[1] < 1e-2
    ref = fem.direct_solve(p)[:, 0]
    u = s[1].solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    assert s[1].last_stats.converged == 1
    assert _rel(u, ref) < 1e-8
