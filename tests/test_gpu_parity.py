"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64-PCG solutions within 1e-8 relative 2-norm of the oracle (both
sides solved to 1e-12); operator applications in FP64 within 1e-11 (a few hundred FP64
roundings times kappa(K_II) ~ 1e3); the FP32 preconditioner within 1e-3, the size of
kappa(A_i) * 2^-24 for kappa(A_i) <= 1e4 as measured on these subdomains (corner-only
constraints give the largest kappa)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem
from oracle.bddc import Bddc
from paper_1201_5991_gb300 import capi, meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


PROBLEMS = {
    "poisson32": lambda: meshgen.poisson2d(32, 4),
    "elast12": lambda: meshgen.elasticity3d(12, 2, seed=0),
    "elast8_4": lambda: meshgen.elasticity3d(8, 4, seed=4),
    "elast_ragged": lambda: meshgen.elasticity3d(10, 2, seed=9),       # 5^3 subdomains: ragged tiles
    "elast_corners": lambda: meshgen.elasticity3d(6, 2, seed=1, constraints=meshgen.CORNERS),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_solution_matches_direct_solve(name, prec):
    p = PROBLEMS[name]()
    ref = fem.direct_solve(p)[:, 0]
    s = BddcSolver(p, precision=prec)
    u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    assert s.last_stats.converged == 1
    assert _rel(u, ref) < 1e-8


@pytest.mark.parametrize("name", ["poisson32", "elast12", "elast_ragged"])
def test_schur_operator_matches_oracle(name):
    p = PROBLEMS[name]()
    o = Bddc(p)
    x = np.random.default_rng(3).standard_normal(o.n_iface)
    y_ref = o.schur(x)
    for prec in ("fp64", "mixed"):
        s = BddcSolver(p, precision=prec)
        y = s.apply_schur(_dev(x)).cpu().numpy()
        assert _rel(y, y_ref) < 1e-11, prec


@pytest.mark.parametrize("name", ["poisson32", "elast12", "elast8_4", "elast_corners"])
def test_preconditioner_matches_oracle(name):
    p = PROBLEMS[name]()
    o = Bddc(p)
    r = np.random.default_rng(4).standard_normal(o.n_iface)
    z_ref = o.precond(r)
    z64 = BddcSolver(p, precision="fp64").apply_precond(_dev(r)).cpu().numpy()
    assert _rel(z64, z_ref) < 1e-10
    z32 = BddcSolver(p, precision="mixed").apply_precond(_dev(r)).cpu().numpy()
    assert _rel(z32, z_ref) < 1e-3


def test_iterations_match_oracle_fp64():
    p = PROBLEMS["elast8_4"]()
    _, info = Bddc(p).solve(p.f[:, 0], tol=1e-10)
    s = BddcSolver(p, precision="fp64")
    s.solve(_dev(p.f[:, 0]), tol=1e-10)
    assert abs(s.last_stats.iterations - info[0].iterations) <= 1
    lmin, lmax = info[0].lanczos()
    assert s.last_stats.lambda_min >= 1 - 1e-6
    assert abs(s.last_stats.lambda_max - lmax) <= 1e-3 * lmax


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_three_levels_match_direct_solve(prec):
    p = meshgen.elasticity3d(8, 4, seed=4, group=2)
    ref = fem.direct_solve(p)[:, 0]
    s = BddcSolver(p, precision=prec)
    u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    assert s.last_stats.n_levels == 3
    assert _rel(u, ref) < 1e-8
    o = Bddc(p)
    r = np.random.default_rng(5).standard_normal(o.n_iface)
    z = BddcSolver(p, precision="fp64").apply_precond(_dev(r)).cpu().numpy()
    assert _rel(z, o.precond(r)) < 1e-10


def test_multiple_rhs_and_host_entry_point():
    p = meshgen.elasticity3d(6, 2, seed=5, nrhs=3)
    ref = fem.direct_solve(p)
    s = BddcSolver(p, precision="mixed")
    U = s.solve(_dev(p.f.T), tol=1e-12).cpu().numpy()
    for k in range(3):
        assert _rel(U[k], ref[:, k]) < 1e-8
    Uh = s.solve_host(np.ascontiguousarray(p.f.T), tol=1e-12)
    np.testing.assert_array_equal(Uh, U)


def test_bitwise_reproducible():
    p = PROBLEMS["elast12"]()
    a = BddcSolver(p, precision="mixed").solve(_dev(p.f[:, 0]), tol=1e-10).cpu().numpy()
    b = BddcSolver(p, precision="mixed").solve(_dev(p.f[:, 0]), tol=1e-10).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_gradient_matches_oracle():
    from oracle import grad as og
    p = meshgen.elasticity3d(6, 2, seed=7, nrhs=2)
    u_ref = fem.direct_solve(p)
    w = np.random.default_rng(8).standard_normal(u_ref.shape)
    g_ref, lam_ref = og.adjoint_gradient(p, u_ref, w)
    s = BddcSolver(p, precision="mixed")
    u = s.solve(_dev(p.f.T), tol=1e-12)
    gc, gr = s.grad(_dev(w.T), u, tol=1e-12)
    assert _rel(gc.cpu().numpy(), g_ref) < 1e-5
    assert _rel(gr.cpu().numpy().T, lam_ref) < 1e-8


def test_error_codes():
    p = PROBLEMS["poisson32"]()
    s = BddcSolver(p, precision="fp64", maxit=2)
    with pytest.raises(capi.BddcError) as ei:
        s.solve(_dev(p.f[:, 0]), tol=1e-12)
    assert ei.value.code == capi.ERR_NOT_CONVERGED
    s = BddcSolver(p, precision="fp64")
    f = p.f[:, 0].copy()
    f[5] = np.nan
    with pytest.raises(capi.BddcError) as ei:
        s.solve(_dev(f), tol=1e-8)
    assert ei.value.code == capi.ERR_NAN
