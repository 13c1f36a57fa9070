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


def test_tensor_core_factor_matches_cuda_core_factor():
    # 12^3-element subdomains (n ~ 6k, 25 super-panels of 256).  Both FP32 factorisations (the
    # tcgen05 trailing update from two scaled FP16 parts and the CUDA-core update) carry FP32
    # rounding amplified by kappa(A_i) ~ 1e4.  Against the FP64 preconditioner (itself pinned to
    # the oracle at 1e-10) the tensor-core error may exceed the CUDA-core one by the split's extra
    # rounding: the low parts keep 11 more bits than the high parts, so each product carries
    # ~2^-22 relative (the dropped lo lo term and the rounding of lo), about one FP32 rounding more
    # than an FMA, so at most 4x; a misplaced tile or wrong sign gives O(1).
    # The tensor-core path must still solve to 1e-8.
    p = meshgen.elasticity3d(24, 2, seed=2)
    ref = fem.direct_solve(p)[:, 0]
    s_tc = BddcSolver(p, precision="mixed", tensor_cores=1)
    s_cc = BddcSolver(p, precision="mixed", tensor_cores=0)
    s_64 = BddcSolver(p, precision="fp64")
    r = torch.tensor(np.random.default_rng(6).standard_normal(s_tc.n_iface), dtype=torch.float64, device="cuda")
    z_tc = s_tc.apply_precond(r).cpu().numpy()
    z_cc = s_cc.apply_precond(r).cpu().numpy()
    z_64 = s_64.apply_precond(r).cpu().numpy()
    e_tc, e_cc = _rel(z_tc, z_64), _rel(z_cc, z_64)
    print(f"FP32 preconditioner error vs FP64: tensor cores {e_tc:.3e}, CUDA cores {e_cc:.3e}")
    assert e_tc < 4.0 * e_cc + 1e-7
    assert e_tc < 1e-2
    u = s_tc.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    assert _rel(u, ref) < 1e-8


def test_graph_iteration_matches_eager_and_profiles():
    # the captured PCG iteration replays exactly the eager kernels: bit-identical iterates
    p = PROBLEMS["elast8_4"]()
    f = _dev(p.f[:, 0])
    a = BddcSolver(p, precision="mixed", use_graph=1).solve(f, tol=1e-10).cpu().numpy()
    b = BddcSolver(p, precision="mixed", use_graph=0).solve(f, tol=1e-10).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    s = BddcSolver(p, precision="mixed", use_graph=1, profile=1)
    s.reset_profile()
    s.solve(f, tol=1e-10)
    st = s.stats()
    # every inner iteration sweeps the interface rows forward and backward (preconditioner),
    # applies the factor-based Schur operator once and the explicit inverse of the coarsest
    # factor once
    assert st.prof_launches[capi.PROF_TRSV_IFACE] >= 2 * st.iterations
    assert st.prof_launches[capi.PROF_TRMV] >= st.iterations
    assert st.prof_launches[capi.PROF_COARSE] >= st.iterations
    assert st.prof_launches[capi.PROF_TRSV] > 0   # FP64 operator of the outer iteration
    assert st.prof_ms[capi.PROF_TRSV_IFACE] > 0 and st.prof_ms[capi.PROF_TRMV] > 0


@pytest.mark.parametrize("inner", [-1, 0, 1, 2])
def test_outer_refinement_variants_match_direct_solve(inner):
    # mixed PCG with (inner >= 0) or without (-1) the FP64 outer refinement loop around an
    # inner PCG whose Schur operator comes from the stored factor (0) or uses `inner`
    # interior-solve steps
    p = PROBLEMS["elast8_4"]()
    ref = fem.direct_solve(p)[:, 0]
    s = BddcSolver(p, precision="mixed", inner_steps=inner)
    u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    st = s.last_stats
    assert st.converged == 1
    assert _rel(u, ref) < 1e-8
    if inner == -1:
        assert st.outer_iterations == 0 and st.inner_steps == -1
    elif inner < st.refine_steps:
        assert st.outer_iterations >= 2 and st.inner_steps == inner


def test_autotuned_sweeps_are_bitwise_equal_to_defaults():
    # the tuner only picks launch variants (CTAs per SM, tile-ring depth, task order) of sweeps
    # whose per-row summation order is fixed, so the solution must not change in any bit
    p = meshgen.elasticity3d_kmeans(12, 20, 4, seed=3, seed2=33)   # uneven subdomains, 3 levels
    f = _dev(p.f[:, 0])
    a = BddcSolver(p, precision="mixed", autotune=0)
    ua = a.solve(f, tol=1e-10).cpu().numpy()
    b = BddcSolver(p, precision="mixed", autotune=1)
    ub = b.solve(f, tol=1e-10).cpu().numpy()
    np.testing.assert_array_equal(ua, ub)
    st = b.last_stats
    for l in range(st.n_levels):
        for part in range(2):
            k = 2 * l + part
            assert st.sweep_ctas[k] in (1, 2) and st.sweep_deep[k] in (0, 1) and st.sweep_order[k] in (0, 1)
    assert all(a.last_stats.sweep_ctas[k] == 2 and a.last_stats.sweep_deep[k] == 1 for k in range(2 * st.n_levels))


def test_batching_ablation_leaves_the_handle_unchanged():
    p = PROBLEMS["elast8_4"]()
    f = _dev(p.f[:, 0])
    s = BddcSolver(p, precision="mixed")
    u0 = s.solve(f, tol=1e-10).cpu().numpy()
    ab = s.batching_ablation()
    assert all(v > 0 for v in ab.values())
    u1 = s.solve(f, tol=1e-10).cpu().numpy()
    np.testing.assert_array_equal(u0, u1)   # the factors were recomputed bit for bit
