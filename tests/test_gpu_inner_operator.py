"""The inner operator of the mixed form's outer refinement in its two forms: products with the
stored interface factor (L_GG S L_GG^T - C^T R C) and the explicit augmented Schur complement
copied from the tiles once the interior is eliminated (the interior block count padded to a
multiple of 4 tiles, so that every subdomain reaches that point at a sub-panel boundary; the
super-panel in which an interior ends after its first half takes two rank-256 updates).

Both equal S_i + C_i^T R C_i - C_i^T R C_i in exact arithmetic; they differ by the interface
Cholesky's backward error applied to x and by FP32 rounding of the products.  Measured on these
cases: 1.6e-7 to 2.2e-7 (relative 2-norm), and each is within 3.5e-7 of the FP64 operator.  The
test allows 1e-5.  A dropped or doubled tile contribution changes the result by about a tile's
share of a row sum (1 / n_Gb, a few per cent here), a missing mirror of a diagonal tile more.
The outer refinement corrects with the FP64 operator, so solutions with either form match the
direct solve to 1e-8 (both solved to 1e-12).  Padding the interior must not change the local
coarse matrices beyond the FP32 factorisation's error: each is within max(kappa_2(A_i), 64) 2^-24
of the exact K_Ci (the bound of the coarse-matrix tests), so the two differ by at most twice that,
below 1e-3 for kappa_2(A_i) up to 8e3."""
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
    "elast24": lambda: meshgen.elasticity3d(24, 2, seed=2),                 # 12^3 subdomains
    "tet": lambda: meshgen.elasticity3d_tet(12, 8, seed=1),                 # irregular interiors
    "elast8_3lev": lambda: meshgen.elasticity3d(8, 4, seed=4, group=2),     # three levels
}


@pytest.mark.parametrize("name", list(CASES))
def test_explicit_and_factor_forms(name):
    p = CASES[name]()
    ref = fem.direct_solve(p)[:, 0]
    x = np.random.default_rng(5).standard_normal(BddcSolver(p, precision="mixed").n_iface)
    out = {}
    for form in (1, 2):
        s = BddcSolver(p, precision="mixed", inner_operator=form)
        u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
        st = s.last_stats
        assert st.converged == 1 and st.inner_operator == form
        assert _rel(u, ref) < 1e-8
        out[form] = (s.apply_inner_schur(_dev(x)).cpu().numpy(), s.apply_schur(_dev(x)).cpu().numpy(),
                     np.concatenate([k.ravel() for k in s.coarse_matrices(1)]), st.iterations)
    y1, s1, kc1, it1 = out[1]
    y2, s2, kc2, it2 = out[2]
    d = _rel(y2, y1)
    print(f"{name}: explicit vs factor form {d:.2e}; vs FP64 S {_rel(y2, s2):.2e} / {_rel(y1, s1):.2e}; "
          f"iterations {it2} / {it1}")
    assert d < 1e-5
    # the padded factorisation leaves the FP64 Schur operator and the coarse matrices unchanged up to
    # the FP32 factor's error (the FP64 operator refines its interior solves to FP64 accuracy)
    assert _rel(s2, s1) < 1e-11
    assert _rel(kc2, kc1) < 1e-3
    assert abs(it2 - it1) <= max(3, it1 // 10)


def test_automatic_choice_and_blocks():
    # 12^3 subdomains: padding the interior to a multiple of 4 tiles costs < 8 %: explicit form
    p = meshgen.elasticity3d(24, 2, seed=2, nrhs=5)
    s = BddcSolver(p, precision="mixed")
    U = s.solve(_dev(p.f.T), tol=1e-12).cpu().numpy()
    assert s.last_stats.inner_operator == 2
    ref = fem.direct_solve(p)
    for k in range(5):
        assert _rel(U[k], ref[:, k]) < 1e-8
    # a block of 5 columns (groups 4 + 1 in the symmetric product) equals the columns one by one
    # (the same FP32 operations per column; 1e-6 leaves room for a different contraction into FMAs)
    X = np.random.default_rng(9).standard_normal((5, s.n_iface))
    Y = s.apply_inner_schur(_dev(X)).cpu().numpy()
    for k in range(5):
        np.testing.assert_allclose(Y[k], s.apply_inner_schur(_dev(X[k])).cpu().numpy(), rtol=1e-6, atol=0)
    # 6^3 subdomains: padding 6 -> 8 interior tile rows would cost 70 %: factor products
    q = meshgen.elasticity3d(12, 2, seed=0)
    t = BddcSolver(q, precision="mixed")
    t.solve(_dev(q.f[:, 0]), tol=1e-10)
    assert t.last_stats.inner_operator == 1
    # FP64 handles have no inner operator
    f = BddcSolver(q, precision="fp64")
    f.solve(_dev(q.f[:, 0]), tol=1e-10)
    assert f.last_stats.inner_operator == 0
