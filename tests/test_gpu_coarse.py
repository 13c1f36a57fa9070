"""Local coarse matrices K_Ci of the CUDA path (read back through bddc_get_coarse) against the
oracle's K_Ci = -Lambda_i, which solves the unmodified saddle-point system of Eq. psi_def by dense
LU (Sec. 2; K_Ci = Psi_i^T K_i Psi_i).

Tolerances, per subdomain, relative Frobenius norm:
  * FP64 form: 1e-10 (FP64 factors; the oracle's own LU carries kappa * 2^-53).
  * Mixed form: the library forms K_Ci = G_i^{-1} - R from G_i = C_i A_i^{-1} C_i^T, and the
    Cholesky factor of A_i = K_i + rho_i C_i^T C_i is FP32.  FP32 Cholesky is backward stable,
    (A_i + dA) = L L^T with ||dA|| ~ 2^-24 ||A_i||, so G_i and with it K_Ci carry a relative
    error of order kappa_2(A_i) 2^-24: the tolerance is max(kappa_2(A_i), 64) 2^-24, with
    kappa_2(A_i) computed here in FP64 from the oracle's K_i, C_i and the library's
    rho_i = mean diag K_i; the floor covers well-conditioned tiny subdomains, where the roundings
    of the small dense steps (G_i, its inverse) of order n_c 2^-24 dominate.
    On level l > 1 the element matrices are the level-(l-1) K_Ci, so their relative error e
    perturbs A_i by e ||A_i||: the tolerance there is max(kappa_2(A_i), 64) (2^-24 + e) with e
    the largest error measured on the level below.
A dropped term (R not subtracted, a missing constraint row, a transposed G) gives O(1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.bddc import Bddc
from paper_1201_5991_gb300 import meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _kappa(A):
    if A.shape[0] <= 2500:
        ev = np.abs(np.linalg.eigvalsh(A))
        return float(ev.max() / ev.min())
    import scipy.sparse.linalg as spla
    hi = spla.eigsh(A, k=1, which="LM", return_eigenvectors=False)[0]
    lo = spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return float(abs(hi) / abs(lo))


def _augmented(d, s, rigid_comps):
    """A_i = K_i + rho_i C_i^T diag(c) C_i with c = 1 on the rows of the floating components."""
    K, C = d.K[s], d.maps.sub_C[s]
    comp = d.maps.coarse_comp[d.maps.sub_coarse[s]]
    c = np.isin(comp, rigid_comps).astype(float)
    rho = float(np.mean(np.diag(K)))
    return K + rho * (C.T * c) @ C


def _errors(p, prec, sample=None):
    o = Bddc(p)
    s = BddcSolver(p, precision=prec)
    out = []
    for lev in range(1, p.n_levels):
        d = o.levels[lev - 1]
        kc = s.coarse_matrices(lev)
        assert len(kc) == len(d.KC)
        subs = range(len(kc)) if sample is None else sample
        out.append([(si, np.linalg.norm(kc[si] - d.KC[si]) / np.linalg.norm(d.KC[si])) for si in subs])
    return o, out


PROBLEMS = {
    "elast12": lambda: meshgen.elasticity3d(12, 2, seed=0),
    "elast_corners": lambda: meshgen.elasticity3d(6, 2, seed=1, constraints=meshgen.CORNERS),
    "elast_3lev": lambda: meshgen.elasticity3d(8, 4, seed=4, group=2),
    "cavity4_2": lambda: meshgen.stokes_cavity(4, 2),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_coarse_matrices_fp64(name):
    p = PROBLEMS[name]()
    _, errs = _errors(p, "fp64")
    worst = max(e for lev in errs for _, e in lev)
    print(f"{name}: FP64 K_Ci max relative error {worst:.2e}")
    assert worst < 1e-10


def _mixed_check(p, sample=None, label=""):
    o, errs = _errors(p, "mixed", sample)
    rigid = (0, 1, 2) if p.physics != meshgen.POISSON else (0,)
    prev = 0.0
    for lev, lerr in enumerate(errs, start=1):
        d = o.levels[lev - 1]
        worst_ratio = 0.0
        for si, e in lerr:
            bound = max(_kappa(_augmented(d, si, rigid)), 64.0) * (U32 + prev)
            worst_ratio = max(worst_ratio, e / bound)
            assert e <= bound, (lev, si, e, bound)
        prev = max(e for _, e in lerr)
        print(f"{label} level {lev}: mixed K_Ci max relative error {prev:.2e}, "
              f"max error / (max(kappa(A_i), 64) (2^-24 + e_prev)) = {worst_ratio:.3f}")


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_coarse_matrices_mixed(name):
    _mixed_check(PROBLEMS[name](), label=name)


def test_coarse_matrices_mixed_tensor_cores():
    # 12^3-element subdomains (n ~ 6.1k-6.6k): the factor's trailing updates run on tcgen05
    p = meshgen.elasticity3d(24, 2, seed=2)
    _mixed_check(p, sample=[0, 7], label="elast24 (tensor cores)")
