"""Oracle multilevel BDDC with PCG on the reduced interface problem.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2 and Algorithms 1-2 of the paper step by step, in FP64, with dense LAPACK
per subdomain:

  * reduced interface problem  S u_hat = g_hat;  S applied through independent discrete
    Dirichlet problems (interior solves with K_II), g_hat the condensed right-hand side.
  * coarse basis Psi_i and Lambda_i from the saddle-point system Eq. psi_def, solved with
    the UNMODIFIED matrix [[K_i, C_i^T], [C_i, 0]] (dense LU with partial pivoting);
    local coarse matrix K_Ci = -Lambda_i; global coarse matrix by assembly with R_Ci.
  * one application (Algorithm 2): r_i = E_i^T r_hat, subdomain correction Eq. sub_cor,
    coarse residual r_C = sum R_Ci^T Psi_i^T E_i^T r_hat, coarse correction, then
    z_hat = sum E_i (Psi_i R_Ci z_C + z_i).  E_i^T = D_i R_i (weights D_i on the interface).
  * levels l > 1 (Sec. 2 last paragraph; Algorithm 2): the coarse problem of level l-1 is
    replaced by one BDDC step of level l with interior pre-correction and post-correction.
    Reading taken (the paper gives no formula): static condensation around the interface
    step -- u1 = R_I^T A_II^{-1} r_I, r' = r - A u1, z_G = BDDC_G(r'_G),
    z = u1 + [-A_II^{-1} A_IG z_G ; z_G].
  * PCG (Sec. 4): x0 = 0, stop when ||r||/||g_hat|| <= tol on the recursively updated
    residual, confirmed once with the true residual.  The condition number is estimated
    from the Lanczos tridiagonal T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    T_{j,j+1} = sqrt(beta_j)/alpha_j.
  * BiCGstab (Sec. 4, the Stokes experiments): right preconditioned, van der Vorst's
    recurrences; flexible GMRES (Saad) as the alternative for an inexact preconditioner.

Weights: diagonal-stiffness D_i(j) = K_i(jj) / sum_k K_k(jj) (default) or multiplicity; DOFs
whose diagonal sum is zero (Stokes pressures) take the multiplicity weight.

Parity: pinned in ``tests/test_oracle_bddc.py`` against the direct solve, an explicitly
formed Schur complement, one-subdomain exactness, the all-interface-corners case, K_Ci =
-Lambda_i = Psi_i^T K_i Psi_i, C_i Psi_i = I, and lambda_min(M^{-1} S) >= 1; the Krylov
methods against LAPACK solves; the Stokes cavity against the direct solve and the discrete
divergence-free condition.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem
from .maps import LevelMaps, LevelMesh, analyze, mesh_level1, next_level_mesh


@dataclasses.dataclass
class LevelData:
    maps: LevelMaps
    K: List[np.ndarray]            # dense local matrices, local order (interior, interface)
    KII: List[object]              # LU factors of the interior blocks
    saddle: List[object]           # LU factors of [[K_i, C_i^T], [C_i, 0]]
    Psi: List[np.ndarray]          # [n_local, n_c]
    Lam: List[np.ndarray]          # [n_c, n_c]
    KC: List[np.ndarray]           # -Lambda_i
    w: List[np.ndarray]            # weights of the local interface DOFs
    A: Optional[sp.csr_matrix]     # assembled level matrix (levels > 1)


def _local_matrices(mesh: LevelMesh, maps: LevelMaps, Ke) -> List[np.ndarray]:
    """Sub-assembly of element matrices into K_i (Sec. 2: 'sub-assembling')."""
    out = []
    for s in range(mesh.n_sub):
        dofs = maps.sub_dofs[s]
        loc = {int(d): k for k, d in enumerate(dofs)}
        K = np.zeros((dofs.size, dofs.size))
        for e in maps.sub_elems[s]:
            ed = mesh.elem_dofs[int(e)]
            idx = np.array([loc.get(int(d), -1) if d >= 0 else -1 for d in ed])
            keep = idx >= 0
            K[np.ix_(idx[keep], idx[keep])] += Ke[int(e)][np.ix_(keep, keep)]
        out.append(K)
    return out


def _assemble_level(mesh: LevelMesh, Ke) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    for e, ed in enumerate(mesh.elem_dofs):
        ed = np.asarray(ed)
        keep = ed >= 0
        d = ed[keep]
        rows.append(np.repeat(d, d.size))
        cols.append(np.tile(d, d.size))
        vals.append(Ke[e][np.ix_(keep, keep)].ravel())
    n = mesh.n_dof
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def setup_level(mesh: LevelMesh, Ke, constraints: int, weights: str, assembled: bool,
                all_corners: bool = False) -> LevelData:
    """One pass of Algorithm 1's loop body for a level."""
    maps = analyze(mesh, constraints, all_corners)
    K = _local_matrices(mesh, maps, Ke)
    KII, saddle, Psi, Lam, KC, w = [], [], [], [], [], []
    diag_sum = np.zeros(maps.iface_dofs.size)
    for s in range(mesh.n_sub):
        nI = maps.sub_nI[s]
        d = np.diag(K[s])[nI:]
        np.add.at(diag_sum, maps.sub_iface[s], d)
    for s in range(mesh.n_sub):
        Ks = K[s]
        nI = maps.sub_nI[s]
        n = Ks.shape[0]
        KII.append(sla.lu_factor(Ks[:nI, :nI]) if nI else None)
        C = maps.sub_C[s]
        nc = C.shape[0]
        Sd = np.zeros((n + nc, n + nc))
        Sd[:n, :n] = Ks
        Sd[:n, n:] = C.T
        Sd[n:, :n] = C
        lu = sla.lu_factor(Sd)
        saddle.append(lu)
        rhs = np.zeros((n + nc, nc))
        rhs[n:, :] = np.eye(nc)
        sol = sla.lu_solve(lu, rhs)                     # Eq. psi_def
        Psi.append(sol[:n])
        Lam.append(sol[n:])
        KC.append(-sol[n:])                             # K_Ci = -Lambda_i
        if weights == "multiplicity":
            w.append(maps.sub_wmult[s].copy())
        else:
            ds = diag_sum[maps.sub_iface[s]]
            dw = np.diag(Ks)[nI:]
            # DOFs with a zero diagonal (Stokes pressures) fall back to multiplicity weights
            w.append(np.where(ds > 0, dw / np.where(ds > 0, ds, 1.0), maps.sub_wmult[s]))
    A = _assemble_level(mesh, Ke) if assembled else None
    return LevelData(maps, K, KII, saddle, Psi, Lam, KC, w, A)


class Bddc:
    """Multilevel BDDC for a Problem; ``n_levels`` counts the coarsest direct solve as a level."""

    def __init__(self, prob, weights: str = "stiffness", n_levels: Optional[int] = None,
                 constraints: Optional[int] = None, Ke=None, all_corners_levels=()):
        self.prob = prob
        self.L = int(n_levels or prob.n_levels)
        cons = prob.constraints if constraints is None else constraints
        if Ke is None:
            Ke = fem.element_matrices(prob)
        self.Ke1 = Ke
        mesh = mesh_level1(prob)
        self.levels: List[LevelData] = []
        for lev in range(1, self.L):
            if lev > 1:
                prev = self.levels[-1]
                mesh = next_level_mesh(prev.maps, prob.parts[lev - 1], prob.n_parts[lev - 1])
                Ke = prev.KC
            self.levels.append(setup_level(mesh, Ke, cons, weights, assembled=lev > 1,
                                           all_corners=lev in all_corners_levels))
        last = self.levels[-1]
        nC = last.maps.n_coarse
        KC = np.zeros((nC, nC))
        for s, rc in enumerate(last.maps.sub_coarse):   # K_C = sum R_Ci^T K_Ci R_Ci
            KC[np.ix_(rc, rc)] += last.KC[s]
        self.KC = KC
        self.KC_chol = sla.lu_factor(KC) if nC else None

    # ------------------------------------------------------------------ level-1 operators
    @property
    def l1(self) -> LevelData:
        return self.levels[0]

    @property
    def n_iface(self) -> int:
        return int(self.l1.maps.iface_dofs.size)

    def schur(self, x: np.ndarray) -> np.ndarray:
        """S x = sum_i R_i^T (K_GG x_i - K_GI K_II^{-1} K_IG x_i)  (Sec. 2)."""
        d = self.l1
        y = np.zeros_like(x)
        for s in range(len(d.K)):
            nI = d.maps.sub_nI[s]
            K = d.K[s]
            xi = x[d.maps.sub_iface[s]]
            yi = K[nI:, nI:] @ xi
            if nI:
                yi -= K[nI:, :nI] @ sla.lu_solve(d.KII[s], K[:nI, nI:] @ xi)
            np.add.at(y, d.maps.sub_iface[s], yi)
        return y

    def condensed_rhs(self, f: np.ndarray) -> np.ndarray:
        """g_hat = f_G - sum_i R_i^T K_GI K_II^{-1} f_I,i."""
        d = self.l1
        g = f[d.maps.iface_dofs].copy()
        for s in range(len(d.K)):
            nI = d.maps.sub_nI[s]
            if nI:
                fI = f[d.maps.sub_dofs[s][:nI]]
                np.add.at(g, d.maps.sub_iface[s], -(d.K[s][nI:, :nI] @ sla.lu_solve(d.KII[s], fI)))
        return g

    def recover(self, f: np.ndarray, uG: np.ndarray) -> np.ndarray:
        """u_I,i = K_II^{-1} (f_I,i - K_IG u_G,i); u_G = u_hat."""
        d = self.l1
        u = np.zeros((d.maps.mesh.n_dof,) + f.shape[1:])
        u[d.maps.iface_dofs] = uG
        for s in range(len(d.K)):
            nI = d.maps.sub_nI[s]
            if nI:
                dofs = d.maps.sub_dofs[s]
                rhs = f[dofs[:nI]] - d.K[s][:nI, nI:] @ uG[d.maps.sub_iface[s]]
                u[dofs[:nI]] = sla.lu_solve(d.KII[s], rhs)
        return u

    # ------------------------------------------------------------------ Algorithm 2
    def _interface_step(self, lev: int, r_hat: np.ndarray) -> np.ndarray:
        d = self.levels[lev]
        m = d.maps
        nC = m.n_coarse
        r_C = np.zeros((nC,) + r_hat.shape[1:])
        z_loc = []
        for s in range(len(d.K)):
            nI = m.sub_nI[s]
            n = d.K[s].shape[0]
            nc = d.Psi[s].shape[1]
            r_i = np.zeros((n,) + r_hat.shape[1:])
            r_i[nI:] = (d.w[s] * r_hat[m.sub_iface[s]].T).T           # r_i = E_i^T r_hat
            sol = sla.lu_solve(d.saddle[s], np.concatenate([r_i, np.zeros((nc,) + r_hat.shape[1:])]))
            z_loc.append(sol[:n])                                     # Eq. sub_cor
            np.add.at(r_C, m.sub_coarse[s], d.Psi[s].T @ r_i)         # r_C
        if lev == len(self.levels) - 1:
            z_C = sla.lu_solve(self.KC_chol, r_C) if nC else r_C
        else:
            z_C = self._full_step(lev + 1, r_C)
        z_hat = np.zeros_like(r_hat)
        for s in range(len(d.K)):
            nI = m.sub_nI[s]
            zi = d.Psi[s][nI:] @ z_C[m.sub_coarse[s]] + z_loc[s][nI:]
            np.add.at(z_hat, m.sub_iface[s], (d.w[s] * zi.T).T)       # sum E_i (...)
        return z_hat

    def _full_step(self, lev: int, r: np.ndarray) -> np.ndarray:
        """Levels l > 1: interior pre-correction, interface BDDC step, post-correction."""
        d = self.levels[lev]
        m = d.maps
        u1 = np.zeros_like(r)
        for s in range(len(d.K)):
            nI = m.sub_nI[s]
            if nI:
                I = m.sub_dofs[s][:nI]
                u1[I] = sla.lu_solve(d.KII[s], r[I])
        rp = r - d.A @ u1
        zG = self._interface_step(lev, rp[m.iface_dofs])
        z = u1.copy()
        z[m.iface_dofs] += zG
        for s in range(len(d.K)):
            nI = m.sub_nI[s]
            if nI:
                I = m.sub_dofs[s][:nI]
                z[I] -= sla.lu_solve(d.KII[s], d.K[s][:nI, nI:] @ zG[m.sub_iface[s]])
        return z

    def precond(self, r_hat: np.ndarray) -> np.ndarray:
        """One application of the L-level BDDC preconditioner to an interface residual."""
        return self._interface_step(0, r_hat)

    # ------------------------------------------------------------------ solve
    def solve(self, f: Optional[np.ndarray] = None, tol: float = 1e-12, maxit: int = 1000,
              flexible: bool = False, krylov: Optional[str] = None):
        """Krylov solve of S u_hat = g_hat for each right-hand side column; returns (u, info).

        PCG (Sec. 4) for the SPD problems, BiCGstab (Sec. 4, Stokes) for the indefinite one;
        ``krylov="fgmres"`` selects flexible GMRES.
        """
        if f is None:
            f = self.prob.f
        if krylov is None:
            krylov = "bicgstab" if self.prob.physics == 2 else "pcg"
        f = np.asarray(f, dtype=np.float64)
        squeeze = f.ndim == 1
        F = f[:, None] if squeeze else f
        U = np.zeros_like(F)
        infos = []
        for k in range(F.shape[1]):
            g = self.condensed_rhs(F[:, k])
            if krylov == "pcg":
                uG, info = pcg(self.schur, self.precond, g, tol, maxit, flexible)
            elif krylov == "fgmres":
                uG, info = fgmres(self.schur, self.precond, g, tol, maxit)
            else:
                uG, info = bicgstab(self.schur, self.precond, g, tol, maxit)
            U[:, k] = self.recover(F[:, k], uG)
            infos.append(info)
        return (U[:, 0] if squeeze else U), infos


@dataclasses.dataclass
class PcgInfo:
    iterations: int
    rel_residual: float
    alphas: np.ndarray
    betas: np.ndarray
    converged: bool

    def lanczos(self):
        return lanczos_extremes(self.alphas, self.betas)


def pcg(A, M, b, tol: float, maxit: int, flexible: bool = False):
    """Preconditioned CG; Fletcher-Reeves beta, or Polak-Ribiere (flexible) beta."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, PcgInfo(0, 0.0, np.zeros(0), np.zeros(0), True)
    r = b.copy()
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    it = 0
    rel = 1.0
    checked = False
    converged = False
    while it < maxit:
        it += 1
        q = A(p)
        alpha = rz / float(p @ q)
        alphas.append(alpha)
        x += alpha * p
        r_new = r - alpha * q
        rel = np.linalg.norm(r_new) / nb
        if rel <= tol:
            rt = b - A(x)
            rel_true = np.linalg.norm(rt) / nb
            if rel_true <= tol or checked:
                rel = rel_true
                converged = rel_true <= tol
                break
            checked = True
            r_new = rt
        z_new = M(r_new)
        if flexible:
            beta = float(z_new @ (r_new - r)) / rz
        else:
            beta = float(r_new @ z_new) / rz
        betas.append(beta)
        rz = float(r_new @ z_new)
        p = z_new + beta * p
        r = r_new
    return x, PcgInfo(it, float(rel), np.array(alphas), np.array(betas), converged)


def bicgstab(A, M, b, tol: float, maxit: int):
    """Right-preconditioned BiCGstab (van der Vorst); stops on ||r|| / ||b|| <= tol, confirmed
    with the true residual."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, PcgInfo(0, 0.0, np.zeros(0), np.zeros(0), True)
    r = b.copy()
    rh = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    rel = 1.0
    it = 0
    converged = False
    while it < maxit:
        it += 1
        rho_new = float(rh @ r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = M(p)
        v = A(ph)
        alpha = rho_new / float(rh @ v)
        s = r - alpha * v
        sh = M(s)
        t = A(sh)
        omega = float(t @ s) / float(t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho = rho_new
        rel = np.linalg.norm(r) / nb
        if rel <= tol:
            rel = np.linalg.norm(b - A(x)) / nb
            if rel <= tol:
                converged = True
                break
    return x, PcgInfo(it, float(rel), np.zeros(0), np.zeros(0), converged)


def fgmres(A, M, b, tol: float, maxit: int, restart: int = 50):
    """Flexible GMRES(restart) with right preconditioning (Saad 1993): the preconditioned
    vectors z_j = M(v_j) are stored and x is updated with Z y, so M may change between calls.
    Modified Gram-Schmidt; stops when the true residual ||b - A x|| / ||b|| <= tol."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, PcgInfo(0, 0.0, np.zeros(0), np.zeros(0), True)
    it = 0
    rel = 1.0
    while it < maxit:
        r = b - A(x)
        beta = np.linalg.norm(r)
        rel = beta / nb
        if rel <= tol:
            return x, PcgInfo(it, float(rel), np.zeros(0), np.zeros(0), True)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        k = 0
        while k < restart and it < maxit:
            Z.append(M(V[k]))
            w = A(Z[k])
            for i in range(k + 1):
                H[i, k] = float(V[i] @ w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            V.append(w / H[k + 1, k] if H[k + 1, k] > 0 else w)
            k += 1
            it += 1
            e1 = np.zeros(k + 1)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
            if np.linalg.norm(H[:k + 1, :k] @ y - e1) / nb <= tol or H[k, k - 1] == 0:
                break
        x = x + np.column_stack(Z) @ y
    rel = np.linalg.norm(b - A(x)) / nb
    return x, PcgInfo(it, float(rel), np.zeros(0), np.zeros(0), rel <= tol)


def lanczos_extremes(alphas: np.ndarray, betas: np.ndarray):
    """Extreme eigenvalues of the Lanczos tridiagonal built from PCG's alpha, beta."""
    k = alphas.size
    if k == 0:
        return 1.0, 1.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(max(betas[j], 0.0)) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])
