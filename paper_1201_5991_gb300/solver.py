"""Python binding of the BDDC library: marshalling between numpy/torch and the C ABI.

Every numerical step runs inside libbddc_gb300.so; this module only passes pointers,
sizes and streams.  Device vectors are torch CUDA tensors (FP64).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import capi


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class _HostMesh:
    """Keeps the host arrays of a mesh / partition alive while the C structs point at them."""

    def __init__(self, dim, nodes_per_elem, dofs_per_node, physics, coords, conn, coef, nu, dirichlet, parts,
                 n_parts, n_levels, dir_values=None):
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.conn = np.ascontiguousarray(conn, dtype=np.int32)
        self.coef = np.ascontiguousarray(coef, dtype=np.float64)
        self.dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
        self.dir_values = None if dir_values is None else np.ascontiguousarray(dir_values, dtype=np.float64)
        self.parts = [np.ascontiguousarray(p, dtype=np.int32) for p in parts]
        dv = _ptr(self.dir_values, C.c_double) if self.dir_values is not None else None
        self.mesh = capi.Mesh(dim, nodes_per_elem, dofs_per_node, physics, self.coords.shape[0], self.conn.shape[0],
                              _ptr(self.coords, C.c_double), _ptr(self.conn, C.c_int32), _ptr(self.coef, C.c_double),
                              float(nu), _ptr(self.dirichlet, C.c_uint8), dv)
        self.part = capi.Partition()
        self.part.n_levels = int(n_levels)
        for l, p in enumerate(self.parts):
            self.part.part[l] = _ptr(p, C.c_int32)
            self.part.n_parts[l] = int(n_parts[l])


def host_mesh(prob, n_levels: Optional[int] = None) -> _HostMesh:
    L = int(n_levels or prob.n_levels)
    return _HostMesh(prob.dim, prob.nodes_per_elem, prob.dofs_per_node, prob.physics, prob.coords, prob.conn,
                     prob.coef, prob.nu, prob.dirichlet, prob.parts[:L - 1], prob.n_parts[:L - 1], L,
                     getattr(prob, "dir_values", None))


def make_opts(precision="mixed", weights="stiffness", all_corners=0, maxit=500, refine_steps=0, flexible=-1,
              use_graph=1, profile=0, tensor_cores=1, inner_steps=0, inner_tol=0.0, krylov=0,
              autotune=1, verbose=0, wait_probe=0, inner_operator=0, retain_host_memory=1) -> capi.Opts:
    o = capi.Opts()
    capi.lib().bddc_default_opts(C.byref(o))
    o.precision = capi.PREC_MIXED if precision == "mixed" else capi.PREC_FP64
    o.weights = capi.WEIGHTS_MULTIPLICITY if weights == "multiplicity" else capi.WEIGHTS_STIFFNESS
    o.all_corners = int(all_corners)
    o.maxit = int(maxit)
    o.refine_steps = int(refine_steps)
    o.flexible = int(flexible)
    o.use_graph = int(use_graph)
    o.profile = int(profile)
    o.tensor_cores = int(tensor_cores)
    o.inner_steps = int(inner_steps)
    o.inner_tol = float(inner_tol)
    o.krylov = int(krylov)
    o.autotune = int(autotune)
    o.verbose = int(verbose)
    o.wait_probe = int(wait_probe)
    o.inner_operator = int(inner_operator)
    o.retain_host_memory = int(retain_host_memory)
    return o


def _maps_to_numpy(m: capi.LevelMaps) -> dict:
    def arr(p, n, dt):
        if n == 0:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(p, shape=(int(n),)).astype(dt, copy=True)

    ns = int(m.n_sub)
    sub_dof_ptr = arr(m.sub_dof_ptr, ns + 1, np.int64)
    nloc = int(sub_dof_ptr[-1])
    cptr = arr(m.sub_coarse_ptr, ns + 1, np.int64)
    nrows = int(cptr[-1])
    c_ptr = arr(m.c_ptr, nrows + 1, np.int64)
    nent = int(c_ptr[-1])
    gptr = arr(m.glob_ptr, int(m.n_globs) + 1, np.int64)
    return dict(
        n_dof=int(m.n_dof), n_sub=ns, n_iface=int(m.n_iface), n_coarse=int(m.n_coarse), n_globs=int(m.n_globs),
        n_promoted=int(m.n_promoted), iface_dofs=arr(m.iface_dofs, m.n_iface, np.int64), sub_dof_ptr=sub_dof_ptr,
        sub_dofs=arr(m.sub_dofs, nloc, np.int64), sub_nI=arr(m.sub_nI, ns, np.int64),
        sub_iface=arr(m.sub_iface, nloc, np.int64), sub_wmult=arr(m.sub_wmult, nloc, np.float64),
        sub_coarse_ptr=cptr, sub_coarse=arr(m.sub_coarse, nrows, np.int64), c_ptr=c_ptr,
        c_col=arr(m.c_col, nent, np.int64), c_val=arr(m.c_val, nent, np.float64), glob_ptr=gptr,
        glob_nodes=arr(m.glob_nodes, int(gptr[-1]), np.int64), glob_kind=arr(m.glob_kind, m.n_globs, np.int32),
        glob_promoted=arr(m.glob_promoted, m.n_globs, np.int32),
        coarse_glob=arr(m.coarse_glob, m.n_coarse, np.int64), coarse_comp=arr(m.coarse_comp, m.n_coarse, np.int32))


class _Handle:
    def __init__(self):
        self.h = C.c_void_p()

    def __del__(self):
        try:
            if self.h:
                capi.lib().bddc_free(self.h)
                self.h = C.c_void_p()
        except Exception:
            pass


def analyze(prob, n_levels: Optional[int] = None, constraints: Optional[int] = None, **opts) -> list:
    """Index maps of every BDDC level (no GPU needed): list of dicts of numpy arrays."""
    hm = host_mesh(prob, n_levels)
    o = make_opts(**opts)
    hd = _Handle()
    cons = prob.constraints if constraints is None else constraints
    capi.check(capi.lib().bddc_analyze(C.byref(hm.mesh), C.byref(hm.part), cons, C.byref(o), C.byref(hd.h)))
    out = []
    for lev in range(1, hm.part.n_levels):
        m = capi.LevelMaps()
        capi.check(capi.lib().bddc_get_maps(hd.h, lev, C.byref(m)))
        out.append(_maps_to_numpy(m))
    return out


class BddcSolver:
    """Set-up (Algorithm 1) on construction; solve / apply / grad on CUDA FP64 tensors."""

    def __init__(self, prob, precision: str = "mixed", n_levels: Optional[int] = None,
                 constraints: Optional[int] = None, stream=None, **opts):
        import torch
        self.torch = torch
        self.prob = prob
        self.hm = host_mesh(prob, n_levels)
        self.opts = make_opts(precision=precision, **opts)
        self.hd = _Handle()
        cons = prob.constraints if constraints is None else constraints
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        capi.check(capi.lib().bddc_setup(C.byref(self.hm.mesh), C.byref(self.hm.part), cons, C.byref(self.opts),
                                         C.c_void_p(st.cuda_stream), C.byref(self.hd.h)))
        nf, ni = C.c_int64(), C.c_int64()
        capi.check(capi.lib().bddc_sizes(self.hd.h, C.byref(nf), C.byref(ni)))
        self.n_free, self.n_iface = int(nf.value), int(ni.value)

    @staticmethod
    def _dptr(t) -> C.c_void_p:
        return C.c_void_p(t.data_ptr())

    def _check_vec(self, t, n):
        torch = self.torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected a contiguous CUDA float64 tensor")
        if t.shape[-1] != n:
            raise ValueError(f"last dimension must be {n}")

    def solve(self, rhs, tol: float = 1e-8, allow_not_converged: bool = False):
        """u = K^{-1} f; rhs [n_free] or [nrhs, n_free] CUDA float64."""
        self._check_vec(rhs, self.n_free)
        nrhs = 1 if rhs.dim() == 1 else rhs.shape[0]
        x = self.torch.empty_like(rhs)
        st = capi.Stats()
        allow = (capi.ERR_NOT_CONVERGED,) if allow_not_converged else ()
        capi.check(capi.lib().bddc_solve(self.hd.h, self._dptr(rhs), self._dptr(x), nrhs, float(tol), C.byref(st)),
                   allow)
        self.last_stats = st
        return x

    def solve_host(self, rhs: np.ndarray, tol: float = 1e-8) -> np.ndarray:
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.empty_like(rhs)
        nrhs = 1 if rhs.ndim == 1 else rhs.shape[0]
        st = capi.Stats()
        capi.check(capi.lib().bddc_solve_host(self.hd.h, _ptr(rhs, C.c_double), _ptr(x, C.c_double), nrhs, float(tol),
                                              C.byref(st)))
        self.last_stats = st
        return x

    def apply_precond(self, r):
        self._check_vec(r, self.n_iface)
        z = self.torch.empty_like(r)
        capi.check(capi.lib().bddc_apply_precond(self.hd.h, self._dptr(r), self._dptr(z), 1 if r.dim() == 1 else r.shape[0]))
        return z

    def apply_schur(self, x):
        self._check_vec(x, self.n_iface)
        y = self.torch.empty_like(x)
        capi.check(capi.lib().bddc_apply_schur(self.hd.h, self._dptr(x), self._dptr(y), 1 if x.dim() == 1 else x.shape[0]))
        return y

    def apply_inner_schur(self, x):
        """The mixed form's inner operator S~ (factor products or explicit Schur complement)."""
        self._check_vec(x, self.n_iface)
        y = self.torch.empty_like(x)
        capi.check(capi.lib().bddc_apply_inner_schur(self.hd.h, self._dptr(x), self._dptr(y),
                                                     1 if x.dim() == 1 else x.shape[0]))
        return y

    def grad(self, dJdu, u, tol: float = 1e-10, want_coef: bool = True, want_rhs: bool = True):
        self._check_vec(dJdu, self.n_free)
        self._check_vec(u, self.n_free)
        nrhs = 1 if u.dim() == 1 else u.shape[0]
        torch = self.torch
        gc = torch.empty(self.prob.n_elems, dtype=torch.float64, device=u.device) if want_coef else None
        gr = torch.empty_like(u) if want_rhs else None
        capi.check(capi.lib().bddc_grad(self.hd.h, self._dptr(dJdu), self._dptr(u), nrhs, float(tol),
                                        self._dptr(gc) if gc is not None else None,
                                        self._dptr(gr) if gr is not None else None))
        return gc, gr

    def update_coef(self, coef: np.ndarray):
        c = np.ascontiguousarray(coef, dtype=np.float64)
        capi.check(capi.lib().bddc_update_coef(self.hd.h, _ptr(c, C.c_double)))

    def coarse_matrices(self, level: int = 1) -> list:
        """Local coarse matrices K_Ci of every subdomain of a BDDC level (host numpy, FP64)."""
        m = self.maps(level)
        nc = np.diff(m["sub_coarse_ptr"])
        buf = np.empty(int((nc * nc).sum()), dtype=np.float64)
        capi.check(capi.lib().bddc_get_coarse(self.hd.h, level, _ptr(buf, C.c_double), buf.size))
        out, off = [], 0
        for k in nc:
            out.append(buf[off:off + k * k].reshape(k, k).copy())
            off += k * k
        return out

    def maps(self, level: int = 1) -> dict:
        m = capi.LevelMaps()
        capi.check(capi.lib().bddc_get_maps(self.hd.h, level, C.byref(m)))
        return _maps_to_numpy(m)

    def reset_profile(self):
        capi.check(capi.lib().bddc_reset_profile(self.hd.h))

    def batching_ablation(self) -> dict:
        """Level-1 sweeps and CUDA-core factorisation, batched vs one launch per subdomain (ms)."""
        ms = (C.c_double * 4)()
        capi.check(capi.lib().bddc_batching_ablation(self.hd.h, ms))
        return {"sweep_pair_batched_ms": ms[0], "sweep_pair_per_subdomain_ms": ms[1],
                "cuda_core_factor_batched_ms": ms[2], "cuda_core_factor_per_subdomain_ms": ms[3]}

    def stats(self) -> capi.Stats:
        st = capi.Stats()
        capi.check(capi.lib().bddc_get_stats(self.hd.h, C.byref(st)))
        return st


def _make_autograd():
    import torch

    class BddcSolve(torch.autograd.Function):
        """u = K(coef)^{-1} f as a differentiable op.  Backward: adjoint solve with the same
        BDDC factors, grad_f = lambda, grad_coef_e = -lambda_e^T (K_e / coef_e) u_e."""

        @staticmethod
        def forward(ctx, rhs, coef, solver, tol):
            c = coef.detach().to("cpu", torch.float64).numpy()
            if not np.array_equal(c, solver.hm.coef):
                solver.update_coef(c)
                solver.hm.coef = c.copy()
            u = solver.solve(rhs.contiguous(), tol)
            ctx.solver = solver
            ctx.tol = tol
            ctx.coef_device = coef.device
            ctx.save_for_backward(u)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            (u,) = ctx.saved_tensors
            gc, gr = ctx.solver.grad(grad_u.contiguous(), u, ctx.tol, want_coef=ctx.needs_input_grad[1],
                                     want_rhs=ctx.needs_input_grad[0])
            if gc is not None:
                gc = gc.to(ctx.coef_device)   # the coefficients may live on the host
            return gr, gc, None, None

    return BddcSolve


_autograd_fn = None


def bddc_solve(rhs, coef, solver: BddcSolver, tol: float = 1e-10):
    """Differentiable solve: gradients flow to ``rhs`` and the per-element ``coef``."""
    global _autograd_fn
    if _autograd_fn is None:
        _autograd_fn = _make_autograd()
    return _autograd_fn.apply(rhs, coef, solver, tol)


def tc_update_check(a: np.ndarray, rank: int = 512):
    """a (n x n FP32) with a[i, j] -= sum_{q < rank} a[i, q] a[j, q] on the tile lower triangle of the
    trailing part (rank 256 or 512), through the tensor-core kernels of the factorisation.
    Returns (result, ms)."""
    a = np.ascontiguousarray(a, dtype=np.float32).copy()
    ms = C.c_double()
    capi.check(capi.lib().bddc_tc_update_check(a.shape[0], int(rank), _ptr(a, C.c_float), C.byref(ms)))
    return a, ms.value
