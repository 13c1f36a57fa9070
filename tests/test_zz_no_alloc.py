"""bddc_grad_noalloc through the C ABI: the gradient entry point for callers that cannot let
the library allocate device memory (a caller-owned memory pool holding the device, or a
latency-critical loop that must not hit cudaMalloc / cudaFree).  Its output must match
bddc_grad, call after call, since the fixed scratch array keeps the previous call's contents.

Collected last on purpose (file name), so a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1201_5991_gb300 import capi, meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_grad_noalloc_matches_grad_on_two_calls():
    p = meshgen.elasticity3d(6, 2, seed=7, nrhs=2)
    s = BddcSolver(p, precision="mixed")
    f = torch.tensor(np.ascontiguousarray(p.f.T), dtype=torch.float64, device="cuda")
    u = s.solve(f, tol=1e-12)
    w = torch.tensor(np.random.default_rng(8).standard_normal(u.shape), dtype=torch.float64, device="cuda")
    gc_ref, gr_ref = s.grad(w, u, tol=1e-12)
    L = capi.lib()
    for _ in range(2):   # the second call runs on the scratch the first call left behind
        gc = torch.full((p.n_elems,), float("nan"), dtype=torch.float64, device="cuda")
        gr = torch.full_like(u, float("nan"))
        rc = L.bddc_grad_noalloc(s.hd.h, C.c_void_p(w.data_ptr()), C.c_void_p(u.data_ptr()), 2, 1e-12,
                                 C.c_void_p(gc.data_ptr()), C.c_void_p(gr.data_ptr()))
        capi.check(rc)
        # same adjoint solve, contraction summed in another order: agreement to round-off
        assert _rel(gr, gr_ref) < 1e-12
        assert _rel(gc, gc_ref) < 1e-10
