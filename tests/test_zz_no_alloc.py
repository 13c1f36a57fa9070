"""bddc_grad_noalloc through the C ABI: the gradient entry point for callers that cannot let
the library allocate device memory (a caller-owned memory pool holding the device, or a
latency-critical loop that must not hit cudaMalloc / cudaFree).  Its output must match
bddc_grad, call after call, since the fixed scratch array keeps the previous call's contents;
once the handle is warm, a call must leave the device's free memory and the memory in use in
the default pool unchanged.

Collected last on purpose (file name), so a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import ctypes as C
import ctypes.util

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1201_5991_gb300 import capi, meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _default_pool_used():
    """Bytes in use in the current device's default memory pool (cudaMemPoolAttrUsedMemCurrent),
    or None when the CUDA runtime cannot be opened here."""
    for name in (ctypes.util.find_library("cudart"), "libcudart.so", "libcudart.so.13", "libcudart.so.12"):
        if not name:
            continue
        try:
            rt = C.CDLL(name)
            break
        except OSError:
            continue
    else:
        return None
    pool = C.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(C.byref(pool), C.c_int(torch.cuda.current_device())) != 0:
        return None
    used = C.c_uint64()
    attr_used_mem_current = 0x7   # cudaMemPoolAttrUsedMemCurrent
    if rt.cudaMemPoolGetAttribute(pool, C.c_int(attr_used_mem_current), C.byref(used)) != 0:
        return None
    return int(used.value)


def _check_against_grad(p, nrhs, tol):
    s = BddcSolver(p, precision="mixed")
    f = torch.tensor(np.ascontiguousarray(p.f.T), dtype=torch.float64, device="cuda")
    u = s.solve(f, tol=tol)
    w = torch.tensor(np.random.default_rng(8).standard_normal(u.shape), dtype=torch.float64, device="cuda")
    gc_ref, gr_ref = s.grad(w, u, tol=tol)
    L = capi.lib()
    for call in range(2):   # the second call runs on the scratch the first call left behind
        gc = torch.full((p.n_elems,), float("nan"), dtype=torch.float64, device="cuda")
        gr = torch.full_like(u, float("nan"))
        torch.cuda.synchronize()
        free0, used0 = torch.cuda.mem_get_info()[0], _default_pool_used()
        rc = L.bddc_grad_noalloc(s.hd.h, C.c_void_p(w.data_ptr()), C.c_void_p(u.data_ptr()), nrhs, tol,
                                 C.c_void_p(gc.data_ptr()), C.c_void_p(gr.data_ptr()))
        capi.check(rc)
        torch.cuda.synchronize()
        if call == 1:   # the handle is warm: nothing allocated or freed by the call
            assert torch.cuda.mem_get_info()[0] == free0
            if used0 is not None:
                assert _default_pool_used() == used0
        # same adjoint solve, contraction summed in another order: agreement to round-off
        assert _rel(gr, gr_ref) < 1e-12
        assert _rel(gc, gc_ref) < 1e-10


def test_grad_noalloc_matches_grad_on_two_calls():
    _check_against_grad(meshgen.elasticity3d(6, 2, seed=7, nrhs=2), 2, 1e-12)


def test_grad_noalloc_with_prescribed_values():
    # non-zero prescribed displacements: the contraction adds u_d on the prescribed DOFs
    p = meshgen.elasticity3d(6, 2, seed=1, nrhs=2)
    p.dir_values = np.where(p.dirichlet == 1, np.random.default_rng(4).standard_normal(p.dirichlet.size), 0.0)
    _check_against_grad(p, 2, 1e-12)
