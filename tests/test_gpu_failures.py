"""Failure detection without a GPU fault: the error codes the C ABI documents for a breakdown of a
subdomain factorisation and for a bounded device-side wait that gives up, made on the host.

* BDDC_ERR_BREAKDOWN: the elements of one subdomain get Young's modulus 1e40.  Their element and
  local matrices are finite in FP64, but the mixed form stores the subdomain factor in FP32, whose
  range ends at 3.4e38: the densified tiles overflow, the pivots of that subdomain become NaN and
  the factorisation flags that subdomain (and only it: the other local matrices hold only their
  own elements).  The library must name the level and the subdomain, keep the CUDA context usable
  and, after bddc_update_coef with sane coefficients, solve again.
* BDDC_ERR_TIMEOUT: the test-only option wait_probe makes every wait of the streaming sweeps for a
  published solution block poll a device word that nothing sets, with a short limit.  Each wait then takes its
  error path (flag the timeout, stage the block as it is, go on), so every tile copy is still
  consumed and the sweep ends by itself; the host must report BDDC_ERR_TIMEOUT, and a later
  handle on the same context must solve correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem
from paper_1201_5991_gb300 import capi, meshgen
from paper_1201_5991_gb300.solver import BddcSolver

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _overflowing(p, sub):
    coef = p.coef.copy()
    coef[p.parts[0] == sub] = 1e40
    return coef


def test_breakdown_reports_level_and_subdomain():
    p = meshgen.elasticity3d(12, 2, seed=0)
    ref = fem.direct_solve(p)[:, 0]
    bad_sub = 5
    # at set-up: the handle is not created, the message names level 1 and the subdomain
    q = meshgen.elasticity3d(12, 2, seed=0)
    q.coef = _overflowing(q, bad_sub)
    with pytest.raises(capi.BddcError) as ei:
        BddcSolver(q, precision="mixed")
    assert ei.value.code == capi.ERR_BREAKDOWN
    assert "level 1 subdomain 5" in str(ei.value)
    # on an existing handle: bddc_update_coef fails, the statistics name the level and subdomain
    s = BddcSolver(p, precision="mixed")
    with pytest.raises(capi.BddcError) as ei:
        s.update_coef(_overflowing(p, bad_sub))
    assert ei.value.code == capi.ERR_BREAKDOWN
    st = s.stats()
    assert (st.breakdown_level, st.breakdown_sub) == (1, bad_sub)
    with pytest.raises(capi.BddcError) as ei:   # no numeric set-up until the next successful one
        s.solve(_dev(p.f[:, 0]), tol=1e-12)
    assert ei.value.code == capi.ERR_INVALID
    s.update_coef(p.coef)
    u = s.solve(_dev(p.f[:, 0]), tol=1e-12).cpu().numpy()
    assert _rel(u, ref) < 1e-8


def test_bounded_wait_reports_timeout():
    p = meshgen.elasticity3d(12, 2, seed=0)   # 6^3-element subdomains: several block rows per sweep
    ref = fem.direct_solve(p)[:, 0]
    f = _dev(p.f[:, 0])
    # FP64 form without autotuning runs no sweep at set-up: the solve meets the probe
    s = BddcSolver(p, precision="fp64", autotune=0, wait_probe=1)
    with pytest.raises(capi.BddcError) as ei:
        s.solve(f, tol=1e-10)
    assert ei.value.code == capi.ERR_TIMEOUT
    assert "bounded device-side wait" in str(ei.value)
    # mixed form: the set-up's own sweeps (refinement probe, autotuner) meet it
    with pytest.raises(capi.BddcError) as ei:
        BddcSolver(p, precision="mixed", wait_probe=1)
    assert ei.value.code == capi.ERR_TIMEOUT
    # the context is still usable: fresh handles solve correctly
    for prec in ("fp64", "mixed"):
        u = BddcSolver(p, precision=prec).solve(f, tol=1e-12).cpu().numpy()
        assert _rel(u, ref) < 1e-8
    torch.cuda.synchronize()
