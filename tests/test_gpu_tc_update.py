"""The tensor-core trailing update of the mixed factorisation (two row-scaled FP16 parts, three
tcgen05 products, FP32 accumulation) against an FP64 product, through bddc_tc_update_check.

Error bound of the scheme, entry by entry, for C - P P^T with K = 256 or 512 panel columns (the
rank-256 update of a super-panel's second half and the rank-512 trailing update): each entry a
of a row scaled into [2^14, 2^15) is split as a = hi + 2^-11 lo + r with |r| <= 2^-22 |a|, the
dropped lo lo term is at most 2^-22 |a||b|, and the FP32 accumulation (tensor-core MMAs of K = 16,
then FP32 adds of every 64-wide chunk) adds at most about 2 (K + 16) 2^-24 sum_q |a_q||b_q|.  So
    |fl(c_ij) - c_ij| <= (3 2^-22 + 2 (K + 16) 2^-24) sum_q |p_iq| |p_jq| + 2^-24 |c_ij|.
A dropped or mis-signed cross product or a mis-scaled low part gives about 2^-11 sum |p||p|, a
wrong row scale O(1); both are far above the bound.  Norm-wise the error must stay within a few
times that of an FP32 GEMM of the same data.  The entries outside the updated tile triangle must
come back unchanged."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_1201_5991_gb300.solver import tc_update_check

pytestmark = pytest.mark.gpu


def _factor_like(n, K, seed):
    # panel rows spanning four decades (as factor rows of a stiffness matrix with E in [1, 1e3])
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)).astype(np.float32)
    rows = (10.0 ** rng.uniform(-2, 2, size=n)).astype(np.float32)
    a[:, :K] *= rows[:, None]
    return a


@pytest.mark.parametrize("K,n", [(256, 64 * 5), (256, 64 * 12), (256, 64 * 21),
                                 (512, 64 * 9), (512, 64 * 16), (512, 64 * 25)])
def test_split_update_error_bound(K, n):
    a = _factor_like(n, K, seed=n)
    out, ms = tc_update_check(a, rank=K)
    P = a[:, :K].astype(np.float64)
    exact = a.astype(np.float64) - P @ P.T
    absprod = np.abs(P) @ np.abs(P).T
    gamma = 3 * 2.0 ** -22 + 2 * (K + 16) * 2.0 ** -24
    tiles = np.arange(n) // 64
    upd = (tiles[:, None] >= tiles[None, :]) & (np.arange(n)[:, None] >= K) & (np.arange(n)[None, :] >= K)
    err = np.abs(out.astype(np.float64) - exact)
    bound = gamma * absprod + 2.0 ** -24 * np.abs(exact)
    assert np.all(err[upd] <= bound[upd]), float((err[upd] / bound[upd]).max())
    np.testing.assert_array_equal(out[~upd], a[~upd])
    rel = float((err[upd] / absprod[upd]).max())
    # norm-wise against an FP32 GEMM of the same panel (BLAS sgemm, FMA accumulation): the split
    # keeps about one FP32 rounding more per product, so at most a few times the FP32 error
    P32 = a[:, :K]
    e32 = np.abs((a - P32 @ P32.T).astype(np.float64) - exact)
    ratio = float(np.linalg.norm(err[upd]) / np.linalg.norm(e32[upd]))
    print(f"K={K} n={n}: max |error| / sum |p||p| = {rel:.2e} (bound {gamma:.2e}); "
          f"||error|| / ||FP32 GEMM error|| = {ratio:.2f}; update {ms:.3f} ms")
    assert ratio < 4.0
