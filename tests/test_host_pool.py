"""The host side of the set-up on its persistent worker pool (no GPU): index analyses started
from several threads at once must give exactly the maps of one analysis run alone.  The pool
runs one parallel region at a time (a second caller waits for the first region to end) and every
region writes its results by item, so the maps cannot depend on which threads take which items or
on how callers interleave; a race in the region hand-over (a worker still in the previous region,
a stale job pointer) would corrupt or mix maps.  Also: the heap-retention option off and on gives
the same maps (it only changes how glibc returns freed memory)."""
import threading

import numpy as np

from paper_1201_5991_gb300 import meshgen, solver


def _flat(maps):
    return [(k, v) for lev in maps for k, v in sorted(lev.items())]


def _same(a, b):
    assert len(a) == len(b)
    for (ka, va), (kb, vb) in zip(a, b):
        assert ka == kb
        if isinstance(va, np.ndarray):
            np.testing.assert_array_equal(va, vb, err_msg=ka)
        else:
            assert va == vb, ka


def test_concurrent_analyses_match_serial():
    probs = [meshgen.elasticity3d(16, 4, seed=3, group=2),          # three levels
             meshgen.elasticity3d_tet(12, 8, seed=1),               # irregular k-means subdomains
             meshgen.stokes_cavity(6, 3)]                            # Stokes, velocities before pressures
    ref = [_flat(solver.analyze(p)) for p in probs]
    out, errors = {}, []

    def work(t):
        try:
            for r in range(3):
                k = (t + r) % len(probs)
                out[(t, r)] = (k, _flat(solver.analyze(probs[k])))
        except Exception as e:   # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(t,)) for t in range(6)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert len(out) == 18
    for k, flat in out.values():
        _same(flat, ref[k])


def test_retain_host_memory_option_keeps_maps():
    p = meshgen.elasticity3d(12, 2, seed=0)
    a = _flat(solver.analyze(p, retain_host_memory=0))
    b = _flat(solver.analyze(p, retain_host_memory=1))
    _same(a, b)
