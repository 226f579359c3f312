"""The allocation-free tracking entry point against the ordinary one.

xt_track_noalloc serves callers that cannot allocate device memory while they
track (an application whose device memory is owned by its own allocator or
budget, or a real-time loop that cannot wait for cudaMalloc): its scratch is
a static device array instead of the tracker's cudaMalloc'd workspace.  It
must give exactly what xt_track gives, call after call, refuse particle
counts above its fixed capacity, and report a cycle-budget stop through
xt_noalloc_status.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import xtgb

pytestmark = pytest.mark.gpu

FIELDS = xtgb.FLOAT_FIELDS + xtgb.INT_FIELDS
MAX_PARTICLES = 1048576  # XT_NOALLOC_MAX_PARTICLES in include/xtgb.h


def _noalloc(tracker, particles, n_turns, start_turn):
    import torch
    L = xtgb.lib()
    L.xt_track_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_void_p]
    L.xt_track_noalloc.restype = ctypes.c_int32
    s = particles.c_struct()
    return L.xt_track_noalloc(tracker.handle, ctypes.byref(s), start_turn, n_turns,
                              torch.cuda.current_stream().cuda_stream)


def test_noalloc_equals_track_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available()
    el, ref = I.lhc_ring(n_cells=20)
    r = np.random.default_rng(31)
    n = 5000 + 13  # ragged tail
    p = I.make_particles(ref, r.normal(0, 4e-3, n), r.normal(0, 2e-5, n), r.normal(0, 4e-3, n),
                         r.normal(0, 2e-5, n), r.normal(0, 0.1, n), r.normal(0, 5e-4, n))
    p["state"][::11] = 0  # some already lost on entry
    ta, tb = xtgb.Tracker(el, ref), xtgb.Tracker(el, ref)
    A, B = xtgb.Particles.from_numpy(p), xtgb.Particles.from_numpy(p)
    for start, turns in ((0, 6), (6, 5)):
        ta.track(A, turns, start)
        assert _noalloc(tb, B, turns, start) == xtgb.XT_OK, xtgb.last_error()
        torch.cuda.synchronize()
        a, b = A.to_numpy(), B.to_numpy()
        for k in FIELDS:
            assert np.array_equal(a[k], b[k]), (start, k)
    assert np.any(a["state"] != 1) and np.any(a["state"] == 1)
    ta.close()
    tb.close()


def test_noalloc_rejects_more_particles_than_its_capacity():
    import torch
    el, ref = I.fodo10()
    tr = xtgb.Tracker(el, ref)
    one = xtgb.Particles.from_numpy(I.make_particles(ref, [0.0], [0.0], [0.0], [0.0], [0.0], [0.0]))
    s = one.c_struct()
    s.n = MAX_PARTICLES + 1  # never dereferenced: the size check comes first
    L = xtgb.lib()
    L.xt_track_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_void_p]
    L.xt_track_noalloc.restype = ctypes.c_int32
    rc = L.xt_track_noalloc(tr.handle, ctypes.byref(s), 0, 1, torch.cuda.current_stream().cuda_stream)
    assert rc == xtgb.XT_ERR_INVALID
    assert "at most 1048576" in xtgb.last_error()
    tr.close()


def test_noalloc_status_reports_a_cycle_budget_stop():
    """A tracker whose cycle budget runs out stops at a turn boundary; the
    allocation-free call records that in the static array's status word,
    xt_noalloc_status returns XT_ERR_TIMEOUT once and then XT_OK, and a
    normal call afterwards reports XT_OK."""
    import torch
    el, ref = I.fodo10()
    p = I.matched_gaussian(el, ref, 2000, 2.5e-6, 3e-4, seed=8)
    L = xtgb.lib()
    L.xt_noalloc_status.argtypes = [ctypes.c_void_p]
    L.xt_noalloc_status.restype = ctypes.c_int32
    stream = torch.cuda.current_stream().cuda_stream
    tr = xtgb.Tracker(el, ref, max_cycles=200000)
    P = xtgb.Particles.from_numpy(p)
    assert _noalloc(tr, P, 200000, 0) == xtgb.XT_OK, xtgb.last_error()
    assert L.xt_noalloc_status(stream) == xtgb.XT_ERR_TIMEOUT
    assert L.xt_noalloc_status(stream) == xtgb.XT_OK
    out = P.to_numpy()
    assert np.all(out["state"] == 1) and np.all((out["at_turn"] > 0) & (out["at_turn"] < 200000))
    tr.close()
    tr = xtgb.Tracker(el, ref)
    P = xtgb.Particles.from_numpy(p)
    assert _noalloc(tr, P, 20, 0) == xtgb.XT_OK, xtgb.last_error()
    assert L.xt_noalloc_status(stream) == xtgb.XT_OK
    tr.close()
