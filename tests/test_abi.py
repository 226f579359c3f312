"""The C-ABI library builds, loads on a machine without a GPU and exports
every entry point that include/xtgb.h declares; argument validation happens
before any CUDA call (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2310_00317_gb300 import build, inputs as I, xtgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return xtgb.lib()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "xtgb.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(xt_[a-z_0-9]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s


def test_options_default_and_version(L):
    o = xtgb.options_default()
    assert o == dict(radiation=0, block=0, chunk_bytes=0, segment_turns=0, seed=0, max_cycles=0)
    assert "sm_103a" in xtgb.version()


def test_create_rejects_bad_arguments_before_cuda(L):
    el, ref = I.fodo10()
    h = ctypes.c_void_p()
    r = xtgb._Reference(*ref)
    # null table
    assert L.xt_tracker_create(None, 10, ctypes.byref(r), None, ctypes.byref(h)) == xtgb.XT_ERR_INVALID
    # zero elements
    assert L.xt_tracker_create(el.ctypes.data, 0, ctypes.byref(r), None, ctypes.byref(h)) == xtgb.XT_ERR_INVALID
    # bad reference
    bad = xtgb._Reference(0.0, 1.0, 1e9)
    assert L.xt_tracker_create(el.ctypes.data, el.shape[0], ctypes.byref(bad), None,
                               ctypes.byref(h)) == xtgb.XT_ERR_INVALID
    # bad options
    o = xtgb._Options(3, 0, 0, 0, 0, 0)
    assert L.xt_tracker_create(el.ctypes.data, el.shape[0], ctypes.byref(r), ctypes.byref(o),
                               ctypes.byref(h)) == xtgb.XT_ERR_INVALID
    o = xtgb._Options(0, 48, 0, 0, 0, 0)
    assert L.xt_tracker_create(el.ctypes.data, el.shape[0], ctypes.byref(r), ctypes.byref(o),
                               ctypes.byref(h)) == xtgb.XT_ERR_INVALID
    assert "block" in xtgb.last_error()
    # unsupported order / type
    t = el.copy()
    t[1]["order"] = 11
    assert L.xt_tracker_create(t.ctypes.data, t.shape[0], ctypes.byref(r), None,
                               ctypes.byref(h)) == xtgb.XT_ERR_UNSUPPORTED
    t = el.copy()
    t[2]["type"] = 42
    assert L.xt_tracker_create(t.ctypes.data, t.shape[0], ctypes.byref(r), None,
                               ctypes.byref(h)) == xtgb.XT_ERR_UNSUPPORTED
    assert not h.value


def test_track_rejects_null_tracker(L):
    p = xtgb._Particles()
    assert L.xt_track(None, ctypes.byref(p), 0, 1, None) == xtgb.XT_ERR_INVALID
    assert L.xt_track_batched(None, None, 0, 0, 1, 1, None) == xtgb.XT_ERR_INVALID


def test_traversed_element_count():
    p = dict(state=np.array([1, 0, -2, 1], np.int32), at_turn=np.array([7, 5, 6, 3], np.int32),
             at_element=np.array([0, 10, 0, 0], np.int32))
    before = np.array([1, 1, 1, 0], np.int32)
    # survivor: 2 turns x 20; lost at (5,10): 0*20+11; lost at (6,0): 20+1; not alive before: 0
    assert xtgb.traversed_elements(p, 20, 5, 2, before) == 40 + 11 + 21


def test_create_rejects_bad_element_parameters_before_cuda(L):
    """Every parameter rule of the element rows is checked by the lattice
    compiler before any CUDA call: XT_ERR_INVALID, with the row named."""
    el, ref = I.fodo10()
    r = xtgb._Reference(*ref)
    bad_rows = [
        I.quadrupole(0.1, -1.0),                      # negative length
        I.quadrupole(float("nan"), 1.0),              # non-finite gradient
        I._row(I.BEND, 0, [0.1, 0.1, 1.0, 0.0, 2.0]),  # unknown model
        I.bend(0.1, 0.1, 1.0, k1=0.2, full=True, kicks=65),   # too many gradient kicks
        I._row(I.BEND, 0, [0.1, 0.1, 1.0, 0.2, 1.0, 1.5]),  # a fractional number of kicks
        I.bend(0.1, 0.1, -1.0),                       # negative length
        I.bend(0.1, float("inf"), 1.0),               # non-finite curvature
        I._row(I.DIPEDGE, 0, [0.1, 0.1, 0.0, 0.0, 3.0, 0.0]),  # unknown edge model
        I._row(I.DIPEDGE, 0, [0.1, 0.1, 0.0, 0.0, 1.0, 3.0]),  # unknown face
        I.spacecharge(1e10, 0.0, 0.0, 1e-3, 1.0),     # zero sigma_x
        I.spacecharge(-1e10, 0.0, 1e-3, 1e-3, 1.0),   # negative line density
        I.spacecharge(1e10, -0.1, 1e-3, 1e-3, 1.0),   # negative sigma_z
        I.beambeam4d(1e11, 1.5, 1e-3, 1e-3),          # beta_s > 1
        I.aperture_ellipse(0.0, 0.01),                # zero semi-axis
        I.aperture_rect(0.01, -0.01, -0.01, 0.01),    # x_min > x_max
    ]
    for row in bad_rows:
        t = I.table(list(el)[:3] + [row] + list(el)[3:])
        h = ctypes.c_void_p()
        rc = L.xt_tracker_create(t.ctypes.data, t.shape[0], ctypes.byref(r), None, ctypes.byref(h))
        assert rc == xtgb.XT_ERR_INVALID, (row, rc)
        assert "element 3" in xtgb.last_error(), xtgb.last_error()
        assert not h.value


def test_every_call_rejects_null_arguments_before_cuda(L):
    """Each entry point checks its pointers and sizes first and returns
    XT_ERR_INVALID with a message, without touching CUDA (this machine has no
    GPU, so any CUDA call would fail with a different code)."""
    P = ctypes.c_void_p
    i32, i64, u64, dbl, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_float
    sig = {
        "xt_track_host": [P, P, i64, i64, P], "xt_sync_status": [P, P], "xt_cancel": [P], "xt_reset_cancel": [P],
        "xt_set_profiling": [P, i32], "xt_kernel_time": [P, P, P], "xt_fp64_peak": [P, P, P],
        "xt_refine_losses": [P, P, dbl, i32, P, P], "xt_track_monitor": [P, P, i64, P, P],
        "xt_element_flops": [P, P, i64], "xt_autotune": [P, P, i64, P], "xt_batched_sync_status": [P, P, i32, P],
        "xt_track_noalloc": [P, P, i64, i64, P], "xt_tracker_set_options": [P, P], "xt_tracker_get_options": [P, P],
        "xs_mlp_create": [u64, P], "xs_mlp_set_params": [P, P, i64, P], "xs_mlp_get_params": [P, P, i64, P],
        "xs_mlp_forward": [P, P, P, i64, P], "xs_da_select": [P, i32, i32, f32, i32, i32, P, P, P, P, P],
        "xs_da_combine": [P, P, i32, i32, P, P, P],
    }
    # a CDLL object of its own, so these prototypes do not replace the binding's
    C = ctypes.CDLL(xtgb.library_path())
    for name, args in sig.items():
        f = getattr(C, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    p = xtgb._Particles()  # all pointers null, n = 0
    o = xtgb._Options()
    d, k = ctypes.c_double(), ctypes.c_int64()
    calls = [
        ("xt_track_host", (None, ctypes.byref(p), 0, 1, None)),
        ("xt_sync_status", (None, None)),
        ("xt_cancel", (None,)),
        ("xt_reset_cancel", (None,)),
        ("xt_set_profiling", (None, 1)),
        ("xt_kernel_time", (None, ctypes.byref(d), ctypes.byref(k))),
        ("xt_fp64_peak", (None, None, None)),
        ("xt_refine_losses", (None, ctypes.byref(p), 0.01, 128, None, None)),
        ("xt_track_monitor", (None, ctypes.byref(p), 0, None, None)),
        ("xt_element_flops", (None, None, 0)),
        ("xt_autotune", (None, ctypes.byref(p), 2, None)),
        ("xt_batched_sync_status", (None, None, 0, None)),
        ("xt_track_noalloc", (None, ctypes.byref(p), 0, 1, None)),
        ("xt_tracker_set_options", (None, ctypes.byref(o))),
        ("xt_tracker_get_options", (None, ctypes.byref(o))),
        ("xs_mlp_create", (1, None)),
        ("xs_mlp_set_params", (None, None, 202242, None)),
        ("xs_mlp_get_params", (None, None, 202242, None)),
        ("xs_mlp_forward", (None, None, None, 16, None)),
        ("xs_da_select", (None, 9, 40, 0.2, 5, 5, None, None, None, None, None)),
        ("xs_da_combine", (None, None, 9, 40, None, None, None)),
    ]
    for name, args in calls:
        rc = getattr(C, name)(*args)
        assert rc == xtgb.XT_ERR_INVALID, (name, rc)
