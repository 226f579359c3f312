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
        I.bend(0.1, 0.1, 1.0, k1=0.2, full=True),     # gradient in the full model
        I.bend(0.1, 0.1, -1.0),                       # negative length
        I.bend(0.1, float("inf"), 1.0),               # non-finite curvature
        I._row(I.DIPEDGE, 0, [0.1, 0.1, 0.0, 0.0, 2.0, 0.0]),  # unknown edge model
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
