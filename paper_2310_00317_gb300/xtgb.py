"""Python binding of ``libxtgb.so`` (argument marshalling only).

Every step of the tracking path runs in the library's CUDA kernels; this
module only converts numpy/torch objects to the C structures of
``include/xtgb.h`` and raises on error codes.  PyTorch provides device memory
and streams.  There is no CPU fallback: if the library is missing or no GPU
is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build
from .inputs import ELEMENT_DTYPE

XT_OK, XT_ERR_INVALID, XT_ERR_UNSUPPORTED, XT_ERR_CUDA, XT_ERR_TIMEOUT, XT_ERR_CANCELLED, XT_ERR_NOMEM = (
    0, -1, -2, -3, -4, -5, -6)
RAD_OFF, RAD_MEAN, RAD_QUANTUM = 0, 1, 2

FLOAT_FIELDS = ("x", "px", "y", "py", "zeta", "delta", "ptau", "rpp", "rvv")
INT_FIELDS = ("state", "at_turn", "at_element")
ALL_FIELDS = FLOAT_FIELDS + INT_FIELDS + ("particle_id",)


class XtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("xtgb error %d: %s" % (code, msg))
        self.code = code


class _Particles(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ALL_FIELDS] + [("n", ctypes.c_int64)]


class _Reference(ctypes.Structure):
    _fields_ = [("mass0", ctypes.c_double), ("q0", ctypes.c_double), ("p0c", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("radiation", ctypes.c_int32), ("block", ctypes.c_int32),
                ("chunk_bytes", ctypes.c_int32), ("segment_turns", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("max_cycles", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Loads the in-tree library (build it with ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("libxtgb.so is not built (%s); run __graft_entry__.build()" % path)
            L = ctypes.CDLL(path)
            P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            L.xt_options_default.argtypes = [P]
            L.xt_options_default.restype = None
            L.xt_last_error.restype = ctypes.c_char_p
            L.xt_version.restype = ctypes.c_char_p
            L.xt_tracker_create.argtypes = [P, i64, P, P, P]
            L.xt_tracker_destroy.argtypes = [P]
            L.xt_tracker_destroy.restype = None
            L.xt_tracker_set_options.argtypes = [P, P]
            L.xt_tracker_get_options.argtypes = [P, P]
            L.xt_track.argtypes = [P, P, i64, i64, P]
            L.xt_track_host.argtypes = [P, P, i64, i64, P]
            L.xt_sync_status.argtypes = [P, P]
            L.xt_cancel.argtypes = [P]
            L.xt_reset_cancel.argtypes = [P]
            L.xt_element_flops.argtypes = [P, P, i64]
            L.xt_autotune.argtypes = [P, P, i64, P]
            L.xt_refine_losses.argtypes = [P, P, ctypes.c_double, ctypes.c_int32, P, P]
            L.xt_track_monitor.argtypes = [P, P, ctypes.c_int64, P, P]
            L.xt_track_batched.argtypes = [P, P, i32, i64, i64, i32, P]
            L.xt_batched_sync_status.argtypes = [P, P, i32, P]
            L.xt_set_profiling.argtypes = [P, i32]
            L.xt_kernel_time.argtypes = [P, P, P]
            L.xt_fp64_peak.argtypes = [P, P, P]
            L.xt_batched_release.argtypes = []
            L.xt_batched_release.restype = None
            for name in ("xt_tracker_create", "xt_tracker_set_options", "xt_tracker_get_options",
                         "xt_track", "xt_track_host", "xt_sync_status", "xt_cancel", "xt_reset_cancel",
                         "xt_element_flops", "xt_autotune", "xt_track_batched", "xt_batched_sync_status",
                         "xt_set_profiling", "xt_kernel_time", "xt_fp64_peak", "xt_refine_losses"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def _check(code: int) -> int:
    if code != XT_OK:
        raise XtError(code, lib().xt_last_error().decode())
    return code


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def last_error() -> str:
    return lib().xt_last_error().decode()


def version() -> str:
    return lib().xt_version().decode()


# ----------------------------------------------------------------------------
class Particles:
    """Particle arrays (SoA) as torch tensors on one device."""

    def __init__(self, tensors: dict):
        self.t = tensors
        self.n = int(tensors["x"].shape[0])

    @classmethod
    def from_numpy(cls, d: dict, device="cuda") -> "Particles":
        import torch
        t = {}
        for k in FLOAT_FIELDS:
            t[k] = torch.as_tensor(np.ascontiguousarray(d[k], dtype=np.float64)).to(device)
        for k in INT_FIELDS:
            t[k] = torch.as_tensor(np.ascontiguousarray(d[k], dtype=np.int32)).to(device)
        t["particle_id"] = torch.as_tensor(np.ascontiguousarray(d["particle_id"], dtype=np.int64)).to(device)
        return cls(t)

    def to_numpy(self) -> dict:
        return {k: v.cpu().numpy() for k, v in self.t.items()}

    def clone(self) -> "Particles":
        return Particles({k: v.clone() for k, v in self.t.items()})

    def c_struct(self) -> _Particles:
        s = _Particles()
        for k in ALL_FIELDS:
            v = self.t[k]
            assert v.is_contiguous() and v.shape[0] == self.n
            setattr(s, k, v.data_ptr())
        s.n = self.n
        return s


class HostParticles:
    """Particle arrays (SoA) as numpy arrays in host memory."""

    def __init__(self, d: dict, copy: bool = True):
        """Copies the arrays unless copy=False and they already have the right
        dtype and layout (then results are written into the caller's arrays)."""
        self.a = {k: np.array(d[k], dtype=(np.float64 if k in FLOAT_FIELDS else
                                           np.int64 if k == "particle_id" else np.int32),
                              copy=copy, order="C")
                  for k in ALL_FIELDS}
        self.n = int(self.a["x"].shape[0])

    def c_struct(self) -> _Particles:
        s = _Particles()
        for k in ALL_FIELDS:
            setattr(s, k, self.a[k].ctypes.data)
        s.n = self.n
        return s


def options_default() -> dict:
    o = _Options()
    lib().xt_options_default(ctypes.byref(o))
    return {f: getattr(o, f) for f, _ in _Options._fields_}


class Tracker:
    """Owns an ``xt_tracker`` compiled from a lattice table (numpy rows)."""

    def __init__(self, table, ref, radiation: int = RAD_OFF, block: int = 0, chunk_bytes: int = 0,
                 segment_turns: int = 0, seed: int = 0, max_cycles: int = 0):
        self._h = ctypes.c_void_p()
        self.table = np.ascontiguousarray(table, dtype=ELEMENT_DTYPE)
        self.ref = tuple(float(v) for v in ref)
        o = _Options(radiation, block, chunk_bytes, segment_turns, seed, max_cycles)
        r = _Reference(*self.ref)
        _check(lib().xt_tracker_create(self.table.ctypes.data, self.table.shape[0], ctypes.byref(r),
                                       ctypes.byref(o), ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().xt_tracker_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def options(self) -> dict:
        o = _Options()
        _check(lib().xt_tracker_get_options(self._h, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in _Options._fields_}

    def set_options(self, **kw):
        o = _Options()
        _check(lib().xt_tracker_get_options(self._h, ctypes.byref(o)))
        for k, v in kw.items():
            setattr(o, k, v)
        _check(lib().xt_tracker_set_options(self._h, ctypes.byref(o)))

    def track(self, particles: Particles, n_turns: int, start_turn: int = 0, stream=None):
        s = particles.c_struct()
        _check(lib().xt_track(self._h, ctypes.byref(s), start_turn, n_turns, _stream_handle(stream)))

    def track_host(self, particles: HostParticles, n_turns: int, start_turn: int = 0, stream=None):
        s = particles.c_struct()
        _check(lib().xt_track_host(self._h, ctypes.byref(s), start_turn, n_turns, _stream_handle(stream)))

    def sync_status(self, stream=None) -> int:
        """Returns XT_OK, XT_ERR_TIMEOUT or XT_ERR_CANCELLED (does not raise for those)."""
        return lib().xt_sync_status(self._h, _stream_handle(stream))

    def cancel(self):
        _check(lib().xt_cancel(self._h))

    def reset_cancel(self):
        _check(lib().xt_reset_cancel(self._h))

    def element_flops(self) -> np.ndarray:
        out = np.zeros(self.table.shape[0], dtype=np.int64)
        _check(lib().xt_element_flops(self._h, out.ctypes.data, out.shape[0]))
        return out

    def set_profiling(self, enable: bool):
        _check(lib().xt_set_profiling(self._h, 1 if enable else 0))

    def kernel_time(self):
        """(summed duration [ms], launches) of the tracking kernels since the last query."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().xt_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def refine_losses(self, particles: Particles, ds: float, n_angles: int = 128, stream=None):
        """Loss positions [m from the start of the table] of the particles
        lost at apertures, to within ds, as a CUDA float64 tensor (NaN for the
        others); see xt_refine_losses."""
        import torch
        out = torch.empty(particles.n, dtype=torch.float64, device=particles.t["x"].device)
        s = particles.c_struct()
        _check(lib().xt_refine_losses(self._h, ctypes.byref(s), float(ds), int(n_angles), out.data_ptr(),
                                      _stream_handle(stream)))
        return out

    def monitor(self, particles: Particles, turn: int = 0, stream=None):
        """One pass of the table with the particles' state after every row:
        a CUDA float64 tensor [n_elements, 8, n] of (x, px, y, py, zeta, ptau,
        delta, state); the particles advance by one turn as in track()."""
        import torch
        out = torch.empty((self.table.shape[0], 8, particles.n), dtype=torch.float64, device=particles.t["x"].device)
        s = particles.c_struct()
        _check(lib().xt_track_monitor(self._h, ctypes.byref(s), int(turn), out.data_ptr(), _stream_handle(stream)))
        return out

    def autotune(self, probe: Particles, probe_turns: int, stream=None) -> dict:
        s = probe.c_struct()
        _check(lib().xt_autotune(self._h, ctypes.byref(s), probe_turns, _stream_handle(stream)))
        return self.options


def _batch_structs(trackers, particles):
    n = len(trackers)
    H = (ctypes.c_void_p * n)(*[t.handle.value for t in trackers])
    P = (_Particles * n)(*[p.c_struct() for p in particles])
    return H, P, n


def track_batched(trackers, particles, n_turns: int, start_turn: int = 0, graph: bool = True, stream=None):
    """All seeds in one persistent launch per segment (captured in a CUDA graph)."""
    H, P, n = _batch_structs(trackers, particles)
    _check(lib().xt_track_batched(H, P, n, start_turn, n_turns, 1 if graph else 0, _stream_handle(stream)))


def batched_sync_status(trackers, particles, stream=None) -> int:
    H, P, n = _batch_structs(trackers, particles)
    return lib().xt_batched_sync_status(H, P, n, _stream_handle(stream))


def fp64_peak(stream=None):
    """Measured FP64 fma throughput of the current device [flop/s]."""
    f = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().xt_fp64_peak(ctypes.byref(f), ctypes.byref(ms), _stream_handle(stream)))
    return f.value


def batched_release():
    lib().xt_batched_release()


# C-ABI names
def tracker_create(table, ref, **options) -> Tracker:
    return Tracker(table, ref, **options)


def tracker_destroy(tracker: Tracker):
    tracker.close()


def track(tracker: Tracker, particles: Particles, n_turns: int, start_turn: int = 0, stream=None):
    tracker.track(particles, n_turns, start_turn, stream)


def track_host(tracker: Tracker, particles: HostParticles, n_turns: int, start_turn: int = 0, stream=None):
    tracker.track_host(particles, n_turns, start_turn, stream)


def autotune(tracker: Tracker, probe: Particles, probe_turns: int, stream=None) -> dict:
    return tracker.autotune(probe, probe_turns, stream)


def traversed_elements(particles: dict, n_el: int, start_turn: int, n_turns: int,
                       state_before: np.ndarray | None = None) -> int:
    """Particle-element passes made during a call (the throughput metric's
    counting rule): survivors n_turns * n_el; a particle lost at (turn, element)
    (turn - start_turn) * n_el + element + 1; particles lost before the call 0."""
    st = particles["state"]
    at = particles["at_turn"].astype(np.int64)
    ae = particles["at_element"].astype(np.int64)
    alive_before = np.ones(st.shape, bool) if state_before is None else (state_before == 1)
    surv = (st == 1) & alive_before
    lost = (st != 1) & alive_before
    return int(surv.sum()) * n_turns * n_el + int(((at[lost] - start_turn) * n_el + ae[lost] + 1).sum())


# ----------------------------------------------------------------------------
# Dynamic-aperture surrogate network and scan glue.
XS_N_PARAMS = 202242
XS_STATE_PREDICTED = 2
XS_STATE_SURVIVED = 3
XS_WIDEN_INWARD = 1
XS_WIDEN_VERIFY = 2
_xs_ready = False


def _xs_lib():
    global _xs_ready
    L = lib()
    if not _xs_ready:
        P, i32, i64, u64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
        L.xs_mlp_create.argtypes = [u64, P]
        L.xs_mlp_destroy.argtypes = [P]
        L.xs_mlp_destroy.restype = None
        L.xs_mlp_set_params.argtypes = [P, P, i64, P]
        L.xs_mlp_get_params.argtypes = [P, P, i64, P]
        L.xs_mlp_forward.argtypes = [P, P, P, i64, P]
        L.xs_mlp_loss_grad.argtypes = [P, P, P, P, P, i64, f32, P, P, P]
        L.xs_mlp_train_step.argtypes = [P, P, P, P, P, i64, f32, f32, P, P]
        L.xs_last_error.restype = ctypes.c_char_p
        L.xs_da_select.argtypes = [P, i32, i32, f32, i32, i32, P, P, P, P, P]
        L.xs_da_combine.argtypes = [P, P, i32, i32, P, P, P]
        L.xs_da_last_error.restype = ctypes.c_char_p
        for n in ("xs_mlp_create", "xs_mlp_set_params", "xs_mlp_get_params", "xs_mlp_forward",
                  "xs_mlp_loss_grad", "xs_mlp_train_step", "xs_da_select", "xs_da_combine"):
            getattr(L, n).restype = i32
        _xs_ready = True
    return L


def _xs_check(code, which="xs_last_error"):
    if code != XT_OK:
        raise XtError(code, getattr(_xs_lib(), which)().decode())


def _ptr(t):
    return None if t is None else t.data_ptr()


class Surrogate:
    """The surrogate network (``xs_mlp``): FP32 master weights on the device."""

    def __init__(self, seed: int = 0):
        self._h = ctypes.c_void_p()
        _xs_check(_xs_lib().xs_mlp_create(seed, ctypes.byref(self._h)))

    def close(self):
        if self._h:
            _xs_lib().xs_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _xs_check(_xs_lib().xs_mlp_set_params(self._h, a.ctypes.data, a.shape[0], _stream_handle(None)))

    def get_params(self) -> np.ndarray:
        a = np.zeros(XS_N_PARAMS, dtype=np.float32)
        _xs_check(_xs_lib().xs_mlp_get_params(self._h, a.ctypes.data, a.shape[0], _stream_handle(None)))
        return a

    def forward(self, X):
        """X: CUDA float32 tensor (B, 16) -> (B, 2)."""
        import torch
        X = X.contiguous()
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _xs_check(_xs_lib().xs_mlp_forward(self._h, X.data_ptr(), out.data_ptr(), X.shape[0],
                                           _stream_handle(None)))
        return out

    def loss_grad(self, X, y, t, mask, lam: float):
        import torch
        g = torch.empty(XS_N_PARAMS, dtype=torch.float32, device=X.device)
        L = torch.empty(1, dtype=torch.float32, device=X.device)
        _xs_check(_xs_lib().xs_mlp_loss_grad(self._h, _ptr(X.contiguous()), _ptr(y), _ptr(t), _ptr(mask),
                                             X.shape[0], lam, g.data_ptr(), L.data_ptr(), _stream_handle(None)))
        return L, g

    def train_step(self, X, y, t, mask, lr: float, lam: float, loss_out=None):
        _xs_check(_xs_lib().xs_mlp_train_step(self._h, _ptr(X), _ptr(y), _ptr(t), _ptr(mask), X.shape[0],
                                              lr, lam, _ptr(loss_out), _stream_handle(None)))


def da_select(out2, n_rays: int, n_r: int, p_lo: float, margin: int, window: int, state, r_lo, widen=None,
              da_prev=None):
    _xs_check(_xs_lib().xs_da_select(_ptr(out2), n_rays, n_r, p_lo, margin, window, _ptr(widen), _ptr(da_prev),
                                     _ptr(state), _ptr(r_lo), _stream_handle(None)), "xs_da_last_error")


def da_combine(out2, state, n_rays: int, n_r: int, da, widen=None):
    _xs_check(_xs_lib().xs_da_combine(_ptr(out2), _ptr(state), n_rays, n_r, _ptr(da), _ptr(widen),
                                      _stream_handle(None)), "xs_da_last_error")
