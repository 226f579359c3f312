"""Oracle tracker (test infrastructure only).

A plain, slow, single-threaded FP64 CPU implementation of the tracking path of
the Xsuite paper (section "Lattice modelling and single particle tracking"),
written in ``xtoracle.cpp`` and loaded here through ctypes.  It is the
independent reference that the CUDA tracker is checked against.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
in ``paper_2310_00317_gb300``; the two meet only through the flat lattice
table layout (type, order, 48 parameters) and the particle arrays.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "xtoracle.cpp")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_FUSED = os.path.join(_BUILD, "liboracle_fused.so")
_lock = threading.Lock()
_lib = None
_lib_fused = None

# Lattice-table row: the same memory layout the library's public header uses.
ELEMENT_DTYPE = np.dtype([("type", "<i4"), ("order", "<i4"), ("p", "<f8", (48,))], align=True)
DRIFT, MULTIPOLE, CAVITY, DIPEDGE, LINEARMAP, APERTURE, MARKER = 1, 2, 3, 4, 5, 6, 0
XYSHIFT, SROTATION, APERTURE_RECT, APERTURE_ELLIPSE = 7, 8, 9, 10
BEAMBEAM4D = 11
QUAD = 12
BEND = 13
SPACECHARGE = 14

FLOAT_FIELDS = ("x", "px", "y", "py", "zeta", "delta", "ptau", "rpp", "rvv")
INT_FIELDS = ("state", "at_turn", "at_element")


def build(force: bool = False, fused: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (g++, no
    contraction: every product and sum rounded on its own).

    ``fused=True`` builds the same source as ``liboracle_fused.so`` with the
    compiler free to contract a*b + c into fused multiply-adds.  That build
    differs from the plain one by rounding alone, so the distance between
    the two after many turns is the floor below which no FP64 tracker can be
    expected to reproduce the oracle; the long-run tests measure it."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_FUSED if fused else _SO
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC)):
        return so
    tmp = so + ".tmp%d" % os.getpid()
    if fused:
        flags = ["-ffp-contract=fast"] + (["-mfma"] if platform.machine() in ("x86_64", "AMD64") else [])
    else:
        flags = ["-ffp-contract=off", "-fno-fast-math"]
    cmd = ["g++", "-std=c++17", "-O2", *flags, "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def lib(fused: bool = False) -> ctypes.CDLL:
    global _lib, _lib_fused
    with _lock:
        if (_lib_fused if fused else _lib) is None:
            path = build(fused=fused)
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            L.xo_track.argtypes = [P, i64, P, i32, u64] + [P] * 13 + [i64, i64, i64]
            L.xo_track.restype = i32
            L.xo_track_jacobian.argtypes = [P, i64, P, i32, P, i64, P, P, P]
            L.xo_track_jacobian.restype = i32
            L.xo_closed_orbit.argtypes = [P, i64, P, i32, i32, P]
            L.xo_closed_orbit.restype = i32
            L.xo_philox4x64_10.argtypes = [P, P, P]
            L.xo_philox4x64_10.restype = None
            L.xo_uniform.argtypes = [u64, u64, u64, u64, i64]
            L.xo_uniform.restype = dbl
            L.xo_spectrum_size.restype = i32
            L.xo_spectrum_table.argtypes = [P, P]
            L.xo_spectrum_sample.argtypes = [dbl]
            L.xo_spectrum_sample.restype = dbl
            L.xo_ref_constants.argtypes = [P, P]
            L.xo_refine_losses.argtypes = [P, i64, P] + [P] * 11 + [i64, dbl, i32, P]
            L.xo_refine_losses.restype = i32
            L.xo_gauss_field.argtypes = [dbl, dbl, P, P, P, P, i64]
            L.xo_gauss_field.restype = None
            L.xo_gauss_legendre.argtypes = [P, P]
            L.xo_gauss_legendre.restype = i32
            L.xo_osc_funcs.argtypes = [P, P, i64]
            L.xo_osc_funcs.restype = None
            L.xo_lyapunov.argtypes = [P, i64, P, i32, P, P, P, i64, i64, i64, P, P, P]
            L.xo_lyapunov.restype = i32
            if fused:
                _lib_fused = L
            else:
                _lib = L
    return _lib_fused if fused else _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _ref_arr(ref) -> np.ndarray:
    return np.array([ref[0], ref[1], ref[2]], dtype=np.float64)


def _elements(elements) -> np.ndarray:
    el = np.ascontiguousarray(elements)
    if el.dtype != ELEMENT_DTYPE:
        el = el.astype(ELEMENT_DTYPE)
    return el


def refine_losses(elements, ref, particles: dict, ds: float, n_angles: int = 128) -> np.ndarray:
    """Loss positions [m] of the particles lost at apertures (state 0), NaN
    for the others; see xo_refine_losses."""
    el = _elements(elements)
    r = _ref_arr(ref)
    a = {k: np.ascontiguousarray(particles[k], dtype=np.float64) for k in FLOAT_FIELDS}
    st = np.ascontiguousarray(particles["state"], dtype=np.int32)
    ae = np.ascontiguousarray(particles["at_element"], dtype=np.int32)
    n = st.shape[0]
    out = np.empty(n)
    rc = lib().xo_refine_losses(_ptr(el), el.shape[0], _ptr(r), *[_ptr(a[k]) for k in FLOAT_FIELDS], _ptr(st),
                                _ptr(ae), n, float(ds), int(n_angles), _ptr(out))
    if rc != 0:
        raise ValueError("oracle refine_losses rejected its arguments")
    return out


def track(elements, ref, particles: dict, n_turns: int, start_turn: int = 0,
          rad_mode: int = 0, seed: int = 0, fused: bool = False) -> dict:
    """Track a copy of ``particles`` (dict of numpy arrays); returns the new
    dict.  ``fused`` runs the contracted build (see ``build``)."""
    el = _elements(elements)
    r = _ref_arr(ref)
    out = {}
    for k in FLOAT_FIELDS:
        out[k] = np.ascontiguousarray(particles[k], dtype=np.float64).copy()
    for k in INT_FIELDS:
        out[k] = np.ascontiguousarray(particles[k], dtype=np.int32).copy()
    out["particle_id"] = np.ascontiguousarray(particles["particle_id"], dtype=np.int64).copy()
    n = out["x"].shape[0]
    rc = lib(fused).xo_track(_ptr(el), el.shape[0], _ptr(r), rad_mode, seed,
                        *[_ptr(out[k]) for k in FLOAT_FIELDS],
                        *[_ptr(out[k]) for k in INT_FIELDS], _ptr(out["particle_id"]),
                        n, start_turn, n_turns)
    if rc != 0:
        raise ValueError("oracle track rejected its arguments")
    return out


def track_jacobian(elements, ref, z0, n_turns: int = 1, rad_mode: int = 0, along: bool = False):
    """Final canonical coordinates, the 6x6 Jacobian, and optionally the
    orbit and cumulative Jacobian after each element of the first turn."""
    el = _elements(elements)
    r = _ref_arr(ref)
    z = np.ascontiguousarray(z0, dtype=np.float64)
    zo = np.zeros(6)
    M = np.zeros(36)
    al = np.zeros(el.shape[0] * 42) if along else None
    rc = lib().xo_track_jacobian(_ptr(el), el.shape[0], _ptr(r), rad_mode, _ptr(z), n_turns,
                                 _ptr(zo), _ptr(M), _ptr(al) if along else None)
    if rc != 0:
        raise ValueError("oracle jacobian: particle lost or bad input (%d)" % rc)
    if along:
        al = al.reshape(el.shape[0], 42)
        return zo, M.reshape(6, 6), al[:, :6].copy(), al[:, 6:].reshape(-1, 6, 6).copy()
    return zo, M.reshape(6, 6)


def closed_orbit(elements, ref, rad_mode: int = 0, dim: int = 6, guess=None) -> np.ndarray:
    el = _elements(elements)
    r = _ref_arr(ref)
    z = np.zeros(6) if guess is None else np.array(guess, dtype=np.float64)
    it = lib().xo_closed_orbit(_ptr(el), el.shape[0], _ptr(r), rad_mode, dim, _ptr(z))
    if it < 0:
        raise ValueError("closed orbit search failed")
    return z


def lyapunov(elements, ref, z0, dz0, n_turns: int, every: int = 10, metric=None,
             rad_mode: int = 0, growth: float = 1e3) -> dict:
    """Chaos marker (twin-particle finite-time Lyapunov estimate, xo_lyapunov).

    z0: (n, 6) canonical starts (x, px, y, py, zeta, pzeta); dz0: the twin's
    offset (6,); metric: 6x6 matrix A of the distance |A dz| (identity if
    None).  Returns sum_log, turns, lost (0 both survived, 1 only one lost or
    lost at different turns, 2 both lost in the same turn), lam = sum_log /
    turns, and chaotic: the twin was lost alone, or the separation grew by
    more than ``growth`` times the turn count, sum_log > ln(growth * turns).
    A regular orbit separates at most linearly in the turn count, so the
    default leaves it three orders of magnitude of room."""
    el = _elements(elements)
    r = _ref_arr(ref)
    z = np.ascontiguousarray(np.asarray(z0, dtype=np.float64).reshape(-1, 6))
    d = np.ascontiguousarray(np.asarray(dz0, dtype=np.float64).reshape(6))
    A = None if metric is None else np.ascontiguousarray(np.asarray(metric, dtype=np.float64).reshape(36))
    n = z.shape[0]
    S = np.zeros(n)
    T = np.zeros(n, dtype=np.int32)
    L = np.zeros(n, dtype=np.int32)
    rc = lib().xo_lyapunov(_ptr(el), el.shape[0], _ptr(r), rad_mode, _ptr(z), _ptr(d),
                           None if A is None else _ptr(A), n, int(n_turns), int(every),
                           _ptr(S), _ptr(T), _ptr(L))
    if rc != 0:
        raise ValueError("oracle lyapunov rejected its arguments")
    lam = S / np.maximum(T, 1)
    chaotic = (L == 1) | (S > np.log(growth * np.maximum(T, 1)))
    return dict(sum_log=S, turns=T, lost=L, lam=lam, chaotic=chaotic)


def _track_job(args):
    elements, ref, particles, n_turns, fused = args
    return track(elements, ref, particles, n_turns, fused=fused)


def _lyapunov_job(args):
    elements, ref, z0, dz0, n_turns, every, metric = args
    return lyapunov(elements, ref, z0, dz0, n_turns, every=every, metric=metric)


def _chunks(n: int, procs: int):
    k = max(1, min(procs, n))
    return [c for c in np.array_split(np.arange(n), k) if c.size]


def track_parallel(elements, ref, particles: dict, n_turns: int, procs: int | None = None,
                   fused: bool = False) -> dict:
    """``track`` split over ``procs`` spawned processes (one particle slice
    each; the particles are independent, so the result is the same)."""
    import multiprocessing as mp
    lib(fused)  # built once here, not by every worker
    n = np.asarray(particles["x"]).shape[0]
    if n == 0:
        return track(elements, ref, particles, n_turns, fused=fused)
    procs = procs or os.cpu_count() or 1
    parts = _chunks(n, procs)
    jobs = [(elements, ref, {k: np.asarray(particles[k])[c] for k in FLOAT_FIELDS + INT_FIELDS + ("particle_id",)},
             n_turns, fused) for c in parts]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_track_job, jobs)
    return {k: np.concatenate([r[k] for r in res]) for k in res[0]}


def lyapunov_parallel(elements, ref, z0, dz0, n_turns: int, every: int = 10, metric=None,
                      procs: int | None = None) -> dict:
    """``lyapunov`` split over ``procs`` spawned processes."""
    import multiprocessing as mp
    lib()
    z = np.asarray(z0, dtype=np.float64).reshape(-1, 6)
    if z.shape[0] == 0:
        return lyapunov(elements, ref, z, dz0, n_turns, every=every, metric=metric)
    procs = procs or os.cpu_count() or 1
    parts = _chunks(z.shape[0], procs)
    jobs = [(elements, ref, z[c], dz0, n_turns, every, metric) for c in parts]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_lyapunov_job, jobs)
    return {k: np.concatenate([r[k] for r in res]) for k in res[0]}


def canonical(particles: dict, ref) -> np.ndarray:
    """(n, 6) canonical coordinates (x, px, y, py, zeta, pzeta = ptau/beta0)."""
    beta0 = ref_constants(ref)["beta0"]
    return np.stack([np.asarray(particles[k], dtype=np.float64) for k in ("x", "px", "y", "py", "zeta")]
                    + [np.asarray(particles["ptau"], dtype=np.float64) / beta0], axis=1)


def gauss_field(sx: float, sy: float, x, y):
    """Field shape (f_x, f_y) of a unit bi-Gaussian line charge."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y)]
    fx, fy = np.empty_like(a[0]), np.empty_like(a[0])
    lib().xo_gauss_field(float(sx), float(sy), a[0].ctypes.data, a[1].ctypes.data, fx.ctypes.data,
                         fy.ctypes.data, a[0].size)
    return fx, fy


def gauss_legendre():
    """Nodes and weights of the oracle's quadrature rule on [-1, 1]."""
    x = np.zeros(64)
    w = np.zeros(64)
    n = lib().xo_gauss_legendre(_ptr(x), _ptr(w))
    return x[:n].copy(), w[:n].copy()


def osc_funcs(z) -> np.ndarray:
    """(n, 4) array of the thick maps' C, S, S2, S3 at z."""
    z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.float64)
    out = np.empty((z.size, 4))
    lib().xo_osc_funcs(_ptr(z), _ptr(out), z.size)
    return out


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().xo_philox4x64_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniform(seed: int, pid: int, turn: int, elem: int, index: int) -> float:
    return lib().xo_uniform(seed, pid, turn, elem, index)


def spectrum_table():
    n = lib().xo_spectrum_size()
    xi = np.zeros(n)
    F = np.zeros(n)
    lib().xo_spectrum_table(_ptr(xi), _ptr(F))
    return xi, F


def spectrum_sample(u: float) -> float:
    return lib().xo_spectrum_sample(float(u))


def ref_constants(ref) -> dict:
    r = _ref_arr(ref)
    o = np.zeros(6)
    lib().xo_ref_constants(_ptr(r), _ptr(o))
    return dict(E0=o[0], beta0=o[1], gamma0=o[2], crad=o[3], kq=o[4], uc15=o[5])
