"""Twiss by tracking on the GPU (section "Twiss module" of the paper).

The paper's Twiss module finds the closed orbit with a root finder on the
one-turn map, takes the one-turn Jacobian by central differences of tracked
particles, and derives the lattice functions from it.  Here every turn of
every particle is tracked by the library's kernel (``xt_track``); the host
only solves 6x6 (or 4x4) linear systems and eigenvalue problems.

Coordinates are canonical: z = (x, px, y, py, zeta, pzeta), pzeta =
ptau/beta0.  Four-dimensional mode (``dim=4``) tracks the line with its RF
cavities switched off and solves for (x, px, y, py) at fixed zeta and pzeta;
six-dimensional mode (``dim=6``) keeps the RF and, with mean radiation,
gives the damping decrements.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I
from . import xtgb

# step of the central differences per coordinate (m, rad, m, rad, m, 1)
EPS = np.array([1e-8, 1e-10, 1e-8, 1e-10, 1e-7, 1e-9])


def without_cavities(table):
    el = np.array(table, copy=True)
    for i in range(el.shape[0]):
        if int(el[i]["type"]) == I.CAVITY:
            el[i]["p"][0] = 0.0
    return el


def particles_from_z(ref, Z: np.ndarray) -> dict:
    """Particle arrays for canonical coordinates Z (n x 6), with delta, rpp and
    rvv from ptau = beta0 pzeta by the kinematic relations
    (1+delta)^2 = 1 + 2 ptau/beta0 + ptau^2 and rvv = (1+delta)/(1+beta0 ptau)."""
    m0, _, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))
    n = Z.shape[0]
    ptau = beta0 * Z[:, 5]
    u = ptau * (ptau + 2.0 / beta0)
    delta = u / (np.sqrt(1.0 + u) + 1.0)
    return dict(x=Z[:, 0].copy(), px=Z[:, 1].copy(), y=Z[:, 2].copy(), py=Z[:, 3].copy(), zeta=Z[:, 4].copy(),
                delta=delta, ptau=ptau, rpp=1.0 / (1.0 + delta), rvv=(1.0 + delta) / (1.0 + beta0 * ptau),
                state=np.ones(n, np.int32), at_turn=np.zeros(n, np.int32), at_element=np.zeros(n, np.int32),
                particle_id=np.arange(n, dtype=np.int64))


def track_z(tracker, ref, Z: np.ndarray, n_turns: int = 1) -> np.ndarray:
    """Tracks the rows of Z for n_turns turns on the GPU; returns the final
    canonical coordinates (NaN rows for lost particles)."""
    m0, _, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    P = xtgb.Particles.from_numpy(particles_from_z(ref, Z))
    tracker.track(P, n_turns)
    o = P.to_numpy()
    out = np.stack([o["x"], o["px"], o["y"], o["py"], o["zeta"], o["ptau"] / beta0], 1)
    out[o["state"] != 1] = np.nan
    return out


def jacobian(tracker, ref, z0, eps=EPS):
    """One-turn map at z0 and its Jacobian by central differences: the
    centre and the 12 displaced particles are tracked in one launch."""
    z0 = np.asarray(z0, dtype=np.float64)
    Z = np.tile(z0, (13, 1))
    for i in range(6):
        Z[1 + 2 * i, i] += eps[i]
        Z[2 + 2 * i, i] -= eps[i]
    out = track_z(tracker, ref, Z)
    if np.any(np.isnan(out)):
        raise RuntimeError("a particle of the Jacobian stencil was lost")
    R = np.empty((6, 6))
    for i in range(6):
        R[:, i] = (out[1 + 2 * i] - out[2 + 2 * i]) / (2.0 * eps[i])
    return out[0], R


def closed_orbit(tracker, ref, dim: int = 4, guess=None, tol: float = 1e-14, max_iter: int = 30):
    """Newton's method on z -> M(z) - z: the first `dim` coordinates are
    solved for, the others stay at the guess (zeta = pzeta = 0 by default)."""
    z = np.zeros(6) if guess is None else np.array(guess, dtype=np.float64)
    k = dim
    for _ in range(max_iter):
        z1, R = jacobian(tracker, ref, z)
        F = z1[:k] - z[:k]
        dz = np.linalg.solve(R[:k, :k] - np.eye(k), -F)
        z[:k] += dz
        if np.max(np.abs(dz)) < tol:
            return z
    return z


def _tune(A):
    c = 0.5 * np.trace(A)
    s = math.copysign(math.sqrt(max(0.0, 1.0 - c * c)), A[0, 1])
    return (math.atan2(s, c) / (2 * math.pi)) % 1.0, s


def twiss(table, ref, dim: int = 4, delta0: float = 0.0, radiation: int = 0) -> dict:
    """Closed orbit, one-turn matrix, tunes, beta, alpha and dispersion at the
    start of the line (uncoupled reading of the 2x2 blocks).  dim=4: RF off,
    the closed orbit at pzeta for delta = delta0."""
    m0, _, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    el = without_cavities(table) if dim == 4 else table
    tr = xtgb.Tracker(el, ref, radiation=radiation)
    try:
        E0 = math.sqrt(p0c * p0c + m0 * m0)
        E = math.sqrt((p0c * (1 + delta0)) ** 2 + m0 * m0)
        guess = np.zeros(6)
        guess[5] = (E - E0) / p0c / beta0
        z = closed_orbit(tr, ref, dim=dim, guess=guess)
        _, M = jacobian(tr, ref, z)
    finally:
        tr.close()
    qx, sx = _tune(M[:2, :2])
    qy, sy = _tune(M[2:4, 2:4])
    D = np.linalg.solve(np.eye(4) - M[:4, :4], M[:4, 5])
    return dict(closed_orbit=z, M=M, qx=qx, qy=qy, betx=M[0, 1] / sx, alfx=(M[0, 0] - M[1, 1]) / (2 * sx),
                bety=M[2, 3] / sy, alfy=(M[2, 2] - M[3, 3]) / (2 * sy), dx=D[0], dpx=D[1], dy=D[2], dpy=D[3])


def chromaticity(table, ref, d: float = 1e-5) -> tuple:
    """dQ/ddelta from the tunes at delta = +d and -d (RF off)."""
    a, b = twiss(table, ref, 4, d), twiss(table, ref, 4, -d)
    dq = lambda qa, qb: ((qa - qb + 0.5) % 1.0 - 0.5) / (2 * d)
    return dq(a["qx"], b["qx"]), dq(a["qy"], b["qy"])


def damping(table, ref) -> dict:
    """With mean radiation: the 6D closed orbit and the damping decrements
    per turn, -ln|lambda| of the one-turn matrix's eigenvalues, one per plane
    (each complex pair assigned to the plane holding most of its
    eigenvector)."""
    t = twiss(table, ref, dim=6, radiation=xtgb.RAD_MEAN)
    w, V = np.linalg.eig(t["M"])
    planes = np.argmax(np.abs(V[[0, 2, 4], :]) ** 2 + np.abs(V[[1, 3, 5], :]) ** 2, axis=0)
    alpha = np.array([np.mean(-np.log(np.abs(w[planes == k]))) for k in range(3)])
    return dict(alpha=alpha, closed_orbit=t["closed_orbit"], M=t["M"])
