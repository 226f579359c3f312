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


def row_lengths(table) -> np.ndarray:
    """Reference length of every table row (drifts, thick quadrupoles, bends)."""
    t = np.asarray(table)
    L = np.zeros(t.shape[0])
    for i in range(t.shape[0]):
        ty = int(t[i]["type"])
        if ty == I.DRIFT:
            L[i] = t[i]["p"][0]
        elif ty == I.QUAD:
            L[i] = t[i]["p"][1]
        elif ty == I.BEND:
            L[i] = t[i]["p"][2]
    return L


def _symplectic_form(n: int) -> np.ndarray:
    S = np.zeros((n, n))
    for k in range(0, n, 2):
        S[k, k + 1], S[k + 1, k] = 1.0, -1.0
    return S


def normal_modes(M: np.ndarray) -> np.ndarray:
    """Eigenvectors of a stable one-turn matrix (n x n, n = 4 or 6), one per
    mode as columns (mode I mostly in x, II in y, III in zeta), each chosen
    from its conjugate pair and scaled so that v^H S v = i (S the symplectic
    form).  For an uncoupled plane this is v = (sqrt(beta), (i - alpha) /
    sqrt(beta)) / sqrt(2) times a phase."""
    n = M.shape[0]
    S = _symplectic_form(n)
    w, V = np.linalg.eig(M)
    modes = []
    for k in range(n):
        v = V[:, k]
        nv = np.vdot(v, S @ v)  # purely imaginary for a symplectic M
        if nv.imag > 0:
            modes.append(v / math.sqrt(nv.imag))
    if len(modes) != n // 2:
        raise RuntimeError("one-turn matrix is not stable (eigenvalues off the unit circle)")
    planes = [int(np.argmax([abs(v[2 * j]) ** 2 + abs(v[2 * j + 1]) ** 2 for j in range(n // 2)])) for v in modes]
    if sorted(planes) != list(range(n // 2)):
        raise RuntimeError("modes cannot be assigned to planes (strong coupling)")
    return np.stack([modes[planes.index(j)] for j in range(n // 2)], 1)


def _stencil_along(tr, ref, z):
    """Orbit and Jacobians from the start to the exit of every row: the
    13-particle central-difference stencil about z tracked once through the
    table by the monitor.  Returns (orbit [n, 6], M [n, 6, 6]) in canonical
    coordinates (pzeta = ptau / beta0)."""
    m0, _, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    Z = np.tile(z, (13, 1))
    for i in range(6):
        Z[1 + 2 * i, i] += EPS[i]
        Z[2 + 2 * i, i] -= EPS[i]
    P = xtgb.Particles.from_numpy(particles_from_z(ref, Z))
    out = tr.monitor(P).cpu().numpy()
    if np.any(out[:, 7, :] != 1.0):
        raise RuntimeError("a particle of the stencil was lost along the line")
    zs = out[:, :6, :].copy()
    zs[:, 5, :] /= beta0  # ptau -> pzeta
    Ms = np.empty((zs.shape[0], 6, 6))
    for k in range(6):
        Ms[:, :, k] = (zs[:, :, 1 + 2 * k] - zs[:, :, 2 + 2 * k]) / (2.0 * EPS[k])
    return zs[:, :, 0], Ms


def _functions_along(el, z, orbit, Ms, Vm, D0) -> dict:
    """Mais-Ripken functions at the start (row -1 of the arrays: index 0)
    and at the exit of every row from the modes Vm at the start carried as
    M_i v: beta_x^I = 2 |v_I,x|^2, alpha_x^I = -2 Re(conj(v_I,x) v_I,px),
    the phase from arg v_I,x (likewise y, mode II), the cross terms
    beta_x^II and beta_y^I, and the dispersion M_i (D_0, 1)."""
    n = Vm.shape[0]
    V = np.einsum("eij,jk->eik", Ms[:, :n, :n], Vm)
    V = np.concatenate([Vm[None], V], 0)
    mux = np.unwrap(np.angle(V[:, 0, 0]))
    muy = np.unwrap(np.angle(V[:, 2, 1]))
    D = np.einsum("eij,j->ei", Ms[:, :4, :4], D0) + Ms[:, :4, 5]
    D = np.concatenate([D0[None], D], 0)
    s = np.concatenate([[0.0], np.cumsum(row_lengths(el))])
    orb = np.concatenate([z[None], orbit], 0)
    return dict(s=s, x=orb[:, 0], px=orb[:, 1], y=orb[:, 2], py=orb[:, 3], zeta=orb[:, 4], pzeta=orb[:, 5],
                betx=2 * np.abs(V[:, 0, 0]) ** 2, bety=2 * np.abs(V[:, 2, 1]) ** 2,
                alfx=-2 * np.real(np.conj(V[:, 0, 0]) * V[:, 1, 0]), alfy=-2 * np.real(np.conj(V[:, 2, 1]) * V[:, 3, 1]),
                mux=(mux - mux[0]) / (2 * math.pi), muy=(muy - muy[0]) / (2 * math.pi),
                betx2=2 * np.abs(V[:, 0, 1]) ** 2, bety1=2 * np.abs(V[:, 2, 0]) ** 2,
                dx=D[:, 0], dpx=D[:, 1], dy=D[:, 2], dpy=D[:, 3], modes_along=V)


def _pzeta_of_delta(ref, delta0):
    m0, _, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    E0 = math.sqrt(p0c * p0c + m0 * m0)
    E = math.sqrt((p0c * (1 + delta0)) ** 2 + m0 * m0)
    return (E - E0) / p0c / beta0


def twiss_along(table, ref, dim: int = 4, delta0: float = 0.0, radiation: int = 0) -> dict:
    """Lattice functions at the exit of every table row of a ring (section
    "Twiss module"): the closed orbit and one-turn Jacobian as in twiss();
    the stencil about the closed orbit tracked once through the line by the
    monitor gives the Jacobian M_i to the exit of every row; the modes of
    the one-turn matrix (normal_modes) are carried along as M_i v and the
    Mais-Ripken functions read from them (_functions_along).  The dispersion
    (per unit pzeta, as in twiss()) is M_i (D_0, 1) with D_0 periodic.
    dim=6 keeps the RF and gives three modes (the third longitudinal)."""
    el = without_cavities(table) if dim == 4 else np.asarray(table)
    tr = xtgb.Tracker(el, ref, radiation=radiation)
    try:
        guess = np.zeros(6)
        guess[5] = _pzeta_of_delta(ref, delta0)
        z = closed_orbit(tr, ref, dim=dim, guess=guess)
        orbit, Ms = _stencil_along(tr, ref, z)
    finally:
        tr.close()
    M = Ms[-1]
    n = 4 if dim == 4 else 6
    Vm = normal_modes(M[:n, :n])
    D0 = np.linalg.solve(np.eye(4) - M[:4, :4], M[:4, 5])
    out = _functions_along(el, z, orbit, Ms, Vm, D0)
    out.update(M=M, modes=Vm, qx=float(out["mux"][-1]) % 1.0, qy=float(out["muy"][-1]) % 1.0)
    return out


def twiss_open(table, ref, betx: float, alfx: float, bety: float, alfy: float, dx: float = 0.0, dpx: float = 0.0,
               dy: float = 0.0, dpy: float = 0.0, orbit=None, delta0: float = 0.0, radiation: int = 0) -> dict:
    """Lattice functions along a line, or a portion of a ring, from given
    initial conditions (section "Twiss module": Twiss on part of a line with
    assigned initial conditions and momentum): uncoupled modes built from
    (beta, alpha) at the start, v_I = (sqrt(betx), (i - alfx)/sqrt(betx), 0, 0)
    / sqrt(2) and likewise v_II, carried through the monitor's per-row
    Jacobians about the given orbit (zeros, at momentum delta0, by default)."""
    z = np.zeros(6) if orbit is None else np.array(orbit, dtype=np.float64)
    if orbit is None:
        z[5] = _pzeta_of_delta(ref, delta0)
    el = np.asarray(table)
    tr = xtgb.Tracker(el, ref, radiation=radiation)
    try:
        orb, Ms = _stencil_along(tr, ref, z)
    finally:
        tr.close()
    Vm = np.zeros((4, 2), dtype=complex)
    Vm[0, 0], Vm[1, 0] = math.sqrt(betx), (1j - alfx) / math.sqrt(betx)
    Vm[2, 1], Vm[3, 1] = math.sqrt(bety), (1j - alfy) / math.sqrt(bety)
    Vm /= math.sqrt(2.0)
    return _functions_along(el, z, orb, Ms, Vm, np.array([dx, dpx, dy, dpy], dtype=np.float64))


def kick_as_closed_orbit(table, ref) -> tuple:
    """The "kick as closed orbit" line of section "Twiss module": with mean
    radiation the 6D closed orbit is found and one particle on it is
    tracked once around by the monitor; at every radiating multipole the
    radiation's share of the change is read off the monitor (the energy step
    dpzeta, and px, py times 1 - 1/f where f = (1+delta_after)/(1+delta_before)
    is the scaling that keeps the angles), and the returned table carries
    those constant kicks as identity linear maps with offsets right after
    each radiating row.  Tracked with radiation off, it gives every particle
    the closed orbit's radiation kicks: a symplectic one-turn matrix that
    includes the energy loss to first order.  Returns (table, closed orbit,
    the position of every original row in the new table)."""
    m0, _, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    el0 = np.asarray(table)
    tr = xtgb.Tracker(el0, ref, radiation=xtgb.RAD_MEAN)
    try:
        co = closed_orbit(tr, ref, dim=6)
        P = xtgb.Particles.from_numpy(particles_from_z(ref, co[None]))
        start = P.to_numpy()
        out = tr.monitor(P).cpu().numpy()[:, :, 0]
    finally:
        tr.close()
    before = np.concatenate([[[start[k][0] for k in ("x", "px", "y", "py", "zeta", "ptau")] + [start["delta"][0]]],
                             out[:-1, :7]], 0)
    rows, index = [], []
    for i in range(el0.shape[0]):
        r = el0[i]
        index.append(len(rows))
        rows.append(r)
        if int(r["type"]) != I.MULTIPOLE or r["p"][23] <= 0.0:
            continue
        f = (1.0 + out[i, 6]) / (1.0 + before[i, 6])
        d = np.zeros(6)
        d[1] = out[i, 1] * (1.0 - 1.0 / f)
        d[3] = out[i, 3] * (1.0 - 1.0 / f)
        d[5] = (out[i, 5] - before[i, 5]) / beta0
        rows.append(I.linear_map(np.eye(6), d))
    return I.table(rows), co, np.array(index)


R_ELECTRON = 2.8179403262e-15        # classical electron radius [m]
LAMBDA_C_ELECTRON = 3.8615926796e-13  # reduced Compton wavelength hbar / (m_e c) [m]


def equilibrium_emittances(table, ref) -> dict:
    """Equilibrium emittances from the linear normal form (section "Twiss
    module", after Chao): the modes of the 6D one-turn matrix without
    radiation are carried along the ring (twiss_along, dim=6); a quantum
    kick of variance s2_i in pzeta at radiating element i raises the action
    of mode k by |v_k,zeta(i)|^2 s2_i (the action of z is |v^H S z|^2), and
    the mode damps at 2 alpha_k per turn (damping()), so
    eps_k = sum_i |v_k,zeta(i)|^2 s2_i / (2 alpha_k).  The energy diffusion
    of a thin radiating slice of curvature h = knl0 / L_rad is the variance of
    its relative energy kick per passage,
    s2 = 55 / (24 sqrt 3) r_e (hbar / m_e c) gamma0^5 |h|^3 L_rad (electrons;
    pzeta = delta for beta0 -> 1).  Also returns the momentum spread
    2 sum_k eps_k |v_k,pzeta|^2 at the start."""
    m0, _, p0c = ref
    gamma0 = math.sqrt(p0c * p0c + m0 * m0) / m0
    t6 = twiss_along(table, ref, dim=6)
    dmp = damping(table, ref)
    el = np.asarray(table)
    V = t6["modes_along"]  # [row + 1, 6, 3]
    c = 55.0 / (24.0 * math.sqrt(3.0)) * R_ELECTRON * LAMBDA_C_ELECTRON * gamma0 ** 5
    growth = np.zeros(3)
    for i in range(el.shape[0]):
        r = el[i]
        if int(r["type"]) != I.MULTIPOLE or r["p"][23] <= 0.0 or r["p"][0] == 0.0:
            continue
        L = r["p"][23]
        h = r["p"][0] / L
        growth += np.abs(V[i + 1, 4, :]) ** 2 * (c * abs(h) ** 3 * L)
    eps = growth / (2.0 * dmp["alpha"])
    sigma_delta = math.sqrt(2.0 * float(np.sum(eps * np.abs(t6["modes"][5, :]) ** 2)))
    return dict(eps=eps, sigma_delta=sigma_delta, alpha=dmp["alpha"], twiss=t6)


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


# --------------------------------------------------------------------------
# Energy-loss compensation ("tapering", section "Twiss module")

def scale_magnets(table, scale) -> np.ndarray:
    """A copy of the table with the field strengths of every magnet row i
    scaled by scale[i]: thin multipole knl and ksl (not the frame curvature
    hxl nor L_rad), thick quadrupole k1, bend k0 and k1 (not h), dipole-edge
    h.  Other rows are unchanged."""
    el = np.array(table, copy=True)
    for i in range(el.shape[0]):
        t, f = int(el[i]["type"]), float(scale[i])
        if t == I.MULTIPOLE:
            el[i]["p"][:22] = el[i]["p"][:22] * f
        elif t == I.QUAD:
            el[i]["p"][0] = el[i]["p"][0] * f
        elif t == I.BEND:
            el[i]["p"][0] = el[i]["p"][0] * f
            el[i]["p"][3] = el[i]["p"][3] * f
        elif t == I.DIPEDGE:
            el[i]["p"][0] = el[i]["p"][0] * f
    return el


def compensate_energy_loss(table, ref, max_iter: int = 40, tol: float = 1e-13) -> dict:
    """The paper's iteration for lepton rings with strong radiation:
    (1) the 4D closed orbit without radiation, energy frozen; (2) with mean
    radiation, one particle from that orbit tracked once around by the
    monitor while every magnet's strength is scaled to the energy
    (1 + delta) of the particle entering it, which measures the energy lost
    along the ring while keeping the orbit and optics; (3) the RF phases set
    so that the cavities restore that loss, shared in proportion to their
    voltages: every cavity runs at the phase phi with
    q V_total sin(phi) = U0, on the side of 90 degrees its lag had, and
    lag = phi + k_rf zeta at the particle's zeta; (4) steps 2-3 repeated,
    the scaling taken from the previous pass, until scaling, lags and the
    energy after one turn settle.  Every turn is tracked on the GPU."""
    m0, q0, p0c = ref
    beta0 = p0c / math.sqrt(p0c * p0c + m0 * m0)
    el0 = np.array(table, copy=True)
    n = el0.shape[0]
    cav = np.array([i for i in range(n) if int(el0[i]["type"]) == I.CAVITY and el0[i]["p"][0] != 0.0])
    if cav.size == 0:
        raise ValueError("no RF cavity to compensate the energy loss")
    volts = np.array([el0[i]["p"][0] for i in cav])
    krf = np.array([2 * math.pi * el0[i]["p"][1] / (beta0 * 2.99792458e8) for i in cav])
    above = np.array([el0[i]["p"][2] > 90.0 for i in cav])
    tr = xtgb.Tracker(without_cavities(el0), ref)
    try:
        z4 = closed_orbit(tr, ref, dim=4)
    finally:
        tr.close()
    scale = np.ones(n)
    lags = np.array([el0[i]["p"][2] for i in cav])
    last = None
    for it in range(1, max_iter + 1):
        el = scale_magnets(el0, scale)
        for j, i in enumerate(cav):
            el[i]["p"][2] = lags[j]
        tr = xtgb.Tracker(el, ref, radiation=xtgb.RAD_MEAN)
        try:
            P = xtgb.Particles.from_numpy(particles_from_z(ref, z4[None]))
            start = P.to_numpy()
            out = tr.monitor(P).cpu().numpy()[:, :, 0]
        finally:
            tr.close()
        if np.any(out[:, 7] != 1.0):
            raise RuntimeError("the closed-orbit particle was lost during compensation")
        delta_in = np.concatenate([[start["delta"][0]], out[:-1, 6]])
        ptau_in = np.concatenate([[start["ptau"][0]], out[:-1, 5]])
        zeta_in = np.concatenate([[start["zeta"][0]], out[:-1, 4]])
        dpt = out[:, 5] - ptau_in
        radiated = -(np.sum(dpt) - np.sum(dpt[cav]))  # in units of p0 c
        u = radiated * p0c / (q0 * np.sum(volts))
        if not abs(u) < 1.0:
            raise RuntimeError("the RF voltage cannot restore the energy loss")
        phi = np.where(above, math.pi - math.asin(u), math.asin(u))
        new_lags = np.degrees(phi + krf * zeta_in[cav])
        new_scale = 1.0 + delta_in
        d_end = out[-1, 6] - start["delta"][0]
        done = (np.max(np.abs(new_scale - scale)) < tol and np.max(np.abs(new_lags - lags)) < 1e-9
                and abs(d_end) < tol)
        scale, lags = new_scale, new_lags
        last = dict(delta=delta_in, x=np.concatenate([[z4[0]], out[:-1, 0]]),
                    y=np.concatenate([[z4[2]], out[:-1, 2]]), delta_end=d_end)
        if done:
            break
    el = scale_magnets(el0, scale)
    for j, i in enumerate(cav):
        el[i]["p"][2] = lags[j]
    return dict(table=el, scale=scale, lags=lags, energy_loss=radiated * p0c, iterations=it,
                converged=done, **last)

