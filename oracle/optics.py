"""Linear optics and radiation integrals from the oracle tracker (test
infrastructure only).

Follows the Twiss procedure of the paper (section "Twiss module"): closed
orbit by a root finder on the one-turn map, the one-turn Jacobian (here exact,
by forward-mode differentiation of the oracle's maps instead of central
differences), lattice functions from its eigen-structure, and their
propagation along the line with the cumulative Jacobians.  The radiation
quantities follow the section "Synchrotron radiation models and
compensation": energy loss, damping from the eigenvalues of the one-turn
matrix with radiation, equilibrium emittance and momentum spread from the
synchrotron integrals (Sands; thin-element sums of this project's model).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

C_Q = 55.0 / (32.0 * math.sqrt(3.0)) * 197.3269804e-9 / 0.51099895000e6  # m (electrons)
C_GAMMA = 4 * math.pi / 3 * 2.8179403262e-15 / (0.51099895000e-3) ** 3  # m / GeV^3


def without_cavities(elements):
    el = np.array(elements, copy=True)
    for i in range(el.shape[0]):
        if int(el[i]["type"]) == oracle.CAVITY:
            el[i]["p"][0] = 0.0
    return el


def twiss_uncoupled(elements, ref):
    """beta, alpha (x, y), dispersion D, D' at the START of every element and
    after the last, for the lattice without RF, radiation off, on momentum."""
    el = without_cavities(elements)
    z0 = oracle.closed_orbit(el, ref, rad_mode=0, dim=4)
    _, M, _, Ms = oracle.track_jacobian(el, ref, z0, along=True)
    n = el.shape[0]

    def cs(A):
        c = 0.5 * np.trace(A)
        s = math.copysign(math.sqrt(1 - c * c), A[0, 1])
        return A[0, 1] / s, (A[0, 0] - A[1, 1]) / (2 * s)

    bx, ax = cs(M[:2, :2])
    by, ay = cs(M[2:4, 2:4])
    # periodic dispersion w.r.t. pzeta (= delta to first order at delta = 0)
    D0 = np.linalg.solve(np.eye(2) - M[:2, :2], M[:2, 5])
    Sx = np.array([[bx, -ax], [-ax, (1 + ax * ax) / bx]])
    Sy = np.array([[by, -ay], [-ay, (1 + ay * ay) / by]])
    out = {k: np.zeros(n + 1) for k in ("betx", "alfx", "bety", "alfy", "dx", "dpx")}
    for i in range(n + 1):
        if i == 0:
            A, B, m5 = np.eye(2), np.eye(2), np.zeros(2)
        else:
            A, B, m5 = Ms[i - 1][:2, :2], Ms[i - 1][2:4, 2:4], Ms[i - 1][:2, 5]
        S1 = A @ Sx @ A.T
        S2 = B @ Sy @ B.T
        Dv = A @ D0 + m5
        out["betx"][i], out["alfx"][i] = S1[0, 0], -S1[0, 1]
        out["bety"][i], out["alfy"][i] = S2[0, 0], -S2[0, 1]
        out["dx"][i], out["dpx"][i] = Dv
    out["M"] = M
    return out


def radiation_integrals(elements, ref, tw=None):
    """Thin-element synchrotron integrals over the radiating multipoles, with
    the local curvature h = knl0/L_rad of the design orbit:
    I2 = sum h^2 L, I3 = sum |h|^3 L, I5 = sum H |h|^3 L, with
    H = gamma_x D^2 + 2 alpha_x D D' + beta_x D'^2 at the kick."""
    if tw is None:
        tw = twiss_uncoupled(elements, ref)
    I2 = I3 = I5 = 0.0
    for i in range(elements.shape[0]):
        r = elements[i]
        if int(r["type"]) != oracle.MULTIPOLE or r["p"][23] <= 0:
            continue
        L = r["p"][23]
        h = r["p"][0] / L
        b, a, D, Dp = tw["betx"][i], tw["alfx"][i], tw["dx"][i], tw["dpx"][i]
        g = (1 + a * a) / b
        H = g * D * D + 2 * a * D * Dp + b * Dp * Dp
        I2 += h * h * L
        I3 += abs(h) ** 3 * L
        I5 += H * abs(h) ** 3 * L
    return I2, I3, I5


def damping(elements, ref):
    """Damping decrements per turn and partition numbers from the eigenvalues of
    the one-turn matrix at the 6D closed orbit with mean radiation, and the
    energy loss per turn U0 [eV] = the RF energy gain on that orbit."""
    co = oracle.closed_orbit(elements, ref, rad_mode=1, dim=6)
    _, M, zs, _ = oracle.track_jacobian(elements, ref, co, rad_mode=1, along=True)
    w, V = np.linalg.eig(M)
    # each complex pair belongs to the plane holding most of its eigenvector
    planes = np.argmax(np.abs(V[[0, 2, 4], :]) ** 2 + np.abs(V[[1, 3, 5], :]) ** 2, axis=0)
    alpha = np.array([np.mean(-np.log(np.abs(w[planes == k]))) for k in range(3)])
    rc = oracle.ref_constants(ref)
    U0 = 0.0
    for i in range(elements.shape[0]):
        if int(elements[i]["type"]) == oracle.CAVITY:
            before = co[5] if i == 0 else zs[i - 1][5]
            U0 += (zs[i][5] - before) * rc["beta0"] * ref[2]
    J = 2 * alpha * rc["E0"] / U0
    return dict(alpha=alpha, J=J, U0=U0, E0=rc["E0"], M=M, closed_orbit=co)


def equilibrium(elements, ref):
    """Equilibrium emittance and momentum spread (Sands):
    eps_x = C_q gamma^2 I5 / (J_x I2), sigma_delta^2 = C_q gamma^2 I3 / (J_z I2)."""
    tw = twiss_uncoupled(elements, ref)
    I2, I3, I5 = radiation_integrals(elements, ref, tw)
    d = damping(elements, ref)
    rc = oracle.ref_constants(ref)
    g = rc["gamma0"]
    Jx, Jz = d["J"][0], d["J"][2]
    eps = C_Q * g * g * I5 / (Jx * I2)
    sd2 = C_Q * g * g * I3 / (Jz * I2)
    return dict(eps_x=eps, sigma_delta=math.sqrt(sd2), I2=I2, I3=I3, I5=I5, twiss=tw, **d)
