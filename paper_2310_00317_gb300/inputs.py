"""Seeded synthetic inputs: lattice tables and particle ensembles.

This module builds the inputs both the CUDA tracker and the oracle consume:
flat lattice tables (one row per element: type, order, 48 parameters) and
particle arrays.  It contains none of the tracking maps.  To place particles
in normalised phase space it uses the textbook linear optics of thin lenses
(2x2 and 3x3 transfer matrices of drifts, thin quadrupoles and thin dipole
kicks, Courant-Snyder parameters from the one-turn matrix), which is input
preparation only.

The paper's machines (LHC, FCC-ee, ...) are not available; the synthetic rings
below stand in for them with LHC-like and FCC-like shapes, sizes and element
mixes (section "Lattice modelling and single particle tracking": a line is a
sequence of thin elements with multipolar errors; section "Particle-matter
interaction": aperture elements along the line).
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# Table layout and element constructors.

ELEMENT_DTYPE = np.dtype([("type", "<i4"), ("order", "<i4"), ("p", "<f8", (48,))], align=True)
MARKER, DRIFT, MULTIPOLE, CAVITY, DIPEDGE, LINEARMAP, APERTURE = 0, 1, 2, 3, 4, 5, 6
XYSHIFT, SROTATION, APERTURE_RECT, APERTURE_ELLIPSE = 7, 8, 9, 10
BEAMBEAM4D, QUAD, BEND, SPACECHARGE = 11, 12, 13, 14
MAX_ORDER = 10

C_LIGHT = 299792458.0
PROTON_MASS_EV = 938.27208816e6
ELECTRON_MASS_EV = 0.51099895000e6
BASE_SEED = 20231001


def _row(t: int, order: int = 0, params=()) -> np.ndarray:
    r = np.zeros((), dtype=ELEMENT_DTYPE)
    r["type"] = t
    r["order"] = order
    p = np.zeros(48)
    p[: len(params)] = params
    r["p"] = p
    return r


def drift(length: float):
    return _row(DRIFT, 0, [length])


def multipole(knl=(), ksl=(), hxl: float = 0.0, lrad: float = 0.0, order: int | None = None):
    """Thin multipole; knl/ksl are integrated strengths K_n L (m^-n), n = 0..10."""
    kn = np.zeros(MAX_ORDER + 1)
    ks = np.zeros(MAX_ORDER + 1)
    kn[: len(knl)] = knl
    ks[: len(ksl)] = ksl
    if order is None:
        nz = [n for n in range(MAX_ORDER + 1) if kn[n] != 0.0 or ks[n] != 0.0]
        order = max(nz) if nz else 0
    return _row(MULTIPOLE, order, list(kn) + list(ks) + [hxl, lrad])


def cavity(voltage: float, frequency: float, lag_deg: float):
    return _row(CAVITY, 0, [voltage, frequency, lag_deg])


def dipedge(h: float, e1: float, hgap: float = 0.0, fint: float = 0.0, nonlinear: bool = False,
            exit: bool = False, wedge: bool = False):
    """Dipole edge of field h [1/m] with face angle e1 [rad] and fringe
    extent hgap [m] x fint; nonlinear=True selects the non-linear model and
    wedge=True the non-linear fringe on the face between exact changes of
    plane (the exact wedge); for both, exit=True marks the magnet's exit face."""
    model = 2.0 if wedge else (1.0 if nonlinear else 0.0)
    return _row(DIPEDGE, 0, [h, e1, hgap, fint, model, 1.0 if exit else 0.0])


def linear_map(M, d=None):
    """6x6 map on (x, px, y, py, zeta, pzeta) plus an offset d."""
    M = np.asarray(M, dtype=np.float64).reshape(36)
    d = np.zeros(6) if d is None else np.asarray(d, dtype=np.float64)
    return _row(LINEARMAP, 0, list(M) + list(d))


def aperture(radius: float):
    return _row(APERTURE, 0, [radius])


def marker():
    return _row(MARKER)


def xy_shift(dx: float, dy: float):
    """Change of reference frame: displaced by (dx, dy)."""
    return _row(XYSHIFT, 0, [dx, dy])


def s_rotation(angle: float):
    """Change of reference frame: rotated by `angle` [rad] about the orbit."""
    return _row(SROTATION, 0, [angle])


def quadrupole(k1: float, length: float):
    """Thick quadrupole: k1 [m^-2] (> 0 focuses x), length [m]."""
    return _row(QUAD, 0, [k1, length])


def bend(k0: float, h: float, length: float, k1: float = 0.0, full: bool = False, kicks: int = 0):
    """Thick sector bend: field k0 = B / (B rho) [1/m], frame curvature h
    [1/m] (k0 = h on the design orbit), reference length [m], gradient k1
    [m^-2]; full=True selects the exact model, in which a gradient is applied
    as `kicks` thin quadrupole kicks (0 means 1) between exact bodies."""
    return _row(BEND, 0, [k0, h, length, k1, 1.0 if full else 0.0, float(kicks)])


def beambeam4d(q_n: float, beta_s: float, sigma_x: float, sigma_y: float, x_c: float = 0.0, y_c: float = 0.0):
    """4D weak-strong beam-beam lens: strong bunch of q_n = charge x particles
    [e] at speed beta_s against the beam, Gaussian sigma_x, sigma_y, centre."""
    return _row(BEAMBEAM4D, 0, [q_n, beta_s, sigma_x, sigma_y, x_c, y_c])


def spacecharge(line_density: float, sigma_z: float, sigma_x: float, sigma_y: float, length: float,
                x_c: float = 0.0, y_c: float = 0.0):
    """Frozen space-charge lens: the beam's own Gaussian charge, peak line
    density [particles/m], bunch length sigma_z [m] (0: coasting beam),
    transverse sigma_x, sigma_y [m], for `length` [m] of ring, centre."""
    return _row(SPACECHARGE, 0, [line_density, sigma_z, sigma_x, sigma_y, length, x_c, y_c])


def aperture_rect(x_min: float, x_max: float, y_min: float, y_max: float):
    return _row(APERTURE_RECT, 0, [x_min, x_max, y_min, y_max])


def aperture_ellipse(a: float, b: float):
    return _row(APERTURE_ELLIPSE, 0, [a, b])


def misaligned(rows, dx: float = 0.0, dy: float = 0.0, tilt: float = 0.0):
    """Rows of one element seen from a frame displaced by (dx, dy) and then
    rotated by `tilt`: shift, rotation, the element, and the inverse
    rotation and shift."""
    rows = list(rows) if isinstance(rows, (list, tuple)) else [rows]
    return ([xy_shift(dx, dy), s_rotation(tilt)] + rows + [s_rotation(-tilt), xy_shift(-dx, -dy)])


def table(rows) -> np.ndarray:
    return np.array(rows, dtype=ELEMENT_DTYPE)


# ----------------------------------------------------------------------------
# Reference particles and particle arrays.

def proton_reference(p0c: float = 450e9):
    """(mass0 [eV], q0 [e], p0c [eV]); 450 GeV read as the momentum p0c."""
    return (PROTON_MASS_EV, 1.0, p0c)


def electron_reference(E0: float = 45.6e9):
    """45.6 GeV read as the total energy E0 of the electron beam."""
    return (ELECTRON_MASS_EV, 1.0, math.sqrt(E0 * E0 - ELECTRON_MASS_EV ** 2))


def make_particles(ref, x, px, y, py, zeta, delta, particle_id=None) -> dict:
    """SoA particle arrays with ptau, rpp, rvv set from delta by the kinematic
    definitions ptau = (E-E0)/(P0 c), rpp = 1/(1+delta), rvv = beta/beta0."""
    m0, _, p0c = ref
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    delta = np.asarray(delta, dtype=np.float64) * np.ones(n)
    E0 = math.sqrt(p0c * p0c + m0 * m0)
    beta0 = p0c / E0
    opd = 1.0 + delta
    E = np.sqrt((p0c * opd) ** 2 + m0 * m0)
    # (E - E0)/p0c written without cancellation
    ptau = p0c * delta * (2.0 + delta) / (E + E0)
    rvv = opd / (1.0 + beta0 * ptau)
    out = dict(
        x=x.copy(), px=np.asarray(px, np.float64) * np.ones(n), y=np.asarray(y, np.float64) * np.ones(n),
        py=np.asarray(py, np.float64) * np.ones(n), zeta=np.asarray(zeta, np.float64) * np.ones(n),
        delta=delta.copy(), ptau=ptau, rpp=1.0 / opd, rvv=rvv,
        state=np.ones(n, np.int32), at_turn=np.zeros(n, np.int32), at_element=np.zeros(n, np.int32),
        particle_id=np.arange(n, dtype=np.int64) if particle_id is None else np.asarray(particle_id, np.int64),
    )
    return out


# ----------------------------------------------------------------------------
# Linear design optics of a table (input preparation only).

def _linear_matrices(row, ref):
    """(Mx 3x3 on (x, px, delta), My 2x2) of one element, to first order."""
    t = int(row["type"])
    p = row["p"]
    Mx = np.eye(3)
    My = np.eye(2)
    if t == DRIFT:
        Mx[0, 1] = p[0]
        My[0, 1] = p[0]
    elif t == MULTIPOLE:
        k1 = p[1]
        hxl, lrad = p[22], p[23]
        Mx[1, 0] = -k1 - (p[0] * hxl / lrad if lrad > 0 else 0.0)
        Mx[1, 2] = hxl
        My[1, 0] = k1
    elif t == DIPEDGE:
        h, e1, hgap, fint = p[0], p[1], p[2], p[3]
        psi = 2.0 * h * hgap * fint * (1.0 + math.sin(e1) ** 2) / math.cos(e1)
        Mx[1, 0] = h * math.tan(e1)
        My[1, 0] = -h * math.tan(e1 - psi)
    elif t == LINEARMAP:
        M = p[:36].reshape(6, 6)
        Mx[:2, :2] = M[:2, :2]
        My[:, :] = M[2:4, 2:4]
    return Mx, My


def design_optics(elements, ref):
    """Courant-Snyder beta/alpha in x and y, dispersion D, D' at the start of
    every element, the tunes, and the momentum-compaction estimate."""
    n = len(elements)
    mats = [_linear_matrices(elements[i], ref) for i in range(n)]
    Mx = np.eye(3)
    My = np.eye(2)
    for a, b in mats:
        Mx = a @ Mx
        My = b @ My

    def cs(M):
        c = 0.5 * (M[0, 0] + M[1, 1])
        if abs(c) >= 1.0:
            raise ValueError("design optics unstable (|cos mu| >= 1)")
        s = math.copysign(math.sqrt(1.0 - c * c), M[0, 1])
        beta = M[0, 1] / s
        alpha = (M[0, 0] - M[1, 1]) / (2.0 * s)
        mu = math.atan2(s, c) % (2 * math.pi)
        return beta, alpha, mu

    bx, ax, mux = cs(Mx)
    by, ay, muy = cs(My)
    # periodic dispersion: (I - M2) D = m
    D = np.linalg.solve(np.eye(2) - Mx[:2, :2], Mx[:2, 2])
    betx = np.zeros(n); alfx = np.zeros(n); bety = np.zeros(n); alfy = np.zeros(n)
    dx = np.zeros(n); dpx = np.zeros(n)
    phx = np.zeros(n); phy = np.zeros(n)
    Bx = np.array([[bx, -ax], [-ax, (1 + ax * ax) / bx]])
    By = np.array([[by, -ay], [-ay, (1 + ay * ay) / by]])
    Dv = np.array([D[0], D[1], 1.0])
    mx = my = 0.0
    for i in range(n):
        betx[i], alfx[i] = Bx[0, 0], -Bx[0, 1]
        bety[i], alfy[i] = By[0, 0], -By[0, 1]
        dx[i], dpx[i] = Dv[0], Dv[1]
        phx[i], phy[i] = mx, my
        a, b = mats[i]
        if a[0, 1] != 0.0:
            mx += math.atan2(a[0, 1], Bx[0, 0] + a[0, 1] * Bx[0, 1])
            my += math.atan2(b[0, 1], By[0, 0] + b[0, 1] * By[0, 1])
        a2 = a[:2, :2]
        Bx = a2 @ Bx @ a2.T
        By = b @ By @ b.T
        Dv = a @ Dv
    # momentum compaction from the thin dipole path lengths: sum hxl * D / C
    C = sum(float(r["p"][0]) for r in elements if int(r["type"]) == DRIFT)
    ac = sum(float(elements[i]["p"][22]) * dx[i] for i in range(n)
             if int(elements[i]["type"]) == MULTIPOLE) / C
    return dict(betx=betx, alfx=alfx, bety=bety, alfy=alfy, dx=dx, dpx=dpx,
                mux=phx, muy=phy, qx=mux / (2 * math.pi), qy=muy / (2 * math.pi),
                alpha_c=ac, length=C)


def longitudinal_beta(elements, ref, optics):
    """Linear synchrotron beta_z = sigma_zeta/sigma_delta from the slip
    eta*C and the summed linear RF slope (input preparation only)."""
    m0, q0, p0c = ref
    E0 = math.sqrt(p0c * p0c + m0 * m0)
    beta0, gamma0 = p0c / E0, E0 / m0
    eta = optics["alpha_c"] - 1.0 / gamma0 ** 2
    C = optics["length"]
    K = 0.0
    for r in elements:
        if int(r["type"]) == CAVITY:
            V, f, lag = r["p"][0], r["p"][1], r["p"][2]
            k = 2 * math.pi * f / (beta0 * C_LIGHT)
            K += q0 * V / p0c * k * math.cos(math.radians(lag)) / beta0
    S = np.array([[1.0, -eta * C], [0.0, 1.0]])
    R = np.array([[1.0, 0.0], [-K, 1.0]])
    M = S @ R
    c = 0.5 * (M[0, 0] + M[1, 1])
    if abs(c) >= 1.0 or K == 0.0:
        raise ValueError("longitudinal motion not stable")
    s = math.copysign(math.sqrt(1 - c * c), M[0, 1])
    return M[0, 1] / s, eta


# ----------------------------------------------------------------------------
# Matched beams and dynamic-aperture grids.

def matched_gaussian(elements, ref, n: int, emit_n: float, sigma_delta: float, seed: int,
                     optics=None, emit_x: float | None = None, emit_y: float | None = None) -> dict:
    """Gaussian 6D beam matched at element 0 to the design optics: normalised
    Gaussian coordinates times the Courant-Snyder matrices, plus the
    dispersion term, zeta from the linear synchrotron beta."""
    m0, _, p0c = ref
    if optics is None:
        optics = design_optics(elements, ref)
    bg0 = p0c / m0
    ex = emit_n / bg0 if emit_x is None else emit_x
    ey = emit_n / bg0 if emit_y is None else emit_y
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((6, n))
    bx, ax = optics["betx"][0], optics["alfx"][0]
    by, ay = optics["bety"][0], optics["alfy"][0]
    delta = sigma_delta * g[4]
    x = math.sqrt(ex * bx) * g[0] + optics["dx"][0] * delta
    px = math.sqrt(ex / bx) * (g[1] - ax * g[0]) + optics["dpx"][0] * delta
    y = math.sqrt(ey * by) * g[2]
    py = math.sqrt(ey / by) * (g[3] - ay * g[2])
    try:
        bz, _ = longitudinal_beta(elements, ref, optics)
    except ValueError:
        bz = 0.0
    zeta = bz * sigma_delta * g[5]
    return make_particles(ref, x, px, y, py, zeta, delta)


def da_grid(elements, ref, n_r: int = 22222, n_theta: int = 9, deltas=(-2, -1, 0, 1, 2),
            sigma_delta: float = 3e-4, r_max: float = 20.0, emit_n: float = 2.5e-6,
            optics=None) -> dict:
    """Polar grid in normalised amplitude: r uniform in (0, r_max] sigma,
    theta_j = 90 deg (j+1)/(n_theta+1), delta in deltas*sigma_delta, placed on
    the dispersive orbit at element 0 with zero normalised momenta.  Ordered
    ray-major (consecutive particles: neighbouring radii on one ray).
    Returns the particles plus ``grid`` = (r, theta_index, delta_index)."""
    m0, _, p0c = ref
    if optics is None:
        optics = design_optics(elements, ref)
    eps = emit_n / (p0c / m0)
    bx, ax = optics["betx"][0], optics["alfx"][0]
    by, ay = optics["bety"][0], optics["alfy"][0]
    r = r_max * (np.arange(n_r) + 1) / n_r
    th = np.radians(90.0 * (np.arange(n_theta) + 1) / (n_theta + 1))
    dl = np.asarray(deltas, dtype=np.float64) * sigma_delta
    R, T, Dd = np.meshgrid(r, np.arange(n_theta), np.arange(len(dl)), indexing="ij")
    # ray-major ordering: (delta, theta) outer, r inner
    R = R.transpose(2, 1, 0).reshape(-1)
    T = T.transpose(2, 1, 0).reshape(-1)
    Dd = Dd.transpose(2, 1, 0).reshape(-1)
    delta = dl[Dd]
    xn = R * np.cos(th[T])
    yn = R * np.sin(th[T])
    x = math.sqrt(eps * bx) * xn + optics["dx"][0] * delta
    px = -ax * math.sqrt(eps / bx) * xn + optics["dpx"][0] * delta
    y = math.sqrt(eps * by) * yn
    py = -ay * math.sqrt(eps / by) * yn
    p = make_particles(ref, x, px, y, py, np.zeros_like(x), delta)
    p["grid"] = (R, T, Dd)
    return p


# ----------------------------------------------------------------------------
# The synthetic rings.

def fodo10(seed: int = BASE_SEED):
    """FODO-10 ring: cells [QF thin knl1=+0.2 (f=5 m), SX thin knl2 = 0.05*N(0,1),
    drift 2 m, QD thin knl1=-0.2, drift 2 m] x 10, plus one thin 400 MHz, 1 MV
    RF cavity (lag 0: below transition) at index 0 -> 51 elements, C = 40 m,
    450 GeV protons."""
    rng = np.random.default_rng(seed)
    rows = [cavity(1e6, 400e6, 0.0)]
    for _ in range(10):
        rows += [multipole(knl=[0, 0.2]), multipole(knl=[0, 0, 0.05 * rng.standard_normal()]),
                 drift(2.0), multipole(knl=[0, -0.2]), drift(2.0)]
    return table(rows), proton_reference(450e9)


def _cell_layout(kf: float, kd: float, k2f: float, k2d: float, theta: float, l_quad: float = 3.1,
                 l_dip: float = 14.3, gap: float = 1.49, quad_slices: int = 4, dip_per_half: int = 3,
                 dip_slices: int = 4, **_):
    """One FODO cell as (kind, main strength, drift after) triples: QF,
    dip_per_half dipoles, SF, QD, dip_per_half dipoles, SD; every magnet split
    into thin slices at the centres of equal parts, every slice followed by a
    drift.  LHC-like defaults: 4 quad slices, 3 x 4 dipole slices per half."""
    seq = []

    def magnet(kind, k, length, n, gap_after):
        for j in range(n):
            d = length / n if j < n - 1 else length / (2 * n) + gap_after
            seq.append((kind, k, d))

    for kq, k2, kq_name, s_name in ((kf, k2f, "QF", "SF"), (kd, k2d, "QD", "SD")):
        magnet(kq_name, kq / quad_slices, l_quad, quad_slices, gap + l_dip / (2 * dip_slices))
        for b in range(dip_per_half):
            last = b == dip_per_half - 1
            magnet("MB", theta, l_dip, dip_slices, gap + (0.0 if last else l_dip / (2 * dip_slices)))
        seq.append((s_name, k2, gap + l_quad / (2 * quad_slices)))
    return seq


def _ring_rows(n_cells, kf, kd, k2f, k2d, theta, l_dip, rf_cells, rf_v, rf_f, rf_lag,
               error_rng=None, error_scale=None, aperture_r=0.02, r_ref=0.017, cell=None):
    """Rows of n_cells cells.  An aperture follows the drift of every
    quadrupole and dipole slice (or where cell["_ap"](kind, dipole slice index
    in the half cell) says); the first aperture of the cells in rf_cells is an
    RF cavity instead."""
    cell = cell or {}
    seq = _cell_layout(kf, kd, k2f, k2d, theta, l_dip=l_dip, **cell)
    ap_rule = cell.get("_ap", None)
    rows = []
    for c in range(n_cells):
        first_ap = True
        mb_in_half = 0
        for kind, k, dlen in seq:
            knl = np.zeros(MAX_ORDER + 1)
            ksl = np.zeros(MAX_ORDER + 1)
            hxl = lrad = 0.0
            if kind in ("QF", "QD"):
                knl[1] = k
                bref = abs(k) * r_ref
            elif kind == "MB":
                knl[0] = k
                hxl = k
                lrad = l_dip / cell.get("dip_slices", 4)
                bref = abs(k)
            else:
                knl[2] = k
                bref = abs(k) * r_ref ** 2 / 2
            order = 2 if kind in ("SF", "SD") else (1 if kind[0] == "Q" else 0)
            if error_rng is not None:
                # b_n, a_n at r_ref relative to the main field, orders 2..10
                g = error_rng.standard_normal((2, MAX_ORDER - 1))
                for n in range(2, MAX_ORDER + 1):
                    fac = bref * 1e-4 * math.factorial(n) / r_ref ** n
                    knl[n] += fac * error_scale[0][n] * g[0, n - 2]
                    ksl[n] += fac * error_scale[1][n] * g[1, n - 2]
                order = MAX_ORDER
            rows.append(multipole(knl=knl, ksl=ksl, hxl=hxl, lrad=lrad, order=order))
            rows.append(drift(dlen))
            if kind == "MB":
                mb_in_half += 1
            elif kind in ("SF", "SD"):
                mb_in_half = 0
            want = kind in ("QF", "QD", "MB") if ap_rule is None else ap_rule(kind, mb_in_half)
            if want:
                if first_ap and c in rf_cells:
                    rows.append(cavity(rf_v, rf_f, rf_lag))
                else:
                    rows.append(aperture(aperture_r))
                first_ap = False
    return table(rows)


def _match_cell(n_cells, qx, qy, theta, l_dip, cell=None, k0=0.0265):
    """Thin-lens FODO strengths giving the requested tunes (design optics)."""
    ref = proton_reference()
    target = np.array([qx, qy])
    k = np.array([k0, -k0])  # integrated per quadrupole, 1/m

    def tunes(kk):
        rows = _ring_rows(1, kk[0], kk[1], 0.0, 0.0, theta, l_dip, (), 0, 0, 0, cell=cell)
        o = design_optics(rows, ref)
        return np.array([o["qx"], o["qy"]]) * n_cells

    for _ in range(30):
        q = tunes(k)
        r = q - target
        if np.max(np.abs(r)) < 1e-10:
            break
        J = np.zeros((2, 2))
        for j in range(2):
            dk = np.zeros(2)
            dk[j] = 1e-7
            J[:, j] = (tunes(k + dk) - q) / 1e-7
        k = k - np.linalg.solve(J, r)
    return k


def _match_chroma(rows_cell, ref, n_cells, target=2.0):
    """Sextupole strengths for the requested linear chromaticity from the
    textbook thin-lens sums over one cell (design optics)."""
    o = design_optics(rows_cell, ref)
    nat_x = nat_y = 0.0
    sx = {"F": [0.0, 0.0], "D": [0.0, 0.0]}
    seen = 0
    for i, r in enumerate(rows_cell):
        if int(r["type"]) != MULTIPOLE:
            continue
        k1 = r["p"][1]
        nat_x += -o["betx"][i] * k1
        nat_y += o["bety"][i] * k1
        if r["p"][2] != 0.0 or (k1 == 0 and r["p"][0] == 0):
            key = "F" if seen == 0 else "D"
            sx[key] = [o["betx"][i] * o["dx"][i], -o["bety"][i] * o["dx"][i]]
            seen += 1
    A = np.array([[sx["F"][0], sx["D"][0]], [sx["F"][1], sx["D"][1]]]) * n_cells / (4 * math.pi)
    b = np.array([target, target]) - np.array([nat_x, nat_y]) * n_cells / (4 * math.pi)
    return np.linalg.solve(A, b)


def lhc_ring(seed: int = BASE_SEED, n_cells: int = 200, error_scales=None,
             with_errors: bool = True, qx: float | None = None, qy: float | None = None,
             rf_voltage: float = 2e6):
    """LHC-scale synthetic ring: n_cells x 100 thin elements (200 cells ->
    20,000): per cell 8 thin quadrupole slices, 24 thin dipole slices
    (theta = 2 pi/(24 n_cells), L_rad = 14.3/4 m), 2 thin sextupoles (linear
    chromaticity ~ +2), 34 drifts and 32 circular apertures (r = 20 mm), of
    which 8 ring-wide are replaced by 400 MHz RF cavities (2 MV each, lag 180
    deg, above transition).  Field errors on every multipole slice, orders
    2..10 normal and skew, Gaussian at 1e-4 of the main field at R_ref = 17 mm,
    times per-(order, normal/skew) scales ``error_scales`` (2 x 11, default 1).
    Cell length 106.9 m; 450 GeV protons; default tunes 49.31/49.32 for
    200 cells (the same phase advance per cell for other cell counts)."""
    ref = proton_reference(450e9)
    theta = 2 * math.pi / (24 * n_cells)
    l_dip = 14.3
    qx = 49.31 * n_cells / 200 if qx is None else qx
    qy = 49.32 * n_cells / 200 if qy is None else qy
    kf, kd = _match_cell(n_cells, qx, qy, theta, l_dip)
    cell0 = _ring_rows(1, kf, kd, 1e-9, -1e-9, theta, l_dip, (), 0, 0, 0)
    k2f, k2d = _match_chroma(cell0, ref, n_cells)
    rf_cells = tuple(int(round(i * n_cells / 8)) for i in range(8))
    scale = np.ones((2, MAX_ORDER + 1)) if error_scales is None else np.asarray(error_scales)
    rng = np.random.default_rng(seed) if with_errors else None
    rows = _ring_rows(n_cells, kf, kd, k2f, k2d, theta, l_dip, rf_cells, rf_voltage, 400e6, 180.0,
                      error_rng=rng, error_scale=scale)
    return rows, ref


def _lepton_aperture(kind, dipole_slice):
    return kind in ("QF", "QD") or (kind == "MB" and dipole_slice == 1)


LEPTON_CELL = dict(quad_slices=2, dip_per_half=2, dip_slices=4, l_quad=2.0, gap=1.0, _ap=_lepton_aperture)


def lepton_ring(n_cells: int = 200, E0: float = 45.6e9, v_total: float = 500e6, rf_every: int = 1):
    """Lepton ring with radiation: 200 FODO cells of 50 thin elements
    (10,000): per cell QF and QD in 2 slices, 2 dipoles of 4 slices per half
    cell (theta = 2 pi/(16 n_cells), L_rad = 10.7/4 m, bending radius 1.36 km),
    2 sextupoles (linear chromaticity ~ +2), 22 drifts and 6 apertures
    (r = 20 mm), of which one per cell is an RF cavity.  45.6 GeV electrons,
    no field errors.  The RF (400 MHz, V_total = 500 MV) is phased at
    180 deg - arcsin(U0/V_total) with the design energy loss
    U0 = C_gamma E0^4 I2 / (2 pi), C_gamma = 8.846e-5 m/GeV^3,
    I2 = sum theta^2 / L_rad.  The ring has no dispersion-free straights, so
    the RF is spread over every cell: a few lumped stations would make the
    radiation energy sawtooth jump the dispersive orbit at each station and
    excite betatron motion; rf_every > 1 lumps the RF into stations every
    rf_every cells (the case that energy-loss compensation addresses)."""
    ref = electron_reference(E0)
    theta = 2 * math.pi / (16 * n_cells)
    l_dip = 10.7
    cell = LEPTON_CELL
    mu = 0.2466  # phase advance per cell [2 pi], about 89 degrees
    base = round(mu * n_cells)
    kf, kd = _match_cell(n_cells, base + 0.31, base + 0.32, theta, l_dip, cell=cell, k0=0.05)
    cell0 = _ring_rows(1, kf, kd, 1e-9, -1e-9, theta, l_dip, (), 0, 0, 0, cell=cell)
    k2f, k2d = _match_chroma(cell0, electron_reference(E0), n_cells)
    I2 = 16 * n_cells * theta ** 2 / (l_dip / 4)
    U0 = 8.846e-5 * (E0 / 1e9) ** 4 * I2 / (2 * math.pi) * 1e9
    lag = 180.0 - math.degrees(math.asin(U0 / v_total))
    rf_cells = tuple(range(0, n_cells, rf_every))
    rows = _ring_rows(n_cells, kf, kd, k2f, k2d, theta, l_dip, rf_cells, v_total / len(rf_cells),
                      400e6, lag, cell=cell)
    return rows, ref, dict(U0=U0, I2=I2, lag=lag)


def seed_error_scales(i: int):
    """Per-seed error scales for the batched-seed workload: log-uniform in
    [0.5, 2] for normal and skew orders 2..6 (10 descriptors), 1 elsewhere.
    Returns (scales 2x11, descriptors = log(scales) at those 10 entries)."""
    rng = np.random.default_rng(BASE_SEED + 7919 * (i + 1))
    s = np.ones((2, MAX_ORDER + 1))
    desc = rng.uniform(math.log(0.5), math.log(2.0), size=(2, 5))
    s[:, 2:7] = np.exp(desc)
    return s, desc.reshape(-1)


def batched_seed_counts(n_seeds: int = 64, seed: int = BASE_SEED) -> np.ndarray:
    """Uneven particle counts per seed: round(10**U(3, 5))."""
    rng = np.random.default_rng(seed + 1)
    return np.round(10.0 ** rng.uniform(3.0, 5.0, size=n_seeds)).astype(np.int64)


def polar_sample(elements, ref, n: int, seed: int, r_max: float = 20.0, emit_n: float = 2.5e-6,
                 sigma_delta: float = 3e-4, optics=None) -> dict:
    """Random amplitudes for the batched-seed workload: r uniform in
    [0, r_max] sigma, theta uniform in (0, 90) deg, delta ~ N(0, sigma_delta),
    zero normalised momenta, zeta = 0.  Returns particles plus ``norm`` =
    (r, theta, delta)."""
    m0, _, p0c = ref
    if optics is None:
        optics = design_optics(elements, ref)
    eps = emit_n / (p0c / m0)
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, r_max, n)
    th = rng.uniform(0.0, 0.5 * math.pi, n)
    delta = np.clip(rng.standard_normal(n), -3, 3) * sigma_delta
    bx, ax = optics["betx"][0], optics["alfx"][0]
    by, ay = optics["bety"][0], optics["alfy"][0]
    xn, yn = r * np.cos(th), r * np.sin(th)
    x = math.sqrt(eps * bx) * xn + optics["dx"][0] * delta
    px = -ax * math.sqrt(eps / bx) * xn + optics["dpx"][0] * delta
    y = math.sqrt(eps * by) * yn
    py = -ay * math.sqrt(eps / by) * yn
    p = make_particles(ref, x, px, y, py, np.zeros(n), delta)
    p["norm"] = (r, th, delta)
    return p


def subset(particles: dict, idx) -> dict:
    idx = np.asarray(idx, dtype=np.int64)
    return {k: (v[idx].copy() if isinstance(v, np.ndarray) else v)
            for k, v in particles.items() if k not in ("grid", "norm")}
