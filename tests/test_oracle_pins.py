"""Pins of the oracle tracker against closed forms, invariants, special cases,
independent libraries and high-precision brute force (CPU only).

Each test checks the oracle against something other than itself, chosen so
that a dropped term, a wrong sign or index, or a transposed operand in one of
its maps fails at least one of them.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from paper_2310_00317_gb300 import inputs as I

J6 = np.zeros((6, 6))
for k in range(3):
    J6[2 * k, 2 * k + 1] = 1.0
    J6[2 * k + 1, 2 * k] = -1.0

PROTON = I.proton_reference(450e9)


def one(ref, x=0.0, px=0.0, y=0.0, py=0.0, zeta=0.0, delta=0.0):
    return I.make_particles(ref, [x], [px], [y], [py], [zeta], [delta])


def hp_kin(ref, delta):
    """High-precision kinematics (mpmath) of a particle with momentum deviation delta."""
    m0, _, p0c = [mpmath.mpf(v) for v in ref]
    d = mpmath.mpf(delta)
    E0 = mpmath.sqrt(p0c ** 2 + m0 ** 2)
    E = mpmath.sqrt((p0c * (1 + d)) ** 2 + m0 ** 2)
    beta0 = p0c / E0
    beta = p0c * (1 + d) / E
    ptau = (E - E0) / p0c
    return dict(E0=E0, beta0=beta0, beta=beta, ptau=ptau, rvv=beta / beta0)


# --------------------------------------------------------------------------
# Exact drift

def test_drift_closed_form_highprec():
    """Drift against the straight-line closed form in 40-digit arithmetic."""
    mpmath.mp.dps = 40
    rng = np.random.default_rng(1)
    for _ in range(20):
        x, px, y, py, z = rng.normal(0, [1e-3, 1e-4, 1e-3, 1e-4, 1e-2])
        d = rng.normal(0, 1e-3)
        L = float(rng.uniform(0.1, 20.0))
        p = one(PROTON, x, px, y, py, z, d)
        el = I.table([I.drift(L)])
        o = oracle.track(el, PROTON, p, 1)
        k = hp_kin(PROTON, p["delta"][0])
        opd = 1 + mpmath.mpf(p["delta"][0])
        PX, PY = mpmath.mpf(p["px"][0]), mpmath.mpf(p["py"][0])
        pz = mpmath.sqrt(opd ** 2 - PX ** 2 - PY ** 2)
        # path length L(1+delta)/pz travelled at beta: zeta += L - beta0/beta * path
        xe = mpmath.mpf(p["x"][0]) + PX * L / pz
        ye = mpmath.mpf(p["y"][0]) + PY * L / pz
        ze = mpmath.mpf(p["zeta"][0]) + L - (k["beta0"] / k["beta"]) * L * opd / pz
        # rounding bound scales with the operands (the sum may cancel)
        assert abs(o["x"][0] - float(xe)) <= 4e-16 * (abs(x) + abs(px) * L)
        assert abs(o["y"][0] - float(ye)) <= 4e-16 * (abs(y) + abs(py) * L)
        # zeta change is a small difference of O(L) terms: absolute bound
        assert abs(o["zeta"][0] - float(ze)) <= 8e-16 * L
        assert o["px"][0] == p["px"][0] and o["delta"][0] == p["delta"][0]


@pytest.mark.parametrize("d", [0.0, 3e-4, -2e-3, 4e-3, -6e-3, 0.02, -0.05, 0.3])
def test_drift_over_momentum_range(d):
    """x and the zeta increment against 40-digit arithmetic from near
    momentum to 30 % off it.  The increment is formed from ptau, which the
    stored (delta, ptau, rvv) satisfy to rounding, hence the absolute
    2e-16 L term."""
    mpmath.mp.dps = 40
    L = 3.7
    x, px, y, py = 1e-3, 2e-4, -1e-3, -1e-4
    p = one(PROTON, x, px, y, py, 0.0, d)
    o = oracle.track(I.table([I.drift(L)]), PROTON, p, 1)
    k = hp_kin(PROTON, p["delta"][0])
    opd = 1 + mpmath.mpf(p["delta"][0])
    pz = mpmath.sqrt(opd ** 2 - mpmath.mpf(px) ** 2 - mpmath.mpf(py) ** 2)
    xe = x + mpmath.mpf(px) * L / pz
    dz = L - (k["beta0"] / k["beta"]) * L * opd / pz
    assert abs(o["x"][0] - float(xe)) <= 4e-16 * (abs(x) + abs(px) * L)
    assert abs(o["zeta"][0] - float(dz)) <= 2e-16 * L + 1e-15 * abs(float(dz))


@pytest.mark.parametrize("d", [0.0, 1e-9, -3e-7, 2e-5, -6e-4, 1e-3])
def test_drift_zeta_increment_relative_accuracy(d):
    """The zeta increment L (1 - (1+delta)/(rvv pz)) is a small difference of
    O(L) terms (about 1e-9 L near momentum at 450 GeV).  Against 40-digit
    arithmetic it must hold to 1e-14 of itself for small angles and small
    momentum deviations, so that 1000 turns of a ring do not accumulate a
    cancellation error; a dropped 1/gamma0^2 or a sign slip in the
    cancellation-free form fails here.  ptau is given and delta, rvv
    derived from it in 40 digits, so the stored state is consistent."""
    mpmath.mp.dps = 40
    L = 2.7
    m0, _, p0c = [mpmath.mpf(v) for v in PROTON]
    E0 = mpmath.sqrt(p0c ** 2 + m0 ** 2)
    beta0 = p0c / E0
    for px, py in [(0.0, 0.0), (1e-6, 0.0), (3e-5, -2e-5), (2e-4, 1e-4)]:
        ptau = float(mpmath.mpf(d) * beta0)
        PT = mpmath.mpf(ptau)
        opd = mpmath.sqrt(1 + 2 * PT / beta0 + PT ** 2)
        rvv = opd / (1 + beta0 * PT)
        p = one(PROTON, 0.0, px, 0.0, py, 0.0, 0.0)
        p["ptau"][0] = ptau
        p["delta"][0] = float(opd - 1)
        p["rpp"][0] = float(1 / opd)
        p["rvv"][0] = float(rvv)
        o = oracle.track(I.table([I.drift(L)]), PROTON, p, 1)
        PX, PY = mpmath.mpf(px), mpmath.mpf(py)
        pz = mpmath.sqrt(opd ** 2 - PX ** 2 - PY ** 2)
        dz = L - L * opd / (rvv * pz)
        if dz == 0:
            assert o["zeta"][0] == 0.0
        else:
            assert abs(o["zeta"][0] - float(dz)) <= 1e-14 * abs(float(dz)), (px, py, o["zeta"][0], float(dz))


def test_drift_reversible():
    """A drift of -L undoes a drift of +L to rounding."""
    rng = np.random.default_rng(2)
    n = 200
    p = I.make_particles(PROTON, rng.normal(0, 1e-3, n), rng.normal(0, 1e-4, n),
                         rng.normal(0, 1e-3, n), rng.normal(0, 1e-4, n),
                         rng.normal(0, 0.1, n), rng.normal(0, 1e-3, n))
    el = I.table([I.drift(7.3), I.drift(-7.3)])
    o = oracle.track(el, PROTON, p, 1)
    for k in ("x", "y"):
        assert np.max(np.abs(o[k] - p[k])) <= 4e-18 + 4 * np.spacing(np.max(np.abs(p[k])))
    assert np.max(np.abs(o["zeta"] - p["zeta"])) < 1e-15


def test_drift_invalid_momentum_lost():
    p = one(PROTON, px=0.8, py=0.7)  # px^2 + py^2 > (1+delta)^2
    o = oracle.track(I.table([I.drift(1.0), I.drift(1.0)]), PROTON, p, 3)
    assert o["state"][0] == -2 and o["at_turn"][0] == 0 and o["at_element"][0] == 0
    assert o["x"][0] == p["x"][0] and o["zeta"][0] == p["zeta"][0]


# --------------------------------------------------------------------------
# Thin multipole

@pytest.mark.parametrize("order", list(range(11)))
def test_multipole_kick_vs_bruteforce(order):
    """Horner kick vs the term-by-term sum with mpmath powers."""
    mpmath.mp.dps = 40
    rng = np.random.default_rng(10 + order)
    knl = rng.normal(0, 1, order + 1) * 10.0 ** -np.arange(order + 1)
    ksl = rng.normal(0, 1, order + 1) * 10.0 ** -np.arange(order + 1)
    el = I.table([I.multipole(knl=knl, ksl=ksl, order=order)])
    for _ in range(5):
        x, y = rng.normal(0, 0.01, 2)
        px, py = rng.normal(0, 1e-4, 2)
        p = one(PROTON, x, px, y, py, 0.0, 1e-4)
        o = oracle.track(el, PROTON, p, 1)
        z = mpmath.mpc(x, y)
        b = mpmath.mpc(0)
        scale = mpmath.mpf(0)
        for n in range(order + 1):
            term = mpmath.mpc(knl[n], ksl[n]) * z ** n / math.factorial(n)
            b += term
            scale += abs(term)
        tol = 8e-16 * float(scale) + 1e-20
        assert abs(o["px"][0] - float(px - b.real)) <= tol + 1e-16 * abs(px)
        assert abs(o["py"][0] - float(py + b.imag)) <= tol + 1e-16 * abs(py)
        assert o["x"][0] == x and o["y"][0] == y


def test_multipole_sign_conventions():
    """Normal quad focuses x (dpx=-kx, dpy=+ky); skew quad dpx=+ky, dpy=+kx;
    sextupole dpx=-(k2/2)(x^2-y^2), dpy=k2 x y."""
    x, y = 3e-3, -2e-3
    cases = [
        (I.multipole(knl=[0, 0.1]), -0.1 * x, 0.1 * y),
        (I.multipole(ksl=[0, 0.1]), 0.1 * y, 0.1 * x),
        (I.multipole(knl=[0, 0, 0.4]), -0.2 * (x * x - y * y), 0.4 * x * y),
        (I.multipole(knl=[1e-4]), -1e-4, 0.0),
        (I.multipole(ksl=[1e-4]), 0.0, 1e-4),
    ]
    for row, dpx, dpy in cases:
        o = oracle.track(I.table([row]), PROTON, one(PROTON, x=x, y=y), 1)
        assert o["px"][0] == pytest.approx(dpx, rel=1e-14, abs=1e-22)
        assert o["py"][0] == pytest.approx(dpy, rel=1e-14, abs=1e-22)


def test_multipole_curvature_terms():
    """Thin dipole of the curved frame: px += hxl(1+delta) - knl0 hxl x/L,
    zeta -= hxl x / rvv (evaluated in high precision)."""
    mpmath.mpf.dps = 40
    hxl, L = 1.3e-3, 3.575
    el = I.table([I.multipole(knl=[hxl], hxl=hxl, lrad=L)])
    for d in (-2e-3, 0.0, 1.5e-3):
        x = 4e-3
        p = one(PROTON, x=x, delta=d)
        o = oracle.track(el, PROTON, p, 1)
        k = hp_kin(PROTON, d)
        px = -hxl + hxl * (1 + mpmath.mpf(p["delta"][0])) - hxl * hxl * x / L
        zeta = -hxl * x / k["rvv"]
        assert o["px"][0] == pytest.approx(float(px), rel=1e-12, abs=1e-19)
        assert o["zeta"][0] == pytest.approx(float(zeta), rel=1e-13)


# --------------------------------------------------------------------------
# Linear optics: FODO phase advance, symplecticity, invariants

def test_fodo_cell_phase_advance():
    """Thin FODO with f = 5 m and 2 m drifts: cos mu = 1 - L^2/(2 f^2) = 0.92."""
    cell = I.table([I.multipole(knl=[0, 0.2]), I.drift(2.0), I.multipole(knl=[0, -0.2]), I.drift(2.0)])
    _, M = oracle.track_jacobian(cell, PROTON, np.zeros(6))
    assert 0.5 * np.trace(M[:2, :2]) == pytest.approx(0.92, abs=1e-14)
    assert 0.5 * np.trace(M[2:4, 2:4]) == pytest.approx(0.92, abs=1e-14)


def test_fodo10_ring_tune():
    """The FODO-10 ring (sextupoles off the closed orbit do not act linearly)
    has Q = 10 arccos(0.92)/(2 pi) = 0.6408..."""
    el, ref = I.fodo10()
    co = oracle.closed_orbit(el, ref, dim=6)
    _, M = oracle.track_jacobian(el, ref, co)
    # cos(2 pi Q) with Q = 10 arccos(0.92)/(2 pi); the trace fixes Q up to 1-Q
    assert 0.5 * np.trace(M[:2, :2]) == pytest.approx(math.cos(10 * math.acos(0.92)), abs=1e-12)
    assert 0.5 * np.trace(M[2:4, 2:4]) == pytest.approx(math.cos(10 * math.acos(0.92)), abs=1e-12)
    assert np.max(np.abs(co)) < 1e-14


@pytest.mark.parametrize("which", ["fodo10", "lhc_cells"])
def test_symplectic_one_turn(which):
    """M^T J M = J to 1e-13 for the analytic one-turn Jacobian in canonical
    (x, px, y, py, zeta, pzeta), radiation off, at an off-axis point."""
    if which == "fodo10":
        el, ref = I.fodo10()
        z0 = np.array([2e-4, 1e-5, -1e-4, 2e-5, 0.05, 2e-4])
    else:
        full, ref = I.lhc_ring(n_cells=8)
        el = full
        z0 = np.array([1e-3, 1e-5, 1e-3, -1e-5, 0.01, 1e-4])
    _, M = oracle.track_jacobian(el, ref, z0)
    E = M.T @ J6 @ M - J6
    assert np.max(np.abs(E)) < 1e-13 * max(1.0, np.max(np.abs(M)) ** 2)


def _rot6(mu, beta=1.0):
    M = np.eye(6)
    c, s = math.cos(mu), math.sin(mu)
    M[0, 0], M[0, 1], M[1, 0], M[1, 1] = c, beta * s, -s / beta, c
    return M


def test_courant_snyder_action_conserved():
    """Linear lattice (linear-map elements and thin quadrupoles, delta = 0):
    the Courant-Snyder action from the one-turn matrix is conserved to 1e-13
    over 1e4 turns.  The linear maps are exact shears (dyadic entries, det = 1
    exactly) so only the tracker's own rounding can change the action."""
    S = np.eye(6)
    S[0, 1] = 2.0
    S[2, 3] = 2.0
    el = I.table([I.multipole(knl=[0, 0.25]), I.linear_map(S), I.multipole(knl=[0, -0.25]), I.linear_map(S)])
    _, M = oracle.track_jacobian(el, PROTON, np.zeros(6))
    A = M[:2, :2]
    c = 0.5 * np.trace(A)
    s = math.copysign(math.sqrt(1 - c * c), A[0, 1])
    beta, alpha = A[0, 1] / s, (A[0, 0] - A[1, 1]) / (2 * s)
    gamma = (1 + alpha ** 2) / beta
    rng = np.random.default_rng(3)
    n = 16
    p = I.make_particles(PROTON, rng.normal(0, 1e-3, n), rng.normal(0, 1e-4, n),
                         np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n))
    J0 = gamma * p["x"] ** 2 + 2 * alpha * p["x"] * p["px"] + beta * p["px"] ** 2
    o = oracle.track(el, PROTON, p, 10000)
    J1 = gamma * o["x"] ** 2 + 2 * alpha * o["x"] * o["px"] + beta * o["px"] ** 2
    assert np.all(o["state"] == 1)
    assert np.max(np.abs(J1 / J0 - 1)) < 1e-13


def test_henon_map():
    """Rotation by mu (beta = 1, alpha = 0) + thin sextupole k2 on y = 0 is the
    Henon map: with X = (k2/2) x, P = (k2/2) px, (X, P) -> R(mu)(X, P - X^2).
    Iterates agree with a 40-digit evaluation to 1e-12 relative for 1000 turns."""
    mpmath.mp.dps = 40
    mu, k2 = 2 * math.pi * 0.2114, 2.0
    el = I.table([I.multipole(knl=[0, 0, k2]), I.linear_map(_rot6(mu))])
    starts = [0.05, 0.1, 0.2]
    p = I.make_particles(PROTON, [s / (k2 / 2) for s in starts], np.zeros(3), np.zeros(3),
                         np.zeros(3), np.zeros(3), np.zeros(3))
    o = oracle.track(el, PROTON, p, 1000)
    c, s = mpmath.cos(mpmath.mpf(mu)), mpmath.sin(mpmath.mpf(mu))
    for i, X0 in enumerate(starts):
        X, P = mpmath.mpf(p["x"][i]) * k2 / 2, mpmath.mpf(0)
        for _ in range(1000):
            P = P - X * X
            X, P = c * X + s * P, -s * X + c * P
        assert o["state"][i] == 1
        assert o["x"][i] * k2 / 2 == pytest.approx(float(X), rel=1e-12, abs=1e-14)
        assert o["px"][i] * k2 / 2 == pytest.approx(float(P), rel=1e-12, abs=1e-14)


def test_linear_map_element():
    rng = np.random.default_rng(4)
    M = np.eye(6) + rng.normal(0, 1e-2, (6, 6))
    d = rng.normal(0, 1e-6, 6)
    el = I.table([I.linear_map(M, d)])
    z0 = np.array([1e-3, 2e-5, -1e-3, 1e-5, 0.02, 3e-4])
    z1, J = oracle.track_jacobian(el, PROTON, z0)
    assert np.allclose(z1, M @ z0 + d, rtol=1e-14, atol=1e-19)
    assert np.allclose(J, M, rtol=1e-13, atol=1e-15)


def test_dipedge_matrix():
    h, e1, hgap, fint = 1 / 500.0, 0.03, 0.02, 0.5
    el = I.table([I.dipedge(h, e1, hgap, fint)])
    _, M = oracle.track_jacobian(el, PROTON, np.zeros(6))
    psi = 2 * h * hgap * fint * (1 + math.sin(e1) ** 2) / math.cos(e1)
    assert M[1, 0] == pytest.approx(h * math.tan(e1), rel=1e-15)
    assert M[3, 2] == pytest.approx(-h * math.tan(e1 - psi), rel=1e-15)
    assert np.linalg.det(M) == pytest.approx(1.0, abs=1e-15)
    M2 = M.copy(); M2[1, 0] = 0; M2[3, 2] = 0
    assert np.array_equal(M2, np.eye(6))


# --------------------------------------------------------------------------
# RF cavity and energy variables

def test_rf_energy_identity():
    """After an RF kick: (1+delta)^2 = 1 + 2 ptau/beta0 + ptau^2, rpp (1+delta) = 1,
    rvv = beta/beta0 of the particle (high-precision kinematics)."""
    mpmath.mp.dps = 40
    el = I.table([I.cavity(5e6, 400e6, 30.0)])
    rng = np.random.default_rng(5)
    n = 50
    p = I.make_particles(PROTON, np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n),
                         rng.normal(0, 0.2, n), rng.normal(0, 1e-3, n))
    o = oracle.track(el, PROTON, p, 1)
    rc = oracle.ref_constants(PROTON)
    for i in range(n):
        pt = mpmath.mpf(o["ptau"][i])
        lhs = (1 + mpmath.mpf(o["delta"][i])) ** 2
        rhs = 1 + 2 * pt / mpmath.mpf(rc["beta0"]) + pt ** 2
        assert abs(float(lhs - rhs)) < 4e-16
        assert o["rpp"][i] * (1 + o["delta"][i]) == pytest.approx(1.0, abs=3e-16)
        k = hp_kin(PROTON, o["delta"][i])
        assert o["rvv"][i] == pytest.approx(float(k["rvv"]), rel=2e-15)
        # energy gain: q V sin(lag - k zeta)
        phi = math.radians(30.0) - 2 * math.pi * 400e6 / (rc["beta0"] * I.C_LIGHT) * p["zeta"][i]
        assert o["ptau"][i] - p["ptau"][i] == pytest.approx(5e6 / 450e9 * math.sin(phi), rel=1e-9, abs=1e-18)


def test_fodo10_synchrotron_tune():
    """Small-amplitude synchrotron tune of FODO-10 against
    cos(2 pi Qs) = 1 + eta C q V omega cos(lag) / (2 beta0^2 p0c c),
    eta = -1/gamma0^2 (no bends)."""
    el, ref = I.fodo10()
    co = oracle.closed_orbit(el, ref, dim=6)
    _, M = oracle.track_jacobian(el, ref, co)
    rc = oracle.ref_constants(ref)
    eta = -1.0 / rc["gamma0"] ** 2
    C = 40.0
    omega = 2 * math.pi * 400e6
    cs = 1 + eta * C * 1e6 * omega * 1.0 / (2 * rc["beta0"] ** 2 * ref[2] * I.C_LIGHT)
    assert 0.5 * np.trace(M[4:, 4:]) == pytest.approx(cs, abs=1e-13)


# --------------------------------------------------------------------------
# Aperture and loss bookkeeping

def test_aperture_and_guard():
    r = 0.02
    el = I.table([I.aperture(r), I.drift(1.0)])
    xs = [0.0, r, 0.019, 0.014, 0.0142, float("nan"), 0.5]
    ys = [0.0, 0.0, 0.0, 0.014, 0.0142, 0.0, 0.0]
    p = I.make_particles(PROTON, xs, np.zeros(7), ys, np.zeros(7), np.zeros(7), np.zeros(7))
    p["state"][:] = 1
    o = oracle.track(el, PROTON, p, 2, start_turn=5)
    # on the circle survives; 0.014*sqrt(2) < r survives; 0.0142*sqrt(2) > r lost
    assert list(o["state"]) == [1, 1, 1, 1, 0, -1, 0]
    assert list(o["at_turn"]) == [7, 7, 7, 7, 5, 5, 5]
    assert o["x"][4] == 0.0142 and o["at_element"][4] == 0
    # end-of-turn guard (|x| > 1 m) with no aperture
    p2 = one(PROTON, x=1.5)
    o2 = oracle.track(I.table([I.drift(1.0)]), PROTON, p2, 3)
    assert o2["state"][0] == -3 and o2["at_turn"][0] == 0 and o2["at_element"][0] == 0


# --------------------------------------------------------------------------
# Misalignments and tilts (changes of reference frame) and aperture shapes

def _track_xy(elements, xs, ys, pxs=None, pys=None, n_turns=1):
    n = len(xs)
    pxs = np.zeros(n) if pxs is None else np.asarray(pxs, float)
    pys = np.zeros(n) if pys is None else np.asarray(pys, float)
    p = I.make_particles(PROTON, np.asarray(xs, float), pxs, np.asarray(ys, float), pys, np.zeros(n), np.zeros(n))
    return oracle.track(I.table(elements), PROTON, p, n_turns)


def test_srotation_identities():
    """A rotation about s keeps x^2 + y^2 and px^2 + py^2, rotations compose
    additively, theta then -theta returns to the start, a quarter turn maps
    (x, y) to (y, -x), and the map is symplectic."""
    rng = np.random.default_rng(21)
    n = 50
    xs, ys, pxs, pys = (rng.normal(0, s, n) for s in (1e-3, 1e-3, 1e-4, 1e-4))
    th1, th2 = 0.37, -1.21
    a = _track_xy([I.s_rotation(th1), I.s_rotation(th2)], xs, ys, pxs, pys)
    b = _track_xy([I.s_rotation(th1 + th2)], xs, ys, pxs, pys)
    for k, sc in (("x", 1e-3), ("y", 1e-3), ("px", 1e-4), ("py", 1e-4)):
        assert np.max(np.abs(a[k] - b[k])) < 8e-16 * sc * 10
    np.testing.assert_allclose(a["x"] ** 2 + a["y"] ** 2, xs ** 2 + ys ** 2, rtol=1e-14)
    np.testing.assert_allclose(a["px"] ** 2 + a["py"] ** 2, pxs ** 2 + pys ** 2, rtol=1e-14)
    c = _track_xy([I.s_rotation(th1), I.s_rotation(-th1)], xs, ys, pxs, pys)
    assert np.max(np.abs(c["x"] - xs)) < 1e-18 and np.max(np.abs(c["py"] - pys)) < 1e-19
    q = _track_xy([I.s_rotation(math.pi / 2)], xs, ys, pxs, pys)
    assert np.max(np.abs(q["x"] - ys)) < 1e-18 and np.max(np.abs(q["y"] + xs)) < 1e-18
    _, M = oracle.track_jacobian(I.table([I.s_rotation(th1), I.drift(2.0), I.s_rotation(th2)]), PROTON,
                                 np.array([1e-3, 1e-5, -2e-3, 3e-5, 0.0, 1e-4]))
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-14


def test_xyshift_round_trip():
    rng = np.random.default_rng(22)
    xs, ys = rng.normal(0, 1e-3, 40), rng.normal(0, 1e-3, 40)
    o = _track_xy([I.xy_shift(2.5e-3, -1.25e-3), I.xy_shift(-2.5e-3, 1.25e-3)], xs, ys)
    assert np.max(np.abs(o["x"] - xs)) <= np.max(np.spacing(np.abs(xs) + 2.5e-3))
    assert np.max(np.abs(o["y"] - ys)) <= np.max(np.spacing(np.abs(ys) + 1.25e-3))
    o1 = _track_xy([I.xy_shift(2.5e-3, -1.25e-3)], [2.5e-3], [-1.25e-3])
    assert o1["x"][0] == 0.0 and o1["y"][0] == 0.0


def test_rect_aperture_edges():
    """One ulp inside each edge survives, one ulp outside is lost, corners and
    edges survive, a non-finite coordinate is lost with state -1."""
    x0, x1, y0, y1 = -0.01, 0.02, -0.004, 0.006
    el = [I.aperture_rect(x0, x1, y0, y1)]
    up, dn = (lambda v: np.nextafter(v, np.inf)), (lambda v: np.nextafter(v, -np.inf))
    xs = [x0, x1, x0, x1, dn(x0), up(x1), 0.0, 0.0, up(x0), dn(x1), 0.0, float("nan")]
    ys = [y0, y1, y1, y0, 0.0, 0.0, dn(y0), up(y1), 0.0, 0.0, float("inf"), 0.0]
    o = _track_xy(el + [I.drift(0.5)], xs, ys)
    assert list(o["state"]) == [1, 1, 1, 1, 0, 0, 0, 0, 1, 1, -1, -1]


def test_ellipse_aperture_boundary():
    a, b = 0.03, 0.012
    t = np.linspace(0.0, 2 * math.pi, 37)[:-1]
    xs, ys = a * np.cos(t), b * np.sin(t)
    inside = _track_xy([I.aperture_ellipse(a, b)], xs * (1 - 1e-12), ys * (1 - 1e-12))
    outside = _track_xy([I.aperture_ellipse(a, b)], xs * (1 + 1e-12), ys * (1 + 1e-12))
    assert np.all(inside["state"] == 1) and np.all(outside["state"] == 0)


def test_tilted_shifted_apertures_geometry():
    """A rectangle and an ellipse displaced by (dx, dy) and tilted by theta
    (the aperture transition of the paper's loss-location figure): the loss
    decision of random points away from the boundary equals a half-plane test
    against the rectangle's corners in the laboratory frame, and the
    laboratory-frame quadratic form (p - d)^T Q (p - d) <= 1 of the ellipse."""
    rng = np.random.default_rng(23)
    dx, dy, th = 1.5e-3, -0.8e-3, 0.35
    x0, x1, y0, y1 = -0.012, 0.010, -0.006, 0.007
    n = 4000
    xs, ys = rng.uniform(-0.02, 0.02, n), rng.uniform(-0.015, 0.015, n)
    o = _track_xy(I.misaligned([I.aperture_rect(x0, x1, y0, y1)], dx, dy, th), xs, ys)
    # corners in the lab frame: d + R(-theta) (u, v), counter-clockwise
    c, s = math.cos(th), math.sin(th)
    corners = [(dx + c * u - s * v, dy + s * u + c * v) for u, v in ((x0, y0), (x1, y0), (x1, y1), (x0, y1))]
    cross = np.stack([(bx - ax) * (ys - ay) - (by - ay) * (xs - ax)
                      for (ax, ay), (bx, by) in zip(corners, corners[1:] + corners[:1])])
    sure_in = np.all(cross > 1e-12, axis=0)
    sure_out = np.any(cross < -1e-12, axis=0)
    assert sure_in.sum() > 500 and sure_out.sum() > 500
    assert np.all(o["state"][sure_in] == 1) and np.all(o["state"][sure_out] == 0)
    a, b = 0.011, 0.006
    o = _track_xy(I.misaligned([I.aperture_ellipse(a, b)], dx, dy, th), xs, ys)
    R = np.array([[c, s], [-s, c]])
    Q = R.T @ np.diag([1 / a ** 2, 1 / b ** 2]) @ R
    d = np.stack([xs - dx, ys - dy])
    f = np.einsum("in,ij,jn->n", d, Q, d)
    assert np.all(o["state"][f < 1 - 1e-9] == 1) and np.all(o["state"][f > 1 + 1e-9] == 0)


def test_misaligned_quadrupole_is_a_dipole_kick():
    """A thin quadrupole displaced by dx kicks a particle on the axis by
    px = k1 L dx (feed-down).  Tilted by +pi/4 (frame x' = x cos + y sin,
    y' = -x sin + y cos) it kicks a particle at (0, y) by px = -k1 L y,
    py = 0, worked out by hand: the skew quadrupole ksl1 = -k1 L of the
    multipole convention (b = (knl + i ksl)(x + i y), px -= Re b)."""
    k1l, dx = 0.05, 2e-3
    o = _track_xy(I.misaligned([I.multipole(knl=[0.0, k1l])], dx=dx), [0.0], [0.0])
    assert o["px"][0] == pytest.approx(k1l * dx, rel=1e-15) and o["x"][0] == pytest.approx(0.0, abs=1e-19)
    y = 1e-3
    o = _track_xy(I.misaligned([I.multipole(knl=[0.0, k1l])], tilt=math.pi / 4), [0.0], [y])
    assert o["px"][0] == pytest.approx(-k1l * y, rel=1e-14) and abs(o["py"][0]) < 1e-19
    sk = _track_xy([I.multipole(ksl=[0.0, -k1l])], [0.0], [y])
    assert o["px"][0] == pytest.approx(sk["px"][0], rel=1e-14)


# --------------------------------------------------------------------------
# Loss-location refinement

def _lost_at(el, xs, pxs, ys=None, pys=None):
    n = len(xs)
    ys = np.zeros(n) if ys is None else np.asarray(ys, float)
    pys = np.zeros(n) if pys is None else np.asarray(pys, float)
    p = I.make_particles(PROTON, np.asarray(xs, float), np.asarray(pxs, float), ys, pys, np.zeros(n), np.zeros(n))
    return oracle.track(I.table(el), PROTON, p, 1)


def _first_root(a2, a1, a0):
    """Smallest positive root of a2 s^2 + a1 s + a0 = 0."""
    r = np.roots([a2, a1, a0])
    r = np.real(r[np.isreal(r)])
    return float(np.min(r[r > 0]))


@pytest.mark.parametrize("r2", [0.01, 0.006])
def test_refine_straight_line_through_cylinder_and_cone(r2):
    """Circular apertures r1 = 10 mm at s = 0 and r2 at s = 20 m with drifts
    between: the interpolated polygon is a regular polygon of circumradius
    r1 + (r2 - r1) s / 20 m, so a straight trajectory leaves it where
    |x0 + a s, y0 + b s| = r(s) (a quadratic, a = px/pz, b = py/pz), less the
    polygon's sag; the refined position lies within one step after that."""
    r1, Ls, ds, n_ang = 0.01, 20.0, 0.01, 1024
    el = [I.aperture(r1), I.drift(7.0), I.drift(13.0), I.aperture(r2)]
    rng = np.random.default_rng(41)
    n = 60
    phi = rng.uniform(0, 2 * math.pi, n)
    rad = rng.uniform(0.0, 0.6 * min(r1, r2), n)
    xs, ys = rad * np.cos(phi), rad * np.sin(phi)
    th = rng.uniform(0, 2 * math.pi, n)
    ang = rng.uniform(6e-4, 1.2e-3, n)
    pxs, pys = ang * np.cos(th), ang * np.sin(th)
    o = _lost_at(el, xs, pxs, ys, pys)
    lost = o["state"] == 0
    assert lost.sum() > 40 and np.all(o["at_element"][lost] == 3)
    s = oracle.refine_losses(I.table(el), PROTON, o, ds, n_ang)
    assert np.all(np.isnan(s[~lost]))
    sag = 1 - math.cos(math.pi / n_ang)
    for i in np.flatnonzero(lost):
        pz = math.sqrt(1 - pxs[i] ** 2 - pys[i] ** 2)
        a, b = pxs[i] / pz, pys[i] / pz
        k = (r2 - r1) / Ls
        # (x0 + a s)^2 + (y0 + b s)^2 - (r1 + k s)^2 = 0
        s_star = _first_root(a * a + b * b - k * k, 2 * (xs[i] * a + ys[i] * b) - 2 * r1 * k,
                             xs[i] ** 2 + ys[i] ** 2 - r1 ** 2)
        if s_star >= Ls:
            continue
        v_r = (xs[i] + a * s_star) * a + (ys[i] + b * s_star) * b
        v_r = v_r / (r1 + k * s_star) - k
        early = sag * r1 / max(v_r, 1e-12)
        assert s_star - early - 1e-9 <= s[i] <= s_star + ds + 1e-9, (i, s[i], s_star)


def test_refine_backtracks_through_a_kick():
    """A thin quadrupole halfway between two circular apertures: the particle
    lost at the second aperture is backtracked through the drift, the inverse
    kick and the first drift, then re-tracked; the crossing on the second
    straight segment is x1 + (px1 / pz1)(s - 10) = r, worked out by hand."""
    r, k = 0.01, 0.02
    el = [I.aperture(r), I.drift(10.0), I.multipole(knl=[0.0, -k]), I.drift(10.0), I.aperture(r)]
    xs = np.array([0.002, 0.004, -0.003, 0.0])
    pxs = np.array([6e-4, 4e-4, -6e-4, 7e-4])
    o = _lost_at(el, xs, pxs)
    s = oracle.refine_losses(I.table(el), PROTON, o, 0.005, 1024)
    for i in range(len(xs)):
        pz = math.sqrt(1 - pxs[i] ** 2)
        x1 = xs[i] + pxs[i] / pz * 10.0
        assert abs(x1) < r
        px1 = pxs[i] + k * x1
        pz1 = math.sqrt(1 - px1 ** 2)
        x2 = x1 + px1 / pz1 * 10.0
        assert o["state"][i] == 0 and abs(x2) > r
        s_star = 10.0 + (math.copysign(r, px1) - x1) * pz1 / px1
        early = (1 - math.cos(math.pi / 1024)) * r * pz1 / abs(px1)
        assert s_star - early - 1e-9 <= s[i] <= s_star + 0.005 + 1e-9, (i, s[i], s_star)


def test_refine_steps_through_a_thick_quadrupole():
    """A defocusing thick quadrupole (k1 = -0.05 m^-2 over 6 m) between 1 m
    drifts and two circular apertures: inside the magnet x(t) = x1 cosh(w t)
    + (px1 / w) sinh(w t), w = sqrt(0.05), t = s - 1 m (on momentum).  The
    refined loss lies within one step after the crossing x(s) = r found here
    by bisection, less the 1024-gon's sag."""
    r, k1, Lq, ds = 0.01, -0.05, 6.0, 0.005
    el = [I.aperture(r), I.drift(1.0), I.quadrupole(k1, Lq), I.drift(1.0), I.aperture(r)]
    xs = np.array([0.006, 0.007, -0.008, 0.0065, -0.0062])
    pxs = np.array([1e-4, -2e-4, 3e-4, 0.0, -1e-4])
    o = _lost_at(el, xs, pxs)
    assert np.all(o["state"] == 0) and np.all(o["at_element"] == 4)
    s = oracle.refine_losses(I.table(el), PROTON, o, ds, 1024)
    w = math.sqrt(-k1)
    for i in range(len(xs)):
        pz = math.sqrt(1 - pxs[i] ** 2)
        x1, px1 = xs[i] + pxs[i] / pz, pxs[i]
        xq = lambda t: x1 * math.cosh(w * t) + px1 / w * math.sinh(w * t)
        def cross(rr):
            lo, hi = 0.0, Lq
            assert abs(xq(lo)) < rr < abs(xq(hi))
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if abs(xq(mid)) < rr else (lo, mid)
            return 1.0 + hi
        s_star, s_early = cross(r), cross(r * math.cos(math.pi / 1024))
        assert s_early - 1e-9 <= s[i] <= s_star + ds + 1e-9, (i, s[i], s_star)


def _winding_inside(px, py, vx, vy):
    """Winding number of the closed polygon (vx, vy) about (px, py) != 0."""
    ang = np.arctan2(vy - py, vx - px)
    d = np.diff(np.append(ang, ang[0]))
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return abs(np.sum(d)) > np.pi


def test_refine_rect_to_ellipse_transition_bruteforce():
    """The paper's loss-location example: a rectangular aperture, then 5 m
    further an elliptic one, shifted and tilted with respect to each other.
    Straight trajectories scanned every 1 mm against the interpolated polygon
    (built here from the two shapes and tested by winding number): the
    refined position is the first outside point to within the step."""
    n_ang, ds = 256, 0.01
    dx, dy, th = 1.2e-3, -0.7e-3, 0.25
    el = (I.misaligned([I.aperture_rect(-0.010, 0.012, -0.006, 0.005)], 0.0, 0.0, 0.0) + [I.drift(2.0), I.drift(3.0)]
          + I.misaligned([I.aperture_ellipse(0.009, 0.0045)], dx, dy, th))
    ap_e = len(el) - 3
    rng = np.random.default_rng(43)
    n = 40
    xs, ys = rng.uniform(-0.004, 0.004, n), rng.uniform(-0.002, 0.002, n)
    t = rng.uniform(0, 2 * math.pi, n)
    pxs, pys = 1.6e-3 * np.cos(t), 1.6e-3 * np.sin(t)
    o = _lost_at(el, xs, pxs, ys, pys)
    lost = (o["state"] == 0) & (o["at_element"] == ap_e)
    assert lost.sum() > 10
    s = oracle.refine_losses(I.table(el), PROTON, o, ds, n_ang)
    phis = 2 * np.pi * np.arange(n_ang) / n_ang
    c, sn = np.cos(phis), np.sin(phis)
    with np.errstate(divide="ignore"):
        tx = np.where(c > 0, 0.012 / c, np.where(c < 0, -0.010 / c, np.inf))
        ty = np.where(sn > 0, 0.005 / sn, np.where(sn < 0, -0.006 / sn, np.inf))
    rr = np.minimum(tx, ty)
    A = np.stack([rr * c, rr * sn], 1)
    re = 1 / np.sqrt(c ** 2 / 0.009 ** 2 + sn ** 2 / 0.0045 ** 2)
    loc = np.stack([re * c, re * sn], 1)
    B = np.stack([math.cos(th) * loc[:, 0] - math.sin(th) * loc[:, 1] + dx,
                  math.sin(th) * loc[:, 0] + math.cos(th) * loc[:, 1] + dy], 1)
    for i in np.flatnonzero(lost):
        pz = math.sqrt(1 - pxs[i] ** 2 - pys[i] ** 2)
        first = None
        for sv in np.arange(0.001, 5.0 + 1e-9, 0.001):
            w = sv / 5.0
            V = A + w * (B - A)
            if not _winding_inside(xs[i] + pxs[i] / pz * sv, ys[i] + pys[i] / pz * sv, V[:, 0], V[:, 1]):
                first = sv
                break
        first = 5.0 if first is None else first
        assert first - 0.001 - 1e-9 <= s[i] <= first + ds + 1e-9, (i, s[i], first)


# --------------------------------------------------------------------------
# 4D beam-beam kick: the field of a bi-Gaussian line charge

def test_gauss_legendre_rule():
    """The oracle's 16-point rule: nodes symmetric in (-1, 1), weights
    summing to 2, and exact (to rounding) for every monomial up to degree
    31 = 2n - 1, against the exact integral 2/(k+1) for even k."""
    x, w = oracle.gauss_legendre()
    assert x.size == 16 and np.all(np.abs(x) < 1) and np.all(w > 0)
    assert np.allclose(np.sort(x), -np.sort(x)[::-1], rtol=0, atol=1e-16)
    for k in range(32):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) <= 1e-15, k
    # degree 32 is the first the rule misses
    assert abs(np.sum(w * x ** 32) - 2.0 / 33) > 1e-12


def test_gauss_field_vs_bassetti_erskine_with_scipy():
    """The oracle's field (quadrature of the single-integral form) against
    the closed form of Bassetti and Erskine evaluated with scipy's Faddeeva
    function: f_y + i f_x = sqrt(pi)/S [w(z1) - e^(-x^2/2sx^2 - y^2/2sy^2) w(z2)],
    S = sqrt(2 (sx^2 - sy^2)), z1 = (x + i y)/S, z2 = (x sy/sx + i y sx/sy)/S,
    for sx > sy and x, y >= 0 (the other quadrants by symmetry), within
    1e-12 of the field's size away from the centre, where the closed form
    does not cancel."""
    from scipy.special import wofz
    rng = np.random.default_rng(54)
    for sx, sy in [(2e-3, 1e-3), (1.2e-3, 0.3e-3), (1e-3, 0.999e-3)]:
        pts = np.abs(np.concatenate([rng.normal(0, 2, (200, 2)), rng.normal(0, 8, (100, 2))]) * [sx, sy])
        pts = pts[np.hypot(pts[:, 0] / sx, pts[:, 1] / sy) > 0.1]
        x, y = pts[:, 0], pts[:, 1]
        S = math.sqrt(2 * (sx * sx - sy * sy))
        w1 = wofz((x + 1j * y) / S)
        w2 = wofz((x * sy / sx + 1j * y * sx / sy) / S)
        f = math.sqrt(math.pi) / S * (w1 - np.exp(-x * x / (2 * sx * sx) - y * y / (2 * sy * sy)) * w2)
        fx, fy = oracle.gauss_field(sx, sy, x, y)
        err = np.hypot(fx - f.imag, fy - f.real) / np.hypot(f.imag, f.real)
        assert err.max() <= 1e-12, (sx, sy, err.max())
    # signs: the field points away from the centre in every quadrant
    fx, fy = oracle.gauss_field(2e-3, 1e-3, np.array([1e-3, -1e-3, -1e-3, 1e-3]), np.array([5e-4, 5e-4, -5e-4, -5e-4]))
    assert np.array_equal(np.sign(fx), [1, -1, -1, 1]) and np.array_equal(np.sign(fy), [1, 1, -1, -1])


@pytest.mark.parametrize("sx,sy", [(2e-3, 1e-3), (0.4e-3, 1.2e-3), (1.0005e-3, 1e-3), (0.7e-3, 0.7e-3)])
def test_gauss_field_vs_integral(sx, sy):
    """Field of a unit bi-Gaussian line charge against its single-integral
    form f_x = x int_0^inf exp(-x^2/(2sx^2+q) - y^2/(2sy^2+q)) /
    ((2sx^2+q)^(3/2) (2sy^2+q)^(1/2)) dq (and f_y with the roles swapped),
    integrated by mpmath at points near the centre, at a few sigma and far."""
    rng = np.random.default_rng(53)
    pts = np.concatenate([rng.normal(0, 1, (20, 2)) * [sx, sy], rng.normal(0, 4, (20, 2)) * [sx, sy],
                          [[30 * sx, 5 * sy], [-2e-9, 1e-9], [sx, 0.0], [0.0, -sy]]])
    fx, fy = oracle.gauss_field(sx, sy, pts[:, 0], pts[:, 1])
    mpmath.mp.dps = 25
    ax, ay = mpmath.mpf(2 * sx * sx), mpmath.mpf(2 * sy * sy)
    m = min(ax, ay)
    cuts = [0, m / 1000, m / 10, m, 10 * m, 1000 * m, 1e6 * m, mpmath.inf]
    for (x, y), gx, gy in zip(pts, fx, fy):
        X, Y = mpmath.mpf(float(x)), mpmath.mpf(float(y))
        e = lambda q: mpmath.exp(-X * X / (ax + q) - Y * Y / (ay + q))
        ix = float(mpmath.quad(lambda q: e(q) / ((ax + q) ** 1.5 * (ay + q) ** 0.5), cuts))
        iy = float(mpmath.quad(lambda q: e(q) / ((ax + q) ** 0.5 * (ay + q) ** 1.5), cuts))
        scale = math.hypot(x * ix, y * iy) + 1e-300
        assert abs(gx - x * ix) <= 5e-14 * scale and abs(gy - y * iy) <= 5e-14 * scale, (x, y, gx, x * ix)


def test_gauss_field_round_limits():
    """Round beam: f = (x, y)/(2 sigma^2) near the centre and (x, y)/r^2 far
    away (all the charge enclosed)."""
    s = 1e-3
    x, y = np.array([1e-9, -3e-10, 40 * s]), np.array([2e-9, 1e-10, 30 * s])
    fx, fy = oracle.gauss_field(s, s, x, y)
    assert fx[0] == pytest.approx(x[0] / (2 * s * s), rel=1e-12) and fy[1] == pytest.approx(y[1] / (2 * s * s), rel=1e-12)
    r2 = x[2] ** 2 + y[2] ** 2
    assert fx[2] == pytest.approx(x[2] / r2, rel=1e-15) and fy[2] == pytest.approx(y[2] / r2, rel=1e-15)


def test_beambeam_linear_tune_shift():
    """A ring (linear map: tune 0.31, beta* = 0.55 m) with a head-on round
    proton bunch at the IP: the small-amplitude tune, from central differences
    of oracle tracking, obeys the thin-lens relation
    cos 2 pi Q = cos 2 pi Q0 + (beta k / 2) sin 2 pi Q0 with the textbook
    defocusing strength k = N r_p / (gamma sigma^2) (like charges, beta = 1,
    so to within 1/(2 gamma^2)): -Delta Q is the beam-beam parameter
    N r_p beta / (4 pi gamma sigma^2)."""
    ref = PROTON
    m0, _, p0c = ref
    gamma = math.sqrt(p0c ** 2 + m0 ** 2) / m0
    N, sig, beta, Q0 = 1.15e11, 50e-6, 0.55, 0.31
    mu = 2 * math.pi * Q0
    M = np.eye(6)
    for k in (0, 2):
        M[k, k], M[k, k + 1], M[k + 1, k], M[k + 1, k + 1] = math.cos(mu), beta * math.sin(mu), -math.sin(mu) / beta, math.cos(mu)
    bb = I.beambeam4d(N, 1.0, sig, sig)
    el = I.table([I.linear_map(M), bb])
    eps = 1e-9
    xs = np.array([eps, -eps])
    o = oracle.track(el, ref, I.make_particles(ref, xs, np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2)), 1)
    o2 = oracle.track(el, ref, I.make_particles(ref, np.zeros(2), xs * 1e-2, np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2)), 1)
    R = np.array([[(o["x"][0] - o["x"][1]) / (2 * eps), (o2["x"][0] - o2["x"][1]) / (2e-2 * eps)],
                  [(o["px"][0] - o["px"][1]) / (2 * eps), (o2["px"][0] - o2["px"][1]) / (2e-2 * eps)]])
    r_p = 2.8179403262e-15 * 0.51099895000e6 / m0
    k = N * r_p / (gamma * sig * sig)
    shift = beta * k / 2 * math.sin(mu)
    # the textbook strength takes beta0 = 1: allow its relative error 1/(2 gamma^2)
    beta0 = p0c / math.sqrt(p0c ** 2 + m0 ** 2)
    assert abs(0.5 * np.trace(R) - (math.cos(mu) + shift)) <= 1.5 * (1 - beta0) * abs(shift) + 1e-10
    xi = N * r_p * beta / (4 * math.pi * gamma * sig * sig)
    dq = math.acos(0.5 * np.trace(R)) / (2 * math.pi) - Q0
    assert dq == pytest.approx(-xi, rel=0.05) and 0.001 < xi < 0.01


# --------------------------------------------------------------------------
# Thick quadrupole

@pytest.mark.parametrize("k1", [0.08, -0.05])
def test_thick_quad_linear_matrix(k1):
    """On momentum at the origin the Jacobian is the textbook thick
    quadrupole: [[cos wL, sin(wL)/w], [-w sin wL, cos wL]] in the focusing
    plane and cosh/sinh in the other, w = sqrt|k1|."""
    L = 3.1
    _, M = oracle.track_jacobian(I.table([I.quadrupole(k1, L)]), PROTON, np.zeros(6))
    w = math.sqrt(abs(k1))
    foc = np.array([[math.cos(w * L), math.sin(w * L) / w], [-w * math.sin(w * L), math.cos(w * L)]])
    dfo = np.array([[math.cosh(w * L), math.sinh(w * L) / w], [w * math.sinh(w * L), math.cosh(w * L)]])
    fx, fy = (foc, dfo) if k1 > 0 else (dfo, foc)
    assert np.max(np.abs(M[:2, :2] - fx)) < 1e-14 and np.max(np.abs(M[2:4, 2:4] - fy)) < 1e-14


def test_osc_funcs_vs_40_digits():
    """The thick maps' entire functions of z = +-a^2: C = cos a (cosh a),
    S = sin(a)/a (sinh(a)/a), S2 = (1 - C)/z, S3 = (1 - S)/z, from 1e-12 to
    30 in |z| on both sides of the series/closed-form switch at |z| = 1/2,
    against 40-digit arithmetic, to 1e-14 relative."""
    mpmath.mp.dps = 40
    mag = np.concatenate([np.logspace(-12, np.log10(30.0), 60), [0.4999999, 0.5, 0.5000001]])
    z = np.concatenate([mag, -mag, [0.0]])
    got = oracle.osc_funcs(z)
    for zi, row in zip(z, got):
        Z = mpmath.mpf(float(zi))
        if Z == 0:
            ref = [1, 1, mpmath.mpf(1) / 2, mpmath.mpf(1) / 6]
        else:
            a = mpmath.sqrt(abs(Z))
            C = mpmath.cos(a) if Z > 0 else mpmath.cosh(a)
            Sv = (mpmath.sin(a) if Z > 0 else mpmath.sinh(a)) / a
            ref = [C, Sv, (1 - C) / Z, (1 - Sv) / Z]
        for g, r in zip(row, ref):
            assert abs(g - float(r)) <= 1e-14 * abs(float(r)), (zi, row, [float(v) for v in ref])


def test_thick_quad_without_gradient_is_the_expanded_drift():
    """k1 = 0: x += L px / (1+delta) in both planes, with finite derivatives."""
    L, d = 1.7, 2e-3
    z0 = np.array([1e-3, 2e-4, -5e-4, 1e-4, 0.0, d])
    zo, M = oracle.track_jacobian(I.table([I.quadrupole(0.0, L)]), PROTON, z0)
    p = oracle.track(I.table([I.quadrupole(0.0, L)]), PROTON,
                     I.make_particles(PROTON, [1e-3], [2e-4], [-5e-4], [1e-4], [0.0], [d]), 1)
    opd = 1.0 + p["delta"][0]
    assert abs(p["x"][0] - (1e-3 + L * 2e-4 / opd)) < 1e-18 and abs(p["y"][0] - (-5e-4 + L * 1e-4 / opd)) < 1e-18
    assert np.all(np.isfinite(M))
    b0 = PROTON[2] / math.hypot(PROTON[0], PROTON[2])
    pt = b0 * d  # z0[5] is pzeta = ptau / beta0
    opd_z = math.sqrt(1.0 + 2.0 * pt / b0 + pt * pt)
    assert abs(M[0, 1] - L / opd_z) < 1e-15 and abs(M[2, 3] - L / opd_z) < 1e-15 and M[1, 0] == 0.0


def test_thick_quad_symplectic_and_reversible():
    el = I.table([I.quadrupole(0.07, 2.3), I.drift(1.0), I.quadrupole(-0.07, 2.3)])
    z0 = np.array([2e-3, 1e-4, -1.5e-3, -2e-4, 0.02, 3e-3])
    _, M = oracle.track_jacobian(el, PROTON, z0)
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-13
    p = I.make_particles(PROTON, [2e-3], [1e-4], [-1.5e-3], [-2e-4], [0.02], [3e-3])
    o = oracle.track(I.table([I.quadrupole(0.07, 2.3), I.quadrupole(0.07, -2.3)]), PROTON, p, 1)
    for k, sc in (("x", 2e-3), ("px", 1e-4), ("y", 1.5e-3), ("py", 2e-4), ("zeta", 0.02)):
        assert abs(o[k][0] - p[k][0]) < 1e-14 * sc


@pytest.mark.parametrize("delta", [0.0, 1.5e-3])
def test_thick_quad_is_the_limit_of_thin_slices(delta):
    """N drift-kick-drift slices (exact drifts, thin kicks k1 L / N) converge
    to the thick map at second order: the gap falls four-fold from N = 500
    to N = 1000.  At 10 um amplitudes the exact drift's terms beyond the
    expanded Hamiltonian are ~1e-11 relative, far below the slicing gap."""
    k1, L = 0.09, 2.7
    rng = np.random.default_rng(61)
    n = 20
    p = I.make_particles(PROTON, rng.normal(0, 1e-5, n), rng.normal(0, 5e-7, n), rng.normal(0, 1e-5, n),
                         rng.normal(0, 5e-7, n), np.zeros(n), np.full(n, delta))
    a = oracle.track(I.table([I.quadrupole(k1, L)]), PROTON, p, 1)
    gaps = []
    for N in (500, 1000):
        thin = []
        for _ in range(N):
            thin += [I.drift(L / (2 * N)), I.multipole(knl=[0.0, k1 * L / N]), I.drift(L / (2 * N))]
        b = oracle.track(I.table(thin), PROTON, p, 1)
        dz = np.max(np.abs(b["zeta"] - p["zeta"]))
        gaps.append(max(np.max(np.abs(a[k] - b[k])) / sc for k, sc in (("x", 1e-5), ("px", 1e-6), ("y", 1e-5),
                                                                         ("py", 1e-6), ("zeta", dz))))
    assert gaps[1] < 2e-6
    assert 3.5 < gaps[0] / gaps[1] < 4.5


# --------------------------------------------------------------------------
# Thick bends

def _bend_matrix_want(h, L, Md56):
    mp = mpmath.mp
    mp.dps = 40
    th = mpmath.mpf(h) * L
    c, s = mpmath.cos(th), mpmath.sin(th)
    omc = 2 * mpmath.sin(th / 2) ** 2
    W = np.eye(6)
    W[0, 0], W[0, 1], W[1, 0], W[1, 1] = float(c), float(s / h), float(-h * s), float(c)
    W[0, 5], W[1, 5], W[4, 0], W[4, 1] = float(omc / h), float(s), float(-s), float(-omc / h)
    W[2, 3] = L
    W[4, 5] = Md56 - float(L - s / h)
    return W


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("h,L", [(1 / 1.5, 1.2), (1 / 2800.0, 14.3)])
def test_sector_bend_linear_matrix(full, h, L):
    """On the design orbit (k0 = h) both models have the textbook sector-bend
    matrix: cos, sin(theta)/h, -h sin in x; R16 = (1 - cos)/h, R26 = sin,
    R51 = -sin, R52 = -(1 - cos)/h; R34 = L; and R56 = the drift's R56 less
    L - sin(theta)/h, the path length saved by the dispersive orbit."""
    _, M = oracle.track_jacobian(I.table([I.bend(h, h, L, full=full)]), PROTON, np.zeros(6))
    _, Md = oracle.track_jacobian(I.table([I.drift(L)]), PROTON, np.zeros(6))
    W = _bend_matrix_want(h, L, Md[4, 5])
    assert np.max(np.abs(M - W)) < 1e-12, np.max(np.abs(M - W))


def test_combined_function_bend_matrix():
    """Expanded model with a gradient on the design orbit: Kx = h^2 + k1 in
    x, R11 = cos(w L), R12 = sin(w L)/w, R16 = h (1 - cos)/Kx, R26 = h
    sin(w L)/w; y defocused by k1 > 0: cosh and sinh."""
    h, L, k1 = 0.2, 1.5, 0.3
    _, M = oracle.track_jacobian(I.table([I.bend(h, h, L, k1=k1)]), PROTON, np.zeros(6))
    w, wy = math.sqrt(h * h + k1), math.sqrt(k1)
    c, s = math.cos(w * L), math.sin(w * L)
    want = {(0, 0): c, (0, 1): s / w, (1, 0): -w * s, (1, 1): c, (0, 5): h * (1 - c) / (w * w), (1, 5): h * s / w,
            (2, 2): math.cosh(wy * L), (2, 3): math.sinh(wy * L) / wy, (3, 2): wy * math.sinh(wy * L),
            (3, 3): math.cosh(wy * L)}
    for (i, j), v in want.items():
        assert abs(M[i, j] - v) < 1e-13, (i, j, M[i, j], v)


@pytest.mark.parametrize("full", [False, True])
def test_bend_symplectic_and_reversible(full):
    """Field and frame curvature mismatched (k0 != h), off axis and off
    momentum: M^T J M = J, and the same bend with -L brings the particle back."""
    k1 = 0.0 if full else 0.12
    b = I.bend(0.55, 0.5, 1.3, k1=k1, full=full)
    z0 = np.array([2e-3, 1e-3, -1.5e-3, -2e-4, 0.02, 3e-3])
    _, M = oracle.track_jacobian(I.table([b]), PROTON, z0)
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-12
    p = I.make_particles(PROTON, [2e-3], [1e-3], [-1.5e-3], [-2e-4], [0.02], [3e-3])
    o = oracle.track(I.table([b, I.bend(0.55, 0.5, -1.3, k1=k1, full=full)]), PROTON, p, 1)
    for k, sc in (("x", 2e-3), ("px", 1e-3), ("y", 1.5e-3), ("py", 2e-4), ("zeta", 0.02)):
        assert abs(o[k][0] - p[k][0]) < 1e-13 * sc + 1e-15, k


@pytest.mark.parametrize("delta", [0.0, 1e-5])
def test_expanded_bend_is_the_limit_of_thin_slices(delta):
    """N drift-kick-drift slices (exact drifts; thin kicks with knl = (k0, k1)
    L/N and frame curvature hxl = h L/N) converge to the expanded bend at
    second order (field and curvature mismatched, with a gradient): the gap
    falls four-fold from N = 400 to N = 800, zeta included.  Orbits stay at
    the micron level, where the exact drift's terms beyond the expansion are
    far below the slicing gap."""
    k0, h, k1, L = 0.050002, 0.05, 0.03, 2.0
    rng = np.random.default_rng(67)
    n = 20
    p = I.make_particles(PROTON, rng.normal(0, 1e-5, n), rng.normal(0, 5e-7, n), rng.normal(0, 1e-5, n),
                         rng.normal(0, 5e-7, n), np.zeros(n), np.full(n, delta))
    a = oracle.track(I.table([I.bend(k0, h, L, k1=k1)]), PROTON, p, 1)
    gaps = []
    for N in (400, 800):
        ds = L / N
        kick = I.multipole(knl=[k0 * ds, k1 * ds], hxl=h * ds, lrad=ds)
        b = oracle.track(I.table([I.drift(ds / 2), kick, I.drift(ds / 2)] * N), PROTON, p, 1)
        dz = np.max(np.abs(b["zeta"] - p["zeta"]))
        sc = {k: np.max(np.abs(b[k] - p[k])) + np.max(np.abs(p[k])) for k in ("x", "px", "y", "py")}
        sc["zeta"] = dz
        gaps.append(max(np.max(np.abs(a[k] - b[k])) / sc[k] for k in sc))
    assert gaps[1] < 1e-5
    assert 3.5 < gaps[0] / gaps[1] < 4.5


def _bend_by_geometry(k0, h, L, x, px, y, py, delta, zeta):
    """Exit coordinates of the full bend by plane geometry in 40 digits: the
    particle's circle (centre P0 + (1/k0) (-pz, px), radius p_h / k0) is cut
    with the exit ray of the sector, the exit momentum is the circle's
    tangent there, and the arc length is radius times the swept angle."""
    mp = mpmath.mp
    mp.dps = 40
    m0, _, p0c = PROTON
    b0 = mpmath.mpf(p0c) / mpmath.sqrt(mpmath.mpf(p0c) ** 2 + mpmath.mpf(m0) ** 2)
    opd = 1 + mpmath.mpf(delta)
    g0 = 1 / mpmath.sqrt(1 - b0 * b0)
    E = mpmath.sqrt((opd * p0c) ** 2 + mpmath.mpf(m0) ** 2)
    beta = opd * p0c / E
    rv0v = b0 / beta
    k0, h, L, x, px, y, py = [mpmath.mpf(v) for v in (k0, h, L, x, px, y, py)]
    pz = mpmath.sqrt(opd ** 2 - px ** 2 - py ** 2)
    ph = mpmath.sqrt(px ** 2 + pz ** 2)
    R = 1 / h
    P0 = mpmath.matrix([R + x, 0])
    th = h * L
    e = mpmath.matrix([mpmath.cos(th), mpmath.sin(th)])
    et = mpmath.matrix([-mpmath.sin(th), mpmath.cos(th)])
    Cp = P0 + mpmath.matrix([-pz, px]) / k0
    rho = ph / k0
    ec = e[0] * Cp[0] + e[1] * Cp[1]
    disc = mpmath.sqrt(ec ** 2 - (Cp[0] ** 2 + Cp[1] ** 2) + rho ** 2)
    r = min((ec - disc, ec + disc), key=lambda v: abs(v - (R + x)))
    P1 = r * e
    a0, a1 = P0 - Cp, P1 - Cp
    v1 = mpmath.matrix([-a1[1], a1[0]]) * (ph / rho)  # counter-clockwise tangent
    phi = mpmath.atan2(a0[0] * a1[1] - a0[1] * a1[0], a0[0] * a1[0] + a0[1] * a1[1])
    lh = rho * phi
    out = dict(x=r - R, px=v1[0] * e[0] + v1[1] * e[1], y=y + py * lh / ph,
               zeta=mpmath.mpf(zeta) + L - rv0v * opd * lh / ph, pzf=v1[0] * et[0] + v1[1] * et[1])
    return {k: float(v) for k, v in out.items()}


@pytest.mark.parametrize("h,L,k0", [(1 / 1.5, 1.2, 1 / 1.5), (1 / 1.5, 1.2, 1.1 / 1.5), (0.05, 2.0, 0.04),
                                    (1 / 2800.0, 14.3, 1 / 2800.0)])
def test_full_bend_against_plane_geometry(h, L, k0):
    """The full model against the circle-and-ray construction: a small-ring
    dipole (theta = 0.8: the trigonometric branch and two halvings in
    asin(u)/u), a mismatched field, a weak field in a curved frame and an
    LHC-like dipole, over random particles off axis and off momentum."""
    rng = np.random.default_rng(71)
    n = 12
    xs, pxs = rng.normal(0, 2e-3, n), rng.normal(0, 1e-3, n)
    ys, pys = rng.normal(0, 2e-3, n), rng.normal(0, 1e-3, n)
    ds_ = rng.normal(0, 2e-3, n)
    p = I.make_particles(PROTON, xs, pxs, ys, pys, np.full(n, 0.01), ds_)
    o = oracle.track(I.table([I.bend(k0, h, L, full=True)]), PROTON, p, 1)
    assert np.all(o["state"] == 1)
    for i in range(n):
        g = _bend_by_geometry(k0, h, L, xs[i], pxs[i], ys[i], pys[i], p["delta"][i], 0.01)
        for k in ("x", "px", "y"):
            assert abs(o[k][i] - g[k]) < 2e-15 * L + 1e-15 * abs(g[k]), (k, i, o[k][i], g[k])
        assert abs(o["zeta"][i] - g["zeta"]) < 1e-14 * L, (i, o["zeta"][i], g["zeta"])


def test_full_bend_without_field_or_curvature_is_the_exact_drift():
    rng = np.random.default_rng(73)
    n = 10
    p = I.make_particles(PROTON, rng.normal(0, 2e-3, n), rng.normal(0, 1e-3, n), rng.normal(0, 2e-3, n),
                         rng.normal(0, 1e-3, n), np.zeros(n), rng.normal(0, 1e-3, n))
    a = oracle.track(I.table([I.bend(0.0, 0.0, 3.0, full=True)]), PROTON, p, 1)
    b = oracle.track(I.table([I.drift(3.0)]), PROTON, p, 1)
    for k in ("x", "px", "y", "py"):
        assert np.max(np.abs(a[k] - b[k])) < 1e-17 + 1e-15 * np.max(np.abs(b[k]))
    assert np.max(np.abs(a["zeta"] - b["zeta"])) < 1e-15


def test_full_and_expanded_bends_agree_to_first_order():
    """The models differ by the Hamiltonian terms the expansion drops, the
    leading one h x (px^2 + py^2) / (2 (1+delta)), of third order: the maps
    then differ at second order in the amplitudes, and halving them cuts the
    gap four-fold."""
    h, L = 0.5, 1.0
    gaps = []
    for amp in (2e-3, 1e-3):
        rng = np.random.default_rng(79)
        n = 20
        p = I.make_particles(PROTON, rng.normal(0, amp, n), rng.normal(0, amp, n), rng.normal(0, amp, n),
                             rng.normal(0, amp, n), np.zeros(n), rng.normal(0, amp, n))
        a = oracle.track(I.table([I.bend(h, h, L, full=True)]), PROTON, p, 1)
        b = oracle.track(I.table([I.bend(h, h, L)]), PROTON, p, 1)
        gaps.append(max(np.max(np.abs(a[k] - b[k])) for k in ("x", "px", "y", "py")))
    assert gaps[0] < 1e-5
    assert 3.6 < gaps[0] / gaps[1] < 4.4


def _gradient_bend_by_ode(k0, h, k1, L, z, ep):
    """The flow of H = -(1 + h x) pz + k0 (x + h x^2 / 2) + k1 (x^2 - y^2) / 2,
    pz = sqrt((1+delta)^2 - px^2 - py^2), integrated over s (DOP853 at
    rtol 1e-13): x' = (1 + h x) px / pz, px' = h pz - k0 (1 + h x) - k1 x,
    y' = (1 + h x) py / pz, py' = k1 y, zeta' = 1 - (1 + h x) ep / pz with
    ep = (1+delta) beta0 / beta."""
    from scipy.integrate import solve_ivp
    x, px, y, py, zeta, opd = z

    def rhs(_, u):
        x_, px_, y_, py_, _z = u
        pz = math.sqrt(opd * opd - px_ * px_ - py_ * py_)
        f = 1.0 + h * x_
        return [f * px_ / pz, h * pz - k0 * f - k1 * x_, f * py_ / pz, k1 * y_, 1.0 - f * ep / pz]

    r = solve_ivp(rhs, (0.0, L), [x, px, y, py, zeta], method="DOP853", rtol=1e-13, atol=1e-16)
    return r.y[:, -1]


def test_full_bend_gradient_kicks_converge_to_the_exact_flow():
    """The full model with a gradient (thin quadrupole kicks between exact
    bodies) against the integrated equations of motion of the full bend's
    Hamiltonian plus k1 (x^2 - y^2) / 2: the splitting is symmetric, so the
    gap falls four-fold from 8 to 16 kicks (a wrong sign or strength of the
    kick, or a body of the wrong length, leaves a gap that does not fall)."""
    k0, h, k1, L = 0.52, 0.5, 0.35, 1.2
    rng = np.random.default_rng(83)
    n = 6
    p = I.make_particles(PROTON, rng.normal(0, 2e-3, n), rng.normal(0, 1e-3, n), rng.normal(0, 2e-3, n),
                         rng.normal(0, 1e-3, n), np.full(n, 0.01), rng.normal(0, 2e-3, n))
    want = []
    for i in range(n):
        opd = 1.0 + p["delta"][i]
        ep = opd / p["rvv"][i]
        want.append(_gradient_bend_by_ode(k0, h, k1, L, (p["x"][i], p["px"][i], p["y"][i], p["py"][i],
                                                        p["zeta"][i], opd), ep))
    want = np.array(want)
    gaps = []
    for nk in (8, 16):
        o = oracle.track(I.table([I.bend(k0, h, L, k1=k1, full=True, kicks=nk)]), PROTON, p, 1)
        assert np.all(o["state"] == 1)
        got = np.stack([o[k] for k in ("x", "px", "y", "py", "zeta")], 1)
        gaps.append(np.max(np.abs(got - want) / (np.abs(want).max(0) + 1e-3)))
    assert gaps[1] < 3e-4
    assert 3.9 < gaps[0] / gaps[1] < 4.1, gaps


def test_full_bend_gradient_linear_matrix():
    """On the design orbit the full model with a gradient linearises to the
    combined-function sector matrix (Kx = h^2 + k1 in x, cosh/sinh in y for
    k1 > 0), the kicks' gap falling four-fold from 16 to 32 kicks."""
    h, L, k1 = 0.2, 1.5, 0.3
    w, wy = math.sqrt(h * h + k1), math.sqrt(k1)
    c, s = math.cos(w * L), math.sin(w * L)
    want = {(0, 0): c, (0, 1): s / w, (1, 0): -w * s, (1, 1): c, (0, 5): h * (1 - c) / (w * w), (1, 5): h * s / w,
            (2, 2): math.cosh(wy * L), (2, 3): math.sinh(wy * L) / wy, (3, 2): wy * math.sinh(wy * L),
            (3, 3): math.cosh(wy * L)}
    gaps = []
    for nk in (16, 32):
        _, M = oracle.track_jacobian(I.table([I.bend(h, h, L, k1=k1, full=True, kicks=nk)]), PROTON, np.zeros(6))
        gaps.append(max(abs(M[i, j] - v) for (i, j), v in want.items()))
    assert gaps[1] < 2e-4
    assert 3.8 < gaps[0] / gaps[1] < 4.2, gaps


@pytest.mark.parametrize("nk", [1, 7])
def test_full_bend_gradient_symplectic_and_reversible(nk):
    """Off axis, off momentum, field and frame mismatched: M^T J M = J, and
    the same element with -L brings the particle back."""
    b = I.bend(0.55, 0.5, 1.3, k1=-0.4, full=True, kicks=nk)
    z0 = np.array([2e-3, 1e-3, -1.5e-3, -2e-4, 0.02, 3e-3])
    _, M = oracle.track_jacobian(I.table([b]), PROTON, z0)
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-12
    p = I.make_particles(PROTON, [2e-3], [1e-3], [-1.5e-3], [-2e-4], [0.02], [3e-3])
    o = oracle.track(I.table([b, I.bend(0.55, 0.5, -1.3, k1=-0.4, full=True, kicks=nk)]), PROTON, p, 1)
    for k, sc in (("x", 2e-3), ("px", 1e-3), ("y", 1.5e-3), ("py", 2e-4), ("zeta", 0.02)):
        assert abs(o[k][0] - p[k][0]) < 1e-13 * sc + 1e-15, k


# --------------------------------------------------------------------------
# Non-linear dipole edge

@pytest.mark.parametrize("exit_face", [False, True])
def test_nonlinear_edge_linearises_to_the_linear_edge(exit_face):
    """At the origin the non-linear edge's Jacobian is the linear edge's
    (face angle, fringe extent fint * hgap included)."""
    kw = dict(hgap=0.02, fint=0.5)
    _, Mn = oracle.track_jacobian(I.table([I.dipedge(0.08, 0.15, nonlinear=True, exit=exit_face, **kw)]), PROTON,
                                  np.zeros(6))
    _, Ml = oracle.track_jacobian(I.table([I.dipedge(0.08, 0.15, **kw)]), PROTON, np.zeros(6))
    assert np.max(np.abs(Mn - Ml)) < 1e-15 and abs(Ml[3, 2]) > 1e-3


@pytest.mark.parametrize("exit_face", [False, True])
def test_nonlinear_edge_is_symplectic(exit_face):
    """Off axis and steep (x, y ~ 8 mm, px ~ 30 mrad), off momentum."""
    el = I.table([I.dipedge(0.3, 0.2, hgap=0.03, fint=0.4, nonlinear=True, exit=exit_face)])
    z0 = np.array([8e-3, 3e-2, -7e-3, 1e-2, 0.01, 2e-3])
    _, M = oracle.track_jacobian(el, PROTON, z0)
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-14
    assert abs(M[0, 2]) > 1e-6  # the fringe's x shift depends on y


def _soft_fringe(k0, e, lam, a, z, exit_face):
    """A particle (x, y, px, py) at s = -a integrated to s = +a through a
    tanh fringe of length lam, the face at angle e: the field k0 f(sigma) with
    sigma = s - tan(e) x at an entrance (field for sigma > 0) or
    sigma = -(s + tan(e) x) at an exit, and the fields that Maxwell's
    equations attach to it to second order in y (B_s = y dB_y/ds,
    B_x = y dB_y/dx, B_y - y^2/2 (d2/ds2 + d2/dx2) B_y), by the Lorentz force
    with s as the independent variable (DOP853, rtol 1e-13)."""
    from scipy.integrate import solve_ivp
    t = math.tan(e)

    def rhs(s, u):
        x, y, px, py = u
        sig = -(s + t * x) if exit_face else s - t * x
        th = math.tanh(sig / lam)
        f, f1, f2 = 0.5 * (1 + th), 0.5 * (1 - th * th) / lam, -(1 - th * th) * th / (lam * lam)
        ds, dx = (-1.0, -t) if exit_face else (1.0, -t)  # d sigma / ds, d sigma / dx
        by = k0 * (f - 0.5 * y * y * (ds * ds + dx * dx) * f2)
        bs, bx = k0 * y * f1 * ds, k0 * y * f1 * dx
        pz = math.sqrt(1.0 - px * px - py * py)
        return [px / pz, py / pz, py * bs / pz - by, bx - px * bs / pz]

    r = solve_ivp(rhs, (-a, a), list(z), method="DOP853", rtol=1e-13, atol=1e-16, max_step=lam / 4)
    return r.y[:, -1]


@pytest.mark.parametrize("exit_face", [False, True])
def test_nonlinear_edge_against_soft_fringe_integration(exit_face):
    """A weak field (k0 = 0.01 /m, so that second-order effects of the field
    stay small) and steep particles (px up to 20 mrad, y up to 5 mm).  The
    hard-edge models are compared with the soft fringe integrated through,
    each composed with a 5 cm drift and 5 cm of uniform field (the full bend
    with h = 0) on the two sides.  At normal incidence the non-linear edge
    converges to the integration as the fringe shortens (the x gap falls
    four-fold per halving of its length; px exact), and its vertical errors
    are under 2 % of the linear model's, which misses the angle dependence
    of the vertical kick and the fringe's shift of x and y.  At a face angle
    of 0.12 rad its py error stays under 2 % of the linear model's; px and y
    keep a first-order residual from the wedge between face and normal
    plane, whose kick is taken without its angle factor
    1 / (1 - tan(e) px/pz) (y under 20 % of the linear model's error)."""
    k0, a = 0.01, 0.05
    rng = np.random.default_rng(89)
    n = 6
    xs, pxs = rng.uniform(-5e-3, 5e-3, n), rng.uniform(-0.02, 0.02, n)
    ys, pys = rng.uniform(-5e-3, 5e-3, n), rng.uniform(-5e-3, 5e-3, n)
    p = I.make_particles(PROTON, xs, pxs, ys, pys, np.zeros(n), np.zeros(n))

    def gaps(e, nl, lam):
        edge = I.dipedge(k0, e, nonlinear=nl, exit=exit_face)
        body = I.bend(k0, 0.0, a, full=True)
        rows = [body, edge, I.drift(a)] if exit_face else [I.drift(a), edge, body]
        o = oracle.track(I.table(rows), PROTON, p, 1)
        g = np.zeros(4)
        for i in range(n):
            u = _soft_fringe(k0, e, lam, a, (xs[i], ys[i], pxs[i], pys[i]), exit_face)
            g = np.maximum(g, np.abs([o["x"][i] - u[0], o["px"][i] - u[2], o["y"][i] - u[1], o["py"][i] - u[3]]))
        return g

    gn = [gaps(0.0, True, lam) for lam in (2e-3, 1e-3)]
    gl = gaps(0.0, False, 1e-3)
    assert 3.0 < gn[0][0] / gn[1][0] < 5.0 and gn[1][0] < 1e-8
    assert gn[1][1] < 1e-14
    assert gn[1][2] < 0.02 * gl[2] and gn[1][3] < 0.02 * gl[3]
    gn_e, gl_e = gaps(0.12, True, 1e-3), gaps(0.12, False, 1e-3)
    assert gn_e[2] < 0.2 * gl_e[2] and gn_e[3] < 0.02 * gl_e[3]


@pytest.mark.parametrize("exit_face", [False, True])
def test_exact_wedge_edge_against_soft_fringe_integration(exit_face):
    """The edge with the exact wedge (the fringe on the face between exact
    changes of plane) against the tanh fringe integrated through, as in the
    test above: at face angles of 0.12 and 0.3 rad it converges like the
    non-linear edge at normal incidence (the x gap falls four-fold per
    halving of the fringe length, px within 1e-10 and falling), and the
    first-order px residual that the non-linear edge's plain wedge kick keeps
    (1e-8 and more) is gone.  At normal incidence it is the non-linear edge."""
    k0, a = 0.01, 0.05
    rng = np.random.default_rng(89)
    n = 6
    xs, pxs = rng.uniform(-5e-3, 5e-3, n), rng.uniform(-0.02, 0.02, n)
    ys, pys = rng.uniform(-5e-3, 5e-3, n), rng.uniform(-5e-3, 5e-3, n)
    p = I.make_particles(PROTON, xs, pxs, ys, pys, np.zeros(n), np.zeros(n))

    def run(e, **kw):
        edge = I.dipedge(k0, e, exit=exit_face, **kw)
        body = I.bend(k0, 0.0, a, full=True)
        rows = [body, edge, I.drift(a)] if exit_face else [I.drift(a), edge, body]
        return oracle.track(I.table(rows), PROTON, p, 1)

    def gaps(o, e, lam):
        g = np.zeros(4)
        for i in range(n):
            u = _soft_fringe(k0, e, lam, a, (xs[i], ys[i], pxs[i], pys[i]), exit_face)
            g = np.maximum(g, np.abs([o["x"][i] - u[0], o["px"][i] - u[2], o["y"][i] - u[1], o["py"][i] - u[3]]))
        return g

    w0, n0 = run(0.0, wedge=True), run(0.0, nonlinear=True)
    for k in ("x", "px", "y", "py", "zeta"):
        assert np.array_equal(w0[k], n0[k]), k
    g_normal = gaps(w0, 0.0, 1e-3)
    for e in (0.12, 0.3):
        ow = run(e, wedge=True)
        gw = [gaps(ow, e, lam) for lam in (2e-3, 1e-3)]
        gn = gaps(run(e, nonlinear=True), e, 1e-3)
        assert 3.0 < gw[0][0] / gw[1][0] < 5.0 and gw[1][0] < 1e-8
        assert gw[1][1] < 1e-10 and gw[1][1] < 1e-3 * gn[1] and gn[1] > 1e-8
        assert gw[1][2] < 2.0 * g_normal[2] + 1e-11 and gw[1][3] < 2.0 * g_normal[3]


@pytest.mark.parametrize("exit_face", [False, True])
def test_exact_wedge_edge_linearises_to_the_linear_edge_and_is_symplectic(exit_face):
    kw = dict(hgap=0.02, fint=0.5)
    _, Mw = oracle.track_jacobian(I.table([I.dipedge(0.08, 0.15, wedge=True, exit=exit_face, **kw)]), PROTON,
                                  np.zeros(6))
    _, Ml = oracle.track_jacobian(I.table([I.dipedge(0.08, 0.15, **kw)]), PROTON, np.zeros(6))
    assert np.max(np.abs(Mw - Ml)) < 1e-15 and abs(Ml[1, 0]) > 1e-3 and abs(Ml[3, 2]) > 1e-3
    el = I.table([I.dipedge(0.3, 0.2, hgap=0.03, fint=0.4, wedge=True, exit=exit_face)])
    _, M = oracle.track_jacobian(el, PROTON, np.array([8e-3, 3e-2, -7e-3, 1e-2, 0.01, 2e-3]))
    assert np.max(np.abs(M.T @ J6 @ M - J6)) < 1e-14
    assert abs(M[1, 1] - 1.0) > 1e-5  # px' depends on px: not the plain wedge kick


def _rect_by_geometry(h, L, e1, e2, x, px, delta, zeta):
    """A dipole of field h between two inclined pole faces, in the midplane,
    by plane geometry in 40 digits.  The reference arc (radius 1/h, length
    L) starts at the origin heading along Z; the entrance face is the line
    through the origin at the angle e1 to the X axis (downstream at X > 0),
    the exit face the line through the arc's end at the angle e2 to the
    radial line (upstream on the outer side).  The particle runs straight to
    the entrance face, on its circle (centre Q + (-pz, px)/h) to the exit
    face, and straight to the plane normal to the arc's end, where x, px and
    the path length are read."""
    mp = mpmath.mp
    mp.dps = 40
    m0, _, p0c = PROTON
    b0 = mpmath.mpf(p0c) / mpmath.sqrt(mpmath.mpf(p0c) ** 2 + mpmath.mpf(m0) ** 2)
    opd = 1 + mpmath.mpf(delta)
    beta = opd * p0c / mpmath.sqrt((opd * p0c) ** 2 + mpmath.mpf(m0) ** 2)
    rv0v = b0 / beta
    h, L, e1, e2, x, px = [mpmath.mpf(v) for v in (h, L, e1, e2, x, px)]
    pz = mpmath.sqrt(opd ** 2 - px ** 2)
    ph = opd
    t = x * mpmath.sin(e1) / (pz * mpmath.cos(e1) - px * mpmath.sin(e1))
    Q = mpmath.matrix([x + t * px, t * pz])
    l1 = t * ph
    Cp = Q + mpmath.matrix([-pz, px]) / h
    rho = ph / h
    th = h * L
    R = 1 / h
    Pe = mpmath.matrix([-R + R * mpmath.cos(th), R * mpmath.sin(th)])
    eX = mpmath.matrix([mpmath.cos(th), mpmath.sin(th)])
    eZ = mpmath.matrix([-mpmath.sin(th), mpmath.cos(th)])
    f = eX * mpmath.cos(e2) - eZ * mpmath.sin(e2)
    d = Pe - Cp
    b = f[0] * d[0] + f[1] * d[1]
    c = d[0] ** 2 + d[1] ** 2 - rho ** 2
    a = min((-b - mpmath.sqrt(b * b - c), -b + mpmath.sqrt(b * b - c)), key=abs)
    F = Pe + a * f
    a0, a1 = Q - Cp, F - Cp
    v1 = mpmath.matrix([-a1[1], a1[0]]) * (ph / rho)
    phi = mpmath.atan2(a0[0] * a1[1] - a0[1] * a1[0], a0[0] * a1[0] + a0[1] * a1[1])
    l2 = rho * phi
    Xf, Zf = (F - Pe)[0] * eX[0] + (F - Pe)[1] * eX[1], (F - Pe)[0] * eZ[0] + (F - Pe)[1] * eZ[1]
    pX, pZ = v1[0] * eX[0] + v1[1] * eX[1], v1[0] * eZ[0] + v1[1] * eZ[1]
    t3 = -Zf / pZ
    l = l1 + l2 + t3 * ph
    out = dict(x=Xf + t3 * pX, px=pX, zeta=mpmath.mpf(zeta) + L - rv0v * opd * l / ph)
    return {k: float(v) for k, v in out.items()}


@pytest.mark.parametrize("h,L,e1,e2", [(1 / 1.5, 0.9, 0.3, 0.3), (1 / 1.5, 0.9, 0.1, 0.45),
                                       (0.05, 2.0, 0.05, -0.02), (1 / 2800.0, 14.3, 14.3 / 5600.0, 14.3 / 5600.0)])
def test_rectangular_bend_with_exact_wedges_against_plane_geometry(h, L, e1, e2):
    """Entrance edge, full sector body and exit edge, the edges with the
    exact wedge, against the straight-circle-straight construction in the
    midplane: a rectangular small-ring dipole, unequal faces, a face inclined
    the other way, and an LHC-like rectangular dipole, over random particles
    off axis, at angles and off momentum."""
    rng = np.random.default_rng(73)
    n = 12
    xs, pxs, ds_ = rng.normal(0, 2e-3, n), rng.normal(0, 1e-3, n), rng.normal(0, 2e-3, n)
    p = I.make_particles(PROTON, xs, pxs, np.zeros(n), np.zeros(n), np.full(n, 0.01), ds_)
    rows = [I.dipedge(h, e1, wedge=True), I.bend(h, h, L, full=True), I.dipedge(h, e2, wedge=True, exit=True)]
    o = oracle.track(I.table(rows), PROTON, p, 1)
    assert np.all(o["state"] == 1)
    for i in range(n):
        g = _rect_by_geometry(h, L, e1, e2, xs[i], pxs[i], p["delta"][i], 0.01)
        for k in ("x", "px"):
            assert abs(o[k][i] - g[k]) < 4e-15 * L + 2e-15 * abs(g[k]), (k, i, o[k][i], g[k])
        assert abs(o["zeta"][i] - g["zeta"]) < 2e-14 * L, (i, o["zeta"][i], g["zeta"])
        assert o["y"][i] == 0.0 and o["py"][i] == 0.0


# --------------------------------------------------------------------------
# Frozen space charge

def test_space_charge_kick_from_the_fields_of_the_beam():
    """A round coasting beam: the kick equals the Lorentz force of the
    beam's own fields integrated over the lens length, worked out in SI
    units here (Gauss's law for the radial field of the Gaussian line
    charge, B = beta E / c, so the force is q E / gamma^2; time L / (beta c);
    momentum gamma m beta c), in 40-digit arithmetic."""
    mp = mpmath.mp
    mp.dps = 40
    lam, sig, L = 5e10, 1.2e-3, 3.0
    ref = PROTON
    el = I.table([I.spacecharge(lam, 0.0, sig, sig, L)])
    xs = np.array([3e-4, -1.1e-3, 2.5e-3, 4e-6])
    ys = np.array([1e-4, 7e-4, -1.9e-3, -2e-6])
    n = len(xs)
    p = I.make_particles(ref, xs, np.zeros(n), ys, np.zeros(n), np.zeros(n), np.zeros(n))
    o = oracle.track(el, ref, p, 1)
    e, eps0, c = mpmath.mpf("1.602176634e-19"), mpmath.mpf("8.8541878128e-12"), mpmath.mpf(299792458)
    m_kg = mpmath.mpf(ref[0]) * e / c ** 2
    E0 = mpmath.sqrt(mpmath.mpf(ref[2]) ** 2 + mpmath.mpf(ref[0]) ** 2)
    gamma, beta = E0 / ref[0], mpmath.mpf(ref[2]) / E0
    p0 = gamma * m_kg * beta * c
    for i in range(n):
        x, y = mpmath.mpf(xs[i]), mpmath.mpf(ys[i])
        r2 = x * x + y * y
        Er = lam * e / (2 * mpmath.pi * eps0) * (1 - mpmath.exp(-r2 / (2 * sig ** 2))) / r2  # E_x / x
        kick = e * Er * (1 - beta ** 2) * (L / (beta * c)) / p0
        # r_e m_e c^2 and e^2 / (4 pi eps0) from rounded CODATA values agree to ~1e-11
        assert abs(o["px"][i] - float(kick * x)) < 1e-10 * abs(float(kick * x))
        assert abs(o["py"][i] - float(kick * y)) < 1e-10 * abs(float(kick * y))


def test_space_charge_longitudinal_profile():
    """Bunched: the kick at zeta = sigma_z is e^(-1/2) times the kick at the
    bunch centre, at 2 sigma_z e^(-2); coasting (sigma_z = 0): no zeta
    dependence."""
    sz = 0.3
    xs = np.full(3, 1e-3)
    p = I.make_particles(PROTON, xs, np.zeros(3), np.full(3, 5e-4), np.zeros(3), np.array([0.0, sz, -2 * sz]),
                         np.zeros(3))
    o = oracle.track(I.table([I.spacecharge(4e10, sz, 1e-3, 6e-4, 2.0)]), PROTON, p, 1)
    assert abs(o["px"][1] / o["px"][0] - math.exp(-0.5)) < 1e-15
    assert abs(o["px"][2] / o["px"][0] - math.exp(-2.0)) < 1e-15
    assert abs(o["py"][1] / o["py"][0] - math.exp(-0.5)) < 1e-15
    oc = oracle.track(I.table([I.spacecharge(4e10, 0.0, 1e-3, 6e-4, 2.0)]), PROTON, p, 1)
    assert oc["px"][0] == oc["px"][1] == oc["px"][2] and oc["px"][0] == o["px"][0]


def test_space_charge_linear_tune_shift():
    """A 2 GeV/c proton ring (linear, tune Q0) with one round space-charge
    lens: the small-amplitude one-turn matrix (by differences of tracked
    particles) has cos(2 pi Q) = cos(mu0) + (beta k / 2) sin(mu0) with the
    defocusing k = K / (2 sigma^2), K = 2 r_c lambda L / (beta0^2 gamma0^3)."""
    ref = I.proton_reference(2e9)
    lam, sig, L, beta, Q0 = 3e9, 8e-4, 50.0, 12.0, 0.27
    mu = 2 * math.pi * Q0
    M = np.eye(6)
    for k in (0, 2):
        M[k, k], M[k, k + 1], M[k + 1, k], M[k + 1, k + 1] = (math.cos(mu), beta * math.sin(mu),
                                                              -math.sin(mu) / beta, math.cos(mu))
    el = I.table([I.linear_map(M), I.spacecharge(lam, 0.0, sig, sig, L)])
    m0, _, p0c = ref
    E0 = math.hypot(p0c, m0)
    b0, g0 = p0c / E0, E0 / m0
    rc = 2.8179403262e-15 * 0.51099895000e6 / m0
    K = 2 * rc * lam * L / (b0 * b0 * g0 ** 3)
    kdef = K / (2 * sig * sig)
    eps = 1e-9
    p = I.make_particles(ref, [eps, -eps, 0.0, 0.0], [0.0, 0.0, eps / beta, -eps / beta], np.zeros(4),
                         np.zeros(4), np.zeros(4), np.zeros(4))
    o = oracle.track(el, ref, p, 1)
    m11 = (o["x"][0] - o["x"][1]) / (2 * eps)
    m22 = (o["px"][2] - o["px"][3]) / (2 * eps / beta)
    want = math.cos(mu) + beta * kdef / 2 * math.sin(mu)
    assert abs(0.5 * (m11 + m22) - want) < 1e-7
    assert want > math.cos(mu) + 0.05  # defocusing: the tune moves well away


def test_segment_resume_bitwise():
    """track(a) then track(b) from turn a equals track(a+b), radiation included."""
    el, ref, _ = I.lepton_ring(n_cells=4, E0=5e9, v_total=30e6)
    p = I.matched_gaussian(el, ref, 20, 1e-3, 1e-3, seed=7)
    for mode in (0, 1, 2):
        full = oracle.track(el, ref, p, 30, rad_mode=mode, seed=11)
        a = oracle.track(el, ref, p, 12, rad_mode=mode, seed=11)
        b = oracle.track(el, ref, a, 18, start_turn=12, rad_mode=mode, seed=11)
        for k in oracle.FLOAT_FIELDS + oracle.INT_FIELDS:
            assert np.array_equal(full[k], b[k]), (mode, k)


# --------------------------------------------------------------------------
# Random numbers and the photon spectrum

def test_philox_vs_numpy():
    """Philox4x64-10 known answers from numpy's independent implementation
    (numpy increments the counter before each block)."""
    for key0, c0, c1 in [(5, 0, 0), (20231001, 123456789, 7), (2 ** 63 + 11, 2 ** 64 - 2, 99)]:
        bg = np.random.Philox(key=np.array([key0, 0], dtype=np.uint64),
                              counter=np.array([c0, c1, 0, 0], dtype=np.uint64))
        ref = bg.random_raw(4)
        got = oracle.philox4x64_10([c0 + 1, c1, 0, 0], [key0, 0])
        assert np.array_equal(ref.astype(np.uint64), got)


def test_uniforms_statistics():
    from scipy import stats
    u = np.array([oracle.uniform(3, pid, 17, 42, j) for pid in range(2000) for j in range(5)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)


def test_spectrum_cdf_vs_bessel_quadrature():
    """The tabulated CDF of xi against scipy's K_{5/3} integrated by quad:
    F(xi) = (3/(5 pi)) int_0^xi ds int_s^inf K_{5/3}(t) dt
          = (3/(5 pi)) [xi G(xi) + int_0^xi t K_{5/3}(t) dt]  (integration by parts)."""
    from scipy import integrate, special
    xi, F = oracle.spectrum_table()
    G = lambda s: integrate.quad(lambda t: special.kv(5 / 3, t), s, np.inf, limit=200)[0]
    for target in (1e-5, 1e-3, 0.05, 0.3, 1.0, 3.0, 8.0):
        i = int(np.argmin(np.abs(xi - target)))
        s = xi[i]
        val = s * G(s) + integrate.quad(lambda t: t * special.kv(5 / 3, t), 0, s, limit=200)[0]
        assert F[i] == pytest.approx(3 / (5 * math.pi) * val, rel=2e-7, abs=1e-12)


def test_spectrum_table_moments():
    """Mean and second moment of the sampled xi (exactly integrated over the
    piecewise-linear inverse CDF) against <xi> = 8/(15 sqrt 3), <xi^2> = 11/27."""
    xi, F = oracle.spectrum_table()
    # below the first knot xi = xi0 (u/F0)^3: int = xi0 F0/4, int xi^2 = xi0^2 F0/7
    m1 = xi[0] * F[0] / 4
    m2 = xi[0] ** 2 * F[0] / 7
    dF = np.diff(F)
    a, b = xi[:-1], xi[1:]
    m1 += np.sum(dF * (a + b) / 2)
    m2 += np.sum(dF * (a * a + a * b + b * b) / 3)
    m1 += xi[-1] * (1 - F[-1])
    m2 += xi[-1] ** 2 * (1 - F[-1])
    assert m1 == pytest.approx(8 / (15 * math.sqrt(3)), rel=2e-5)
    assert m2 == pytest.approx(11 / 27, rel=2e-4)
    # sampled check
    u = np.random.default_rng(8).random(200000)
    s = np.array([oracle.spectrum_sample(v) for v in u])
    assert s.mean() == pytest.approx(8 / (15 * math.sqrt(3)), rel=5 * s.std() / math.sqrt(s.size) / s.mean())


# --------------------------------------------------------------------------
# Synchrotron radiation

def test_radiation_mean_single_slice():
    """Energy lost in one dipole slice by an on-axis electron:
    U = C_gamma E^4 h^2 L / (2 pi), C_gamma = 8.846e-5 m/GeV^3 (beta -> 1)."""
    ref = I.electron_reference(45.6e9)
    theta, L = 2 * math.pi / 2400, 3.575
    el = I.table([I.multipole(knl=[theta], hxl=theta, lrad=L)])
    o = oracle.track(el, ref, one(ref), 1, rad_mode=1)
    E0 = 45.6
    U = 8.846e-5 * E0 ** 4 * (theta / L) ** 2 * L / (2 * math.pi) * 1e9
    assert -o["ptau"][0] * ref[2] == pytest.approx(U, rel=2e-4)
    # angles kept: px/(1+delta) unchanged by the emission (px = 0 here after
    # the curvature kick cancels the field kick on axis)
    assert abs(o["px"][0]) < 1e-18


def test_radiation_damping_partition():
    """Lepton ring with mean radiation: the one-turn eigenvalues at the 6D
    closed orbit give J_x ~ 1, J_y ~ 1, J_z ~ 2 (separated-function thin ring)
    and J_x + J_y + J_z = 4 (Robinson) to O(U0/E0); the energy the RF restores
    on the closed orbit equals C_gamma E^4 I2 / (2 pi) with I2 = sum theta^2/L
    over the table's dipole slices."""
    from oracle import optics as O
    el, ref, info = I.lepton_ring(n_cells=20, E0=10e9, v_total=100e6)
    d = O.damping(el, ref)
    rc = oracle.ref_constants(ref)
    mp = el[el["type"] == I.MULTIPOLE]
    rad = mp[mp["p"][:, 23] > 0]
    I2 = float(np.sum(rad["p"][:, 0] ** 2 / rad["p"][:, 23]))
    U0 = 8.846e-5 * (rc["E0"] / 1e9) ** 4 * I2 / (2 * math.pi) * 1e9
    eps = U0 / rc["E0"]
    assert d["U0"] == pytest.approx(U0, rel=max(2e-4, 3 * eps))
    J = d["J"]
    assert sum(J) == pytest.approx(4.0, rel=3 * eps)
    assert J[0] == pytest.approx(1.0, abs=10 * eps)
    assert J[1] == pytest.approx(1.0, abs=10 * eps)
    assert J[2] == pytest.approx(2.0, abs=10 * eps)
    assert np.linalg.det(d["M"]) == pytest.approx(math.exp(-4 * d["U0"] / rc["E0"]), rel=0.02 * 4 * eps)


def test_radiation_quantum_statistics():
    """One dipole slice, many electrons: mean photon number n = (5/(2 sqrt 3))
    alpha gamma theta, mean loss equal to the mean model, variance of the loss
    n <u^2> = n (11/27) u_c^2."""
    ref = I.electron_reference(45.6e9)
    theta, L = 2 * math.pi / 2400, 3.575
    el = I.table([I.multipole(knl=[theta], hxl=theta, lrad=L)])
    n = 100000
    p = I.make_particles(ref, np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n))
    oq = oracle.track(el, ref, p, 1, rad_mode=2, seed=99)
    om = oracle.track(el, ref, one(ref), 1, rad_mode=1)
    rc = oracle.ref_constants(ref)
    dE = -oq["ptau"] * ref[2]
    mean_model = -om["ptau"][0] * ref[2]
    assert dE.mean() == pytest.approx(mean_model, rel=5 * dE.std() / math.sqrt(n) / dE.mean())
    g = rc["gamma0"]
    h = theta / L
    nbar = 5 / (2 * math.sqrt(3)) * I.C_LIGHT * 0 + 5 / (2 * math.sqrt(3)) * 7.2973525693e-3 * g * h * L
    uc = 1.5 * 197.3269804e-9 * g ** 3 * h
    var = nbar * 11 / 27 * uc ** 2
    assert dE.var() == pytest.approx(var, rel=0.03)
    assert np.mean(dE == 0) == pytest.approx(math.exp(-nbar), abs=5 * math.sqrt(math.exp(-nbar) / n))


# --------------------------------------------------------------------------
# Brute force: whole-ring tracking in 40-digit arithmetic

def _hp_track(el, ref, p, turns):
    """The thin maps evaluated in mpmath for a few particles (drift, multipole,
    cavity only), to bound the oracle's FP64 rounding."""
    mpmath.mp.dps = 40
    m0, q0, p0c = [mpmath.mpf(v) for v in ref]
    E0 = mpmath.sqrt(p0c ** 2 + m0 ** 2)
    b0 = p0c / E0
    out = []
    for i in range(len(p["x"])):
        x, px, y, py, z = [mpmath.mpf(p[k][i]) for k in ("x", "px", "y", "py", "zeta")]
        pt = mpmath.mpf(p["ptau"][i])
        for _ in range(turns):
            for r in el:
                t, pp = int(r["type"]), r["p"]
                d = mpmath.sqrt(1 + 2 * pt / b0 + pt ** 2) - 1
                if t == I.DRIFT:
                    L = mpmath.mpf(pp[0])
                    pz = mpmath.sqrt((1 + d) ** 2 - px ** 2 - py ** 2)
                    rvv = (1 + d) / (1 + b0 * pt)
                    x += px * L / pz
                    y += py * L / pz
                    z += L - (1 + d) / rvv * L / pz
                elif t == I.MULTIPOLE:
                    zz = mpmath.mpc(x, y)
                    b = sum(mpmath.mpc(pp[n], pp[11 + n]) * zz ** n / math.factorial(n)
                            for n in range(int(r["order"]) + 1))
                    px -= b.real
                    py += b.imag
                elif t == I.CAVITY:
                    k = 2 * mpmath.pi * mpmath.mpf(pp[1]) / (b0 * I.C_LIGHT)
                    pt += q0 * mpmath.mpf(pp[0]) / p0c * mpmath.sin(mpmath.mpf(pp[2]) * mpmath.pi / 180 - k * z)
        out.append((x, px, y, py, z, pt))
    return out


def test_fodo10_bruteforce_highprec():
    el, ref = I.fodo10()
    p = I.subset(I.matched_gaussian(el, ref, 1000, 2.5e-6, 3e-4, seed=I.BASE_SEED), [0, 1, 2])
    o = oracle.track(el, ref, p, 5)
    hp = _hp_track(el, ref, p, 5)
    for i, v in enumerate(hp):
        for k, ref_v, scale in zip(("x", "px", "y", "py", "zeta", "ptau"), v,
                                   (1e-3, 1e-4, 1e-3, 1e-4, 1.0, 1e-3)):
            assert abs(o[k][i] - float(ref_v)) < 1e-14 * scale, (i, k)


# --------------------------------------------------------------------------
# The optics helpers of the oracle (oracle/optics.py)

def test_twiss_uncoupled_fodo_closed_forms():
    """FODO-10 (thin f = +-5 m, 2 m drifts, sin(mu/2) = L/(2f) = 0.2): at the
    entry of every thin QF, beta_x = L_c (1 + sin(mu/2))/sin(mu) with the cell
    length L_c = 4 m and alpha_x = -beta_x/(2f) (symmetric point of the thin
    lens); at every QD, beta_x = L_c (1 - sin(mu/2))/sin(mu) and
    alpha_x = +beta_x/(2f); y swaps the two; no bends, so no dispersion."""
    from oracle import optics as O
    el, ref = I.fodo10()
    tw = O.twiss_uncoupled(el, ref)
    f, Lc = 5.0, 4.0
    s2 = Lc / (4 * f)
    mu = 2 * math.asin(s2)
    bmax = Lc * (1 + s2) / math.sin(mu)
    bmin = Lc * (1 - s2) / math.sin(mu)
    qf = [i for i in range(el.shape[0]) if int(el[i]["type"]) == I.MULTIPOLE and el[i]["p"][1] > 0]
    qd = [i for i in range(el.shape[0]) if int(el[i]["type"]) == I.MULTIPOLE and el[i]["p"][1] < 0]
    assert len(qf) == 10 and len(qd) == 10
    for i in qf:
        assert tw["betx"][i] == pytest.approx(bmax, rel=1e-12)
        assert tw["alfx"][i] == pytest.approx(-bmax / (2 * f), rel=1e-12)
        assert tw["bety"][i] == pytest.approx(bmin, rel=1e-12)
        assert tw["alfy"][i] == pytest.approx(bmin / (2 * f), rel=1e-12)
    for i in qd:
        assert tw["betx"][i] == pytest.approx(bmin, rel=1e-12)
        assert tw["alfx"][i] == pytest.approx(bmin / (2 * f), rel=1e-12)
        assert tw["bety"][i] == pytest.approx(bmax, rel=1e-12)
        assert tw["alfy"][i] == pytest.approx(-bmax / (2 * f), rel=1e-12)
    assert np.max(np.abs(tw["dx"])) == 0.0 and np.max(np.abs(tw["dpx"])) == 0.0


def test_radiation_integrals_isomagnetic_and_H_from_local_one_turn_matrices():
    """Lepton ring of 20 cells, every dipole slice of the same curvature
    1/rho: I2 = 2 pi/rho and I3 = 2 pi/rho^2 (isomagnetic ring).  I5 sums
    H |h|^3 L with H = gamma D^2 + 2 alpha D D' + beta D'^2 from lattice
    functions propagated along the line; here H is recomputed at every dipole
    slice from that slice's own one-turn matrix A_i = M_i A M_i^-1 (beta,
    alpha, gamma from its entries, D from (1 - A_i) D = the slice's
    dispersion column), and the two I5 agree.  The constants are the
    textbook C_gamma = 8.846e-5 m/GeV^3 and C_q = 3.832e-13 m."""
    from oracle import optics as O
    el, ref, _ = I.lepton_ring(n_cells=20, E0=10e9, v_total=100e6)
    tw = O.twiss_uncoupled(el, ref)
    I2, I3, I5 = O.radiation_integrals(el, ref, tw)
    rad = [i for i in range(el.shape[0]) if int(el[i]["type"]) == I.MULTIPOLE and el[i]["p"][23] > 0
           and el[i]["p"][0] != 0]
    h = np.array([el[i]["p"][0] / el[i]["p"][23] for i in rad])
    assert np.allclose(h, h[0], rtol=1e-14, atol=0)
    rho = 1 / h[0]
    assert I2 == pytest.approx(2 * math.pi / rho, rel=1e-12)
    assert I3 == pytest.approx(2 * math.pi / rho ** 2, rel=1e-12)
    assert O.C_GAMMA == pytest.approx(8.846e-5, rel=1e-4)
    assert O.C_Q == pytest.approx(3.832e-13, rel=1e-4)
    # H from the local one-turn matrices
    elx = O.without_cavities(el)
    z0 = oracle.closed_orbit(elx, ref, rad_mode=0, dim=4)
    _, M, _, Ms = oracle.track_jacobian(elx, ref, z0, along=True)
    A = M[:2, :2]
    m5 = M[:2, 5]
    I5b = 0.0
    for i in rad:
        T = np.eye(6) if i == 0 else Ms[i - 1]
        Ti = np.linalg.inv(T)
        Mi = T @ M @ Ti           # one-turn matrix starting at the entry of row i
        Ai = Mi[:2, :2]
        c = 0.5 * np.trace(Ai)
        s = math.copysign(math.sqrt(1 - c * c), Ai[0, 1])
        b, a, g = Ai[0, 1] / s, (Ai[0, 0] - Ai[1, 1]) / (2 * s), -Ai[1, 0] / s
        D = np.linalg.solve(np.eye(2) - Ai, Mi[:2, 5])
        H = g * D[0] ** 2 + 2 * a * D[0] * D[1] + b * D[1] ** 2
        L = el[i]["p"][23]
        I5b += H * abs(el[i]["p"][0] / L) ** 3 * L
    assert I5 > 0 and I5b == pytest.approx(I5, rel=1e-9)
    assert np.trace(A) != 2.0 and np.any(m5 != 0)


def test_closed_orbit_of_a_corrector_kick():
    """A thin corrector (knl0 = theta, no curvature: px -= theta) in a linear
    thin FODO ring of 10 cells: the 4D closed orbit found by the oracle's
    Newton iteration sits, at the corrector, at x = theta_k beta/(2 tan(pi Q))
    with theta_k = -theta (textbook closed-orbit distortion of a single kick);
    beta and Q are those of the thin FODO in closed form.  The only
    non-linearity left is the exact drift's, of relative order px^2."""
    f, Ld = 5.0, 2.0
    cell = [I.multipole(knl=[0, 1 / f]), I.drift(Ld), I.multipole(knl=[0, -1 / f]), I.drift(Ld)]
    theta = 1e-6
    el = I.table([I.multipole(knl=[theta])] + cell * 10)
    z = oracle.closed_orbit(el, PROTON, dim=4)
    s2 = Ld / (2 * f)
    mu = 2 * math.asin(s2)
    beta = 2 * Ld * (1 + s2) / math.sin(mu)   # at the QF, where the corrector sits
    Q = 10 * mu / (2 * math.pi)
    x_co = -theta * beta / (2 * math.tan(math.pi * Q))
    assert z[0] == pytest.approx(x_co, rel=1e-9)
    assert abs(z[2]) < 1e-20 and abs(z[3]) < 1e-20
    # a fixed point of the one-turn map
    zo, _ = oracle.track_jacobian(el, PROTON, z)
    assert np.allclose(zo[:4], z[:4], rtol=0, atol=1e-15)  # the Newton tolerance


def test_natural_chromaticity_of_a_thin_fodo():
    """Thin FODO cell (f = 5 m, 2 m drifts) off momentum: the exact drift
    turns the quadrupoles' angle kicks into K L/(1+delta), so the first-order
    chromaticity is the textbook -(1/4 pi) sum beta_i K_i L_i = -(beta_max -
    beta_min)/(4 pi f) per cell, in both planes.  Measured by central
    differences of the cell tune at delta = +-1e-5 (4D fixed point at fixed
    pzeta; no bends, so the orbit stays on axis)."""
    f, Ld = 5.0, 2.0
    cell = I.table([I.multipole(knl=[0, 1 / f]), I.drift(Ld), I.multipole(knl=[0, -1 / f]), I.drift(Ld)])
    rc = oracle.ref_constants(PROTON)
    b0 = rc["beta0"]

    def tunes(delta):
        # pzeta of a particle with momentum deviation delta: ptau = (E - E0)/(P0 c)
        E = math.sqrt((PROTON[2] * (1 + delta)) ** 2 + PROTON[0] ** 2)
        ptau = (E - rc["E0"]) / PROTON[2]
        z = np.array([0, 0, 0, 0, 0, ptau / b0])
        _, M = oracle.track_jacobian(cell, PROTON, z)
        return (math.acos(0.5 * np.trace(M[:2, :2])) / (2 * math.pi),
                math.acos(0.5 * np.trace(M[2:4, 2:4])) / (2 * math.pi))

    d = 1e-5
    qp, qm = tunes(d), tunes(-d)
    s2 = Ld / (2 * f)
    mu = 2 * math.asin(s2)
    bmax = 2 * Ld * (1 + s2) / math.sin(mu)
    bmin = 2 * Ld * (1 - s2) / math.sin(mu)
    xi = -(bmax - bmin) / (4 * math.pi * f)
    assert (qp[0] - qm[0]) / (2 * d) == pytest.approx(xi, rel=1e-6)
    assert (qp[1] - qm[1]) / (2 * d) == pytest.approx(xi, rel=1e-6)
    assert tunes(0.0)[0] == pytest.approx(mu / (2 * math.pi), rel=1e-14)


def test_momentum_compaction_on_the_dispersive_closed_orbit():
    """Lepton ring of 20 cells with RF off: a particle on the 4D closed orbit
    of momentum deviation pzeta slips per turn by dzeta = -C (alpha_c -
    1/gamma0^2) pzeta to first order, with the momentum compaction of thin
    dipoles alpha_c = sum theta_i D_i / C (D at each dipole slice from the
    propagated lattice functions) and C the sum of drift lengths.  The slip
    comes from Newton closed orbits at pzeta = +-1e-6 tracked for one turn:
    it checks the curvature path-length term against the dispersion that the
    curvature kick creates, and the drift's 1/gamma^2 term."""
    from oracle import optics as O
    el, ref, _ = I.lepton_ring(n_cells=20, E0=10e9, v_total=100e6)
    elx = O.without_cavities(el)
    tw = O.twiss_uncoupled(elx, ref)
    rc = oracle.ref_constants(ref)
    C = float(np.sum(elx[elx["type"] == I.DRIFT]["p"][:, 0]))
    dip = [i for i in range(elx.shape[0]) if int(elx[i]["type"]) == I.MULTIPOLE and elx[i]["p"][22] != 0]
    alpha_c = sum(elx[i]["p"][22] * tw["dx"][i] for i in dip) / C
    eta = alpha_c - 1.0 / rc["gamma0"] ** 2

    def slip(pz):
        z = oracle.closed_orbit(elx, ref, dim=4, guess=[0, 0, 0, 0, 0, pz])
        zo, _ = oracle.track_jacobian(elx, ref, z)
        return zo[4] - z[4]

    e = 1e-6
    assert (slip(e) - slip(-e)) / (2 * e) == pytest.approx(-C * eta, rel=1e-6)
    assert alpha_c > 0.0


def test_chromaticity_with_sextupoles_and_dispersion():
    """Lepton ring of 20 cells (thin quadrupoles, thin dipoles with their
    k0 h weak focusing, thin sextupoles at dispersion), RF off: the
    chromaticities from the tunes of the Newton closed orbits at
    pzeta = +-1e-6 equal the first-order sums
    xi_x = (1/4 pi) sum beta_x (-(k1 L + k0 h L) + k2 L D),
    xi_y = (1/4 pi) sum beta_y (k1 L - k2 L D), to 1e-6.  This fixes the
    sextupole's sign and factor against the quadrupole's and the drift's
    chromatic terms."""
    from oracle import optics as O
    el, ref, _ = I.lepton_ring(n_cells=20, E0=10e9, v_total=100e6)
    elx = O.without_cavities(el)
    tw = O.twiss_uncoupled(elx, ref)

    def tunes(pz):
        z = oracle.closed_orbit(elx, ref, dim=4, guess=[0, 0, 0, 0, 0, pz])
        _, M = oracle.track_jacobian(elx, ref, z)
        return np.array([math.acos(0.5 * np.trace(M[:2, :2])), math.acos(0.5 * np.trace(M[2:4, 2:4]))]) / (2 * math.pi)

    e = 1e-6
    xi = (tunes(e) - tunes(-e)) / (2 * e)
    sx = sy = 0.0
    n_sext = 0
    for i in range(elx.shape[0]):
        r = elx[i]
        if int(r["type"]) != I.MULTIPOLE:
            continue
        k1, k2, hxl, L = r["p"][1], r["p"][2], r["p"][22], r["p"][23]
        k0h = r["p"][0] * hxl / L if (hxl != 0 and L > 0) else 0.0
        n_sext += k2 != 0
        sx += tw["betx"][i] * (-(k1 + k0h) + k2 * tw["dx"][i])
        sy += tw["bety"][i] * (k1 - k2 * tw["dx"][i])
    assert n_sext > 0
    assert xi[0] == pytest.approx(sx / (4 * math.pi), rel=1e-6)
    assert xi[1] == pytest.approx(sy / (4 * math.pi), rel=1e-6)
    assert xi[0] > 1.0 and xi[1] > 1.0


def _hp_mean_radiation_line(el, ref, p):
    """One pass of drifts and multipoles (curvature and mean radiation
    included) in 40-digit arithmetic, written from the map definitions: the
    field kick b = sum (knl_n + i ksl_n) z^n / n!, the curved frame's
    px += hxl (1+delta) - knl0 hxl x / L_rad and zeta -= hxl x / rvv, then
    the energy loss dE = -(2/3) r_c m0 c^2 beta^3 gamma^4 h^2 L_rad with
    h = |b| / ((1+delta) L_rad) and the particle's own beta and gamma, and
    px, py scaled by (1+delta_new)/(1+delta_old)."""
    mpmath.mp.dps = 40
    mpf = mpmath.mpf
    m0, q0, p0c = [mpf(v) for v in ref]
    E0 = mpmath.sqrt(p0c ** 2 + m0 ** 2)
    b0 = p0c / E0
    r_c = q0 ** 2 * mpf("2.8179403262e-15") * mpf("0.51099895000e6") / m0
    out = []
    for i in range(len(p["x"])):
        x, px, y, py, z, pt = [mpf(p[k][i]) for k in ("x", "px", "y", "py", "zeta", "ptau")]
        for r in el:
            t, pp = int(r["type"]), r["p"]
            d = mpmath.sqrt(1 + 2 * pt / b0 + pt ** 2) - 1
            rvv = (1 + d) / (1 + b0 * pt)
            if t == I.DRIFT:
                L = mpf(pp[0])
                pz = mpmath.sqrt((1 + d) ** 2 - px ** 2 - py ** 2)
                x += px * L / pz
                y += py * L / pz
                z += L - (1 + d) / rvv * L / pz
            elif t == I.MULTIPOLE:
                zz = mpmath.mpc(x, y)
                b = sum(mpmath.mpc(pp[n], pp[11 + n]) * zz ** n / math.factorial(n)
                        for n in range(int(r["order"]) + 1))
                px -= b.real
                py += b.imag
                hxl, Lr = mpf(pp[22]), mpf(pp[23])
                if hxl != 0:
                    px += hxl * (1 + d) - mpf(pp[0]) * hxl * x / Lr
                    z -= hxl * x / rvv
                if Lr > 0:
                    h2 = (b.real ** 2 + b.imag ** 2) / (Lr ** 2 * (1 + d) ** 2)
                    E = E0 + pt * p0c
                    gam, bet = E / m0, (1 + d) * p0c / E
                    dE = -mpf(2) / 3 * r_c * m0 * bet ** 3 * gam ** 4 * h2 * Lr
                    pt = pt + dE / p0c
                    dn = mpmath.sqrt(1 + 2 * pt / b0 + pt ** 2) - 1
                    px *= (1 + dn) / (1 + d)
                    py *= (1 + dn) / (1 + d)
        out.append((x, px, y, py, z, pt))
    return out


def test_mean_radiation_map_against_40_digits():
    """1 GeV electrons (beta^3 differs from 1 by 4e-7, gamma^4 of the
    particle from gamma0^4 by 4 delta) through radiating slices off axis and
    off momentum: a combined-function dipole slice with curvature, a skew
    quadrupole component, a sextupole, and drifts.  The oracle's mean model
    agrees with the 40-digit statement of the map to 1e-13 of each
    coordinate's scale, and its energy loss (about 3e-9 in ptau, against
    ptau itself near 2e-3) to 1e-9."""
    ref = I.electron_reference(1e9)
    theta, L = 0.02, 2.0
    el = I.table([I.multipole(knl=[theta, 0.05], ksl=[0, 0.01], hxl=theta, lrad=L), I.drift(0.7),
                  I.multipole(knl=[0, -0.3], lrad=0.4), I.drift(0.5),
                  I.multipole(knl=[0, 0, 2.0], ksl=[0, 0, 0.5], lrad=0.3), I.drift(0.4)])
    rng = np.random.default_rng(21)
    n = 4
    p = I.make_particles(ref, rng.normal(0, 2e-3, n), rng.normal(0, 2e-4, n), rng.normal(0, 1e-3, n),
                         rng.normal(0, 1e-4, n), rng.normal(0, 1e-2, n), rng.normal(0, 2e-3, n))
    o = oracle.track(el, ref, p, 1, rad_mode=1)
    off = oracle.track(el, ref, p, 1, rad_mode=0)
    hp = _hp_mean_radiation_line(el, ref, p)
    for i, v in enumerate(hp):
        for k, hv, scale in zip(("x", "px", "y", "py", "zeta", "ptau"), v, (1e-3, 1e-4, 1e-3, 1e-4, 1e-2, 1e-3)):
            assert abs(o[k][i] - float(hv)) < 1e-13 * scale, (i, k, o[k][i], float(hv))
        loss = float(v[5] - mpmath.mpf(p["ptau"][i]))
        assert o["ptau"][i] - p["ptau"][i] == pytest.approx(loss, rel=1e-9)
        assert o["ptau"][i] < off["ptau"][i]


def test_quantum_emission_against_40_digits_with_numpy_philox():
    """One radiating dipole slice, 45.6 GeV electrons with particle ids 1..8
    off axis and off momentum.  Restated in 40 digits with random numbers
    drawn by numpy's independent Philox4x64-10 at the counter (particle id,
    turn, element, call) and key (seed, 0), one uniform (w >> 11) 2^-53 per
    64-bit word: the photon count by inversion of the Poisson CDF of
    n = (5/(2 sqrt 3)) alpha q0^2 gamma h L_rad at the first word, the photon
    energies u_c xi with xi from the next words through the spectrum sampler
    (pinned against scipy's Bessel quadrature), u_c = (3/2) hbar c gamma^3 h,
    gamma and h = |b|/((1+delta) L_rad) of the particle, then the energy
    update and the angle-keeping scaling.  The oracle agrees to 1e-13 of each
    coordinate's scale, so the counter layout, the word order and both
    formulas are fixed."""
    mpmath.mp.dps = 40
    mpf = mpmath.mpf
    ref = I.electron_reference(45.6e9)
    theta, L, seed, elem, turn = 2 * math.pi / 2400, 3.575, 77, 0, 0
    el = I.table([I.multipole(knl=[theta, 0.01], hxl=theta, lrad=L)])
    rng = np.random.default_rng(22)
    n = 8
    p = I.make_particles(ref, rng.normal(0, 1e-3, n), rng.normal(0, 1e-5, n), rng.normal(0, 5e-4, n),
                         rng.normal(0, 1e-5, n), rng.normal(0, 1e-3, n), rng.normal(0, 1e-3, n),
                         particle_id=np.arange(1, n + 1))
    o = oracle.track(el, ref, p, 1, rad_mode=2, seed=seed)
    m0, q0, p0c = [mpf(v) for v in ref]
    E0 = mpmath.sqrt(p0c ** 2 + m0 ** 2)
    b0 = p0c / E0
    alpha, hbarc = mpf("7.2973525693e-3"), mpf("197.3269804e-9")
    counts = []
    for i in range(n):
        pid = int(p["particle_id"][i])
        words = []
        for call in range(8):
            bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                                  counter=np.array([pid - 1, turn, elem, call], dtype=np.uint64))
            words += [int(w) for w in bg.random_raw(4)]
        u = [mpf(w >> 11) / mpf(2) ** 53 for w in words]
        x, px, y, py, z, pt = [mpf(p[k][i]) for k in ("x", "px", "y", "py", "zeta", "ptau")]
        d = mpmath.sqrt(1 + 2 * pt / b0 + pt ** 2) - 1
        rvv = (1 + d) / (1 + b0 * pt)
        b = mpf(theta) + mpf(0.01) * mpmath.mpc(x, y)
        px -= b.real
        py += b.imag
        hx = mpf(theta)
        px += hx * (1 + d) - mpf(theta) * hx * x / mpf(L)
        z -= hx * x / rvv
        h = abs(b) / ((1 + d) * mpf(L))
        gam = (E0 + pt * p0c) / m0
        nbar = 5 / (2 * mpmath.sqrt(3)) * alpha * q0 ** 2 * gam * h * mpf(L)
        k, term = 0, mpmath.exp(-nbar)
        F = term
        while u[0] > F:
            k += 1
            term = term * nbar / k
            F += term
        assert abs(u[0] - F) > 1e-12 and k < 30
        counts.append(k)
        xi = sum(mpf(oracle.spectrum_sample(float(u[1 + j]))) for j in range(k))
        uc = mpf(3) / 2 * hbarc * gam ** 3 * h
        if k > 0:
            pt_new = pt - uc * xi / p0c
            dn = mpmath.sqrt(1 + 2 * pt_new / b0 + pt_new ** 2) - 1
            px *= (1 + dn) / (1 + d)
            py *= (1 + dn) / (1 + d)
            pt = pt_new
        for key, hv, scale in zip(("x", "px", "y", "py", "zeta", "ptau"), (x, px, y, py, z, pt),
                                  (1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-3)):
            assert abs(o[key][i] - float(hv)) < 1e-13 * scale, (i, key, k, o[key][i], float(hv))
    assert max(counts) >= 2 and len(set(counts)) >= 3  # several photon counts occur
