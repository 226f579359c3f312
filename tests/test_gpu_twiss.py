"""Twiss by tracking on the GPU (section "Twiss module") against the oracle.

The oracle's optics come from exact forward-mode Jacobians of its maps; the
GPU version finds the closed orbit by Newton's method and the one-turn matrix
by central differences of particles tracked by the library's kernel.  Checked
on a FODO ring with misaligned quadrupoles (a non-zero closed orbit): closed
orbit, tunes, beta, alpha and dispersion at the start, and the chromaticity;
and on the lepton ring with mean radiation: the damping decrements from the
eigenvalues of the one-turn matrix.  Tolerances follow the central
differences (steps 1e-8 m, 1e-10 rad)."""
import math

import numpy as np
import pytest

import oracle
from oracle import optics as O
from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import twiss as T

pytestmark = pytest.mark.gpu


def misaligned_fodo():
    el, ref = I.fodo10()
    rows = []
    for k, r in enumerate(list(el)):
        if int(r["type"]) == I.MULTIPOLE and r["p"][1] != 0.0:
            rows += I.misaligned([r], dx=2e-4 * math.sin(1.3 * k), dy=-1e-4 * math.cos(0.7 * k), tilt=2e-3 * (k % 3))
        else:
            rows.append(r)
    return I.table(rows), ref


def oracle_tune(el, ref, delta0):
    m0, _, p0c = ref
    E0 = math.sqrt(p0c ** 2 + m0 ** 2)
    beta0 = p0c / E0
    g = np.zeros(6)
    g[5] = (math.sqrt((p0c * (1 + delta0)) ** 2 + m0 ** 2) - E0) / p0c / beta0
    co = oracle.closed_orbit(T.without_cavities(el), ref, rad_mode=0, dim=4, guess=g)
    _, M = oracle.track_jacobian(T.without_cavities(el), ref, co)
    return T._tune(M[:2, :2])[0], T._tune(M[2:4, 2:4])[0]


def test_closed_orbit_and_optics_of_a_misaligned_ring():
    el, ref = misaligned_fodo()
    t = T.twiss(el, ref)
    co = oracle.closed_orbit(T.without_cavities(el), ref, rad_mode=0, dim=4)
    assert np.max(np.abs(co[:4])) > 1e-5
    assert np.max(np.abs(t["closed_orbit"][:4] - co[:4])) < 1e-12
    tw = O.twiss_uncoupled(el, ref)
    qx, _ = T._tune(tw["M"][:2, :2])
    qy, _ = T._tune(tw["M"][2:4, 2:4])
    assert abs(t["qx"] - qx) < 1e-9 and abs(t["qy"] - qy) < 1e-9
    assert t["betx"] == pytest.approx(tw["betx"][0], rel=1e-7)
    assert t["bety"] == pytest.approx(tw["bety"][0], rel=1e-7)
    assert t["alfx"] == pytest.approx(tw["alfx"][0], abs=1e-7)
    assert t["alfy"] == pytest.approx(tw["alfy"][0], abs=1e-7)
    # tilted quadrupoles couple the planes: the periodic dispersion solves the
    # 4x4 system (I - M4) D = M[:4, 5], here from the oracle's exact matrix
    D = np.linalg.solve(np.eye(4) - tw["M"][:4, :4], tw["M"][:4, 5])
    assert t["dx"] == pytest.approx(D[0], rel=1e-6, abs=1e-10)
    assert t["dy"] == pytest.approx(D[2], rel=1e-6, abs=1e-10)


def test_chromaticity():
    el, ref = misaligned_fodo()
    d = 1e-5
    cx, cy = T.chromaticity(el, ref, d)
    (ax, ay), (bx, by) = oracle_tune(el, ref, d), oracle_tune(el, ref, -d)
    ox, oy = ((ax - bx + 0.5) % 1 - 0.5) / (2 * d), ((ay - by + 0.5) % 1 - 0.5) / (2 * d)
    assert cx == pytest.approx(ox, abs=1e-4) and cy == pytest.approx(oy, abs=1e-4)
    assert abs(cx) > 0.1


def test_damping_decrements_of_the_lepton_ring():
    el, ref, _ = I.lepton_ring()
    g = T.damping(el, ref)
    d = O.damping(el, ref)
    np.testing.assert_allclose(g["alpha"], d["alpha"], rtol=1e-5)
    assert np.max(np.abs(g["closed_orbit"] - d["closed_orbit"])) < 1e-10


def test_beambeam_tune_shift_by_tracking():
    """A linear ring with a head-on round proton lens at the IP: the tune
    from Twiss by tracking on the GPU obeys the thin-lens relation
    cos 2 pi Q = cos 2 pi Q0 + (beta k / 2) sin 2 pi Q0 with the lens's
    linear strength k = K / (2 sigma^2), K = 2 N r_e m_e c^2 / p0 c."""
    ref = I.proton_reference(450e9)
    m0, _, p0c = ref
    N, sig, beta, Q0 = 1.15e11, 50e-6, 0.55, 0.31
    mu = 2 * math.pi * Q0
    M = np.eye(6)
    for k in (0, 2):
        M[k, k], M[k, k + 1], M[k + 1, k], M[k + 1, k + 1] = math.cos(mu), beta * math.sin(mu), -math.sin(mu) / beta, math.cos(mu)
    lens = I.beambeam4d(N, 1.0, sig, sig)
    el = I.table([I.linear_map(M), lens])
    t = T.twiss(el, ref)
    k = 2 * N * 2.8179403262e-15 * 0.51099895000e6 / p0c / (2 * sig * sig)
    assert math.cos(2 * math.pi * t["qx"]) == pytest.approx(math.cos(mu) + beta * k / 2 * math.sin(mu), abs=1e-8)
    assert math.cos(2 * math.pi * t["qy"]) == pytest.approx(math.cos(mu) + beta * k / 2 * math.sin(mu), abs=1e-8)
    assert t["qx"] < Q0 - 0.004


# --------------------------------------------------------------------------
# Lattice functions along the line (eigenvectors propagated by tracking)

def _mixed_lepton_line():
    """Thin and thick elements with mean radiation on: radiating thin dipole
    slices, full and expanded bends, thick quadrupoles, sextupoles, an RF
    cavity and an aperture."""
    h = 1.0 / 30.0
    rows = [I.cavity(50e6, 400e6, 175.0)]
    for c in range(6):
        rows += [I.quadrupole(0.35, 0.5), I.drift(0.4), I.bend(h, h, 1.5, full=True), I.drift(0.3)]
        rows += [I.multipole(knl=[h * 1.0, 0.0, 0.3], hxl=h * 1.0, lrad=1.0), I.drift(0.3)]
        rows += [I.quadrupole(-0.35, 0.5), I.drift(0.4), I.bend(h, h, 1.5, k1=-0.02), I.drift(0.5),
                 I.aperture(0.008)]
    return I.table(rows)


def test_monitor_equals_the_oracle_after_every_row():
    """The monitor's state after every row matches the oracle tracking the
    same particles through that prefix of the table (identical loss state,
    coordinates within 1e-12 relative of the larger of their own size and
    their spread), with mean radiation; the final state equals one turn of
    xt_track bit for bit."""
    import torch
    from paper_2310_00317_gb300 import xtgb
    el = _mixed_lepton_line()
    ref = I.electron_reference(3e9)
    rng = np.random.default_rng(83)
    n = 64
    p = I.make_particles(ref, rng.normal(0, 3e-3, n), rng.normal(0, 1e-3, n), rng.normal(0, 1e-3, n),
                         rng.normal(0, 1e-4, n), rng.normal(0, 1e-3, n), rng.normal(0, 2e-3, n))
    tr = xtgb.Tracker(el, ref, radiation=xtgb.RAD_MEAN)
    P = xtgb.Particles.from_numpy(p)
    out = tr.monitor(P).cpu().numpy()
    Q = xtgb.Particles.from_numpy(p)
    tr.track(Q, 1)
    tr.close()
    fin, one = P.to_numpy(), Q.to_numpy()
    for k in oracle.FLOAT_FIELDS + oracle.INT_FIELDS:
        a, b = fin[k], one[k]
        assert np.all((a == b) | (np.isnan(a) & np.isnan(b))), k
    names = ("x", "px", "y", "py", "zeta", "ptau", "delta")
    for i in range(el.shape[0]):
        o = oracle.track(el[:i + 1], ref, p, 1, rad_mode=1)
        for c, k in enumerate(names):
            a, b = out[i, c], o[k]
            fin = np.isfinite(b)
            scale = np.maximum(np.abs(b), np.sqrt(np.mean(b[fin] ** 2)) if fin.any() else 0.0) + 1e-300
            ok = (np.abs(a - b) <= 1e-12 * scale) | (np.isnan(a) & np.isnan(b))
            assert np.all(ok), (i, k, float(np.max(np.abs(a - b) / scale)))
        assert np.all(out[i, 7] == o["state"]), i
    assert np.any(out[-1, 7] != 1.0) and np.any(out[-1, 7] == 1.0)


def _cs_along(Ms, b0, a0):
    m11, m12, m21, m22 = Ms[:, 0, 0], Ms[:, 0, 1], Ms[:, 1, 0], Ms[:, 1, 1]
    u, v = m11 * b0 - m12 * a0, m21 * b0 - m22 * a0
    return (u * u + m12 * m12) / b0, -(u * v + m12 * m22) / b0


def test_twiss_along_thin_fodo():
    """FODO-10 (thin quadrupoles f = 5 m, 4 m cells): beta at the quadrupoles
    equals the closed forms Lc (1 +- sin(mu/2)) / sin(mu) with
    sin(mu/2) = Lc / (4 f), the phase advance per cell is mu, and beta and
    alpha at every row agree with Courant-Snyder propagation through the
    oracle's exact per-row Jacobians."""
    el, ref = I.fodo10()
    t = T.twiss_along(el, ref)
    mu = 2 * math.asin(0.2)
    bp, bm = 4 * 1.2 / math.sin(mu), 4 * 0.8 / math.sin(mu)
    rows = list(el)
    qf = np.array([i for i, r in enumerate(rows) if int(r["type"]) == I.MULTIPOLE and r["p"][1] > 0])
    qd = np.array([i for i, r in enumerate(rows) if int(r["type"]) == I.MULTIPOLE and r["p"][1] < 0])
    assert np.allclose(t["betx"][qf + 1], bp, rtol=1e-7) and np.allclose(t["bety"][qf + 1], bm, rtol=1e-7)
    assert np.allclose(t["betx"][qd + 1], bm, rtol=1e-7) and np.allclose(t["bety"][qd + 1], bp, rtol=1e-7)
    assert np.allclose(np.diff(t["mux"][qf + 1]), mu / (2 * math.pi), atol=1e-9)
    assert abs(t["qx"] - (10 * mu / (2 * math.pi)) % 1.0) < 1e-9
    assert np.max(t["betx2"]) < 1e-12 and np.max(t["bety1"]) < 1e-12
    elo = T.without_cavities(el)
    _, M, _, Ms = oracle.track_jacobian(elo, ref, np.zeros(6), along=True)
    sx = math.copysign(math.sqrt(1 - (0.5 * np.trace(M[:2, :2])) ** 2), M[0, 1])  # sin(mu)
    bx0, ax0 = M[0, 1] / sx, (M[0, 0] - M[1, 1]) / (2 * sx)
    bx, ax = _cs_along(Ms, bx0, ax0)
    assert np.max(np.abs(t["betx"][1:] / bx - 1)) < 1e-7
    assert np.max(np.abs(t["alfx"][1:] - ax)) < 1e-6


def test_twiss_along_coupled_ring_with_thick_elements():
    """A misaligned FODO ring with a skew quadrupole, thick quadrupoles and
    expanded bends: the GPU's eigenvectors propagated along the line agree
    with those propagated through the oracle's exact per-row Jacobians
    (beta of both modes in both planes, the dispersion), and the coupling
    terms are non-zero."""
    el0, ref = misaligned_fodo()
    h = 0.01
    rows = list(el0)[:26] + [I.multipole(ksl=[0.0, 0.02]), I.quadrupole(0.1, 0.6), I.bend(h, h, 2.0),
                              I.quadrupole(-0.01, 0.6)] + list(el0)[26:]
    el = I.table(rows)
    t = T.twiss_along(el, ref)
    elo = T.without_cavities(el)
    co = oracle.closed_orbit(elo, ref, rad_mode=0, dim=4)
    _, M, _, Ms = oracle.track_jacobian(elo, ref, co, along=True)
    V0 = T.normal_modes(M[:4, :4])
    V = np.einsum("eij,jk->eik", Ms[:, :4, :4], V0)
    for name, j, k in (("betx", 0, 0), ("bety", 2, 1), ("betx2", 0, 1), ("bety1", 2, 0)):
        want = 2 * np.abs(V[:, j, k]) ** 2
        assert np.max(np.abs(t[name][1:] - want)) < 1e-7 * np.max(want), name
    D0 = np.linalg.solve(np.eye(4) - M[:4, :4], M[:4, 5])
    D = np.einsum("eij,j->ei", Ms[:, :4, :4], D0) + Ms[:, :4, 5]
    assert np.max(np.abs(t["dx"][1:] - D[:, 0])) < 1e-6 * np.max(np.abs(D[:, 0]))
    assert np.max(t["betx2"]) > 1e-3 and np.max(t["bety1"]) > 1e-3


# --------------------------------------------------------------------------
# Energy-loss compensation (tapering)

def test_energy_loss_compensation_keeps_the_design_orbit():
    """The 45.6 GeV lepton ring (10,000 rows) with its RF lumped into 4
    stations, so that the radiation energy sawtooth spans about 1.5e-3.
    After the compensation loop the closed-orbit particle comes back with
    the energy it started with, stays on the design orbit while its energy
    follows the sawtooth, and the energy lost per turn is the design
    C_gamma E0^4 I2 / (2 pi) within 0.5 %.  With the same RF phases and
    untapered magnets the orbit strays by millimetres."""
    from paper_2310_00317_gb300 import xtgb
    rows, ref, info = I.lepton_ring(rf_every=50)
    el = I.table(rows)
    c = T.compensate_energy_loss(el, ref)
    assert c["converged"] and c["iterations"] < 40
    assert abs(c["delta_end"]) < 1e-12
    assert np.max(np.abs(c["x"])) < 1e-9 and np.max(np.abs(c["y"])) < 1e-12
    assert 1e-3 < np.ptp(c["delta"]) < 2e-3
    assert abs(c["energy_loss"] / info["U0"] - 1) < 5e-3
    # untapered magnets, compensated RF phases: the sawtooth moves the orbit
    el_u = np.array(c["table"], copy=True)
    el_u = T.scale_magnets(el_u, 1.0 / c["scale"])
    tr = xtgb.Tracker(el_u, ref, radiation=xtgb.RAD_MEAN)
    P = xtgb.Particles.from_numpy(T.particles_from_z(ref, np.zeros((1, 6))))
    out = tr.monitor(P).cpu().numpy()[:, :, 0]
    tr.close()
    assert np.max(np.abs(out[:, 0])) > 1e-4


def test_twiss_open_line_with_periodic_initial_conditions():
    """One cell of FODO-10 as an open line from the ring's periodic
    functions at its start reproduces the ring's beta, alpha and phase
    along the cell; from other initial conditions beta follows
    Courant-Snyder propagation through the oracle's per-row Jacobians."""
    el, ref = I.fodo10()
    ring = T.twiss_along(el, ref)
    cell = T.without_cavities(el)[1:6]
    t = T.twiss_open(cell, ref, ring["betx"][1], ring["alfx"][1], ring["bety"][1], ring["alfy"][1])
    assert np.max(np.abs(t["betx"] - ring["betx"][1:7])) < 1e-7 * np.max(ring["betx"])
    assert np.max(np.abs(t["alfy"] - ring["alfy"][1:7])) < 1e-7
    assert np.max(np.abs(t["mux"] - (ring["mux"][1:7] - ring["mux"][1]))) < 1e-9
    t2 = T.twiss_open(T.without_cavities(el), ref, 20.0, -1.5, 5.0, 0.4)
    _, _, _, Ms = oracle.track_jacobian(T.without_cavities(el), ref, np.zeros(6), along=True)
    bx, ax = _cs_along(Ms, 20.0, -1.5)
    assert np.max(np.abs(t2["betx"][1:] / bx - 1)) < 1e-7 and np.max(np.abs(t2["alfx"][1:] - ax)) < 1e-6


def test_equilibrium_emittances_from_the_normal_form():
    """The 45.6 GeV lepton ring: horizontal emittance and momentum spread
    from the normal form (quantum diffusion carried by the 6D modes, damping
    from the one-turn eigenvalues) agree with the synchrotron-integral values
    C_q gamma^2 I5 / (J_x I2) and C_q gamma^2 I3 / (J_z I2) of the oracle's
    optics within 2 %; the vertical emittance of the uncoupled ring vanishes."""
    el, ref, _ = I.lepton_ring()
    e = T.equilibrium_emittances(el, ref)
    eq = O.equilibrium(el, ref)
    assert abs(e["eps"][0] / eq["eps_x"] - 1) < 0.02, (e["eps"], eq["eps_x"])
    assert abs(e["sigma_delta"] / eq["sigma_delta"] - 1) < 0.02, (e["sigma_delta"], eq["sigma_delta"])
    assert e["eps"][1] < 1e-6 * e["eps"][0]


def test_kick_as_closed_orbit_lattice_functions():
    """The 45.6 GeV lepton ring with mean radiation, by the kick-as-closed-
    orbit line (radiation kicks of the closed orbit applied to every
    particle as constant translations): tracked without radiation it keeps
    the radiation closed orbit, its one-turn matrix is symplectic, its tunes
    equal the eigen-tunes of the non-symplectic one-turn matrix with
    radiation, and its beta functions differ from those without radiation
    by the small amount the energy sawtooth causes."""
    from paper_2310_00317_gb300 import xtgb
    el, ref, _ = I.lepton_ring()
    kt, co, index = T.kick_as_closed_orbit(el, ref)
    tr = xtgb.Tracker(kt, ref)
    z1 = T.track_z(tr, ref, co[None])[0]
    tr.close()
    assert np.max(np.abs(z1 - co)) < 1e-11
    t = T.twiss_along(kt, ref, dim=6)
    S6 = T._symplectic_form(6)
    assert np.max(np.abs(t["M"].T @ S6 @ t["M"] - S6)) < 1e-8
    rad = T.twiss(el, ref, dim=6, radiation=xtgb.RAD_MEAN)
    w = np.linalg.eigvals(rad["M"])
    q_rad = np.sort(np.abs(np.angle(w)) / (2 * math.pi))[[2, 4]]  # the two transverse pairs
    w0 = np.linalg.eigvals(t["M"])
    q_kc = np.sort(np.abs(np.angle(w0)) / (2 * math.pi))[[2, 4]]
    assert np.max(np.abs(q_rad - q_kc)) < 1e-4, (q_rad, q_kc)
    t0 = T.twiss_along(el, ref, dim=6)
    rel = np.abs(t["betx"][index + 1] / t0["betx"][1:] - 1)
    print("max relative beta-x change from radiation: %.2e" % np.max(rel))
    assert np.max(rel) < 1e-2
