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
