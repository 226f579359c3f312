"""The seeded synthetic inputs (paper_2310_00317_gb300/inputs.py) against
their stated recipe (CPU): element counts of the LHC-scale ring, the
generator's design optics against the oracle's lattice functions of the same
table, the matched beam's emittance, the DA grid's layout and the uneven
per-seed particle counts."""
import math

import numpy as np
import pytest

import oracle
from oracle import optics as O
from paper_2310_00317_gb300 import inputs as I


@pytest.fixture(scope="module")
def lhc():
    el, ref = I.lhc_ring()
    return el, ref, I.design_optics(el, ref)


def test_lhc_ring_composition(lhc):
    el, ref, _ = lhc
    t = el["type"]
    assert el.shape[0] == 20000
    assert int(np.sum(t == I.DRIFT)) == 6800
    assert int(np.sum(t == I.MULTIPOLE)) == 6800
    assert int(np.sum(t == I.CAVITY)) == 8
    assert int(np.sum(t == I.APERTURE)) == 6392
    ap = el[t == I.APERTURE]
    assert np.all(ap["p"][:, 0] == 0.02)  # radius [m]
    cav = el[t == I.CAVITY]
    assert np.all(cav["p"][:, 0] == 2e6) and np.all(cav["p"][:, 1] == 400e6) and np.all(cav["p"][:, 2] == 180.0)
    mp = el[t == I.MULTIPOLE]
    assert np.all(mp["order"] == 10)
    assert ref[2] == 450e9
    C = float(np.sum(el[t == I.DRIFT]["p"][:, 0]))
    assert C == pytest.approx(200 * 106.9, rel=1e-3)


def test_design_optics_equal_the_oracle_lattice_functions(lhc):
    """The generator places particles with its own thin-lens 2x2/3x3 optics;
    at element 0 they equal the oracle's lattice functions from the exact
    one-turn Jacobian of the same table (radiation and RF off), and the
    tunes are the stated 49.31 / 49.32."""
    el, ref, d = lhc
    tw = O.twiss_uncoupled(el, ref)
    for k in ("betx", "alfx", "bety", "alfy"):
        assert d[k][0] == pytest.approx(tw[k][0], rel=1e-8, abs=1e-9), k
    assert d["dx"][0] == pytest.approx(tw["dx"][0], rel=1e-6, abs=1e-9)
    M = tw["M"]
    qx = math.acos(0.5 * np.trace(M[:2, :2])) / (2 * math.pi)
    qy = math.acos(0.5 * np.trace(M[2:4, 2:4])) / (2 * math.pi)
    assert min(qx, 1 - qx) == pytest.approx(min(d["qx"] % 1, 1 - d["qx"] % 1), abs=1e-8)
    assert min(qy, 1 - qy) == pytest.approx(min(d["qy"] % 1, 1 - d["qy"] % 1), abs=1e-8)
    # fractional tunes as matched; the phase accumulated along the ring gives the integer part
    assert d["qx"] == pytest.approx(0.31, abs=1e-9) and d["qy"] == pytest.approx(0.32, abs=1e-9)
    assert int(d["mux"][-1] // (2 * math.pi)) == 49 and int(d["muy"][-1] // (2 * math.pi)) == 49


def test_matched_beam_emittance_and_spread():
    """FODO-10, 20,000 protons at eps_n = 2.5 um, sigma_delta = 3e-4: the rms
    emittances (dispersion-free ring) and the momentum spread match within
    the statistical error of the sample."""
    el, ref = I.fodo10()
    n = 20000
    p = I.matched_gaussian(el, ref, n, 2.5e-6, 3e-4, seed=I.BASE_SEED)
    eps = 2.5e-6 / (ref[2] / ref[0])
    tol = 4 * math.sqrt(2.0 / n)
    for u, pu in (("x", "px"), ("y", "py")):
        a, b = p[u] - p[u].mean(), p[pu] - p[pu].mean()
        e = math.sqrt(np.mean(a * a) * np.mean(b * b) - np.mean(a * b) ** 2)
        assert e == pytest.approx(eps, rel=tol)
    assert np.std(p["delta"]) == pytest.approx(3e-4, rel=tol)
    assert np.all(p["state"] == 1) and np.array_equal(p["particle_id"], np.arange(n))


def test_da_grid_layout(lhc):
    """999,990 particles: 22,222 radii uniform in (0, 20] sigma, ray-major
    (neighbouring radii adjacent), 9 angles 90 (j+1)/10 deg, 5 momentum
    offsets; the normalised amplitude recovered from x, y is the grid radius."""
    el, ref, d = lhc
    g = I.da_grid(el, ref, optics=d)
    R, T, D = g["grid"]
    assert g["x"].shape[0] == 999990
    assert np.array_equal(R[:22222], 20.0 * (np.arange(22222) + 1) / 22222)
    assert np.all(T[:22222] == 0) and np.all(T[22222:44444] == 1) and np.all(D[:9 * 22222] == 0)
    eps = 2.5e-6 / (ref[2] / ref[0])
    delta = (np.arange(5) - 2)[D] * 3e-4
    xn = (g["x"] - d["dx"][0] * delta) / math.sqrt(eps * d["betx"][0])
    yn = g["y"] / math.sqrt(eps * d["bety"][0])
    assert np.allclose(np.hypot(xn, yn), R, rtol=1e-12)
    th = np.degrees(np.arctan2(yn, xn))
    assert np.allclose(th, 90.0 * (T + 1) / 10, atol=1e-9)
    assert np.allclose(g["delta"], delta, rtol=0, atol=1e-18)


def test_batched_seed_counts():
    """64 counts round(10^U(3, 5)): within [1e3, 1e5], log-uniform (median of
    log10 near 4), fixed by the base seed."""
    c = I.batched_seed_counts(64)
    assert c.shape == (64,) and c.min() >= 1000 and c.max() <= 100000
    assert int(c.sum()) == 1737245
    assert abs(np.median(np.log10(c)) - 4.0) < 0.35


def test_lepton_ring_recipe():
    """45.6 GeV electrons, 200 cells of 50 rows (10,000), 16 dipole slices
    per cell of theta = 2 pi/3200 and L_rad = 10.7/4 m (rho = 1.36 km), one
    400 MHz cavity per cell adding to 500 MV at 180 deg - arcsin(U0/V), and
    U0 = C_gamma E0^4 / rho (isomagnetic) of about 0.6 % of E0 per turn."""
    el, ref, info = I.lepton_ring()
    t = el["type"]
    assert el.shape[0] == 10000
    rc = oracle.ref_constants(ref)
    assert rc["E0"] == pytest.approx(45.6e9, rel=1e-15)
    mp = el[t == I.MULTIPOLE]
    dip = mp[mp["p"][:, 0] != 0]
    assert dip.shape[0] == 16 * 200
    theta = 2 * math.pi / 3200
    assert np.allclose(dip["p"][:, 0], theta, rtol=1e-15) and np.allclose(dip["p"][:, 22], theta, rtol=1e-15)
    rho = (10.7 / 4) / theta
    assert rho == pytest.approx(1362.5, rel=1e-3)
    cav = el[t == I.CAVITY]
    assert cav.shape[0] == 200 and np.sum(cav["p"][:, 0]) == pytest.approx(500e6, rel=1e-12)
    assert np.all(cav["p"][:, 1] == 400e6)
    U0 = 8.846e-5 * (45.6 ** 4) / rho * 1e9
    assert info["U0"] == pytest.approx(U0, rel=1e-12)
    assert np.all(cav["p"][:, 2] == pytest.approx(180.0 - math.degrees(math.asin(U0 / 500e6)), rel=1e-12))
    assert 0.004 < U0 / 45.6e9 < 0.008
