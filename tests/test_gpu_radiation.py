"""Lepton ring with radiation on the GPU against the synchrotron integrals.

Equilibrium: with mean radiation plus quantum excitation, a beam started at
the predicted equilibrium stays there: the tracked horizontal betatron
emittance and the momentum spread match eps_x = C_q gamma^2 I5 / (J_x I2) and
sigma_delta^2 = C_q gamma^2 I3 / (J_z I2) (I2, I3, I5, J from the oracle's
optics of the same lattice), each within 1 %.  Damping: with the mean model
only, the emittance decays as exp(-2 t / tau_x) with tau_x from the oracle's
one-turn eigenvalues, within 1 %.  The runs are seeded (counter-based
Philox draws) and reproducible bit for bit."""
import math

import numpy as np
import pytest

from oracle import optics as O
from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import xtgb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ring():
    el, ref, info = I.lepton_ring()
    eq = O.equilibrium(el, ref)
    return el, ref, eq


def moments(P, tw):
    import torch
    x, px, d = P.t["x"], P.t["px"], P.t["delta"]
    alive = P.t["state"] == 1
    x, px, d = x[alive], px[alive], d[alive]
    xb = x - tw["dx"][0] * d
    pb = px - tw["dpx"][0] * d
    xb = xb - xb.mean()
    pb = pb - pb.mean()
    eps = torch.sqrt((xb * xb).mean() * (pb * pb).mean() - (xb * pb).mean() ** 2)
    return float(eps), float(d.std()), int(alive.sum())


def test_quantum_equilibrium_emittance(ring):
    el, ref, eq = ring
    n = 20000
    p = I.matched_gaussian(el, ref, n, 0.0, eq["sigma_delta"], seed=41, emit_x=eq["eps_x"],
                           emit_y=0.01 * eq["eps_x"])
    tr = xtgb.Tracker(el, ref, radiation=xtgb.RAD_QUANTUM, seed=2024)
    P = xtgb.Particles.from_numpy(p)
    eps, sd = [], []
    turn = 0
    for seg in range(12):
        tr.track(P, 50, turn)
        turn += 50
        if turn >= 200:
            e, s, alive = moments(P, eq["twiss"])
            eps.append(e)
            sd.append(s)
    assert tr.sync_status() == xtgb.XT_OK
    assert alive == n
    e_m, s_m = float(np.mean(eps)), float(np.mean(sd))
    print("eps_x tracked %.5g predicted %.5g (%.2f%%); sigma_delta tracked %.5g predicted %.5g (%.2f%%)"
          % (e_m, eq["eps_x"], 100 * (e_m / eq["eps_x"] - 1), s_m, eq["sigma_delta"],
             100 * (s_m / eq["sigma_delta"] - 1)))
    assert e_m == pytest.approx(eq["eps_x"], rel=0.01)
    assert s_m == pytest.approx(eq["sigma_delta"], rel=0.01)


def test_mean_radiation_damping_time(ring):
    el, ref, eq = ring
    n = 4000
    p = I.matched_gaussian(el, ref, n, 0.0, 1e-4, seed=43, emit_x=4 * eq["eps_x"], emit_y=4 * eq["eps_x"])
    tr = xtgb.Tracker(el, ref, radiation=xtgb.RAD_MEAN)
    P = xtgb.Particles.from_numpy(p)
    turns, ln_eps = [], []
    turn = 0
    for seg in range(12):
        tr.track(P, 25, turn)
        turn += 25
        e, _, alive = moments(P, eq["twiss"])
        turns.append(turn)
        ln_eps.append(math.log(e))
    assert alive == n
    slope = np.polyfit(turns, ln_eps, 1)[0]
    tau_x = 1.0 / eq["alpha"][0]
    print("tau_x fitted %.2f turns, from eigenvalues %.2f" % (-2.0 / slope, tau_x))
    assert -2.0 / slope == pytest.approx(tau_x, rel=0.01)
