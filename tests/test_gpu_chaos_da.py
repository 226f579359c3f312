"""GPU tracker against the oracle at the dynamic-aperture boundary, with the
oracle's chaos marker, and the DA per ray of the plain GPU scan against the
oracle's.

Ring: error seed 60 of the reduced LHC-scale ring (2,000 elements, multipole
errors to order 10, RF, circular apertures); the on-momentum DA grid of 9
angles x 40 radii up to 20 sigma; 1000 turns.  The FP64 criterion: the
coordinates of regular orbits agree to 1e-12 relative, the loss turns agree
for at least 99.9 % of the particles, and every disagreement is on an orbit
the oracle's twin-particle Lyapunov estimate marks chaotic.  (The two sides
use the same operation order, so the differences are in fact zero; the test
states the weaker criterion, which the marker decides.)  The DA of a ray is
the number of radii before its first loss (section "Particle-matter
interaction and collimation studies": apertures stop the tracking)."""
import math

import numpy as np
import pytest

import oracle
from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import surrogate as S
from paper_2310_00317_gb300 import xtgb

pytestmark = pytest.mark.gpu

N_R, N_THETA, TURNS = 40, 9, 1000


@pytest.fixture(scope="module")
def case():
    el, ref, _ = S.seed_ring(60)
    grid, _, n_rays = S.scan_grid(el, ref, N_R, N_THETA)
    o = oracle.track_parallel(el, ref, grid, TURNS)
    lost_o = (o["state"] != 1).reshape(n_rays, N_R)
    da_o = np.where(lost_o.any(1), lost_o.argmax(1), N_R)

    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    tr = xtgb.Tracker(el, ref)
    P = xtgb.Particles.from_numpy(grid)
    tr.track(P, TURNS)
    assert tr.sync_status() == xtgb.XT_OK
    g = P.to_numpy()
    da_g, _, _ = S.plain_scan(tr, grid, n_rays, N_R, TURNS)
    tr.close()

    # chaos marker: every survivor, the lost particles within 3 radii of
    # their ray's DA, and every particle the two sides disagree on
    opt = I.design_optics(el, ref)
    bx, by = opt["betx"][0], opt["bety"][0]
    A = np.diag([1 / math.sqrt(bx), math.sqrt(bx), 1 / math.sqrt(by), math.sqrt(by), 1.0, 1e3])
    same = (g["state"] == o["state"]) & (g["at_turn"] == o["at_turn"]) & (g["at_element"] == o["at_element"])
    k = np.tile(np.arange(N_R), n_rays)
    near = np.abs(k - np.repeat(da_o, N_R)) <= 3
    pick = np.flatnonzero((o["state"] == 1) | (g["state"] == 1) | near | ~same)
    z = oracle.canonical(I.subset(grid, pick), ref)
    m = oracle.lyapunov_parallel(el, ref, z, np.array([1e-8 * math.sqrt(bx), 0, 0, 0, 0, 0]), TURNS,
                                 every=10, metric=A)
    chaotic = np.zeros(grid["x"].shape[0], bool)
    marked = np.zeros_like(chaotic)
    chaotic[pick] = m["chaotic"]
    marked[pick] = True
    return dict(g=g, o=o, same=same, chaotic=chaotic, marked=marked, da_o=da_o, da_g=da_g, A=A, ref=ref)


def test_loss_turns_agree_and_differences_are_chaotic(case):
    same, chaotic, marked = case["same"], case["chaotic"], case["marked"]
    assert same.mean() >= 0.999, "loss turns agree for %.4f of the particles" % same.mean()
    assert np.all(marked[~same]) and np.all(chaotic[~same])
    # the boundary layer holds chaotic orbits: the marker is not vacuous here
    assert chaotic.sum() >= 5
    assert (case["o"]["state"] != 1).sum() > 50 and (case["o"]["state"] == 1).sum() > 50


def test_regular_survivors_agree_to_1e12(case):
    g, o, A, ref = case["g"], case["o"], case["A"], case["ref"]
    surv = (g["state"] == 1) & (o["state"] == 1) & ~case["chaotic"]
    assert surv.sum() > 100
    zg = oracle.canonical({k: g[k][surv] for k in g}, ref) @ A.T
    zo = oracle.canonical({k: o[k][surv] for k in o}, ref) @ A.T
    err = np.linalg.norm(zg - zo, axis=1) / np.linalg.norm(zo, axis=1)
    assert err.max() <= 1e-12


def test_plain_scan_da_per_ray_equals_the_oracle(case):
    assert case["da_g"].shape == case["da_o"].shape
    assert np.array_equal(case["da_g"], case["da_o"])
    assert np.all(case["da_o"] > 5) and np.all(case["da_o"] < N_R)
