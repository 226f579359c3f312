"""Pins of the oracle's chaos marker (twin-particle finite-time Lyapunov
estimate, Benettin, Galgani and Strelcyn, Phys. Rev. A 14, 2338 (1976)).

The marker separates regular orbits, whose neighbours drift apart at most
linearly in the turn count, from chaotic ones.  It is pinned by the closed
forms of linear maps (a hyperbolic map stretches along its unstable
eigenvector by exactly its eigenvalue; a rotation keeps the normalised
distance), by the growth of the tangent vector computed from the oracle's
exact one-turn Jacobians (dual numbers, pinned elsewhere by the matrices and
symplecticity), and by the loss bookkeeping of a twin that leaves the
aperture alone (CPU only).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_00317_gb300 import inputs as I

PROTON = I.proton_reference(450e9)


def _rot(mux, muy=0.0, bx=1.0, by=1.0):
    M = np.eye(6)
    c, s = math.cos(mux), math.sin(mux)
    M[0:2, 0:2] = [[c, bx * s], [-s / bx, c]]
    c, s = math.cos(muy), math.sin(muy)
    M[2:4, 2:4] = [[c, by * s], [-s / by, c]]
    return M


def _henon(k2=2.0, q=0.2114):
    return I.table([I.multipole(knl=[0, 0, k2]), I.linear_map(_rot(2 * math.pi * q))])


def test_hyperbolic_map_exponent_is_the_log_of_its_eigenvalue():
    """M = [[cosh m, sinh m], [sinh m, cosh m]] in x: along the eigenvector
    (1, 1) every turn multiplies the separation by e^m, so the estimate is m
    (numpy's eigenvalues give the largest |lambda| = e^m independently).
    From (1, 0), whose unstable component has length 1/sqrt(2), the sum of
    logarithms after N turns is m N - ln sqrt(2) up to e^(-2 m N)."""
    m = 0.1
    M = np.eye(6)
    M[0:2, 0:2] = [[math.cosh(m), math.sinh(m)], [math.sinh(m), math.cosh(m)]]
    lam_max = math.log(np.max(np.abs(np.linalg.eigvals(M))))
    el = I.table([I.linear_map(M)])
    d0 = 1e-8
    r = oracle.lyapunov(el, PROTON, np.zeros((1, 6)), np.array([1, 1, 0, 0, 0, 0]) * d0 / math.sqrt(2),
                        1000, every=10)
    assert r["turns"][0] == 1000 and r["lost"][0] == 0
    assert r["lam"][0] == pytest.approx(lam_max, rel=1e-12)
    assert r["chaotic"][0]
    for every in (1, 7, 10):   # 1000 = 142 * 7 + 6: the last, shorter interval counts too
        r = oracle.lyapunov(el, PROTON, np.zeros((1, 6)), np.array([d0, 0, 0, 0, 0, 0]), 1000, every=every)
        assert r["sum_log"][0] == pytest.approx(m * 1000 - math.log(math.sqrt(2.0)), abs=1e-9)
    # no renormalisation before the end: one logarithm of the whole growth
    # (kept short, so that the twin stays inside the 1 m guard)
    r = oracle.lyapunov(el, PROTON, np.zeros((1, 6)), np.array([d0, 0, 0, 0, 0, 0]), 99, every=1000)
    assert r["sum_log"][0] == pytest.approx(m * 99 - math.log(math.sqrt(2.0)), abs=1e-9)


def test_rotation_keeps_the_normalised_distance():
    """A linear ring (rotations with beta_x = 12, beta_y = 3 at the start):
    in the metric diag(1/sqrt(beta), sqrt(beta)) per plane the one-turn map is
    a rotation, so every renormalisation ratio is 1 and the sum stays 0."""
    bx, by = 12.0, 3.0
    el = I.table([I.linear_map(_rot(2 * math.pi * 0.31, 2 * math.pi * 0.27, bx, by))])
    A = np.diag([1 / math.sqrt(bx), math.sqrt(bx), 1 / math.sqrt(by), math.sqrt(by), 1.0, 1.0])
    z = np.array([[1e-3, 2e-5, -5e-4, 1e-5, 0.0, 0.0]])
    r = oracle.lyapunov(el, PROTON, z, np.array([1e-8, 2e-9, -3e-9, 1e-9, 1e-8, 0.0]), 1000, every=10, metric=A)
    assert abs(r["sum_log"][0]) < 1e-11
    assert not r["chaotic"][0]
    # in the plain Euclidean metric the distance only oscillates: bounded logarithms
    r = oracle.lyapunov(el, PROTON, z, np.array([1e-8, 0, 0, 0, 0, 0]), 1000, every=1)
    assert abs(r["sum_log"][0]) < math.log(2 * bx) and not r["chaotic"][0]


@pytest.mark.parametrize("X0", [0.3, 0.585, 0.635, 0.65])
@pytest.mark.parametrize("every", [1, 10])
def test_twin_growth_equals_the_tangent_map_growth(X0, every):
    """On the Henon map (thin sextupole + rotation), the twin started 1e-10
    away follows the linearised motion: its summed logarithms equal
    ln |J_N e_x| of the exact N-turn Jacobian to 1e-2 (the finite-offset and
    rounding error), for regular (X0 = 0.3) and chaotic orbits alike, where
    ln |J_N e_x| reaches 45 after 3000 turns."""
    el = _henon()
    z = np.zeros(6)
    z[0] = X0
    for N in (200, 3000):
        _, J = oracle.track_jacobian(el, PROTON, z, N)
        ref_log = math.log(np.linalg.norm(J[:, 0]))
        r = oracle.lyapunov(el, PROTON, z[None], np.array([1e-10, 0, 0, 0, 0, 0]), N, every=every)
        assert r["lost"][0] == 0 and r["turns"][0] == N
        assert r["sum_log"][0] == pytest.approx(ref_log, abs=1e-2)


def test_henon_orbits_small_amplitudes_regular_edge_chaotic():
    """Over 1e4 turns the small-amplitude Henon orbits stay below the linear
    growth bound, while orbits in the layer just inside the escape boundary
    (X0 = 0.635, 0.65) separate exponentially."""
    el = _henon()
    X0 = np.array([0.05, 0.1, 0.2, 0.3, 0.635, 0.65])
    z = np.zeros((X0.size, 6))
    z[:, 0] = X0
    r = oracle.lyapunov(el, PROTON, z, np.array([1e-9, 0, 0, 0, 0, 0]), 10000, every=10)
    assert np.all(r["lost"] == 0)
    assert not np.any(r["chaotic"][:4])
    assert np.all(r["chaotic"][4:])
    assert np.all(r["lam"][4:] > 10 * r["lam"][:4].max())


def test_twin_lost_alone_marks_the_orbit():
    """A particle just inside a 1 mm aperture survives; a twin displaced
    2e-12 m outwards is lost at turn 0: lost = 1 and chaotic.  Both outside:
    lost together, lost = 2, and the marker leaves the decision to the
    separation."""
    el = I.table([I.drift(1.0), I.aperture(1e-3)])
    z = np.array([[1e-3 - 1e-12, 0, 0, 0, 0, 0], [2e-3, 0, 0, 0, 0, 0]])
    r = oracle.lyapunov(el, PROTON, z, np.array([2e-12, 0, 0, 0, 0, 0]), 10)
    assert list(r["lost"]) == [1, 2]
    assert list(r["turns"]) == [0, 0]
    assert r["chaotic"][0] and not r["chaotic"][1]


def test_rejects_bad_arguments():
    el = _henon()
    z = np.zeros((1, 6))
    with pytest.raises(ValueError):
        oracle.lyapunov(el, PROTON, z, np.zeros(6), 10)
    with pytest.raises(ValueError):
        oracle.lyapunov(el, PROTON, z, np.array([1e-9, 0, 0, 0, 0, 0]), 10, every=0)
    with pytest.raises(ValueError):
        oracle.lyapunov(el, PROTON, z, np.array([1e-9, 0, 0, 0, 0, 0]), 10, rad_mode=2)


def test_parallel_helpers_equal_the_single_process_calls():
    """The spawned-process helpers split the particles into slices; the
    particles are independent, so the results are the same bit for bit."""
    el = _henon()
    X0 = np.linspace(0.05, 0.66, 7)
    z = np.zeros((X0.size, 6))
    z[:, 0] = X0
    dz = np.array([1e-9, 0, 0, 0, 0, 0])
    a = oracle.lyapunov(el, PROTON, z, dz, 300)
    b = oracle.lyapunov_parallel(el, PROTON, z, dz, 300, procs=3)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    p = I.make_particles(PROTON, X0, np.zeros(7), np.zeros(7), np.zeros(7), np.zeros(7), np.zeros(7))
    ta, tb = oracle.track(el, PROTON, p, 300), oracle.track_parallel(el, PROTON, p, 300, procs=3)
    for k in ta:
        assert np.array_equal(ta[k], tb[k]), k
    assert oracle.lyapunov_parallel(el, PROTON, np.zeros((0, 6)), dz, 10)["sum_log"].shape == (0,)
