"""Host logic of the lattice functions (no GPU): the normal modes of a
one-turn matrix and their normalisation."""
import math

import numpy as np
import pytest

from paper_2310_00317_gb300 import twiss as T


def cs_block(beta, alpha, mu):
    g = (1 + alpha * alpha) / beta
    c, s = math.cos(mu), math.sin(mu)
    return np.array([[c + alpha * s, beta * s], [-g * s, c - alpha * s]])


@pytest.mark.parametrize("n", [4, 6])
def test_uncoupled_modes_give_courant_snyder_parameters(n):
    """Block-diagonal one-turn matrices: 2 |v_x|^2 = beta and
    -2 Re(conj(v_x) v_px) = alpha in each plane, v^H S v = i."""
    pars = [(12.3, -1.7, 2 * math.pi * 0.31), (4.1, 0.6, 2 * math.pi * 0.27), (900.0, 0.0, 2 * math.pi * 0.004)]
    M = np.zeros((n, n))
    for k in range(n // 2):
        M[2 * k:2 * k + 2, 2 * k:2 * k + 2] = cs_block(*pars[k])
    V = T.normal_modes(M)
    S = T._symplectic_form(n)
    for k in range(n // 2):
        v = V[:, k]
        assert abs(np.vdot(v, S @ v) - 1j) < 1e-12
        b, a, _ = pars[k]
        assert abs(2 * abs(v[2 * k]) ** 2 - b) < 1e-12 * b
        assert abs(-2 * np.real(np.conj(v[2 * k]) * v[2 * k + 1]) - a) < 1e-12
        # the other planes carry nothing
        assert all(abs(v[2 * j]) < 1e-12 for j in range(n // 2) if j != k)


def test_coupled_modes_are_normalised_and_propagate_with_the_map():
    """A symplectic coupling rotation R applied to an uncoupled matrix:
    the modes of R M R^-1 are R times those of M (up to a phase), each with
    v^H S v = i."""
    M = np.zeros((4, 4))
    M[:2, :2] = cs_block(10.0, 0.5, 2 * math.pi * 0.31)
    M[2:, 2:] = cs_block(6.0, -0.3, 2 * math.pi * 0.18)
    th = 0.2
    c, s = math.cos(th), math.sin(th)
    R = np.array([[c, 0, s, 0], [0, c, 0, s], [-s, 0, c, 0], [0, -s, 0, c]])
    Mc = R @ M @ np.linalg.inv(R)
    V0, V = T.normal_modes(M), T.normal_modes(Mc)
    S = T._symplectic_form(4)
    for k in range(2):
        assert abs(np.vdot(V[:, k], S @ V[:, k]) - 1j) < 1e-12
        w = R @ V0[:, k]
        ph = np.vdot(w, V[:, k]) / np.vdot(w, w)
        assert abs(abs(ph) - 1) < 1e-12 and np.max(np.abs(V[:, k] - ph * w)) < 1e-12
    assert 2 * abs(V[0, 1]) ** 2 > 0.1  # mode II has an x part: coupling


def test_unstable_matrix_is_rejected():
    M = np.eye(4)
    M[:2, :2] = [[2.0, 1.0], [1.0, 1.0]]  # hyperbolic
    M[2:, 2:] = cs_block(6.0, 0.0, 1.0)
    with pytest.raises(RuntimeError):
        T.normal_modes(M)


def test_scale_magnets_scales_fields_not_geometry():
    """Tapering scales field strengths only: thin multipole knl and ksl,
    quadrupole k1, bend k0 and k1, edge h; never the frame curvature hxl,
    L_rad, the bend's h and length, nor other rows."""
    from paper_2310_00317_gb300 import inputs as I
    rows = [I.multipole(knl=[0.01, 0.2, 0.3], ksl=[0.0, 0.05], hxl=0.01, lrad=2.0), I.quadrupole(0.1, 0.5),
            I.bend(0.02, 0.02, 1.0, k1=-0.1), I.dipedge(0.02, 0.1, hgap=0.03, fint=0.5), I.drift(1.0),
            I.cavity(1e6, 4e8, 180.0)]
    el = I.table(rows)
    f = np.array([1.01, 1.02, 1.03, 1.04, 1.05, 1.06])
    sc = T.scale_magnets(el, f)
    assert np.array_equal(sc[0]["p"][:22], el[0]["p"][:22] * 1.01)
    assert sc[0]["p"][22] == el[0]["p"][22] and sc[0]["p"][23] == el[0]["p"][23]
    assert sc[1]["p"][0] == el[1]["p"][0] * 1.02 and sc[1]["p"][1] == el[1]["p"][1]
    assert sc[2]["p"][0] == el[2]["p"][0] * 1.03 and sc[2]["p"][3] == el[2]["p"][3] * 1.03
    assert sc[2]["p"][1] == el[2]["p"][1] and sc[2]["p"][2] == el[2]["p"][2]
    assert sc[3]["p"][0] == el[3]["p"][0] * 1.04 and np.array_equal(sc[3]["p"][1:], el[3]["p"][1:])
    assert np.array_equal(sc[4]["p"], el[4]["p"]) and np.array_equal(sc[5]["p"], el[5]["p"])
    assert np.array_equal(el[1]["p"][:2], [0.1, 0.5])  # the input table is not modified


def test_row_lengths():
    from paper_2310_00317_gb300 import inputs as I
    el = I.table([I.drift(1.5), I.quadrupole(0.1, 0.4), I.bend(0.01, 0.01, 2.5), I.multipole(knl=[0, 0.1]),
                  I.aperture(0.02), I.spacecharge(1e10, 0.0, 1e-3, 1e-3, 3.0)])
    assert np.array_equal(T.row_lengths(el), [1.5, 0.4, 2.5, 0.0, 0.0, 0.0])


def test_functions_along_from_exact_jacobians():
    """The host half of the lattice functions along the line (normal modes of
    the one-turn matrix carried through per-row Jacobians, Mais-Ripken
    readout, dispersion M_i (D_0, 1)) fed with the oracle's exact per-row
    Jacobians of the 20-cell lepton ring instead of the GPU stencil: beta,
    alpha and dispersion equal the oracle's Courant-Snyder propagation at
    every row, the phase advance over the ring equals the tune modulo 1, and
    the cross-plane betas vanish (uncoupled ring)."""
    import oracle
    from oracle import optics as O
    from paper_2310_00317_gb300 import inputs as I
    el, ref, _ = I.lepton_ring(n_cells=20, E0=10e9, v_total=100e6)
    elx = O.without_cavities(el)
    tw = O.twiss_uncoupled(elx, ref)
    z = oracle.closed_orbit(elx, ref, rad_mode=0, dim=4)
    _, M, orbit, Ms = oracle.track_jacobian(elx, ref, z, along=True)
    Vm = T.normal_modes(M[:4, :4])
    D0 = np.linalg.solve(np.eye(4) - M[:4, :4], M[:4, 5])
    f = T._functions_along(elx, z, orbit, Ms, Vm, D0)
    for k in ("betx", "alfx", "bety", "alfy", "dx", "dpx"):
        assert np.allclose(f[k], tw[k], rtol=1e-9, atol=1e-9 * np.max(np.abs(tw[k]))), k
    qx = math.acos(0.5 * np.trace(M[:2, :2])) / (2 * math.pi)
    qy = math.acos(0.5 * np.trace(M[2:4, 2:4])) / (2 * math.pi)
    assert f["mux"][-1] % 1.0 == pytest.approx(qx, abs=1e-10)
    assert f["muy"][-1] % 1.0 == pytest.approx(qy, abs=1e-10)
    assert np.all(np.diff(f["mux"]) >= -1e-12) and np.all(np.diff(f["muy"]) >= -1e-12)
    assert np.max(f["betx2"]) < 1e-20 and np.max(f["bety1"]) < 1e-20
    assert f["s"][-1] == pytest.approx(float(np.sum(elx[elx["type"] == I.DRIFT]["p"][:, 0])), rel=1e-12)
