"""Host logic of the surrogate-guided DA scan on CPU: the network's inputs
describe the very points the tracker is given, in the grid's ray-major
order, and the pass count of a scan follows the throughput metric's rule."""
import math

import numpy as np

from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import surrogate as S
from paper_2310_00317_gb300 import xtgb


def _grid():
    el, ref, desc = S.seed_ring(7, n_cells=20)
    n_r, n_theta, deltas = 7, 3, (-1, 0, 2)
    grid, (R, th, dl), n_rays = S.scan_grid(el, ref, n_r, n_theta, deltas)
    return el, ref, desc, grid, R, th, dl, n_rays, n_r, n_theta, deltas


def test_features_are_the_tracked_points_in_normalised_coordinates():
    el, ref, desc, grid, R, th, dl, n_rays, n_r, n_theta, deltas = _grid()
    X = S.features(R, th, dl, desc)
    assert X.shape == (n_rays * n_r, 16) and X.dtype == np.float32
    # undo the placement on the dispersive orbit and the beam size at element 0
    opt = I.design_optics(el, ref)
    m0, _, p0c = ref
    eps = 2.5e-6 / (p0c / m0)
    xn = (grid["x"] - opt["dx"][0] * grid["delta"]) / math.sqrt(eps * opt["betx"][0])
    yn = grid["y"] / math.sqrt(eps * opt["bety"][0])
    np.testing.assert_allclose(X[:, 0] * S.R_MAX, xn, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(X[:, 2] * S.R_MAX, yn, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(X[:, 5] * 3 * S.SIGMA_DELTA, grid["delta"], rtol=1e-6, atol=1e-12)
    # normalised momenta and zeta are zero on the grid
    assert not X[:, [1, 3, 4]].any()
    # the descriptors, the same on every point, in units of log 2
    np.testing.assert_allclose(X[:, 6:], np.tile(np.asarray(desc) / math.log(2.0), (X.shape[0], 1)), rtol=1e-6)


def test_scan_grid_is_ray_major_with_radii_increasing_along_a_ray():
    el, ref, desc, grid, R, th, dl, n_rays, n_r, n_theta, deltas = _grid()
    assert n_rays == n_theta * len(deltas)
    Rr = R.reshape(n_rays, n_r)
    thr = th.reshape(n_rays, n_r)
    dlr = dl.reshape(n_rays, n_r)
    # every ray: one angle, one momentum offset, radii (0, 20] sigma increasing
    assert np.all(np.diff(Rr, axis=1) > 0)
    np.testing.assert_allclose(Rr[:, -1], S.R_MAX)
    np.testing.assert_allclose(Rr[:, 0], S.R_MAX / n_r)
    assert np.all(thr == thr[:, :1]) and np.all(dlr == dlr[:, :1])
    # rays are (delta, angle) pairs, angles fastest, each pair once
    angles = np.radians(90.0 * (np.arange(n_theta) + 1) / (n_theta + 1))
    np.testing.assert_allclose(thr[:, 0], np.tile(angles, len(deltas)))
    np.testing.assert_allclose(dlr[:, 0], np.repeat(np.asarray(deltas) * S.SIGMA_DELTA, n_theta))


def test_scan_pass_count_follows_the_metric_rule():
    # 6 points: two survive, three are lost at (turn, element), one was not tracked
    n_turns, n_el = 5, 20
    before = np.array([1, 1, 1, 1, 1, 0], dtype=np.int32)
    out = {"state": np.array([1, 1, 0, -1, 0, 0], dtype=np.int32),
           "at_turn": np.array([5, 5, 0, 3, 4, 0], dtype=np.int32),
           "at_element": np.array([0, 0, 7, 0, 19, 0], dtype=np.int32)}
    # survivors: n_turns * n_el each; a particle lost at (t, e): t * n_el + e + 1
    expect = 2 * n_turns * n_el + (0 * n_el + 7 + 1) + (3 * n_el + 0 + 1) + (4 * n_el + 19 + 1)
    assert S._alive_passes(before, out, n_turns, n_el) == expect
    p = dict(out)
    assert xtgb.traversed_elements(p, n_el, 0, n_turns, before) == expect
