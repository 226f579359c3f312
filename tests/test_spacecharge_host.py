"""The space-charge installer's host formula (CPU): the summed first-order
tune shift of lumped lenses against the textbook incoherent (Laslett) tune
shift of a round coasting beam, Delta Q = N r_c / (4 pi beta0^2 gamma0^3 eps),
which does not depend on the number of lenses or on beta."""
import math

import numpy as np
import pytest

from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import spacecharge as SC


@pytest.mark.parametrize("n_lenses", [1, 7, 64])
def test_laslett_round_coasting_beam(n_lenses):
    ref = I.proton_reference(2e9)
    m0, _, p0c = ref
    E0 = math.hypot(p0c, m0)
    b0, g0 = p0c / E0, E0 / m0
    N, C, eps = 1e11, 40.0, 2e-6 / (b0 * g0)
    beta = np.linspace(8.0, 12.0, n_lenses)   # any beta: sigma^2 = eps beta cancels it
    sig = np.sqrt(eps * beta)
    inst = dict(line_density=N / C, length=C / n_lenses, betx=beta, bety=beta, sigma_x=sig, sigma_y=sig)
    dqx, dqy = SC.laslett_tune_shift(inst, ref)
    r_p = 2.8179403262e-15 * 0.51099895000e6 / m0
    expect = N * r_p / (4 * math.pi * b0 ** 2 * g0 ** 3 * eps)
    assert dqx == pytest.approx(expect, rel=1e-12)
    assert dqy == pytest.approx(expect, rel=1e-12)


def test_flat_beam_splits_the_shift():
    """For sigma_x != sigma_y the x and y shifts are in the ratio
    beta_x/(sigma_x) : beta_y/(sigma_y) over (sigma_x + sigma_y)."""
    ref = I.proton_reference(2e9)
    inst = dict(line_density=1e9, length=1.0, betx=np.array([10.0]), bety=np.array([5.0]),
                sigma_x=np.array([2e-3]), sigma_y=np.array([1e-3]))
    dqx, dqy = SC.laslett_tune_shift(inst, ref)
    assert dqx / dqy == pytest.approx((10.0 / 2e-3) / (5.0 / 1e-3), rel=1e-14)
