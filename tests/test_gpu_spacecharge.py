"""Frozen space charge on the GPU (section "Space charge", frozen model):
lenses installed from the lattice functions computed on the GPU shift the
small-amplitude tunes by the first-order (Laslett) amount."""
import math

import numpy as np
import pytest

from paper_2310_00317_gb300 import inputs as I
from paper_2310_00317_gb300 import spacecharge as SC
from paper_2310_00317_gb300 import twiss as T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sigma_z", [0.0, 0.5])
def test_installed_lenses_shift_the_tunes_by_the_laslett_amount(sigma_z):
    """FODO-10 at 2 GeV/c (protons), emittances 2 and 1 um (flat beam), 40
    lenses, peak line densities of 7.5e10 and 3.75e10 per metre (coasting, or
    bunched with sigma_z = 0.5 m): the tunes of the ring with the lenses
    (one-turn matrix of the small-amplitude stencil, which sits at the bunch
    centre) are below the bare tunes by the summed first-order shifts (about
    0.02 and 0.01), and the remainder is second order: it halves with the
    line density and stays under 1.5 % at the lower one."""
    el, _ = I.fodo10()
    ref = I.proton_reference(2e9)
    bare = T.twiss(el, ref)
    dev = []
    for lam in (7.5e10, 3.75e10):
        n = lam * (math.sqrt(2 * math.pi) * sigma_z if sigma_z > 0 else 40.0)
        inst = SC.install_space_charge(el, ref, 40, n, 2e-6, 1e-6, sigma_z=sigma_z)
        assert np.sum(inst["table"]["type"] == I.SPACECHARGE) == 40
        with_sc = T.twiss(inst["table"], ref)
        dqx, dqy = SC.laslett_tune_shift(inst, ref)
        shift_x = (bare["qx"] - with_sc["qx"] + 0.5) % 1.0 - 0.5
        shift_y = (bare["qy"] - with_sc["qy"] + 0.5) % 1.0 - 0.5
        print("line density %.3g: tune shifts tracked %.5f %.5f, first order %.5f %.5f"
              % (lam, shift_x, shift_y, dqx, dqy))
        dev.append(np.array([shift_x / dqx - 1, shift_y / dqy - 1]))
    assert np.all(np.abs(dev[1]) < 0.015)
    assert np.all(np.abs(dev[0] / dev[1] - 2.0) < 0.2)
