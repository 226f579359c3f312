"""Surrogate-guided dynamic-aperture scan end to end on the GPU.

The scan (band selection, FP64 tracking of the band, per-ray DA, widening
passes) trusts the network wherever it is confident that a point survives.
So the guarantee is: if every point the network confidently calls a survivor
does survive (an accurate or a conservative network), the scan returns
exactly the DA of the plain scan, which tracks every grid point; losses
predicted too early are found by widening.  The network is replaced by a
stand-in whose predicted boundary is the true one moved by a chosen number
of grid steps per ray: 0 and +-2 steps (the first band holds the boundary)
and -40 steps (the first band lies well inside the stable region and the scan
must widen outwards).  A boundary predicted too far out is not covered: the
scan then reports the first loss it finds near the prediction.  Ring: a
reduced LHC-scale error seed (2,000 elements), 9 angles x 400 radii up to 20
sigma, 300 turns."""
import numpy as np
import pytest

from paper_2310_00317_gb300 import surrogate as S
from paper_2310_00317_gb300 import xtgb

pytestmark = pytest.mark.gpu


class ShiftedBoundary:
    """forward(X) -> (n, 2): survival logit that changes sign at the given
    per-ray edge (grid index), and a zero loss-turn output."""

    def __init__(self, edge, n_r):
        self.edge = np.asarray(edge, np.float64)
        self.n_r = n_r

    def forward(self, X):
        import torch
        n = X.shape[0]
        k = np.arange(n) % self.n_r
        ray = np.arange(n) // self.n_r
        logit = 2.0 * (self.edge[ray] - k - 0.5)
        out = np.stack([logit, np.zeros(n)], axis=1).astype(np.float32)
        return torch.tensor(out, device="cuda")


@pytest.fixture(scope="module")
def scan_case():
    el, ref, desc = S.seed_ring(60)
    n_r, n_theta, n_turns = 400, 9, 300
    grid, _, n_rays = S.scan_grid(el, ref, n_r, n_theta)
    tr = xtgb.Tracker(el, ref)
    da_p, _, _ = S.plain_scan(tr, grid, n_rays, n_r, n_turns)
    yield tr, grid, n_rays, n_r, n_turns, da_p
    tr.close()


def test_plain_scan_has_a_boundary_on_every_ray(scan_case):
    _, _, n_rays, n_r, _, da_p = scan_case
    assert da_p.shape == (n_rays,)
    assert np.all(da_p > 40) and np.all(da_p < n_r - 40)


@pytest.mark.parametrize("shifts", [(0,), (2, -2), (-40, 0, -40, 2)])
def test_surrogate_scan_equals_plain_scan(scan_case, shifts):
    tr, grid, n_rays, n_r, n_turns, da_p = scan_case
    shift = np.array([shifts[j % len(shifts)] for j in range(n_rays)])
    net = ShiftedBoundary(da_p + shift, n_r)
    X = np.zeros((n_rays * n_r, 16), np.float32)
    da_s, _, tracked, passes = S.surrogate_scan(tr, net, grid, X, n_rays, n_r, n_turns, p_lo=0.02, margin=8,
                                                window=8, max_passes=6)
    assert np.array_equal(da_s, da_p)
    assert tracked < n_rays * n_r // 2
    if max(abs(s) for s in shifts) > 8:
        assert passes > 1
