"""What the trained surrogate gains over the scan without it (reduced scale).

A family of 12 error seeds of the reduced LHC-scale ring gets random-amplitude
labels from the batched tracker (100 turns); the network is trained on them
on the GPU by the library's own kernels; the band limits come from two
validation seeds of the family; then another seed of the family is scanned on
2,222 radii x 45 angles three ways: plain (every point tracked: the method
without the network), guided by the network, and on a coarse grid (every 10th
radius, then the gap before the first coarse loss).  The guided scan must
give the plain scan's DA within 0.2 sigma on every ray while tracking well
under half of the points; the test prints all three."""
import pytest

from paper_2310_00317_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def test_trained_network_reaches_the_plain_da_with_a_fraction_of_the_tracking():
    r = S.da_study(family=(13, 25), test_seeds=(20,), val_seeds=(14, 15), unseen_seed=None, mean_count=8000,
                   n_turns=100, epochs=16, n_r=2222, n_theta=45)
    s = r["per_seed"][0]
    print("plain %.2f s | guided %.2f s, %.1f %% tracked, %d pass(es), DA error max %.3f sigma | "
          "coarse %.2f s, %.1f %% tracked, DA error max %.3f sigma; band -%.2f/+%.2f sigma"
          % (s["plain_seconds"], s["surrogate_seconds"], 100 * s["tracked_fraction"], s["passes"],
             s["da_error_sigma_max"], s["coarse_seconds"], 100 * s["coarse_tracked_fraction"],
             s["coarse_da_error_sigma_max"], r["margin_sigma"], r["window_sigma"]))
    assert r["train_accuracy"] > 0.9
    assert s["da_error_sigma_max"] <= 0.2
    assert s["tracked_fraction"] < 0.4
