"""The benchmark's --only specs on CPU: each measurement's own fields, in the
order its help text gives them, become the keyword arguments of its
function (no GPU call is made)."""
import inspect
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("spec, name, kw", [
    ("da_scan_full:100:1.0:1e6:2", "da_scan_full",
     {"n_turns": 100, "base_mult": 1.0, "total_labels": 1000000, "n_test": 2}),
    ("da_scan_full", "da_scan_full", {}),
    ("da_scan:300", "da_scan", {"n_turns": 300}),
    ("steady:200:50", "steady", {"turns": 200, "window": 50}),
    ("batched_seeds:20:5", "batched_seeds", {"T": 20, "steps": 5}),
    ("lepton_quantum:200000:2", "lepton_quantum", {"n": 200000, "turns": 2}),
    ("thick_elements:100000", "thick_elements", {"n": 100000}),
    ("fodo10", "fodo10", {}),
])
def test_only_specs_parse_into_the_measurements_arguments(spec, name, kw):
    assert bench.only_kwargs(spec) == (name, kw)


def test_every_parsed_argument_is_a_parameter_of_its_measurement():
    fns = {"da_scan_full": bench.measure_da_scan_full, "da_scan": bench.measure_da_scan,
           "steady": bench.measure_steady, "batched_seeds": bench.measure_batched,
           "lepton_quantum": bench.measure_lepton, "thick_elements": bench.measure_thick,
           "beambeam_lens": bench.measure_beambeam, "lepton_equilibrium": bench.measure_lepton_equilibrium,
           "fodo10": bench.measure_fodo}
    specs = ["da_scan_full:100:1.0:1e6:2", "da_scan:300", "steady:200:50", "batched_seeds:20:5",
             "lepton_quantum:1:2", "thick_elements:1:2", "beambeam_lens:1:2", "lepton_equilibrium:1:2",
             "fodo10:1:2"]
    for spec in specs:
        name, kw = bench.only_kwargs(spec)
        params = inspect.signature(fns[name]).parameters
        assert set(kw) <= set(params), (spec, kw)
