"""Workloads as JSON: every built-in workload survives the round trip,
left-out fields take their defaults, unknown fields are errors."""
import json

import pytest

from paper_2102_02286_gb300 import configs


@pytest.mark.parametrize("w", configs.WORKLOADS, ids=[w.name for w in configs.WORKLOADS])
def test_round_trip(w):
    assert configs.workload_from_json(configs.workload_to_json(w)) == w


def test_defaults_and_errors():
    w = configs.workload_from_json(json.dumps({"name": "mine", "index": 9, "n_proteins": 40,
                                               "spectra": {"n_spectra": 12, "tol_da": [25.0]}}))
    assert w.params == configs.SearchParams() and w.mods == ()
    assert w.spectra.tol_da == (25.0,) and w.spectra.n_spectra == 12
    with pytest.raises(TypeError):
        configs.workload_from_json(json.dumps({"name": "x", "index": 0, "n_proteins": 1, "colour": 3,
                                               "spectra": {"n_spectra": 1}}))
    with pytest.raises(TypeError):
        configs.workload_from_json(json.dumps({"name": "x", "index": 0, "n_proteins": 1,
                                               "params": {"bin_width": 0.01}, "spectra": {"n_spectra": 1}}))
    with pytest.raises(ValueError):
        configs.workload_from_json("[1, 2]")
