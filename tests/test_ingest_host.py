"""Host half of the ingest pipeline (no GPU): the MS2 parser on a
hand-written file, the writer/parser round trip, the double exponential
smoothing forecast against closed forms, and the scheduling rules of the
Task Scheduling section as truth tables."""
import os

import numpy as np
import pytest

from paper_2102_02286_gb300 import build as pkg_build
from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return hc.load()


def test_ms2_hand_written_file(lib):
    r = hc.read_ms2(os.path.join(GOLDEN, "example.ms2"))
    # three spectra: the first Z line gives the charge, no Z line = charge 0,
    # "I" and blank lines skipped, tabs / spaces / CRLF accepted
    np.testing.assert_array_equal(r["scan"], [7, 9, 11])
    np.testing.assert_array_equal(r["charge"], [2, 0, 1])
    np.testing.assert_array_equal(r["prec_mz"], [500.25, 612.0, 300.5])
    np.testing.assert_array_equal(r["peak_off"], [0, 3, 4, 5])
    np.testing.assert_array_equal(r["mz"], np.array([101.5, 150.25, 2000.125, 110.0, 120.0], np.float32))
    np.testing.assert_array_equal(r["intensity"], np.array([20, 7.5, 300, 1, 4], np.float32))


@pytest.mark.parametrize("text,line", [("101.5 20\n", 1), ("S\t1\t1\t500\n100 1 2\n", 2),
                                       ("S\t1\t1\n", 1), ("H\tx\nZ\t2\t100\n", 2),
                                       ("S\t1\t1\t500\n100 abc\n", 2), ("S\t1\t1\t500\nH\tlate\n", 2)])
def test_ms2_malformed_lines_are_named(lib, tmp_path, text, line):
    p = tmp_path / "bad.ms2"
    p.write_text(text)
    with pytest.raises(hc.HicopsError) as e:
        hc.read_ms2(str(p))
    assert f"line {line}" in str(e.value)


def test_ms2_missing_file(lib, tmp_path):
    with pytest.raises(hc.HicopsError):
        hc.read_ms2(str(tmp_path / "none.ms2"))


def test_ms2_round_trip(lib, tmp_path):
    w = configs.UNEVEN_BATCHED.with_proteins(60).with_spectra(120)
    prot, spec = synth.make_workload_inputs(w)
    spec.charge[5] = 0
    p = str(tmp_path / "a.ms2")
    synth.write_ms2(spec, p, scan_base=100)
    r = hc.read_ms2(p)
    for k in ("peak_off", "mz", "intensity", "prec_mz", "charge"):
        np.testing.assert_array_equal(r[k], getattr(spec, k if k != "mz" else "mz"))
    np.testing.assert_array_equal(r["scan"], np.arange(100, 100 + spec.n))


def des(xs, alpha):
    L = hc.load()
    st = np.zeros(2, np.float64)
    return [L.hicops_des_step(st.ctypes.data, float(x), alpha, int(i == 0)) for i, x in enumerate(xs)]


def test_double_exponential_smoothing(lib):
    # a constant series forecasts itself
    assert des([3.0] * 10, 0.3) == [3.0] * 10
    # by hand, a = 0.5: s1 = s2 = 0, then x = 1: s1 = 0.5, s2 = 0.25, forecast 3 s1 - 2 s2 = 1
    assert des([0.0, 1.0], 0.5) == [0.0, 1.0]
    # a linear series: the forecast error decays as (1 - a)^t to the next value
    a, b = 2.0, 0.25
    f = des([a + b * t for t in range(200)], 0.4)
    assert abs(f[-1] - (a + b * 200)) < 1e-9
    assert abs(f[20] - (a + b * 21)) > 1e-6          # not yet converged early on


def test_scheduling_rules(lib):
    L = hc.load()
    i2r = L.hicops_sched_i_to_r
    # (t_wait >= t_min and t_cum + t_fct > t_max) or (w1 and no R worker)
    assert i2r(0.002, 0.04, 0.02, 0.001, 0.05, 10, 1) == 1
    assert i2r(0.0005, 0.04, 0.02, 0.001, 0.05, 10, 1) == 0     # wait below t_min
    assert i2r(0.002, 0.02, 0.02, 0.001, 0.05, 10, 1) == 0      # cumulative + forecast within t_max
    assert i2r(0.0, 0.0, 0.0, 0.001, 0.05, 4, 0) == 1           # w1 and no R worker
    assert i2r(0.0, 0.0, 0.0, 0.001, 0.05, 5, 0) == 0           # w2
    assert i2r(0.0, 0.0, 0.0, 0.001, 0.05, 4, 1) == 0           # an R worker exists
    r2i = L.hicops_sched_r_to_i
    # (w3 and more than one R worker) or the queue full
    assert r2i(15, 20, 2) == 1
    assert r2i(15, 20, 1) == 0
    assert r2i(14, 20, 3) == 0
    assert r2i(20, 20, 1) == 1
    assert r2i(3, 3, 1) == 1
