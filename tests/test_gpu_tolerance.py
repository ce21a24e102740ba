"""GPU parity of the fragment tolerance of t bins (R15): the CUDA path's
widened query bins against the oracle at several t, on closed and open
searches, at the (2t+1) * top_n_peaks limit, with ragged peak counts
(both preprocessing kernels), overlapping windows and windows cut by the
end of the fragment range, and through the server."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc
from paper_2102_02286_gb300.configs import SearchParams, SpectraRecipe, Workload

from parity import PAD, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_2102_02286_gb300 import build as pkg_build
    pkg_build.build()
    hc.load()
    return torch


def with_tol(w, t, bin_width_da=0.005, **kw):
    return dataclasses.replace(w, params=dataclasses.replace(w.params, bin_width_da=bin_width_da, tol_bins=t, **kw))


def build_both(oracle_lib, w):
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    return prot, idx, db


def widened_count(oracle_lib, p, spec, q):
    """|union of the retained peaks' windows [b - t, b + t] within [0, n_bins)|"""
    a, e = int(spec.peak_off[q]), int(spec.peak_off[q + 1])
    bins, _, _, valid = oracle_lib.preprocess(p, spec.mz[a:e], spec.intensity[a:e], float(spec.prec_mz[q]),
                                              int(spec.charge[q]), float(spec.tol_da[q]))
    if not valid:
        return 0
    n_bins = math.floor(p.frag_mz_max / p.bin_width_da) + 1
    cover = set()
    for b in bins:
        cover.update(x for x in range(int(b) - p.tol_bins, int(b) + p.tol_bins + 1) if 0 <= x < n_bins)
    return len(cover)


@pytest.mark.parametrize("t", [1, 2, 3])
def test_tolerance_closed(gpu, oracle_lib, t):
    w = with_tol(configs.TINY_CLOSED, t).with_proteins(200).with_spectra(300)
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    ref = db.search(spec)
    n = assert_parity(idx.search(spec), ref, label=f"closed t={t}")
    assert n > 250
    _, _, npk, _ = idx.search_work(spec)
    for q in range(0, spec.n, 23):
        assert npk[q] == widened_count(oracle_lib, w.params, spec, q)


@pytest.mark.parametrize("n_spec", [40, 3])
def test_tolerance_open(gpu, oracle_lib, n_spec):
    """open_medium_tol's parameters on a reduced proteome: windows span
    several 16k-peptide chunks; 3 spectra take the split-window path."""
    w = configs.OPEN_MEDIUM_TOL.with_proteins(300).with_spectra(n_spec)
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    ref = db.search(spec)
    assert (ref.hi - ref.lo).max() > 16384
    n = assert_parity(idx.search(spec), ref, label="open t=1")
    assert n > 0


@pytest.mark.parametrize("t,top_n", [(1, 341), (4, 113)])
def test_tolerance_at_the_bin_limit(gpu, oracle_lib, t, top_n):
    """(2t+1) * top_n_peaks just under 1,024 query bins; 200-500 raw peaks,
    so spectra go through both preprocessing kernels."""
    p = SearchParams(missed_cleavages=1, bin_width_da=0.005, tol_bins=t, top_n_peaks=top_n, min_shared=4, top_k=5)
    w = Workload("limit", 0, 150, (configs.CARBAMIDOMETHYL_C,), p,
                 SpectraRecipe(n_spectra=40, target_peaks=(200, 500), tol_da=(100.0,)))
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    assert_parity(idx.search(spec), db.search(spec), label=f"limit t={t}")
    _, _, npk, _ = idx.search_work(spec)
    assert npk.max() > 800
    for q in range(0, spec.n, 7):
        assert npk[q] == widened_count(oracle_lib, w.params, spec, q)


def test_tolerance_edges(gpu, oracle_lib):
    """Peaks one bin apart (overlapping windows), two peaks in one bin, peaks
    at both ends of the fragment range (windows cut at the last bin), a
    spectrum whose only peaks lie just outside the range, invalid spectra."""
    w = with_tol(configs.TINY_CLOSED, 2).with_proteins(80)
    prot, idx, db = build_both(oracle_lib, w)
    base = synth.make_spectra(prot, w, n=4)
    m0 = [float(x) for x in base.mz[:int(base.peak_off[1])]]
    i0 = [float(x) for x in base.intensity[:int(base.peak_off[1])]]
    step = w.params.bin_width_da
    near = [m0[0] + step, m0[0] + 2 * step, m0[1] + 0.3 * step]
    peaks = [
        (m0, i0),                                                       # ordinary
        (m0 + near, i0 + [5.0, 50.0, 500.0]),                           # overlapping windows, shared bin
        (m0 + [100.0, 100.001, 1999.999, 1999.996], i0 + [7.0, 9.0, 11.0, 3.0]),   # range ends
        ([99.999, 2000.0], [1.0, 1.0]),                                 # nothing in range
        (m0, i0),                                                       # charge 0
        ([], []),                                                       # no peaks
    ]
    p0 = float(base.prec_mz[0])
    z = [int(base.charge[0])] * 6
    z[4] = 0
    spec = synth.spectra_from_lists(peaks, [p0] * 6, z, [500.0, 500.0, 500.0, 10.0, 10.0, 10.0])
    got = idx.search(spec)
    assert_parity(got, db.search(spec), label="tolerance edges")
    for q in (3, 4, 5):
        assert np.all(got.psm["pid"][q] == PAD) and got.n_scored[q] == 0
    _, _, npk, _ = idx.search_work(spec)
    for q in range(spec.n):
        assert npk[q] == widened_count(oracle_lib, w.params, spec, q)


def test_tolerance_server_matches_search(gpu):
    w = with_tol(configs.TINY_CLOSED, 1).with_proteins(150).with_spectra(200)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    one = idx.search(spec)
    server = hc.Server(idx)
    got = server.poll(server.submit(spec), -1)
    server.close()
    np.testing.assert_array_equal(got.psm, one.psm)
    np.testing.assert_array_equal(got.hist, one.hist)
    np.testing.assert_array_equal(got.n_scored, one.n_scored)


@pytest.mark.parametrize("t,top_n", [(5, 100), (1, 342), (1024, 1)])
def test_tolerance_too_wide_is_rejected(gpu, t, top_n):
    w = configs.TINY_CLOSED.with_proteins(10)
    p = dataclasses.replace(w.params, tol_bins=t, top_n_peaks=top_n)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    with pytest.raises(hc.HicopsError):
        hc.Index(prot.seq, prot.off, w.mods, p)
