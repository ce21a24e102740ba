"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs."""
import dataclasses

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc
from paper_2102_02286_gb300.configs import SearchParams

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


def build_both(oracle_lib, w):
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    return prot, idx, db


# ------------------------------------------------------------------ index


def test_index_matches_oracle_ion_bins(gpu, oracle_lib):
    w = configs.OPEN_MEDIUM.with_proteins(120)
    prot, idx, db = build_both(oracle_lib, w)
    off, ent = idx.copy_csr()
    st = idx.stats()
    assert st.n_peptides == db.n
    assert off[-1] == st.n_entries == len(ent)
    pid = ent >> 1
    isy = ent & 1
    bins = np.repeat(np.arange(len(off) - 1), np.diff(off.astype(np.int64)))
    # pid ascending inside every bucket
    same = bins[1:] == bins[:-1]
    assert np.all(pid[1:][same] > pid[:-1][same])
    order = np.lexsort((bins, pid))
    per_pid = np.split(np.stack([bins[order], isy[order]], 1), np.cumsum(np.bincount(pid, minlength=db.n))[:-1])
    total = 0
    for p in range(db.n):
        ob, oy = db.bins(p)
        total += len(ob)
        np.testing.assert_array_equal(per_pid[p][:, 0], ob)
        np.testing.assert_array_equal(per_pid[p][:, 1], oy)
    assert total == st.n_entries


# ------------------------------------------------------------------ search


def test_parity_tiny_closed_full(gpu, oracle_lib):
    """The 500-protein closed search, all 1,000 spectra."""
    w = configs.TINY_CLOSED
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    got = idx.search(spec)
    ref = db.search(spec)
    lo, hi, npk, hits = idx.search_work(spec)
    np.testing.assert_array_equal(lo, ref.lo)
    np.testing.assert_array_equal(hi, ref.hi)
    assert np.all(npk <= w.params.top_n_peaks)
    # H(q) counted from the copied CSR with two binary searches per peak
    off, ent = idx.copy_csr()
    for q in range(0, spec.n, 97):
        a, e = int(spec.peak_off[q]), int(spec.peak_off[q + 1])
        bins, _, _, valid = oracle_lib.preprocess(w.params, spec.mz[a:e], spec.intensity[a:e],
                                                  float(spec.prec_mz[q]), int(spec.charge[q]), float(spec.tol_da[q]))
        assert len(bins) == npk[q]
        h = 0
        for bn in bins:
            bucket = ent[int(off[bn]):int(off[bn + 1])] >> 1
            h += int(np.searchsorted(bucket, ref.hi[q]) - np.searchsorted(bucket, ref.lo[q]))
        assert h == hits[q]
    n = assert_parity(got, ref, label="tiny_closed")
    assert n > 900


@pytest.mark.parametrize("n_prot,n_spec,tol", [(300, 48, 500.0), (300, 3, 500.0), (1000, 30, 100.0)])
def test_parity_open_reduced(gpu, oracle_lib, n_prot, n_spec, tol):
    """Open search with modifications on a reduced proteome: windows span
    several 16k-peptide chunks and end in a ragged tail; 3 spectra exercise
    the split-window path (many segments per spectrum)."""
    w = configs.OPEN_MEDIUM.with_proteins(n_prot)
    w = configs.Workload(w.name, w.index, w.n_proteins, w.mods, w.params,
                         configs.SpectraRecipe(n_spectra=n_spec, target_peaks=(100, 100), tol_da=(tol,)))
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    got = idx.search(spec)
    ref = db.search(spec)
    assert (ref.hi - ref.lo).max() > 16384
    n = assert_parity(got, ref, label="open_reduced")
    assert n > 0 and ref.n_scored.sum() > 10


def test_parity_uneven_peaks_and_tolerances(gpu, oracle_lib):
    """50-500 peaks per spectrum, +-10/100/500 Da windows (top_n 500)."""
    w = configs.UNEVEN_BATCHED.with_proteins(150).with_spectra(60)
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    got = idx.search(spec)
    ref = db.search(spec)
    assert_parity(got, ref, label="uneven")


def test_parity_large_params(gpu, oracle_lib):
    """The large workload's parameters (dF 0.02, z 2-4, three variable mods,
    top-10) on a reduced proteome."""
    w = configs.OPEN_LARGE.with_proteins(60).with_spectra(30)
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    assert_parity(idx.search(spec), db.search(spec), label="large_params")


def test_device_pointer_path_matches_host_path(gpu, oracle_lib):
    torch = gpu
    w = configs.OPEN_MEDIUM.with_proteins(100).with_spectra(50)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    host = idx.search(spec)
    db = hc.DeviceBatch.from_spectra(spec)
    out = hc.DeviceResult.alloc(spec.n, w.params.top_k)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        idx.search_device(db, out, stream)
    stream.synchronize()
    dev = out.to_host(spec.n, w.params.top_k)
    np.testing.assert_array_equal(dev.psm, host.psm)
    np.testing.assert_array_equal(dev.hist, host.hist)
    np.testing.assert_array_equal(dev.n_scored, host.n_scored)


# ------------------------------------------------------------------ edge cases


def test_edge_cases(gpu, oracle_lib):
    w = configs.TINY_CLOSED.with_proteins(80)
    prot, idx, db = build_both(oracle_lib, w)
    base = synth.make_spectra(prot, w, n=6)
    m0, i0 = base.mz[:int(base.peak_off[1])], base.intensity[:int(base.peak_off[1])]
    rng = np.random.default_rng(5)
    peaks = [
        (list(m0), list(i0)),                                  # ordinary
        ([], []),                                              # no peaks
        (list(m0), list(i0)),                                  # charge 0
        (list(m0), list(i0)),                                  # NaN precursor
        (list(m0), list(i0)),                                  # negative tolerance
        ([50.0, 2500.0, 99.999], [1.0, 2.0, 3.0]),             # nothing in range
        (list(rng.uniform(100, 2000, 4096)), list(rng.uniform(1, 100, 4096))),   # one sort's worth of raw peaks
        (list(rng.uniform(100, 2000, 4097)), list(rng.uniform(1, 100, 4097))),   # one more
        (list(m0) + [float("nan"), 150.0], list(i0) + [5.0, float("inf")]),      # non-finite peaks
        (list(m0), list(i0)),                                  # whole database in the window
        (list(m0), list(i0)),                                  # zero tolerance
        # 25,000 raw peaks on the peptide's own m/z values, each repeated in
        # every chunk with other intensities: a bin keeps its largest anywhere
        (list(np.tile(m0, 25000 // len(m0) + 1)[:25000]), list(rng.uniform(1, 1000, 25000))),
        # the peptide's peaks after 9,000 weaker noise peaks: the retained
        # bins all come from the last chunk
        (list(rng.uniform(100, 2000, 9000)) + list(m0), list(rng.uniform(0.01, 0.1, 9000)) + list(i0 + 1.0)),
    ]
    p0 = float(base.prec_mz[0])
    prec = [p0, p0, p0, float("nan"), p0, p0, p0, p0, p0, p0, p0, p0, p0]
    z = [int(base.charge[0])] * 13
    z[2] = 0
    tol = [10.0, 10.0, 10.0, 10.0, -1.0, 10.0, 500.0, 500.0, 10.0, 1e9, 0.0, 500.0, 10.0]
    spec = synth.spectra_from_lists(peaks, prec, z, tol)
    got = idx.search(spec)
    ref = db.search(spec)
    assert_parity(got, ref, label="edge")
    for q in (1, 2, 3, 4, 5):
        assert np.all(got.psm["pid"][q] == PAD) and got.n_scored[q] == 0
    # no raw-peak limit: every such spectrum is searched, with the oracle's
    # retained peaks (count here; bins and intensities through the parity)
    _, _, npk, _ = idx.search_work(spec)
    for q in (0, 6, 7, 11, 12):
        a, b = int(spec.peak_off[q]), int(spec.peak_off[q + 1])
        bins, _, _, _ = oracle_lib.preprocess(w.params, spec.mz[a:b], spec.intensity[a:b], float(spec.prec_mz[q]),
                                              int(spec.charge[q]), float(spec.tol_da[q]))
        assert npk[q] == len(bins) > 0, q
    for q in (0, 11, 12):
        assert got.n_scored[q] >= 1, q
    # the last spectrum retains the peptide's own peaks, so it finds what the first finds
    assert got.psm["pid"][12][0] == got.psm["pid"][0][0]


def test_malformed_peak_offsets(gpu):
    """Spectra whose peak offsets decrease or leave the batch's
    [peak_off[0], peak_off[n]) are invalid: padding rows, an empty
    histogram, none of their peaks read; their neighbours are searched as in
    a well-formed batch, through host and device buffers."""
    w = configs.TINY_CLOSED.with_proteins(80)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    good = synth.make_spectra(prot, w, n=4)
    ref = idx.search(good)
    off = good.peak_off.astype(np.uint64).copy()
    # spectrum 1 ends past peak_off[n]; spectrum 2 starts there and ends lower
    off[2] = off[4] + 1000
    bad = dataclasses.replace(good, peak_off=off)
    for got in (idx.search(bad), _search_device(gpu, idx, bad, w.params.top_k)):
        for q in (1, 2):
            assert np.all(got.psm["pid"][q] == PAD) and got.n_scored[q] == 0 and got.hist[q].sum() == 0
        for q in (0, 3):
            np.testing.assert_array_equal(got.psm[q], ref.psm[q])
            np.testing.assert_array_equal(got.hist[q], ref.hist[q])


def _search_device(gpu, idx, spec, k):
    out = hc.DeviceResult.alloc(spec.n, k)
    idx.search_device(hc.DeviceBatch.from_spectra(spec), out)
    gpu.cuda.synchronize()
    return out.to_host(spec.n, k)


def test_empty_batch(gpu):
    w = configs.TINY_CLOSED.with_proteins(20)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.spectra_from_lists([], [], [], [])
    r = idx.search(spec)
    assert r.psm.shape == (0, w.params.top_k)


@pytest.mark.parametrize("top_k,min_shared", [(1, 4), (32, 1), (17, 2)])
def test_topk_and_threshold_extremes(gpu, oracle_lib, top_k, min_shared):
    p = SearchParams(missed_cleavages=1, top_k=top_k, min_shared=min_shared)
    w = configs.Workload("x", 0, 100, (configs.CARBAMIDOMETHYL_C,), p,
                         configs.SpectraRecipe(n_spectra=25, tol_da=(300.0,)))
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    assert_parity(idx.search(spec), db.search(spec), label=f"k{top_k}")


# ------------------------------------------------------------------ full size


@pytest.mark.slow
def test_parity_open_medium_full_index_sampled(gpu, oracle_lib):
    """The 20k-protein open-search index and the full 100k-spectrum batch in
    one launch (the benchmark's configuration); sampled spectra checked
    against the oracle (about 7 s each on one core)."""
    w = configs.OPEN_MEDIUM
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    got = idx.search(spec)          # through host buffers
    dev = hc.DeviceResult.alloc(spec.n, w.params.top_k)
    idx.search_device(hc.DeviceBatch.from_spectra(spec), dev)   # device buffers, same launch
    gpu.cuda.synchronize()
    whole = dev.to_host(spec.n, w.params.top_k)
    np.testing.assert_array_equal(got.psm, whole.psm)
    np.testing.assert_array_equal(got.hist, whole.hist)
    np.testing.assert_array_equal(got.n_scored, whole.n_scored)
    sel = np.array([0, 1, 12345, 54321, 99999], dtype=np.uint32)
    ref = db.search(spec, sel=sel)
    assert_parity(got, ref, sel=sel, label="open_medium")
    # whole-batch properties that hold at any size
    real = got.psm["pid"] != PAD
    k = got.psm["key"]
    assert np.all((k[:, :-1] > k[:, 1:]) | ((k[:, :-1] == k[:, 1:]) & (got.psm["pid"][:, :-1] < got.psm["pid"][:, 1:]))
                  | ~real[:, 1:])
    np.testing.assert_array_equal(got.hist.sum(1), got.n_scored)
    assert np.all(got.psm["nb"][real].astype(int) + got.psm["ny"][real] >= w.params.min_shared)


@pytest.mark.slow
def test_parity_uneven_batched_full_sampled(gpu, oracle_lib):
    """The uneven 200k-spectrum batch (50-500 peaks, +-10/100/500 Da) on the
    open-search index in the batched form the benchmark times: one plan
    launch with the autotuned shape, replayed as a CUDA graph; spectra of
    every tolerance class and both peak-count extremes checked against the
    oracle."""
    torch = gpu
    w = configs.UNEVEN_BATCHED
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    dbat = hc.DeviceBatch.from_spectra(spec)
    shape, _ = idx.autotune(hc.DeviceBatch.from_spectra(spec.subset(np.arange(20000))))
    plan = idx.plan(spec.n, shape)
    out = hc.DeviceResult.alloc(spec.n, w.params.top_k)
    stream = torch.cuda.Stream()
    for _ in range(2):                       # capture, then replay
        with torch.cuda.stream(stream):
            plan.search(dbat, out, stream, graph=True)
    stream.synchronize()
    got = out.to_host(spec.n, w.params.top_k)
    plan.close()
    npk = np.diff(spec.peak_off.astype(np.int64))
    sel = []
    for tol in (10.0, 100.0, 500.0):
        cls = np.flatnonzero(spec.tol_da == tol)
        sel += [int(cls[np.argmin(npk[cls])]), int(cls[np.argmax(npk[cls])])]
    sel = np.array(sorted(sel), dtype=np.uint32)
    assert_parity(got, db.search(spec, sel=sel), sel=sel, label="uneven_batched")
    np.testing.assert_array_equal(got.hist.sum(1), got.n_scored)
