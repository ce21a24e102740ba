"""The host ingest pipeline on the GPU: spectra written to MS2 files, parsed,
searched and written by the R/I/K workers, give exactly the rows of one
hicops_search of the same spectra, whatever the buffer sizes, worker counts
and scheduling thresholds; a malformed file fails the run with its name and
line."""
import types

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

from parity import EV_RTOL, HS_RTOL

pytestmark = pytest.mark.gpu
PAD = 0xFFFFFFFF


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


def write_files(spec, tmp_path, cuts):
    paths = []
    for i, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
        p = str(tmp_path / f"part{i}.ms2")
        synth.write_ms2(spec, p, sel=range(a, b))
        paths.append(p)
    return paths


def check_rows(rows, ref, cuts):
    q = np.asarray(cuts[:-1], np.int64)[rows["file"]] + rows["spectrum"].astype(np.int64)
    order = np.lexsort((rows["rank"], q))
    rows, q = rows[order], q[order]
    real = ref.psm["pid"] != PAD
    wq, wr = np.nonzero(real)
    np.testing.assert_array_equal(q, wq)
    np.testing.assert_array_equal(rows["rank"], wr)
    want = ref.psm[wq, wr]
    for f in ("pid", "nb", "ny", "hyperscore", "evalue"):
        np.testing.assert_array_equal(rows[f], want[f].astype(rows.dtype[f]), err_msg=f)
    np.testing.assert_array_equal(rows["n_scored"], ref.n_scored[wq])
    np.testing.assert_array_equal(rows["scan"], rows["spectrum"] + 1)


@pytest.mark.parametrize("cfg", [{}, dict(batch_spectra=7, n_buffers=3, n_workers=3),
                                 dict(batch_spectra=50, n_buffers=2, n_workers=2, t_min_s=1e-9, t_max_s=1e-9),
                                 dict(batch_spectra=16, n_buffers=30, n_workers=6, alpha=0.9)])
def test_pipeline_equals_direct_search(gpu, tmp_path, cfg):
    w = configs.TINY_CLOSED.with_proteins(200).with_spectra(500)
    prot, spec = synth.make_workload_inputs(w)
    spec.charge[7] = 0                       # an invalid spectrum: no rows
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    ref = idx.search(spec)
    cuts = [0, 37, 300, 300, 500]            # uneven files, one of them empty
    paths = write_files(spec, tmp_path, cuts)
    out = str(tmp_path / "rows.tsv")
    st = hc.run_files(idx, paths, out, 10.0, **cfg)
    assert st.spectra == 500
    check_rows(hc.read_pipeline_rows(out), ref, cuts)
    idx.close()


def test_pipeline_open_search(gpu, tmp_path):
    w = configs.OPEN_MEDIUM.with_proteins(300).with_spectra(120)
    prot, spec = synth.make_workload_inputs(w)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    ref = idx.search(spec)
    cuts = [0, 60, 120]
    paths = write_files(spec, tmp_path, cuts)
    out = str(tmp_path / "rows.tsv")
    st = hc.run_files(idx, paths, out, 500.0, batch_spectra=16, n_workers=4)
    assert st.spectra == 120 and st.batches == 8
    check_rows(hc.read_pipeline_rows(out), ref, cuts)
    idx.close()


def check_rows_against_oracle(rows, ref, cuts):
    """Rows of the written result file against the oracle: every real PSM
    once, in rank order, with the oracle's peptide, b/y counts and candidate
    count; hyperscore and e-value within the parity tolerances (the file
    holds each number in its shortest round-trip form)."""
    q = np.asarray(cuts[:-1], np.int64)[rows["file"]] + rows["spectrum"].astype(np.int64)
    order = np.lexsort((rows["rank"], q))
    rows, q = rows[order], q[order]
    real = ref.psm["pid"] != PAD
    wq, wr = np.nonzero(real)
    np.testing.assert_array_equal(q, wq)
    np.testing.assert_array_equal(rows["rank"], wr)
    want = ref.psm[wq, wr]
    for f in ("pid", "nb", "ny"):
        np.testing.assert_array_equal(rows[f].astype(np.int64), want[f].astype(np.int64), err_msg=f)
    np.testing.assert_array_equal(rows["n_scored"], ref.n_scored[wq])
    np.testing.assert_allclose(rows["hyperscore"].astype(np.float64), want["hyperscore"], rtol=HS_RTOL, atol=0)
    np.testing.assert_allclose(rows["evalue"].astype(np.float64), want["evalue"], rtol=EV_RTOL, atol=0)
    return len(wq)


@pytest.mark.parametrize("name,tol", [("tiny_closed", 10.0), ("open_medium", 500.0)])
def test_pipeline_rows_match_the_oracle(gpu, oracle_lib, tmp_path, name, tol):
    """File -> parse -> buffer -> search -> result file (the Buffering and
    Task Scheduling sections' R/I/K path) against the oracle on the same
    spectra, read back from the written files."""
    w = configs.BY_NAME[name].with_proteins(200).with_spectra(120)
    prot, spec = synth.make_workload_inputs(w)
    spec.charge[3] = 0                       # an invalid spectrum: no rows on either side
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    cuts = [0, 45, 45, 120]
    paths = write_files(spec, tmp_path, cuts)
    out = str(tmp_path / "rows.tsv")
    st = hc.run_files(idx, paths, out, tol, batch_spectra=24, n_workers=4)
    assert st.spectra == 120
    idx.close()
    # the oracle searches what the files hold, as the library's parser reads
    # them (the same values as the in-memory spectra: shortest round-trip text)
    parsed = [hc.read_ms2(p) for p in paths]
    counts = np.concatenate([np.diff(p["peak_off"].astype(np.int64)) for p in parsed])
    files = types.SimpleNamespace(
        n=len(counts), peak_off=np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64),
        mz=np.concatenate([p["mz"] for p in parsed]), intensity=np.concatenate([p["intensity"] for p in parsed]),
        prec_mz=np.concatenate([p["prec_mz"] for p in parsed]), charge=np.concatenate([p["charge"] for p in parsed]),
        tol_da=np.full(len(counts), tol))
    assert files.n == 120
    np.testing.assert_array_equal(files.mz, spec.mz)
    np.testing.assert_array_equal(files.prec_mz, spec.prec_mz)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    ref = db.search(files)
    assert check_rows_against_oracle(hc.read_pipeline_rows(out), ref, cuts) > 80


def test_pipeline_errors(gpu, tmp_path):
    w = configs.TINY_CLOSED.with_proteins(50).with_spectra(30)
    prot, spec = synth.make_workload_inputs(w)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    good = write_files(spec, tmp_path, [0, 30])
    bad = str(tmp_path / "bad.ms2")
    with open(bad, "w") as f:
        f.write("S\t1\t1\t500.0\nZ\t2\t999.0\n100.0 1.0\n101.0 x\n")
    with pytest.raises(hc.HicopsError) as e:
        hc.run_files(idx, good + [bad], str(tmp_path / "o.tsv"), 10.0)
    assert "bad.ms2" in str(e.value) and "line 4" in str(e.value)
    with pytest.raises(hc.HicopsError):
        hc.run_files(idx, [str(tmp_path / "missing.ms2")], str(tmp_path / "o.tsv"), 10.0)
    with pytest.raises(hc.HicopsError):
        hc.run_files(idx, good, str(tmp_path / "o.tsv"), 10.0, n_workers=1)
    idx.close()
