"""The large modified open search (50k proteins, Met-ox <= 3, STY-phospho <= 2,
N/Q-deamidation <= 1, dF 0.02 Da, top-10) at full index size, and the
serving recipe's spectra on the same index, sampled against the oracle.

The oracle digests the whole database on one core before it can find a
window (minutes) and needs minutes per +-500 Da spectrum of this database,
so one spawned oracle process (no fork after the GPU is in use) searches the
sampled spectra while the GPU runs: one +-500 Da spectrum of the open-search
batch and the serving recipe's largest +-10 Da and +-500 Da spectra
(HICOPS_LARGE=1 adds the batch's last spectrum)."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

from parity import PAD, assert_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


_DB = {}


def _oracle_one(job):
    """One sampled spectrum against the database built by _oracle_all (in a
    child forked from that process, which never touched the GPU; the
    children share the database's pages)."""
    name, n_spectra, q = job
    prot, db = _DB["prot"], _DB["db"]
    w = configs.BY_NAME[name].with_spectra(n_spectra)
    spec = synth.make_spectra(prot, w)
    return db.search(spec, sel=np.array([q], dtype=np.uint32))


def _oracle_all(jobs):
    """(in one spawned process: the oracle holds about 340 B per peptide, so
    one copy of the 237M-entry database is all the host takes) the oracle's
    results for spectra q of the workloads' first n_spectra spectra, one
    forked child per spectrum."""
    import time
    import oracle
    oracle.build()
    t0 = time.time()
    w0 = configs.BY_NAME[jobs[0][0]]
    prot = synth.make_proteome(w0.n_proteins, w0.db_seed, w0.protein_len)
    _DB["prot"] = prot
    _DB["db"] = oracle.OracleDb(prot.seq, prot.off, w0.mods, w0.params)
    t1 = time.time()
    with mp.get_context("fork").Pool(len(jobs)) as pool:
        out = pool.map(_oracle_one, jobs)
    return out, (t1 - t0, time.time() - t1)


def test_open_large_and_serving_recipe_sampled(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_2102_02286_gb300 import build as pkg_build
    pkg_build.build()
    wl = configs.OPEN_LARGE.with_spectra(20000)
    ws = configs.SERVING_STREAM.with_spectra(4096)
    prot = synth.make_proteome(wl.n_proteins, wl.db_seed, wl.protein_len)
    spec_l = synth.make_spectra(prot, wl)
    spec_s = synth.make_spectra(prot, ws)
    npk = np.diff(spec_s.peak_off.astype(np.int64))
    s_sel = [int(np.flatnonzero(spec_s.tol_da == t)[np.argmax(npk[spec_s.tol_da == t])]) for t in (10.0, 500.0)]
    l_sel = [0, 19999] if os.environ.get("HICOPS_LARGE") == "1" else [0]
    jobs = [("open_large", wl.spectra.n_spectra, q) for q in l_sel] + \
           [("serving_stream", ws.spectra.n_spectra, q) for q in s_sel]
    with cf.ProcessPoolExecutor(1, mp_context=mp.get_context("spawn")) as ex:
        fut = ex.submit(_oracle_all, jobs)
        idx = hc.Index(prot.seq, prot.off, wl.mods, wl.params)
        st = idx.stats()
        got_l = idx.search(spec_l)                       # one batch of 20k spectra
        server = hc.Server(idx)
        got_s = server.poll(server.submit(spec_s), -1)   # the serving path
        server.close()
        del idx
        refs, (t_db, t_search) = fut.result()
    print(f"oracle: database {t_db:.0f} s, {len(jobs)} spectra in parallel {t_search:.0f} s")
    assert st.n_peptides > 100_000_000
    for i, q in enumerate(l_sel):
        sel = np.array([q], dtype=np.uint32)
        assert_parity(got_l, refs[i], sel=sel, label=f"open_large spectrum {q}")
    for i, q in enumerate(s_sel):
        sel = np.array([q], dtype=np.uint32)
        assert_parity(got_s, refs[len(l_sel) + i], sel=sel, label=f"serving recipe spectrum {q}")
    real = got_l.psm["pid"] != PAD
    np.testing.assert_array_equal(got_l.hist.sum(1), got_l.n_scored)
    assert np.all(got_l.psm["nb"][real].astype(int) + got_l.psm["ny"][real] >= wl.params.min_shared)
