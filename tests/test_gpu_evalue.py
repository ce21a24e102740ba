"""GPU parity of the e-value options (Superstep 4): the Savitzky-Golay
smoothing of the histogram (R16) and the log-Weibull fit (R17), alone and
together, against the oracle; through the shard merge and the server; and
the rejection of unknown option bits."""
import dataclasses

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

from parity import assert_parity

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


def with_mode(w, ev_mode):
    return dataclasses.replace(w, params=dataclasses.replace(w.params, evalue_mode=ev_mode))


def build_both(oracle_lib, w):
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    return prot, idx, db


@pytest.mark.parametrize("ev_mode", [0, 1, 2, 3])
def test_evalue_options_closed(gpu, oracle_lib, ev_mode):
    w = with_mode(configs.TINY_CLOSED, ev_mode).with_proteins(200).with_spectra(300)
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    assert_parity(idx.search(spec), db.search(spec), label=f"evalue mode {ev_mode}")


@pytest.mark.parametrize("ev_mode", [1, 3])
def test_evalue_options_open(gpu, oracle_lib, ev_mode):
    """Open search with min_shared 2: histograms of thousands of candidates."""
    w = with_mode(configs.OPEN_MEDIUM, ev_mode).with_proteins(300).with_spectra(30)
    w = dataclasses.replace(w, params=dataclasses.replace(w.params, min_shared=2))
    prot, idx, db = build_both(oracle_lib, w)
    spec = synth.make_spectra(prot, w)
    ref = db.search(spec)
    assert ref.n_scored.max() > 1000
    got = idx.search(spec)
    assert_parity(got, ref, label=f"open evalue mode {ev_mode}")
    # same ranking, other e-values than the plain tail fit
    plain = hc.Index(prot.seq, prot.off, w.mods, dataclasses.replace(w.params, evalue_mode=0)).search(spec)
    np.testing.assert_array_equal(got.psm["key"], plain.psm["key"])
    real = got.psm["pid"] != 0xFFFFFFFF
    assert np.mean(got.psm["evalue"][real] != plain.psm["evalue"][real]) > 0.5


def test_evalue_options_shards_and_server(gpu):
    torch = gpu
    from paper_2102_02286_gb300 import shard
    w = with_mode(configs.UNEVEN_BATCHED, 3).with_proteins(300).with_spectra(150)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    ref = idx.search(spec)
    shards = [idx.shard(3, s) for s in range(3)]
    out = shard.local_sharded_search(shards, hc.DeviceBatch.from_spectra(spec))
    torch.cuda.synchronize()
    got = out.to_host(spec.n, w.params.top_k)
    np.testing.assert_array_equal(got.psm, ref.psm)
    parts = [s.search(spec) for s in shards]
    host = hc.merge_shards_host(3, spec.n, w.params.top_k, np.concatenate([p.psm for p in parts]),
                                sum(p.hist for p in parts), sum(p.n_scored for p in parts), 1, evalue_mode=3)
    np.testing.assert_array_equal(host.psm, ref.psm)
    for s in shards:
        s.close()
    server = hc.Server(idx)
    got = server.poll(server.submit(spec), -1)
    server.close()
    np.testing.assert_array_equal(got.psm, ref.psm)


def test_unknown_evalue_bits_are_rejected(gpu):
    w = configs.TINY_CLOSED.with_proteins(10)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    with pytest.raises(hc.HicopsError):
        hc.Index(prot.seq, prot.off, w.mods, dataclasses.replace(w.params, evalue_mode=4))
    psm = np.zeros(2 * 1 * w.params.top_k, hc.PSM_DTYPE)
    with pytest.raises(hc.HicopsError):
        hc.merge_shards_host(2, 1, w.params.top_k, psm, np.zeros((1, 256), np.uint32), np.zeros(1, np.uint32), 1,
                             evalue_mode=8)
