"""Sampled partial score distributions on the GPU (Sampling section: at most
s bins kept around the mean, tails pruned first) against the oracle's
sampling, and the sharded merge from sampled distributions against the
oracle's e-value on the summed samples."""
import dataclasses

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

from parity import EV_RTOL, assert_parity

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


def oracle_records(oracle, hist, s):
    rec = np.zeros((hist.shape[0], s + 1), np.uint32)
    for i, h in enumerate(hist):
        lo, ln, _ = oracle.hist_sample(h, s)
        rec[i, 0] = lo | (ln << 16)
        rec[i, 1:1 + ln] = h[lo:lo + ln]
    return rec


def random_histograms(rng, n):
    h = np.zeros((n, 256), np.uint32)
    for i in range(n):
        kind = i % 5
        if kind == 0:      # binned right-skewed scores, like a search's histogram
            x = rng.gumbel(rng.uniform(10, 200), rng.uniform(0.5, 20), size=int(rng.integers(1, 20000)))
            np.add.at(h[i], np.clip(x.astype(int), 0, 255), 1)
        elif kind == 1:    # equal counts everywhere they occur (tie rules)
            h[i, rng.choice(256, size=int(rng.integers(1, 256)))] = 3
        elif kind == 2:    # broad flat support
            h[i] = rng.integers(0, 5, size=256)
        elif kind == 3:    # one or two bins, at the edges too
            h[i, rng.choice([0, 255, int(rng.integers(256))])] = int(rng.integers(1, 1 << 28))
            if rng.random() < 0.5:
                h[i, int(rng.integers(256))] = 1
        # kind 4: empty
    return h


@pytest.mark.parametrize("s", [1, 2, 7, 64, 120, 256])
def test_device_sampling_equals_the_oracle(gpu, oracle_lib, s):
    torch = gpu
    rng = np.random.default_rng(s)
    h = random_histograms(rng, 500)
    want = oracle_records(oracle_lib, h, s)
    got = hc.hist_sample(torch.from_numpy(h.view(np.int32).reshape(-1)).cuda(), s)
    np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32).reshape(-1, s + 1), want)
    np.testing.assert_array_equal(hc.hist_sample(h, s), want)          # host buffers
    # assembly: the sum of the parts' kept counts
    parts = 3
    recs = np.concatenate([want[p::parts][: len(h) // parts] for p in range(parts)])
    n = len(h) // parts
    exp = sum(np.stack([oracle_lib.sampled(x, s) for x in h[p::parts][:n]]).astype(np.int64) for p in range(parts))
    np.testing.assert_array_equal(hc.hist_unsample(parts, n, recs, s), exp)


def test_unsample_rejects_foreign_records(gpu):
    rec = np.zeros((2, 9), np.uint32)
    rec[1, 0] = 250 | (8 << 16)          # bins 250..257: past the histogram
    with pytest.raises(hc.HicopsError) as e:
        hc.hist_unsample(1, 2, rec, 8)
    assert e.value.status == hc.EINVAL
    with pytest.raises(hc.HicopsError):
        hc.hist_sample(np.zeros((1, 256), np.uint32), 0)


@pytest.mark.parametrize("s", [120, 6])
def test_sampled_shard_merge_against_the_oracle(gpu, oracle_lib, s):
    """Three shards of an open search (thousands of candidates a spectrum)
    merged from their sampled distributions: rows, counts and keys exact;
    the e-value the oracle fits to the sum of the oracle's samples; at
    s = 120 nothing is dropped, so the result is the unsharded search's."""
    from paper_2102_02286_gb300 import shard
    w = configs.OPEN_MEDIUM.with_proteins(250).with_spectra(60)
    w = dataclasses.replace(w, params=dataclasses.replace(w.params, min_shared=2))
    prot, spec = synth.make_workload_inputs(w)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    P = 3
    shards = [idx.shard(P, p) for p in range(P)]
    db = hc.DeviceBatch.from_spectra(spec)
    got = shard.local_sharded_search(shards, db, sample=s).to_host(spec.n, w.params.top_k)
    exact = shard.local_sharded_search(shards, db).to_host(spec.n, w.params.top_k)
    odb = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    full = odb.search(spec)
    assert full.n_scored.max() > 1000
    parts = [odb.search(spec, n_shards=P, shard=p) for p in range(P)]
    hsum = sum(np.stack([oracle_lib.sampled(h, s) for h in p.hist]).astype(np.int64) for p in parts)
    np.testing.assert_array_equal(got.hist, hsum)
    np.testing.assert_array_equal(got.n_scored, full.n_scored)
    for f in ("pid", "key", "nb", "ny"):
        np.testing.assert_array_equal(got.psm[f], full.psm[f], err_msg=f)
    real = full.psm["pid"] != 0xFFFFFFFF
    for q in range(spec.n):
        ev = oracle_lib.evalue(hsum[q].astype(np.uint32), full.psm["key"][q], full.psm["pid"][q], w.params.evalue_mode)
        np.testing.assert_allclose(got.psm["evalue"][q][real[q]], ev[real[q]], rtol=EV_RTOL, atol=0)
    if s == 120:
        assert_parity(got, full, label="sampled merge, s = 120")
        np.testing.assert_array_equal(got.psm, exact.psm)
    else:
        drift = np.abs(got.psm["evalue"][real] / exact.psm["evalue"][real] - 1)
        assert np.any(hsum != full.hist) and drift.max() > 0
    for x in shards:
        x.close()
    idx.close()
