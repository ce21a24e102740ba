"""Database shards on one GPU merged by the device kernel: the combined
result equals the unsharded search bit for bit (paper: partitions searched
independently, partial distributions added; Superstep 3 and 4)."""
import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

from parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_2102_02286_gb300 import build as pkg_build
    pkg_build.build()
    w = configs.UNEVEN_BATCHED.with_proteins(400).with_spectra(200)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    return torch, w, prot, idx, spec, idx.search(spec)


def _same(a, b):
    np.testing.assert_array_equal(a.psm, b.psm)
    np.testing.assert_array_equal(a.hist, b.hist)
    np.testing.assert_array_equal(a.n_scored, b.n_scored)


@pytest.mark.parametrize("n_shards", [2, 3, 5])
def test_device_shards_merge_to_the_unsharded_search(setup, n_shards):
    from paper_2102_02286_gb300 import shard
    torch, w, prot, idx, spec, ref = setup
    shards = [idx.shard(n_shards, s) for s in range(n_shards)]
    assert sum(s.stats().n_peptides for s in shards) == idx.stats().n_peptides
    db = hc.DeviceBatch.from_spectra(spec)
    out = shard.local_sharded_search(shards, db)
    torch.cuda.synchronize()
    _same(out.to_host(spec.n, w.params.top_k), ref)
    # each shard alone: its own candidates, global pids of its residue class
    part = shards[1].search(spec)
    real = part.psm["pid"] != np.iinfo(np.uint32).max
    assert np.all(part.psm["pid"][real] % n_shards == 1)
    for s in shards:
        s.close()


def test_host_merge_and_reduced_histograms(setup):
    torch, w, prot, idx, spec, ref = setup
    shards = [idx.shard(2, s) for s in range(2)]
    parts = [s.search(spec) for s in shards]
    psm = np.concatenate([p.psm for p in parts])
    # per-shard histograms summed by the merge
    got = hc.merge_shards_host(2, spec.n, w.params.top_k, psm, np.concatenate([p.hist for p in parts]),
                               np.concatenate([p.n_scored for p in parts]), 2)
    _same(got, ref)
    # histograms already reduced (as after an all-reduce)
    got = hc.merge_shards_host(2, spec.n, w.params.top_k, psm, parts[0].hist + parts[1].hist,
                               parts[0].n_scored + parts[1].n_scored, 1)
    _same(got, ref)


def test_sharded_against_the_oracle(setup, oracle_lib):
    torch, w, prot, idx, spec, ref = setup
    sub = spec.subset(range(40))
    shards = [idx.shard(3, s) for s in range(3)]
    parts = [s.search(sub) for s in shards]
    got = hc.merge_shards_host(3, sub.n, w.params.top_k, np.concatenate([p.psm for p in parts]),
                               np.concatenate([p.hist for p in parts]),
                               np.concatenate([p.n_scored for p in parts]), 3)
    odb = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    assert_parity(got, odb.search(sub), label="3 shards merged")


def test_shard_peptides_use_global_pids(setup):
    torch, w, prot, idx, spec, ref = setup
    s = idx.shard(4, 3, upload=False)
    for g in (3, 7, 4 * 100 + 3):
        assert s.peptide(g) == idx.peptide(g)
    with pytest.raises(hc.HicopsError):
        s.peptide(4)


def test_shard_and_merge_argument_checks(setup):
    torch, w, prot, idx, spec, ref = setup
    for bad in ((0, 0), (65, 0), (2, 2)):
        with pytest.raises(hc.HicopsError) as e:
            idx.shard(*bad, upload=False)
        assert e.value.status == hc.EINVAL
    s = idx.shard(2, 0, upload=False)
    with pytest.raises(hc.HicopsError):
        s.shard(2, 0, upload=False)          # a shard is not split again
    psm = np.zeros((2 * 3, w.params.top_k), hc.PSM_DTYPE)
    hist = np.zeros((2 * 3, 256), np.uint32)
    ns = np.zeros(2 * 3, np.uint32)
    with pytest.raises(hc.HicopsError) as e:
        hc.merge_shards_host(2, 3, w.params.top_k, psm, hist, ns, 3)   # hist_parts neither 1 nor 2
    assert e.value.status == hc.EINVAL


@pytest.mark.parametrize("n_parts", [3, 8])
def test_lbe_parts_merge_to_the_unsharded_search_and_balance(setup, n_parts):
    """The load-balancing partition (LBE with the Mod Distance): its parts
    merge to the unsharded search bit for bit, and the index entries inside
    the spectra's windows (the search's work) are spread evenly over the
    parts, unlike contiguous mass ranges."""
    from paper_2102_02286_gb300 import shard
    torch, w, prot, idx, spec, ref = setup
    parts = shard.lbe_parts(idx, n_parts)
    P = idx.stats().n_peptides
    assert sum(p.stats().n_peptides for p in parts) == P
    out = shard.local_sharded_search(parts, hc.DeviceBatch.from_spectra(spec))
    torch.cuda.synchronize()
    _same(out.to_host(spec.n, w.params.top_k), ref)
    work = np.array([float(p.search_work(spec)[3].sum()) for p in parts])
    cuts = np.linspace(0, P, n_parts + 1).astype(np.int64)
    chunks = [idx.subset(np.arange(cuts[s], cuts[s + 1], dtype=np.uint32)) for s in range(n_parts)]
    cwork = np.array([float(c.search_work(spec)[3].sum()) for c in chunks])
    assert work.sum() == cwork.sum()
    cv, ccv = work.std() / work.mean(), cwork.std() / cwork.mean()
    assert cv < 0.05 and ccv > 4 * cv, (cv, ccv)
    for s in parts + chunks:
        s.close()


def test_saved_index_searches_like_the_original(setup, tmp_path):
    """A checkpointed index, loaded and uploaded again, gives the same results."""
    torch, w, prot, idx, spec, ref = setup
    path = str(tmp_path / "db.hix")
    idx.save(path)
    back = hc.Index.load(path)
    _same(back.search(spec), ref)
    back.close()
