"""The batched form: launch shapes, reusable plans, CUDA-graph replay and the
autotuner never change results."""
import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

from parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_2102_02286_gb300 import build as pkg_build
    pkg_build.build()
    w = configs.UNEVEN_BATCHED.with_proteins(400).with_spectra(300)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    ref = idx.search(spec)
    return torch, w, prot, idx, spec, ref


def same(a, b):
    np.testing.assert_array_equal(a.psm, b.psm)
    np.testing.assert_array_equal(a.hist, b.hist)
    np.testing.assert_array_equal(a.n_scored, b.n_scored)


@pytest.mark.parametrize("threads", [256, 384, 512])
@pytest.mark.parametrize("chunk_entries", [1, 2, 6, 16])
@pytest.mark.parametrize("seg_pids", [0, 1 << 14, 1 << 16])
def test_launch_shapes_identical(setup, threads, chunk_entries, seg_pids):
    torch, w, prot, idx, spec, ref = setup
    idx.set_config(hc.SearchConfig(threads, chunk_entries, 0, seg_pids))
    try:
        same(idx.search(spec), ref)
    finally:
        idx.set_config(None)


def test_plan_and_graph_replay(setup):
    torch, w, prot, idx, spec, ref = setup
    db = hc.DeviceBatch.from_spectra(spec)
    out = hc.DeviceResult.alloc(spec.n, w.params.top_k)
    stream = torch.cuda.Stream()
    plan = idx.plan(spec.n)
    with torch.cuda.stream(stream):
        plan.search(db, out, stream, graph=False)
    stream.synchronize()
    same(out.to_host(spec.n, w.params.top_k), ref)
    for i in range(3):   # capture, then two replays
        out.psm.zero_()
        out.hist.zero_()
        with torch.cuda.stream(stream):
            plan.search(db, out, stream, graph=True)
        stream.synchronize()
        same(out.to_host(spec.n, w.params.top_k), ref)
    plan.close()


def test_plan_small_batch_splits_windows(setup, oracle_lib):
    torch, w, prot, idx, spec, ref = setup
    sub = spec.subset([3, 7])
    db = hc.DeviceBatch.from_spectra(sub)
    out = hc.DeviceResult.alloc(sub.n, w.params.top_k)
    plan = idx.plan(64)
    plan.search(db, out, torch.cuda.current_stream(), graph=False)
    torch.cuda.synchronize()
    got = out.to_host(sub.n, w.params.top_k)
    exp = ref.psm[[3, 7]].copy()
    exp["query"] = np.arange(2)[:, None]        # rows carry the index within their own batch
    np.testing.assert_array_equal(got.psm, exp)
    np.testing.assert_array_equal(got.hist, ref.hist[[3, 7]])
    odb = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    assert_parity(got, odb.search(sub), label="plan small batch")
    plan.close()


def test_autotune_keeps_results(setup):
    torch, w, prot, idx, spec, ref = setup
    db = hc.DeviceBatch.from_spectra(spec)
    best, ms = idx.autotune(db)
    assert best.threads in (256, 384, 512) and 1 <= best.chunk_entries <= 16 and ms > 0
    try:
        same(idx.search(spec), ref)
    finally:
        idx.set_config(None)


def test_plan_rejects_oversized_batch(setup):
    torch, w, prot, idx, spec, ref = setup
    plan = idx.plan(4)
    db = hc.DeviceBatch.from_spectra(spec.subset(range(5)))
    out = hc.DeviceResult.alloc(5, w.params.top_k)
    with pytest.raises(hc.HicopsError) as e:
        plan.search(db, out, graph=False)
    assert e.value.status == hc.EINVAL
    plan.close()
