"""hicops_search_noalloc: the search with its scratch in a fixed device array
gives exactly what hicops_search gives, call after call, without allocating."""
import dataclasses

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

pytestmark = pytest.mark.gpu

NOALLOC_MAX = 64   # HICOPS_NOALLOC_MAX_SPECTRA


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_2102_02286_gb300 import build as pkg_build
    pkg_build.build()
    w = configs.UNEVEN_BATCHED.with_proteins(400).with_spectra(100)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    return torch, w, idx, spec


def _same(got, exp):
    np.testing.assert_array_equal(got.psm, exp.psm)
    np.testing.assert_array_equal(got.hist, exp.hist)
    np.testing.assert_array_equal(got.n_scored, exp.n_scored)


def test_two_calls_in_a_row_match_hicops_search(setup):
    torch, w, idx, spec = setup
    k = w.params.top_k
    # a full batch, then a ragged one that reuses the same scratch
    parts = [spec.subset(range(0, NOALLOC_MAX)), spec.subset(range(NOALLOC_MAX, spec.n))]
    expected = [idx.search(p) for p in parts]             # hicops_search, host buffers
    batches = [hc.DeviceBatch.from_spectra(p) for p in parts]
    outs = [hc.DeviceResult.alloc(p.n, k) for p in parts]
    torch.cuda.synchronize()
    launches = hc.kernel_launches()
    for db, out in zip(batches, outs):
        idx.search_noalloc(db, out)
    torch.cuda.synchronize()
    assert hc.kernel_launches() > launches
    for p, out, exp in zip(parts, outs, expected):
        _same(out.to_host(p.n, k), exp)
    # a second pass over the same inputs, in the opposite order
    for o in outs:
        o.psm.zero_()
        o.hist.zero_()
        o.n_scored.zero_()
    # steady state: these calls take no device memory (the first calls of a
    # process may load modules, which does)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for db, out in reversed(list(zip(batches, outs))):
        idx.search_noalloc(db, out)
    torch.cuda.synchronize()
    for p, out, exp in zip(parts, outs, expected):
        _same(out.to_host(p.n, k), exp)
    assert torch.cuda.mem_get_info()[0] >= free_before


def test_rows_without_optional_outputs(setup):
    torch, w, idx, spec = setup
    sub = spec.subset(range(5, 25))
    exp = idx.search(sub)
    out = hc.DeviceResult.alloc(sub.n, w.params.top_k, hist=False)
    idx.search_noalloc(hc.DeviceBatch.from_spectra(sub), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.to_host(sub.n, w.params.top_k).psm, exp.psm)


def test_rejects_batches_over_the_limit(setup):
    torch, w, idx, spec = setup
    sub = spec.subset(range(NOALLOC_MAX + 1))
    out = hc.DeviceResult.alloc(sub.n, w.params.top_k)
    with pytest.raises(hc.HicopsError) as e:
        idx.search_noalloc(hc.DeviceBatch.from_spectra(sub), out)
    assert e.value.status == hc.EINVAL
    assert "HICOPS_NOALLOC_MAX_SPECTRA" in str(e.value)
    # an empty batch is a no-op
    empty = spec.subset([])
    idx.search_noalloc(hc.DeviceBatch.from_spectra(empty), hc.DeviceResult.alloc(1, w.params.top_k))


def _limit_case(case):
    """A 64-spectrum batch (the limit) of a configuration that stresses the
    scratch: many work units per spectrum (seg_pids set, so hicops_search
    splits windows into up to 64 units where the fixed array allows 16), or
    the widest query-bin stride (fragment tolerance of 1 bin on 341 retained
    peaks: 1,023 bins a spectrum)."""
    if case == "seg_pids":
        w = configs.UNEVEN_BATCHED.with_proteins(400).with_spectra(NOALLOC_MAX)
        cfg = hc.SearchConfig(0, 0, 0, 1 << 10)
    else:
        w = configs.OPEN_MEDIUM_TOL.with_proteins(300).with_spectra(NOALLOC_MAX)
        w = dataclasses.replace(w, params=dataclasses.replace(w.params, top_n_peaks=341),
                                spectra=dataclasses.replace(w.spectra, target_peaks=(380, 500)))
        cfg = None
    return w, cfg


@pytest.mark.parametrize("case", ["seg_pids", "tol_widest"])
def test_matches_hicops_search_at_the_limit(setup, case):
    torch = setup[0]
    w, cfg = _limit_case(case)
    prot = synth.make_proteome(w.n_proteins, w.db_seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    if cfg is not None:
        idx.set_config(cfg)
    spec = synth.make_spectra(prot, w)
    assert spec.n == NOALLOC_MAX
    exp = idx.search(spec)
    assert int(exp.n_scored.sum()) > 0
    db = hc.DeviceBatch.from_spectra(spec)
    out = hc.DeviceResult.alloc(spec.n, w.params.top_k)
    for _ in range(2):                      # two calls in a row on the shared array
        out.psm.zero_()
        out.hist.zero_()
        out.n_scored.zero_()
        idx.search_noalloc(db, out)
        torch.cuda.synchronize()
        _same(out.to_host(spec.n, w.params.top_k), exp)
    idx.close()
