"""hicops_search_scratch: the search with its scratch in caller memory gives
exactly what hicops_search gives, needs no clearing between calls, and
refuses too little or misaligned scratch before it launches anything."""
import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
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
    return torch, w, idx, spec


def _same(got, exp):
    np.testing.assert_array_equal(got.psm, exp.psm)
    np.testing.assert_array_equal(got.hist, exp.hist)
    np.testing.assert_array_equal(got.n_scored, exp.n_scored)


@pytest.mark.parametrize("n", [1, 37, 300])
def test_matches_hicops_search(setup, n):
    """One spectrum (the most work units per spectrum), a ragged batch and the
    whole set, each in scratch filled with garbage beforehand."""
    torch, w, idx, spec = setup
    k = w.params.top_k
    sub = spec.subset(range(n))
    exp = idx.search(sub)
    need = idx.search_scratch_bytes(n)
    scratch = torch.full((need,), 0xA5, dtype=torch.uint8, device="cuda")
    out = hc.DeviceResult.alloc(n, k)
    idx.search_scratch(hc.DeviceBatch.from_spectra(sub), out, scratch)
    torch.cuda.synchronize()
    _same(out.to_host(n, k), exp)


def test_one_buffer_serves_successive_batches(setup):
    torch, w, idx, spec = setup
    k = w.params.top_k
    parts = [spec.subset(range(0, 200)), spec.subset(range(200, 300)), spec.subset(range(17, 18))]
    need = max(idx.search_scratch_bytes(p.n) for p in parts)
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    for p in parts:
        exp = idx.search(p)
        out = hc.DeviceResult.alloc(p.n, k)
        idx.search_scratch(hc.DeviceBatch.from_spectra(p), out, scratch)
        torch.cuda.synchronize()
        _same(out.to_host(p.n, k), exp)
    # without the optional outputs the rows are the same
    p = parts[1]
    out = hc.DeviceResult.alloc(p.n, k, hist=False)
    idx.search_scratch(hc.DeviceBatch.from_spectra(p), out, scratch)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.to_host(p.n, k).psm, idx.search(p).psm)


def test_refuses_short_or_misaligned_scratch(setup):
    torch, w, idx, spec = setup
    k = w.params.top_k
    sub = spec.subset(range(50))
    need = idx.search_scratch_bytes(sub.n)
    assert idx.search_scratch_bytes(0) == idx.search_scratch_bytes(1)
    # at least the binned peaks of every spectrum and its histogram
    assert need >= sub.n * (8 * w.params.top_n_peaks + 4 * hc.HIST_BINS)
    scratch = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    out = hc.DeviceResult.alloc(sub.n, k)
    db = hc.DeviceBatch.from_spectra(sub)
    launches = hc.kernel_launches()
    with pytest.raises(hc.HicopsError) as e:
        idx.search_scratch(db, out, scratch, nbytes=need - 256)
    assert e.value.status == hc.ENOMEM
    with pytest.raises(hc.HicopsError) as e:
        idx.search_scratch(db, out, scratch[1:], nbytes=need)
    assert e.value.status == hc.EINVAL
    assert hc.kernel_launches() == launches          # nothing was launched
    idx.search_scratch(db, out, scratch, nbytes=need)   # exactly enough
    torch.cuda.synchronize()
    _same(out.to_host(sub.n, k), idx.search(sub))
