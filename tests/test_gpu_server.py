"""The serving loop: continuous batching over a device-memory pool and several
streams; every request's result is the same alone and in the mix."""
import dataclasses
import threading
import time

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
    w = configs.SERVING_STREAM.with_proteins(150).with_spectra(600)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    spec = synth.make_spectra(prot, w)
    return w, idx, spec


def split_requests(n, rng, max_size=64):
    cuts, i = [], 0
    while i < n:
        m = int(min(n - i, np.exp(rng.uniform(0, np.log(max_size)))))
        cuts.append((i, i + max(1, m)))
        i += max(1, m)
    return cuts


def test_identity_alone_vs_mix(setup):
    w, idx, spec = setup
    rng = np.random.default_rng(1)
    reqs = split_requests(spec.n, rng)
    alone = [idx.search(spec.subset(range(a, b))) for a, b in reqs]
    srv = hc.Server(idx, n_slots=3, slot_spectra=256)
    tickets = []
    for a, b in reqs:
        tickets.append(srv.submit(spec.subset(range(a, b))))
    for t, ref in zip(tickets, alone):
        got = srv.poll(t, timeout_ms=120000)
        assert got is not None
        np.testing.assert_array_equal(got.psm, ref.psm)
        np.testing.assert_array_equal(got.hist, ref.hist)
        np.testing.assert_array_equal(got.n_scored, ref.n_scored)
    st = srv.stats()
    assert st.completed == len(reqs) and st.spectra == spec.n
    assert st.launches < len(reqs)          # requests were packed together
    srv.close()


def test_packed_requests_match_the_oracle(setup, oracle_lib):
    """The server's own work (requests packed into shared launches, each
    request's spectrum indices rebased, its histogram rows sliced out)
    against the oracle, on a mix of +-10 / +-500 Da windows and 50-500 peaks:
    parity per request."""
    w, idx, spec = setup
    assert set(np.unique(spec.tol_da)) == {10.0, 500.0}
    npk = np.diff(spec.peak_off.astype(np.int64))
    assert npk.min() < 100 and npk.max() > 400
    rng = np.random.default_rng(7)
    reqs = split_requests(spec.n, rng, max_size=96)
    srv = hc.Server(idx, n_slots=3, slot_spectra=256)
    tickets = [srv.submit(spec.subset(range(a, b))) for a, b in reqs]
    got = [srv.poll(t, timeout_ms=120000) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st.completed == len(reqs) and st.launches < len(reqs)   # packed
    # the oracle (all pairs, +-500 Da windows of a 0.7M-entry database) on
    # each request's first and last spectrum and on the most peaks of each
    # window class
    sel = {a for a, _ in reqs} | {b - 1 for _, b in reqs}
    sel |= {int(np.flatnonzero(spec.tol_da == t)[np.argmax(npk[spec.tol_da == t])]) for t in (10.0, 500.0)}
    sel = np.array(sorted(sel), dtype=np.uint32)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    ref = db.search(spec, sel=sel)
    rows = 0
    for (a, b), g in zip(reqs, got):
        pos = np.flatnonzero((sel >= a) & (sel < b))
        r = oracle_lib.SearchResult(ref.psm[pos], ref.hist[pos], ref.n_scored[pos], ref.lo[pos], ref.hi[pos])
        rows += assert_parity(g, r, sel=sel[pos] - a, label=f"request [{a}, {b})")
    assert rows > len(sel)


def test_concurrent_submitters(setup):
    w, idx, spec = setup
    whole = idx.search(spec)
    srv = hc.Server(idx, n_slots=4, slot_spectra=128)
    results = {}
    errors = []

    def client(c):
        try:
            rng = np.random.default_rng(100 + c)
            for a, b in split_requests(spec.n, rng, 16)[c::4]:
                t = srv.submit(spec.subset(range(a, b)))
                time.sleep(rng.uniform(0, 0.002))
                results[(a, b)] = srv.poll(t, timeout_ms=120000)
        except Exception as e:   # pragma: no cover - reported below
            errors.append(e)

    th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    for (a, b), r in results.items():
        np.testing.assert_array_equal(r.psm["pid"], whole.psm["pid"][a:b])
        np.testing.assert_array_equal(r.psm["key"], whole.psm["key"][a:b])
        np.testing.assert_array_equal(r.hist, whole.hist[a:b])
    srv.close()


def test_errors_and_cancel(setup):
    w, idx, spec = setup
    srv = hc.Server(idx, n_slots=1, slot_spectra=32)
    with pytest.raises(hc.HicopsError) as e:
        srv.submit(spec.subset(range(33)))       # over the slot size
    assert e.value.status == hc.EINVAL
    with pytest.raises(hc.HicopsError):
        load = hc.load()
        st = load.hicops_server_poll(srv.h, 987654321, 0, None, None, None)
        hc._check(st)
    ts = [srv.submit(spec.subset(range(i, i + 30))) for i in range(0, 300, 30)]
    st = srv.cancel(ts[-1])
    assert st in (hc.OK, hc.EBUSY)
    for t in ts[:-1]:
        assert srv.poll(t, timeout_ms=120000) is not None
    if st == hc.OK:
        with pytest.raises(hc.HicopsError) as e:
            srv.poll(ts[-1], timeout_ms=1000)
        assert e.value.status == hc.ECANCELLED
    else:
        assert srv.poll(ts[-1], timeout_ms=120000) is not None
    srv.close()
    with pytest.raises(hc.HicopsError):
        hc.Server(idx, n_slots=2, slot_spectra=1024, memory_budget=1024)   # budget below one launch
    with pytest.raises(hc.HicopsError) as e:
        hc.Server(idx, n_slots=65)                                           # more launches in flight than allowed
    assert e.value.status == hc.EINVAL
    # peak offsets that decrease are refused at submission
    srv = hc.Server(idx, n_slots=1, slot_spectra=32)
    sub = spec.subset(range(4))
    off = sub.peak_off.astype(np.uint64).copy()
    off[2] = off[4] + 1000
    with pytest.raises(hc.HicopsError) as e:
        srv.submit(dataclasses.replace(sub, peak_off=off))
    assert e.value.status == hc.EINVAL and "decrease" in str(e.value)
    srv.close()


def test_admission_by_device_memory(setup):
    """A pool that holds about one and a half of the largest request's
    launches: requests wait for memory that launches in flight give back (the
    server counts the waits), the pool never holds more than its size, every
    result is the one the request gets alone, and a request whose launch
    alone exceeds the pool is refused at submission."""
    w, idx, spec = setup
    k = w.params.top_k
    rng = np.random.default_rng(3)
    reqs = split_requests(spec.n, rng, max_size=64)
    alone = [idx.search(spec.subset(range(a, b))) for a, b in reqs]

    def launch_bound(a, b):
        # the search's scratch, the spectra, the PSM rows, histograms and
        # counts, and the 256-byte rounding of each piece
        n, npk = b - a, int(spec.peak_off[b] - spec.peak_off[a])
        return (idx.search_scratch_bytes(n) + 8 * (n + 1) + 8 * npk + 17 * n + n * (32 * k + 4 * 256 + 4)
                + 9 * 256)

    budget = 3 * max(launch_bound(a, b) for a, b in reqs) // 2
    srv = hc.Server(idx, n_slots=3, slot_spectra=256, memory_budget=budget)
    tickets = [srv.submit(spec.subset(range(a, b))) for a, b in reqs]
    for t, ref in zip(tickets, alone):
        got = srv.poll(t, timeout_ms=120000)
        assert got is not None
        np.testing.assert_array_equal(got.psm, ref.psm)
        np.testing.assert_array_equal(got.hist, ref.hist)
        np.testing.assert_array_equal(got.n_scored, ref.n_scored)
    st = srv.stats()
    assert st.completed == len(reqs) and st.spectra == spec.n
    assert 0 < st.pool_peak <= st.pool_bytes <= budget
    assert st.memory_waits > 0
    with pytest.raises(hc.HicopsError) as e:
        srv.submit(spec.subset(range(256)))
    assert e.value.status == hc.EINVAL and "pool" in str(e.value)
    srv.close()
