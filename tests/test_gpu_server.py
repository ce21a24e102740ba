"""The serving loop: continuous batching across slots; every request's
result is the same alone and in the mix."""
import threading
import time

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
        hc.Server(idx, n_slots=2, slot_spectra=1024, memory_budget=1024)   # budget below one slot
