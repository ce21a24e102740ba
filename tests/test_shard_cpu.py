"""Database sharding on CPU ranks: the sharding invariant on the oracle, the
exchange over gloo (world size 2) and dropped-rank detection.

The paper splits the database across processes, each searching every
spectrum against its partition, and adds the partial score distributions
(Superstep 3 and 4).  With exact integer keys and exact histogram counts, the
combined result must equal the unsharded search bit for bit."""
import dataclasses
import multiprocessing as mp
import os
import socket
import traceback

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth

W = configs.TINY_CLOSED.with_proteins(80).with_spectra(24)
# an open search with min_shared 2: score histograms over a dozen bins, so a
# small s drops some
W_OPEN = dataclasses.replace(configs.OPEN_MEDIUM.with_proteins(60).with_spectra(16),
                             params=dataclasses.replace(configs.OPEN_MEDIUM.params, min_shared=2))


def _inputs(w=W):
    prot = synth.make_proteome(w.n_proteins, w.seed, w.protein_len)
    spec = synth.make_spectra(prot, w)
    return prot, spec


def reference_merge(oracle, parts, hist_sum, k, evalue_mode=W.params.evalue_mode):
    """Top-k by (key desc, pid asc) over the shards' rows and the e-value fit
    on the summed histogram: the combination step written out plainly."""
    n = parts[0].shape[0]
    out = np.zeros((n, k), dtype=oracle.PSM_DTYPE)
    for q in range(n):
        rows = np.concatenate([p[q] for p in parts])
        rows = rows[rows["pid"] != np.iinfo(np.uint32).max]
        order = sorted(range(len(rows)), key=lambda i: (-int(rows[i]["key"]), int(rows[i]["pid"])))
        top = rows[order[:k]]
        out[q]["pid"] = np.iinfo(np.uint32).max
        out[q]["key"] = np.iinfo(np.int64).min
        out[q]["evalue"] = np.inf
        out[q][:len(top)] = top
        ev = oracle.evalue(hist_sum[q], out[q]["key"], out[q]["pid"], evalue_mode)
        out[q]["evalue"] = ev
    return out


def _same_rows(a, b):
    for f in ("pid", "nb", "ny", "S", "key"):
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)
    np.testing.assert_array_equal(a["evalue"], b["evalue"])


@pytest.mark.parametrize("n_shards", [2, 3])
def test_sharding_invariant_on_the_oracle(oracle_lib, n_shards):
    prot, spec = _inputs()
    db = oracle_lib.OracleDb(prot.seq, prot.off, W.mods, W.params)
    full = db.search(spec)
    parts = [db.search(spec, n_shards=n_shards, shard=s) for s in range(n_shards)]
    hist = sum(p.hist.astype(np.int64) for p in parts)
    np.testing.assert_array_equal(hist, full.hist)
    np.testing.assert_array_equal(sum(p.n_scored.astype(np.int64) for p in parts), full.n_scored)
    for s, p in enumerate(parts):   # each shard's rows are its own entries
        real = p.psm["pid"] != np.iinfo(np.uint32).max
        assert np.all(p.psm["pid"][real] % n_shards == s)
    merged = reference_merge(oracle_lib, [p.psm for p in parts], hist.astype(np.uint32), W.params.top_k)
    _same_rows(merged, full.psm)
    assert full.n_scored.sum() > 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def pack_records(hist, s, oracle):
    """The library's record layout (word 0 = lo | len << 16, then the kept
    counts), filled from the oracle's sampling."""
    rec = np.zeros((hist.shape[0], s + 1), np.uint32)
    for i, h in enumerate(hist):
        lo, ln, _ = oracle.hist_sample(h, s)
        rec[i, 0] = lo | (ln << 16)
        rec[i, 1:1 + ln] = h[lo:lo + ln]
    return rec


def unpack_sum(recs, world, n, s):
    out = np.zeros((n, 256), np.int64)
    r = recs.reshape(world, n, s + 1)
    for p in range(world):
        for q in range(n):
            lo, ln = int(r[p, q, 0]) & 0xFFFF, int(r[p, q, 0]) >> 16
            out[q, lo:lo + ln] += r[p, q, 1:1 + ln]
    return out


def _rank_main(rank, world, port, mode, q):
    try:
        import datetime
        import torch
        import torch.distributed as dist
        import oracle
        from paper_2102_02286_gb300 import shard
        store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=30))
        dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
        w = W_OPEN if mode.startswith("sampled") else W
        prot, spec = _inputs(w)
        oracle.build()
        db = oracle.OracleDb(prot.seq, prot.off, w.mods, w.params)
        part = db.search(spec, n_shards=world, shard=rank)
        if mode == "drop" and rank == 1:
            q.put((rank, "dropped"))
            q.close()
            q.join_thread()
            os._exit(0)               # leaves between steps: nothing of it is in flight
        try:
            shard.publish_and_wait(store, step=0, rank=rank, world=world, timeout_s=3.0)
        except shard.ShardMissingError as e:
            q.put((rank, ("missing", e.missing)))
            q.close()
            q.join_thread()
            os._exit(0)
        rows = torch.from_numpy(part.psm.view(np.uint8).reshape(-1).copy())
        ns = torch.from_numpy(part.n_scored.astype(np.int32))
        if mode.startswith("sampled"):
            # the partial distributions leave the rank sampled (Sampling section)
            s = int(mode.split(":")[1])
            rec = torch.from_numpy(pack_records(part.hist, s, oracle).view(np.int32))
            all_rows, recs, ns = shard.exchange_sampled(rows, rec, ns)
            assert recs.shape[0] == world * spec.n
            hsum = unpack_sum(recs.numpy().view(np.uint32), world, spec.n, s)
            parts = all_rows.numpy().view(oracle.PSM_DTYPE).reshape(world, spec.n, w.params.top_k)
            full = db.search(spec)
            mine = [db.search(spec, n_shards=world, shard=r) for r in range(world)]
            want = sum(np.stack([oracle.sampled(h, s) for h in m.hist]).astype(np.int64) for m in mine)
            np.testing.assert_array_equal(hsum, want)
            np.testing.assert_array_equal(ns.numpy(), full.n_scored.astype(np.int32))
            merged = reference_merge(oracle, list(parts), hsum.astype(np.uint32), w.params.top_k, w.params.evalue_mode)
            for f in ("pid", "nb", "ny", "key"):
                np.testing.assert_array_equal(merged[f], full.psm[f], err_msg=f)
            if s >= 120:      # these histograms span fewer bins: nothing was dropped
                np.testing.assert_array_equal(hsum, full.hist.astype(np.int64))
                np.testing.assert_array_equal(merged["evalue"], full.psm["evalue"])
            else:             # some partial distributions lost tail bins
                assert np.any(hsum != full.hist.astype(np.int64))
            dist.barrier()
            dist.destroy_process_group()
            q.put((rank, "ok"))
            return
        hist = torch.from_numpy(part.hist.astype(np.int32))
        all_rows, hist, ns = shard.exchange(rows, hist, ns)
        parts = all_rows.numpy().view(oracle.PSM_DTYPE).reshape(world, spec.n, W.params.top_k)
        full = db.search(spec)
        np.testing.assert_array_equal(hist.numpy(), full.hist.astype(np.int32))
        np.testing.assert_array_equal(ns.numpy(), full.n_scored.astype(np.int32))
        merged = reference_merge(oracle, list(parts), hist.numpy().astype(np.uint32), W.params.top_k)
        _same_rows(merged, full.psm)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, "ok"))
    except Exception:
        q.put((rank, traceback.format_exc()))


def _run(world, mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, mode, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = {}
    for _ in range(world):
        r, v = q.get(timeout=120)
        res[r] = v
    for p in ps:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return res


def test_exchange_over_gloo_matches_unsharded(oracle_lib):
    res = _run(2, "ok")
    assert res == {0: "ok", 1: "ok"}, res


@pytest.mark.parametrize("s", [120, 3])
def test_sampled_exchange_over_gloo(oracle_lib, s):
    """The partial distributions exchanged as s-bin samples: exact rows and
    counts, the e-value fitted to the sum of the samples (equal to the
    unsharded search's when no bin is dropped)."""
    res = _run(2, f"sampled:{s}")
    assert res == {0: "ok", 1: "ok"}, res


def test_dropped_rank_is_an_error_not_a_hang(oracle_lib):
    res = _run(2, "drop")
    assert res[1] == "dropped"
    assert res[0] == ("missing", [1]), res
