"""Database sharding on CPU ranks: the sharding invariant on the oracle, the
exchange over gloo (world size 2) and dropped-rank detection.

The paper splits the database across processes, each searching every
spectrum against its partition, and adds the partial score distributions
(Superstep 3 and 4).  With exact integer keys and exact histogram counts, the
combined result must equal the unsharded search bit for bit."""
import multiprocessing as mp
import os
import socket
import traceback

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth

W = configs.TINY_CLOSED.with_proteins(80).with_spectra(24)


def _inputs():
    prot = synth.make_proteome(W.n_proteins, W.seed, W.protein_len)
    spec = synth.make_spectra(prot, W)
    return prot, spec


def reference_merge(oracle, parts, hist_sum, k):
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
        ev = oracle.evalue(hist_sum[q], out[q]["key"], out[q]["pid"], W.params.evalue_mode)
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


def _rank_main(rank, world, port, mode, q):
    try:
        import datetime
        import torch
        import torch.distributed as dist
        import oracle
        from paper_2102_02286_gb300 import shard
        store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=30))
        dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
        prot, spec = _inputs()
        oracle.build()
        db = oracle.OracleDb(prot.seq, prot.off, W.mods, W.params)
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
        hist = torch.from_numpy(part.hist.astype(np.int32))
        ns = torch.from_numpy(part.n_scored.astype(np.int32))
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


def test_dropped_rank_is_an_error_not_a_hang(oracle_lib):
    res = _run(2, "drop")
    assert res[1] == "dropped"
    assert res[0] == ("missing", [1]), res
