"""Database sharding across processes (paper: every process searches its own
partition of the database, Superstep 3; the partial score distributions are
added and the results assembled, Superstep 4).

One process per shard.  Every rank searches the whole batch against its shard
(``Index.shard``: pid = shard mod n_shards, rows carry global pids), then

1. ``publish_and_wait``: records in the process group's store that its
   partial is ready and waits, with a time limit, for every rank's partial of
   the step.  A rank that never publishes is reported by shard number
   (``ShardMissingError``) before any collective starts, so a dropped rank is
   an error, not a hang.
2. ``exchange``: sum-all-reduce of the per-spectrum histograms and candidate
   counts (the paper's addition of partial distributions) and all-gather of
   the top-k rows (32 B each, global pids keep ties exact).
3. ``hicops.merge_shards`` (device, ``hist_parts = 1``): top-k merge by
   (key desc, pid asc) and the e-value fit to the summed histogram.

``sharded_search`` runs the three steps on a device batch.  The result equals
the unsharded search bit for bit, because keys are exact integers and the
histograms are exact counts.

With ``sample = s`` the partial distributions leave each rank sampled
(Sampling section: at most s bins around the mean, tails pruned first;
``hicops.hist_sample``): the ranks all-gather the s + 1-word records instead
of all-reducing the 256-bin histograms, and ``hicops.hist_unsample`` adds
them up before the merge.  Top-k rows and candidate counts stay exact; the
e-value is fitted to the sum of the sampled distributions.
"""
from __future__ import annotations

import datetime
from typing import List, Optional

import numpy as np

from . import hicops as hc


class ShardMissingError(RuntimeError):
    """Some shard's partial result did not arrive within the time limit."""

    def __init__(self, missing: List[int], step: int, timeout_s: float):
        super().__init__(f"partial results of shard(s) {missing} missing after {timeout_s:g} s (step {step})")
        self.missing = missing
        self.step = step


def _key(step: int, rank: int) -> str:
    return f"hicops/partial/{step}/{rank}"


def publish_and_wait(store, step: int, rank: int, world: int, timeout_s: float) -> None:
    """Marks this rank's partial of `step` ready and waits for all of them."""
    store.set(_key(step, rank), "1")
    keys = [_key(step, r) for r in range(world)]
    try:
        store.wait(keys, datetime.timedelta(seconds=timeout_s))
    except Exception:
        missing = [r for r in range(world) if not store.check([keys[r]])]
        if not missing:       # arrived between the timeout and the check
            return
        raise ShardMissingError(missing, step, timeout_s) from None


def exchange(psm_bytes, hist, n_scored, group=None):
    """Collectives of the merge: returns (rows of every shard, shard-major,
    as one uint8 tensor; summed histograms; summed candidate counts).
    hist and n_scored are reduced in place (int32 tensors)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(psm_bytes) for _ in range(world)]
    dist.all_gather(parts, psm_bytes, group=group)
    dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(n_scored, op=dist.ReduceOp.SUM, group=group)
    return torch.cat(parts), hist, n_scored


def exchange_sampled(psm_bytes, rec, n_scored, group=None):
    """Collectives of the sampled merge: returns (rows of every shard; the
    sampled records of every shard, shard-major; summed candidate counts).
    n_scored is reduced in place."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(psm_bytes) for _ in range(world)]
    dist.all_gather(parts, psm_bytes, group=group)
    recs = [torch.empty_like(rec) for _ in range(world)]
    dist.all_gather(recs, rec, group=group)
    dist.all_reduce(n_scored, op=dist.ReduceOp.SUM, group=group)
    return torch.cat(parts), torch.cat(recs), n_scored


def sharded_search(shard_index: hc.Index, dev_batch: hc.DeviceBatch, store, step: int,
                   timeout_s: float = 30.0, group=None, stream=None, sample: int = 0) -> hc.DeviceResult:
    """This rank's shard search of the batch, the exchange and the merge
    (sample = s > 0: partial distributions exchanged sampled)."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n, k = dev_batch.n, shard_index.top_k
    part = hc.DeviceResult.alloc(n, k)
    shard_index.search_device(dev_batch, part, stream)
    rec = hc.hist_sample(part.hist, sample, stream) if sample else None
    import torch
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    publish_and_wait(store, step, rank, world, timeout_s)
    if sample:
        rows, recs, ns = exchange_sampled(part.psm, rec, part.n_scored, group)
        hist = hc.hist_unsample(world, n, recs, sample, stream)
    else:
        rows, hist, ns = exchange(part.psm, part.hist, part.n_scored, group)
    return hc.merge_shards(world, n, k, rows, hist, ns, 1, stream, shard_index.params.evalue_mode)


def lbe_parts(index: hc.Index, n_parts: int, upload: bool = True) -> List[hc.Index]:
    """The database split by the load-balancing partition (LBE with the Mod
    Distance, Superstep 1): one subset index per part."""
    part = index.partition_lbe(n_parts)
    return [index.subset(np.flatnonzero(part == s).astype(np.uint32), upload) for s in range(n_parts)]


def local_sharded_search(shards: List[hc.Index], dev_batch: hc.DeviceBatch,
                         stream=None, sample: int = 0) -> hc.DeviceResult:
    """All shards on this GPU, one after the other, merged by the device
    kernel from the per-shard histograms (hist_parts = n_shards), or with
    sample = s > 0 from their sampled records, added up first."""
    import torch
    n, k = dev_batch.n, shards[0].top_k
    P = len(shards)
    parts = [hc.DeviceResult.alloc(n, k) for _ in range(P)]
    for s, out in zip(shards, parts):
        s.search_device(dev_batch, out, stream)
    rows = torch.cat([p.psm for p in parts])
    ns = torch.cat([p.n_scored for p in parts])
    if sample:
        recs = torch.cat([hc.hist_sample(p.hist, sample, stream) for p in parts])
        hist = hc.hist_unsample(P, n, recs, sample, stream)
        ns = ns.view(P, n).sum(0, dtype=torch.int32)
        return hc.merge_shards(P, n, k, rows, hist, ns, 1, stream, shards[0].params.evalue_mode)
    hist = torch.cat([p.hist for p in parts])
    return hc.merge_shards(P, n, k, rows, hist, ns, P, stream, shards[0].params.evalue_mode)
