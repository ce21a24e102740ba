#!/usr/bin/env python3
"""Benchmark of the search hot path: spectra searched per second on GB300.

One step = one hicops_search call over the whole query batch of the
workload (preprocessing, precursor window, shared-peak accumulation,
scoring, top-k, histogram, e-value), inputs resident in HBM, L2 flushed
between steps.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload open_medium]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

With N > 1 (torchrun) every rank searches its own batch against a replica
of the index (no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2102_02286_gb300 import configs, synth  # noqa: E402

L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default="open_medium", choices=[w.name for w in configs.WORKLOADS])
    ap.add_argument("--spectra", type=int, default=0, help="override the workload's spectra per step")
    ap.add_argument("--proteins", type=int, default=0, help="override the workload's protein count")
    ap.add_argument("--oracle-spectra", type=int, default=3, help="CPU-baseline sample size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--tune-spectra", type=int, default=20000, help="autotuner sample (0 = default shape)")
    return ap.parse_args()


def workload(args):
    w = configs.BY_NAME[args.workload]
    if args.proteins:
        w = w.with_proteins(args.proteins)
    if args.spectra:
        w = w.with_spectra(args.spectra)
    return w


def workload_desc(w):
    return f"{w.name}: {w.description}"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def search_traffic_record():
    """ncu DRAM bytes per spectrum of the search kernel, valid while the
    search source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "search_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    src = os.path.join(ROOT, "paper_2102_02286_gb300", "csrc", "search.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("search_cu_sha256") != h or rec.get("workload") is None:
        return None
    return rec


def cpu_baseline(w, prot, spec, n_sample: int):
    import oracle
    db = oracle.OracleDb(prot.seq, prot.off, w.mods, w.params)
    rng = np.random.default_rng(11)
    sel = np.sort(rng.choice(spec.n, size=min(n_sample, spec.n), replace=False)).astype(np.uint32)
    t0 = time.perf_counter()
    db.search(spec, sel=sel)
    dt = time.perf_counter() - t0
    return {"value": len(sel) / dt, "unit": "spectra/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(sel)} spectra of {w.name} (same index and spectra as the timed run), "
                      f"single-threaded FP64 all-pairs oracle, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workload(args)
    prot = synth.make_proteome(w.n_proteins, w.seed, w.protein_len)
    spec = synth.make_spectra(prot, w)
    db = oracle.OracleDb(prot.seq, prot.off, w.mods, w.params)
    per_step = max(1, args.oracle_spectra // 3)
    rng = np.random.default_rng(13)
    times = []
    for step in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(spec.n, size=per_step, replace=False)).astype(np.uint32)
        t0 = time.perf_counter()
        db.search(spec, sel=sel)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": "spectra/s searched", "value": value, "unit": "spectra/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(w), "spectra_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "spectra/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} spectra per step of {w.name}"},
            "e2e": {"value": value, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_2102_02286_gb300 import build as pkg_build
    from paper_2102_02286_gb300 import hicops as hc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        pkg_build.build()
    if world > 1:
        dist.barrier()
    hc.load()
    w = workload(args)
    t0 = time.perf_counter()
    prot = synth.make_proteome(w.n_proteins, w.seed, w.protein_len)
    spec = synth.make_spectra(prot, w, seed=w.seed + 7919 * rank)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params)
    t_index = time.perf_counter() - t0
    st = idx.stats()
    n = spec.n
    k = w.params.top_k

    # algorithmic work per spectrum (exact, from the CSR)
    lo, hi, npk, hits = idx.search_work(spec)
    H = int(hits.sum())
    NP = int(npk.sum())
    # search kernel bytes: 4 per index entry in the window, 16 (two bucket
    # offsets) + 8 (bin, iq) per retained peak, 16 per top-k slot, 1 KB histogram
    search_bytes = 4 * H + 24 * NP + (16 * k + 4 * 256) * n
    # whole-step bytes: the above plus the raw peaks in (8 B each) and the
    # precursor fields (17 B), PSM rows out (32 B each)
    raw_peaks = int(spec.peak_off[-1])
    step_bytes = search_bytes + 8 * raw_peaks + 17 * n + 32 * k * n

    dev_batch = hc.DeviceBatch.from_spectra(spec)
    out = hc.DeviceResult.alloc(n, k)
    stream = torch.cuda.current_stream()
    # launch shape from the autotuner, on a sample of the batch
    t0 = time.perf_counter()
    tune_batch = hc.DeviceBatch.from_spectra(spec.subset(np.arange(min(n, args.tune_spectra))))
    shape, tune_ms = idx.autotune(tune_batch) if args.tune_spectra > 0 else (hc.SearchConfig(), 0.0)
    t_tune = time.perf_counter() - t0
    del tune_batch
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    idx.set_timing(True)
    for _ in range(args.warmup):
        idx.search_device(dev_batch, out, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = hc.kernel_launches()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    search_ms, prep_ms, merge_ms = [], [], []
    for i in range(args.steps):
        flush.zero_()                      # L2 flush, outside the step's events
        starts[i].record(stream)
        idx.search_device(dev_batch, out, stream)
        ends[i].record(stream)
        t = idx.last_timing()              # waits for this step
        search_ms.append(t.search_ms)
        prep_ms.append(t.prep_ms)
        merge_ms.append(t.merge_ms)
    torch.cuda.synchronize()
    launches = hc.kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    max_total_ms = float(tt.item())
    value = world * n * args.steps / (max_total_ms / 1000.0)

    # end to end through the C ABI with pinned host buffers (copies inside)
    pinned = {}
    for name, arr in (("peak_off", spec.peak_off), ("mz", spec.mz), ("intensity", spec.intensity),
                      ("prec_mz", spec.prec_mz), ("charge", spec.charge), ("tol_da", spec.tol_da)):
        t = torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
        pinned[name] = t.numpy()
    host_spec = synth.Spectra(pinned["peak_off"], pinned["mz"], pinned["intensity"], pinned["prec_mz"],
                              pinned["charge"], pinned["tol_da"], spec.truth_protein, spec.truth_start,
                              spec.truth_len, spec.truth_modpos)
    idx.set_timing(False)
    e2e_t = []
    for i in range(args.e2e_steps + 1):
        t0 = time.perf_counter()
        res = idx.search(host_spec)
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_t.append(dt)
    h2d = sum(a.nbytes for a in pinned.values())
    d2h = res.psm.nbytes + res.hist.nbytes + res.n_scored.nbytes
    et = torch.tensor([sum(e2e_t)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(et, op=dist.ReduceOp.MAX)
    e2e_value = world * n * len(e2e_t) / float(et.item()) if e2e_t else None

    peak, peak_src = measured_peaks()
    mean_search_s = statistics.mean(search_ms) / 1000.0
    achieved = search_bytes / mean_search_s / 1e9
    rec = search_traffic_record()
    traffic = None
    if rec is not None and rec["workload"] == w.name:
        traffic = float(rec["dram_bytes_per_spectrum"]) * n
    line = {
        "metric": "spectra/s searched at 1 GB300 (% HBM roofline)",
        "value": value,
        "unit": "spectra/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": max_total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {
            "workload": workload_desc(w),
            "spectra_per_step": n,
            "n_peptides": int(st.n_peptides),
            "n_index_entries": int(st.n_entries),
            "index_bytes": int(st.device_bytes),
            "mean_window_peptides": float(np.mean(hi.astype(np.int64) - lo)),
            "mean_hits_per_spectrum": H / n,
            "l2": "index larger than L2; L2 flushed (256 MB write) before every timed step",
            "index_build_s": t_index,
            "index_build_host_ms": st.host_ms,
            "index_build_device_ms": st.device_ms,
            "input_gen_s": t_gen,
            "phase_ms": {"prep": statistics.mean(prep_ms), "search": statistics.mean(search_ms),
                         "merge": statistics.mean(merge_ms)},
            "step_roofline_spectra_per_s": peak * 1e9 / (step_bytes / n),
            "launch_shape": shape.as_dict(),
            "autotune_s": t_tune,
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "search_kernel",
                     "bytes_per_launch": search_bytes,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peak_src == "measured"
                     else "fallback 6.8 TB/s"},
        "e2e": {"value": e2e_value, "unit": "spectra/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, prot, spec, args.oracle_spectra)
    idx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
