"""ctypes binding of ``libhicops.so`` (argument marshalling only).

Every step of the search runs in the library's CUDA kernels; this module
only converts arrays and tensors into pointers.  If the library has not been
built, importing works but every call raises: there is no fallback path.
PyTorch is used only for device memory and streams (``search_device``).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import build as _build
from .configs import SearchParams

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, EBUSY, ECANCELLED = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EOVERFLOW", "EBUSY", "ECANCELLED"]
HIST_BINS = 256


class HicopsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Mod(C.Structure):
    _fields_ = [("residues", C.c_char_p), ("delta_da", C.c_double),
                ("max_per_peptide", C.c_uint32), ("fixed", C.c_uint32)]


class Params(C.Structure):
    _fields_ = [("min_len", C.c_uint32), ("max_len", C.c_uint32), ("missed_cleavages", C.c_uint32),
                ("max_total_mods", C.c_uint32), ("min_mass", C.c_double), ("max_mass", C.c_double),
                ("frag_mz_min", C.c_double), ("frag_mz_max", C.c_double), ("bin_width_da", C.c_double),
                ("top_n_peaks", C.c_uint32), ("min_shared", C.c_uint32), ("top_k", C.c_uint32),
                ("hist_bins", C.c_uint32), ("intensity_scale", C.c_uint32), ("tol_bins", C.c_uint32),
                ("evalue_mode", C.c_uint32), ("reserved", C.c_uint32)]


class Proteins(C.Structure):
    _fields_ = [("n_proteins", C.c_uint64), ("seq", C.c_void_p), ("off", C.c_void_p)]


class Batch(C.Structure):
    _fields_ = [("n", C.c_uint32), ("on_device", C.c_uint32), ("peak_off", C.c_void_p), ("mz", C.c_void_p),
                ("intensity", C.c_void_p), ("prec_mz", C.c_void_p), ("charge", C.c_void_p),
                ("prec_tol_da", C.c_void_p), ("cuda_stream", C.c_void_p)]


class IndexStats(C.Structure):
    _fields_ = [("n_peptides", C.c_uint64), ("n_base_peptides", C.c_uint64), ("n_entries", C.c_uint64),
                ("n_bins", C.c_uint64), ("device_bytes", C.c_uint64), ("max_bucket", C.c_uint64),
                ("host_ms", C.c_double), ("device_ms", C.c_double)]


class SearchConfig(C.Structure):
    _fields_ = [("threads", C.c_uint32), ("chunk_entries", C.c_uint32), ("ctas_per_sm", C.c_uint32),
                ("seg_pids", C.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class ServerCfg(C.Structure):
    _fields_ = [("n_slots", C.c_uint32), ("slot_spectra", C.c_uint32), ("memory_budget", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("launches", C.c_uint64),
                ("spectra", C.c_uint64), ("n_slots", C.c_uint32), ("reserved", C.c_uint32),
                ("pool_bytes", C.c_uint64), ("pool_peak", C.c_uint64), ("memory_waits", C.c_uint64)]


class Timing(C.Structure):
    _fields_ = [("prep_ms", C.c_float), ("plan_ms", C.c_float), ("search_ms", C.c_float),
                ("merge_ms", C.c_float), ("total_ms", C.c_float)]


def kernel_launches() -> int:
    return int(load().hicops_kernel_launches())


PSM_DTYPE = np.dtype([("query", np.uint32), ("pid", np.uint32), ("nb", np.uint8), ("ny", np.uint8),
                      ("reserved", np.uint16), ("hyperscore", np.float32), ("key", np.int64),
                      ("evalue", np.float64)])
assert PSM_DTYPE.itemsize == 32

_lib = None


class PipelineConfig(C.Structure):
    _fields_ = [("batch_spectra", C.c_uint32), ("n_buffers", C.c_uint32), ("n_workers", C.c_uint32),
                ("reserved", C.c_uint32), ("prec_tol_da", C.c_double), ("alpha", C.c_double),
                ("t_min_s", C.c_double), ("t_max_s", C.c_double)]


class PipelineStats(C.Structure):
    _fields_ = [("spectra", C.c_uint64), ("batches", C.c_uint64), ("moves_i_to_r", C.c_uint64),
                ("moves_r_to_i", C.c_uint64), ("seconds", C.c_double), ("wait_seconds", C.c_double)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the library (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libhicops.so is not built ({_build.LIB}); run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(_build.LIB)
    P = C.c_void_p
    st = C.c_int
    sig = {
        "hicops_digest": (st, [C.POINTER(Proteins), P, C.c_uint32, C.POINTER(Params), C.POINTER(P)]),
        "hicops_index_upload": (st, [P]),
        "hicops_build_index": (st, [C.POINTER(Proteins), P, C.c_uint32, C.POINTER(Params), C.POINTER(P)]),
        "hicops_search": (st, [P, C.POINTER(Batch), P, P, P]),
        "hicops_search_noalloc": (st, [P, C.POINTER(Batch), P, P, P]),
        "hicops_search_scratch_bytes": (st, [P, C.c_uint32, C.POINTER(C.c_uint64)]),
        "hicops_search_scratch": (st, [P, C.POINTER(Batch), P, C.c_uint64, P, P, P]),
        "hicops_search_work": (st, [P, C.POINTER(Batch), P, P, P, P]),
        "hicops_index_set_config": (st, [P, C.POINTER(SearchConfig)]),
        "hicops_autotune": (st, [P, C.POINTER(Batch), C.POINTER(SearchConfig), C.POINTER(C.c_double)]),
        "hicops_plan_create": (st, [P, C.c_uint32, C.POINTER(SearchConfig), C.POINTER(P)]),
        "hicops_plan_search": (st, [P, C.POINTER(Batch), P, P, P, C.c_int]),
        "hicops_plan_destroy": (None, [P]),
        "hicops_server_create": (st, [P, C.POINTER(ServerCfg), C.POINTER(P)]),
        "hicops_server_submit": (st, [P, C.POINTER(Batch), C.POINTER(C.c_uint64)]),
        "hicops_server_poll": (st, [P, C.c_uint64, C.c_int, P, P, P]),
        "hicops_server_cancel": (st, [P, C.c_uint64]),
        "hicops_server_get_stats": (st, [P, C.POINTER(ServerStats)]),
        "hicops_server_destroy": (None, [P]),
        "hicops_index_set_timing": (st, [P, C.c_int]),
        "hicops_index_last_timing": (st, [P, C.POINTER(Timing)]),
        "hicops_kernel_launches": (C.c_uint64, []),
        "hicops_index_get_stats": (st, [P, C.POINTER(IndexStats)]),
        "hicops_index_shard": (st, [P, C.c_uint32, C.c_uint32, C.POINTER(P)]),
        "hicops_index_subset": (st, [P, P, C.c_uint64, C.POINTER(P)]),
        "hicops_partition_lbe": (st, [P, C.c_uint32, P]),
        "hicops_index_get_params": (st, [P, C.POINTER(Params)]),
        "hicops_index_save": (st, [P, C.c_char_p]),
        "hicops_index_load": (st, [C.c_char_p, C.POINTER(P)]),
        "hicops_merge_shards": (st, [C.c_uint32, C.c_uint32, C.c_uint32, P, P, P, C.c_uint32, C.c_uint32, C.c_int,
                                     P, P, P, P]),
        "hicops_hist_sample": (st, [C.c_uint32, P, C.c_uint32, P, C.c_int, P]),
        "hicops_hist_unsample": (st, [C.c_uint32, C.c_uint32, C.c_uint32, P, P, C.c_int, P]),
        "hicops_peptide": (st, [P, C.c_uint32, C.c_char_p, C.c_uint32, P, P]),
        "hicops_index_copy_csr": (st, [P, P, P]),
        "hicops_index_free": (None, [P]),
        "hicops_last_error": (C.c_char_p, []),
        "hicops_pipeline_run": (st, [P, P, C.c_uint32, C.c_char_p, C.POINTER(PipelineConfig),
                                     C.POINTER(PipelineStats)]),
        "hicops_ms2_read": (st, [C.c_char_p, C.c_uint32, C.c_uint64, C.POINTER(C.c_uint32),
                                 C.POINTER(C.c_uint64), P, P, P, P, P, P]),
        "hicops_des_step": (C.c_double, [P, C.c_double, C.c_double, C.c_int]),
        "hicops_sched_i_to_r": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.c_uint32, C.c_uint32]),
        "hicops_sched_r_to_i": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != OK:
        raise HicopsError(status, load().hicops_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_params(sp) -> Params:
    return Params(min_len=sp.min_len, max_len=sp.max_len, missed_cleavages=sp.missed_cleavages,
                  max_total_mods=sp.max_total_mods, min_mass=sp.min_mass, max_mass=sp.max_mass,
                  frag_mz_min=sp.frag_mz_min, frag_mz_max=sp.frag_mz_max, bin_width_da=sp.bin_width_da,
                  top_n_peaks=sp.top_n_peaks, min_shared=sp.min_shared, top_k=sp.top_k,
                  hist_bins=sp.hist_bins, intensity_scale=sp.intensity_scale, tol_bins=sp.tol_bins,
                  evalue_mode=sp.evalue_mode, reserved=0)


@dataclass
class SearchResult:
    psm: np.ndarray       # PSM_DTYPE [n, top_k]
    hist: np.ndarray      # uint32 [n, 256]
    n_scored: np.ndarray  # uint32 [n]


class Index:
    """A database (superstep 1) and, once uploaded, its device fragment index."""

    def __init__(self, seq: np.ndarray, off: np.ndarray, mods: Sequence, params, upload: bool = True):
        L = load()
        self.params = params
        self.top_k = params.top_k
        self._keep = [np.ascontiguousarray(seq, np.uint8), np.ascontiguousarray(off, np.uint64)]
        arr = (Mod * max(1, len(mods)))()
        self._mod_res = []
        for i, m in enumerate(mods):
            r = m.residues.encode()
            self._mod_res.append(r)
            arr[i] = Mod(r, m.delta_da, m.max_per_peptide, 1 if m.fixed else 0)
        self._mods = arr
        self._p = make_params(params)
        prot = Proteins(len(self._keep[1]) - 1, _ptr(self._keep[0]).value, _ptr(self._keep[1]).value)
        h = C.c_void_p()
        _check(L.hicops_digest(C.byref(prot), C.cast(arr, C.c_void_p), len(mods), C.byref(self._p), C.byref(h)))
        self.h = h
        self._keep = None
        if upload:
            self.upload()

    @classmethod
    def _from_handle(cls, h, params):
        self = cls.__new__(cls)
        self.params = params
        self.top_k = params.top_k
        self.h = h
        self._keep = None
        return self

    def shard(self, n_shards: int, shard: int, upload: bool = True) -> "Index":
        """hicops_index_shard: entries pid = shard (mod n_shards); results carry global pids."""
        h = C.c_void_p()
        _check(load().hicops_index_shard(self.h, n_shards, shard, C.byref(h)))
        s = Index._from_handle(h, self.params)
        if upload:
            s.upload()
        return s

    def subset(self, pids, upload: bool = True) -> "Index":
        """hicops_index_subset: the entries with the given (strictly ascending)
        global pids; results carry global pids."""
        pids = np.ascontiguousarray(pids, np.uint32)
        h = C.c_void_p()
        _check(load().hicops_index_subset(self.h, _ptr(pids), len(pids), C.byref(h)))
        s = Index._from_handle(h, self.params)
        if upload:
            s.upload()
        return s

    def save(self, path: str):
        """hicops_index_save: the host half of the index to one file."""
        _check(load().hicops_index_save(self.h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, upload: bool = True) -> "Index":
        """hicops_index_load: an index saved by ``save`` (its device half rebuilt
        when upload)."""
        L = load()
        h = C.c_void_p()
        _check(L.hicops_index_load(os.fsencode(path), C.byref(h)))
        p = Params()
        _check(L.hicops_index_get_params(h, C.byref(p)))
        sp = SearchParams(**{f.name: getattr(p, f.name) for f in dataclasses.fields(SearchParams)})
        idx = cls._from_handle(h, sp)
        if upload:
            idx.upload()
        return idx

    def partition_lbe(self, n_parts: int) -> np.ndarray:
        """hicops_partition_lbe: part[pid] of the load-balancing partition."""
        out = np.zeros(self.stats().n_peptides, np.uint32)
        _check(load().hicops_partition_lbe(self.h, n_parts, _ptr(out)))
        return out

    def upload(self):
        _check(load().hicops_index_upload(self.h))

    def close(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.hicops_index_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> IndexStats:
        s = IndexStats()
        _check(load().hicops_index_get_stats(self.h, C.byref(s)))
        return s

    @property
    def n_peptides(self) -> int:
        return int(self.stats().n_peptides)

    def peptide(self, pid: int):
        buf = C.create_string_buffer(80)
        mass = C.c_double()
        mask = C.c_uint64()
        _check(load().hicops_peptide(self.h, pid, buf, 80, C.byref(mass), C.byref(mask)))
        return buf.value.decode(), mass.value, mask.value

    def copy_csr(self):
        st = self.stats()
        off = np.zeros(st.n_bins + 1, np.uint64)
        ent = np.zeros(max(1, st.n_entries), np.uint32)
        _check(load().hicops_index_copy_csr(self.h, _ptr(off), _ptr(ent)))
        return off, ent[:st.n_entries]

    # ---- search through host buffers (the library copies in and out)

    @staticmethod
    def _host_batch(spec):
        arrs = [np.ascontiguousarray(spec.peak_off, np.uint64), np.ascontiguousarray(spec.mz, np.float32),
                np.ascontiguousarray(spec.intensity, np.float32), np.ascontiguousarray(spec.prec_mz, np.float64),
                np.ascontiguousarray(spec.charge, np.uint8), np.ascontiguousarray(spec.tol_da, np.float64)]
        b = Batch(len(arrs[3]), 0, *[_ptr(a).value for a in arrs], None)
        return b, arrs

    def search(self, spec, out: Optional[SearchResult] = None) -> SearchResult:
        """Search through host buffers.  `out` may hold preallocated result
        arrays (e.g. views of page-locked memory) of the batch's size."""
        b, keep = self._host_batch(spec)
        n = b.n
        if out is None:
            out = SearchResult(np.zeros((n, self.top_k), PSM_DTYPE), np.zeros((n, HIST_BINS), np.uint32),
                               np.zeros(n, np.uint32))
        if out.psm.shape != (n, self.top_k) or out.hist.shape != (n, HIST_BINS) or out.n_scored.shape != (n,):
            raise ValueError("out arrays do not match the batch")
        _check(load().hicops_search(self.h, C.byref(b), _ptr(out.psm), _ptr(out.hist), _ptr(out.n_scored)))
        return out

    def search_work(self, spec):
        """Per spectrum: window [lo, hi), retained peaks, index entries in the window (H)."""
        b, keep = self._host_batch(spec)
        n = b.n
        lo = np.zeros(n, np.uint32)
        hi = np.zeros(n, np.uint32)
        npk = np.zeros(n, np.uint32)
        hits = np.zeros(n, np.uint64)
        _check(load().hicops_search_work(self.h, C.byref(b), _ptr(lo), _ptr(hi), _ptr(npk), _ptr(hits)))
        return lo, hi, npk, hits

    def set_config(self, cfg: Optional[SearchConfig] = None):
        _check(load().hicops_index_set_config(self.h, C.byref(cfg) if cfg is not None else None))

    def autotune(self, dev_batch: "DeviceBatch", stream=None):
        """Times the candidate launch shapes on a device batch; keeps the fastest."""
        b = _device_batch_struct(dev_batch, stream)
        best = SearchConfig()
        ms = C.c_double()
        _check(load().hicops_autotune(self.h, C.byref(b), C.byref(best), C.byref(ms)))
        return best, ms.value

    def plan(self, max_spectra: int, cfg: Optional[SearchConfig] = None) -> "Plan":
        return Plan(self, max_spectra, cfg)

    def set_timing(self, enable: bool = True):
        _check(load().hicops_index_set_timing(self.h, 1 if enable else 0))

    def last_timing(self) -> "Timing":
        t = Timing()
        _check(load().hicops_index_last_timing(self.h, C.byref(t)))
        return t

    # ---- search on device tensors (asynchronous on the given stream)

    def search_device(self, dev_batch: "DeviceBatch", out: "DeviceResult", stream=None):
        b = _device_batch_struct(dev_batch, stream)
        _check(load().hicops_search(self.h, C.byref(b), out.psm.data_ptr(),
                                    out.hist.data_ptr() if out.hist is not None else None,
                                    out.n_scored.data_ptr() if out.n_scored is not None else None))

    def search_noalloc(self, dev_batch: "DeviceBatch", out: "DeviceResult", stream=None):
        """hicops_search_noalloc: device tensors, at most NOALLOC_MAX_SPECTRA spectra, no allocation."""
        b = _device_batch_struct(dev_batch, stream)
        _check(load().hicops_search_noalloc(self.h, C.byref(b), out.psm.data_ptr(),
                                            out.hist.data_ptr() if out.hist is not None else None,
                                            out.n_scored.data_ptr() if out.n_scored is not None else None))


    def search_scratch_bytes(self, n: int) -> int:
        """hicops_search_scratch_bytes: device scratch one search of n spectra takes."""
        b = C.c_uint64()
        _check(load().hicops_search_scratch_bytes(self.h, n, C.byref(b)))
        return b.value

    def search_scratch(self, dev_batch: "DeviceBatch", out: "DeviceResult", scratch, nbytes=None, stream=None):
        """hicops_search_scratch: device tensors, scratch a device tensor (256-byte aligned start)."""
        b = _device_batch_struct(dev_batch, stream)
        nbytes = scratch.numel() * scratch.element_size() if nbytes is None else nbytes
        _check(load().hicops_search_scratch(self.h, C.byref(b), scratch.data_ptr(), nbytes, out.psm.data_ptr(),
                                            out.hist.data_ptr() if out.hist is not None else None,
                                            out.n_scored.data_ptr() if out.n_scored is not None else None))


def _device_batch_struct(dev_batch, stream=None) -> Batch:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return Batch(dev_batch.n, 1, dev_batch.peak_off.data_ptr(), dev_batch.mz.data_ptr(),
                 dev_batch.intensity.data_ptr(), dev_batch.prec_mz.data_ptr(), dev_batch.charge.data_ptr(),
                 dev_batch.tol_da.data_ptr(), s.cuda_stream)


class Plan:
    """Reusable search with scratch allocated once; optionally replayed as a CUDA graph."""

    def __init__(self, index: Index, max_spectra: int, cfg: Optional[SearchConfig] = None):
        self.index = index
        h = C.c_void_p()
        _check(load().hicops_plan_create(index.h, max_spectra, C.byref(cfg) if cfg is not None else None,
                                         C.byref(h)))
        self.h = h

    def search(self, dev_batch: "DeviceBatch", out: "DeviceResult", stream=None, graph: bool = True):
        b = _device_batch_struct(dev_batch, stream)
        _check(load().hicops_plan_search(self.h, C.byref(b), out.psm.data_ptr(),
                                         out.hist.data_ptr() if out.hist is not None else None,
                                         out.n_scored.data_ptr() if out.n_scored is not None else None,
                                         1 if graph else 0))

    def close(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.hicops_plan_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class DeviceBatch:
    n: int
    peak_off: "object"
    mz: "object"
    intensity: "object"
    prec_mz: "object"
    charge: "object"
    tol_da: "object"

    @classmethod
    def from_spectra(cls, spec, device="cuda"):
        import torch
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).to(device)   # noqa: E731
        return cls(spec.n, t(spec.peak_off, np.uint64).view(torch.int64), t(spec.mz, np.float32),
                   t(spec.intensity, np.float32), t(spec.prec_mz, np.float64), t(spec.charge, np.uint8),
                   t(spec.tol_da, np.float64))


@dataclass
class DeviceResult:
    psm: "object"        # uint8 tensor [n * top_k * 32]
    hist: Optional["object"]
    n_scored: Optional["object"]

    @classmethod
    def alloc(cls, n, top_k, device="cuda", hist=True):
        import torch
        return cls(torch.empty(n * top_k * PSM_DTYPE.itemsize, dtype=torch.uint8, device=device),
                   torch.empty(n * HIST_BINS, dtype=torch.int32, device=device) if hist else None,
                   torch.empty(n, dtype=torch.int32, device=device) if hist else None)

    def to_host(self, n, top_k) -> SearchResult:
        psm = self.psm.cpu().numpy().view(PSM_DTYPE).reshape(n, top_k)
        hist = self.hist.cpu().numpy().view(np.uint32).reshape(n, HIST_BINS) if self.hist is not None else None
        ns = self.n_scored.cpu().numpy().view(np.uint32) if self.n_scored is not None else None
        return SearchResult(psm, hist, ns)


class Server:
    """Continuous-batching request server over a resident index.

    n_slots: launches in flight at most (one stream each); slot_spectra:
    spectra one launch packs at most; memory_budget: bytes of the device pool
    that launches take their blocks from (requests wait for pool memory).
    Zero takes the library's default."""

    def __init__(self, index: Index, n_slots: int = 0, slot_spectra: int = 0, memory_budget: int = 0):
        self.index = index
        self.top_k = index.top_k
        h = C.c_void_p()
        cfg = ServerCfg(n_slots, slot_spectra, memory_budget)
        _check(load().hicops_server_create(index.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self._n = {}

    def submit(self, spec) -> int:
        b, keep = Index._host_batch(spec)
        t = C.c_uint64()
        _check(load().hicops_server_submit(self.h, C.byref(b), C.byref(t)))
        self._n[t.value] = b.n
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1) -> Optional[SearchResult]:
        """Result of a request, or None if it is not done within timeout_ms."""
        n = self._n[ticket]
        psm = np.zeros((n, self.top_k), PSM_DTYPE)
        hist = np.zeros((n, HIST_BINS), np.uint32)
        ns = np.zeros(n, np.uint32)
        st = load().hicops_server_poll(self.h, ticket, timeout_ms, _ptr(psm), _ptr(hist), _ptr(ns))
        if st == ETIMEOUT:
            return None
        self._n.pop(ticket, None)
        _check(st)
        return SearchResult(psm, hist, ns)

    def cancel(self, ticket: int) -> int:
        """Status of the cancel: OK, or EBUSY when the request is already launched."""
        return load().hicops_server_cancel(self.h, ticket)

    def stats(self) -> ServerStats:
        s = ServerStats()
        _check(load().hicops_server_get_stats(self.h, C.byref(s)))
        return s

    def close(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.hicops_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# the e-value mode of the workloads' search parameters (smoothing, then the tail fit)
EVALUE_DEFAULT = 2


def merge_shards(n_shards: int, n: int, top_k: int, psm, hist, n_scored, hist_parts: int,
                 stream=None, evalue_mode: int = EVALUE_DEFAULT) -> "DeviceResult":
    """hicops_merge_shards on device tensors (asynchronous on the stream):
    psm [n_shards * n * top_k] rows, hist [hist_parts * n * 256], n_scored
    [hist_parts * n]; returns a DeviceResult of the merged search."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = DeviceResult.alloc(n, top_k)
    _check(load().hicops_merge_shards(n_shards, n, top_k, psm.data_ptr(), hist.data_ptr(), n_scored.data_ptr(),
                                      hist_parts, evalue_mode, 1, s.cuda_stream, out.psm.data_ptr(),
                                      out.hist.data_ptr(), out.n_scored.data_ptr()))
    return out


def merge_shards_host(n_shards: int, n: int, top_k: int, psm: np.ndarray, hist: np.ndarray,
                      n_scored: np.ndarray, hist_parts: int, evalue_mode: int = EVALUE_DEFAULT) -> SearchResult:
    """hicops_merge_shards on host arrays (the library copies to the device and back)."""
    psm = np.ascontiguousarray(psm, PSM_DTYPE)
    hist = np.ascontiguousarray(hist, np.uint32)
    n_scored = np.ascontiguousarray(n_scored, np.uint32)
    out = SearchResult(np.zeros((n, top_k), PSM_DTYPE), np.zeros((n, HIST_BINS), np.uint32),
                       np.zeros(n, np.uint32))
    _check(load().hicops_merge_shards(n_shards, n, top_k, _ptr(psm), _ptr(hist), _ptr(n_scored), hist_parts,
                                      evalue_mode, 0, None, _ptr(out.psm), _ptr(out.hist), _ptr(out.n_scored)))
    return out


# ---- sampled partial score distributions (Sampling section)

SAMPLE_S = 120   # HICOPS_SAMPLE_S, the paper's default number of samples


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def hist_sample(hist, s: int = SAMPLE_S, stream=None):
    """hicops_hist_sample: records [n, s + 1] (word 0 = lo | len << 16, then
    the kept bins' counts) of histograms [n, 256] or [n * 256].  A device
    tensor gives a device tensor (asynchronous on the stream), a numpy
    array a numpy array."""
    if _is_device(hist):
        import torch
        n = hist.numel() // HIST_BINS
        out = torch.empty(n * (s + 1), dtype=torch.int32, device=hist.device)
        st = stream if stream is not None else torch.cuda.current_stream()
        _check(load().hicops_hist_sample(n, hist.data_ptr(), s, out.data_ptr(), 1, st.cuda_stream))
        return out
    h = np.ascontiguousarray(hist, np.uint32).reshape(-1, HIST_BINS)
    out = np.zeros((h.shape[0], s + 1), np.uint32)
    _check(load().hicops_hist_sample(h.shape[0], _ptr(h), s, _ptr(out), 0, None))
    return out


def hist_unsample(n_parts: int, n: int, rec, s: int = SAMPLE_S, stream=None):
    """hicops_hist_unsample: the summed histograms [n, 256] of n_parts
    parts' records [n_parts * n, s + 1]."""
    if _is_device(rec):
        import torch
        out = torch.empty(n * HIST_BINS, dtype=torch.int32, device=rec.device)
        st = stream if stream is not None else torch.cuda.current_stream()
        _check(load().hicops_hist_unsample(n_parts, n, s, rec.data_ptr(), out.data_ptr(), 1, st.cuda_stream))
        return out
    r = np.ascontiguousarray(rec, np.uint32).reshape(-1, s + 1)
    out = np.zeros((n, HIST_BINS), np.uint32)
    _check(load().hicops_hist_unsample(n_parts, n, s, _ptr(r), _ptr(out), 0, None))
    return out


# ---- host ingest pipeline


def run_files(index: "Index", paths, out_path: str, prec_tol_da: float, **cfg) -> PipelineStats:
    """hicops_pipeline_run: searches every spectrum of the MS2 files and writes
    the top-k rows to out_path (config fields as keyword arguments)."""
    c = PipelineConfig(prec_tol_da=prec_tol_da, **cfg)
    arr = (C.c_char_p * max(1, len(paths)))(*[os.fsencode(p) for p in paths])
    stats = PipelineStats()
    _check(load().hicops_pipeline_run(index.h, C.cast(arr, C.c_void_p), len(paths), os.fsencode(out_path),
                                      C.byref(c), C.byref(stats)))
    return stats


def read_ms2(path: str) -> dict:
    """hicops_ms2_read: the spectra of one MS2 file as arrays."""
    L = load()
    ns, npk = C.c_uint32(), C.c_uint64()
    _check(L.hicops_ms2_read(os.fsencode(path), 0, 0, C.byref(ns), C.byref(npk), None, None, None, None, None,
                             None))
    n, m = ns.value, npk.value
    out = {"peak_off": np.zeros(n + 1, np.uint64), "mz": np.zeros(m, np.float32),
           "intensity": np.zeros(m, np.float32), "prec_mz": np.zeros(n, np.float64),
           "charge": np.zeros(n, np.uint8), "scan": np.zeros(n, np.uint32)}
    _check(L.hicops_ms2_read(os.fsencode(path), n, m, C.byref(ns), C.byref(npk), _ptr(out["peak_off"]),
                             _ptr(out["mz"]), _ptr(out["intensity"]), _ptr(out["prec_mz"]), _ptr(out["charge"]),
                             _ptr(out["scan"])))
    return out


def read_pipeline_rows(path: str) -> np.ndarray:
    """The rows hicops_pipeline_run wrote, as a structured array."""
    dt = np.dtype([("file", np.uint32), ("scan", np.uint32), ("spectrum", np.uint64), ("rank", np.uint32),
                   ("pid", np.uint32), ("nb", np.uint32), ("ny", np.uint32), ("hyperscore", np.float32),
                   ("evalue", np.float64), ("n_scored", np.uint32)])
    rows = np.loadtxt(path, dtype=dt, delimiter="\t", skiprows=1, ndmin=1)
    return rows
