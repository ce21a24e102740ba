"""ctypes wrapper of the CPU oracle (``hicops_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2102_02286_gb300``) never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hicops_oracle.cpp")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE FP64 semantics (no fast-math, no FMA contraction)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, SRC])
    os.replace(tmp, LIB)
    return LIB


class OrMod(C.Structure):
    _fields_ = [("residues", C.c_char_p), ("delta", C.c_double),
                ("max_per_peptide", C.c_uint32), ("fixed", C.c_uint32)]


class OrParams(C.Structure):
    _fields_ = [("min_len", C.c_uint32), ("max_len", C.c_uint32), ("missed_cleavages", C.c_uint32),
                ("pad0", C.c_uint32), ("min_mass", C.c_double), ("max_mass", C.c_double),
                ("frag_mz_min", C.c_double), ("frag_mz_max", C.c_double), ("bin_width", C.c_double),
                ("top_n_peaks", C.c_uint32), ("min_shared", C.c_uint32), ("top_k", C.c_uint32),
                ("hist_bins", C.c_uint32), ("intensity_scale", C.c_uint32), ("max_total_mods", C.c_uint32),
                ("tol_bins", C.c_uint32), ("evalue_mode", C.c_uint32)]


PSM_DTYPE = np.dtype([("pid", np.uint32), ("nb", np.uint32), ("ny", np.uint32), ("S", np.uint32),
                      ("key", np.int64), ("hyperscore", np.float64), ("evalue", np.float64)])

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.c_void_p
        L.or_db_build.restype = P
        L.or_db_build.argtypes = [P, P, C.c_uint32, P, C.c_uint32, C.POINTER(OrParams)]
        L.or_db_free.argtypes = [P]
        L.or_db_size.restype = C.c_uint64
        L.or_db_size.argtypes = [P]
        L.or_db_peptide.restype = C.c_uint32
        L.or_db_peptide.argtypes = [P, C.c_uint64, C.c_char_p, C.c_uint32, P, P]
        L.or_db_masses.argtypes = [P, P]
        L.or_db_ions.restype = C.c_uint32
        L.or_db_ions.argtypes = [P, C.c_uint64, P, P]
        L.or_db_bins.restype = C.c_uint32
        L.or_db_bins.argtypes = [P, C.c_uint64, P, P]
        L.or_preprocess.restype = C.c_uint32
        L.or_preprocess.argtypes = [C.POINTER(OrParams), P, P, C.c_uint64, C.c_double, C.c_uint8,
                                    C.c_double, P, P, P, P]
        L.or_rank_key.restype = C.c_int64
        L.or_rank_key.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_hyperscore.restype = C.c_double
        L.or_hyperscore.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_evalue.argtypes = [P, C.c_uint32, P, P, C.c_uint32, C.c_uint32, P]
        L.or_search.argtypes = [P, P, P, P, P, P, P, P, C.c_uint32, P, P, P, P, P]
        L.or_search_shard.argtypes = [P, P, P, P, P, P, P, P, C.c_uint32, P, P, P, P, P, C.c_uint32, C.c_uint32]
        L.or_edit_distance.restype = C.c_uint32
        L.or_edit_distance.argtypes = [C.c_char_p, P, C.c_char_p, P]
        L.or_mod_distance.restype = C.c_double
        L.or_mod_distance.argtypes = [C.c_char_p, P, C.c_char_p, P]
        L.or_partition_lbe.argtypes = [P, C.c_uint32, P]
        L.or_hist_sample.restype = C.c_uint32
        L.or_hist_sample.argtypes = [P, C.c_uint32, C.c_uint32, P, P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_params(sp) -> OrParams:
    """Oracle parameter block from a ``configs.SearchParams``."""
    return OrParams(min_len=sp.min_len, max_len=sp.max_len, missed_cleavages=sp.missed_cleavages, pad0=0,
                    min_mass=sp.min_mass, max_mass=sp.max_mass, frag_mz_min=sp.frag_mz_min,
                    frag_mz_max=sp.frag_mz_max, bin_width=sp.bin_width_da, top_n_peaks=sp.top_n_peaks,
                    min_shared=sp.min_shared, top_k=sp.top_k, hist_bins=sp.hist_bins,
                    intensity_scale=sp.intensity_scale, max_total_mods=sp.max_total_mods,
                    tol_bins=sp.tol_bins, evalue_mode=sp.evalue_mode)


@dataclass
class SearchResult:
    psm: np.ndarray      # PSM_DTYPE [n_sel, top_k]
    hist: np.ndarray     # uint32 [n_sel, hist_bins]
    n_scored: np.ndarray # uint32 [n_sel]
    lo: np.ndarray
    hi: np.ndarray


class OracleDb:
    """The oracle's peptide database (digest + variants, sorted; no index)."""

    def __init__(self, seq: np.ndarray, off: np.ndarray, mods, params):
        L = lib()
        self._keep = []
        var_mods = [m for m in mods]
        arr = (OrMod * max(1, len(var_mods)))()
        for i, m in enumerate(var_mods):
            r = m.residues.encode()
            self._keep.append(r)
            arr[i] = OrMod(r, m.delta_da, m.max_per_peptide, 1 if m.fixed else 0)
        self.params = make_params(params)
        self.top_k = params.top_k
        self.hist_bins = params.hist_bins
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        self.h = L.or_db_build(_ptr(seq), _ptr(off), len(off) - 1, arr, len(var_mods), C.byref(self.params))
        self.n = int(L.or_db_size(self.h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_db_free(self.h)
            self.h = None

    def masses(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        lib().or_db_masses(self.h, _ptr(out))
        return out

    def peptide(self, pid: int):
        buf = C.create_string_buffer(128)
        mass = np.zeros(1, np.float64)
        codes = np.zeros(128, np.uint8)
        L = lib().or_db_peptide(self.h, pid, buf, 128, _ptr(mass), _ptr(codes))
        return buf.value.decode(), float(mass[0]), codes[:L].copy()

    def ions(self, pid: int):
        b = np.zeros(128, np.float64)
        y = np.zeros(128, np.float64)
        n = lib().or_db_ions(self.h, pid, _ptr(b), _ptr(y))
        return b[:n].copy(), y[:n].copy()

    def partition_lbe(self, n_parts: int) -> np.ndarray:
        """R18: the LBE partition of the database, part[pid] in [0, n_parts)."""
        out = np.zeros(self.n, np.uint32)
        lib().or_partition_lbe(self.h, n_parts, _ptr(out))
        return out

    def bins(self, pid: int):
        b = np.zeros(256, np.uint32)
        t = np.zeros(256, np.uint8)
        n = lib().or_db_bins(self.h, pid, _ptr(b), _ptr(t))
        return b[:n].copy(), t[:n].copy()

    def search(self, spec, sel=None, n_shards: int = 1, shard: int = 0) -> SearchResult:
        """Search the selected spectra; with n_shards > 1 only the database
        entries pid = shard (mod n_shards) are candidates."""
        n = spec.n
        sel = np.arange(n, dtype=np.uint32) if sel is None else np.ascontiguousarray(sel, dtype=np.uint32)
        k, H = self.top_k, self.hist_bins
        psm = np.zeros((len(sel), k), dtype=PSM_DTYPE)
        hist = np.zeros((len(sel), H), dtype=np.uint32)
        ns = np.zeros(len(sel), dtype=np.uint32)
        lo = np.zeros(len(sel), dtype=np.uint32)
        hi = np.zeros(len(sel), dtype=np.uint32)
        a = [np.ascontiguousarray(x) for x in (spec.peak_off.astype(np.uint64), spec.mz.astype(np.float32),
                                               spec.intensity.astype(np.float32), spec.prec_mz.astype(np.float64),
                                               spec.charge.astype(np.uint8), spec.tol_da.astype(np.float64))]
        lib().or_search_shard(self.h, *[_ptr(x) for x in a], _ptr(sel), len(sel), _ptr(psm), _ptr(hist),
                              _ptr(ns), _ptr(lo), _ptr(hi), n_shards, shard)
        return SearchResult(psm, hist, ns, lo, hi)


def preprocess(params, mz, inten, prec_mz, z, tol):
    p = make_params(params)
    mz = np.ascontiguousarray(mz, np.float32)
    inten = np.ascontiguousarray(inten, np.float32)
    bins = np.zeros(max(1, len(mz)), np.uint32)
    iq = np.zeros(max(1, len(mz)), np.uint32)
    Mq = np.zeros(1, np.float64)
    valid = np.zeros(1, np.int32)
    n = lib().or_preprocess(C.byref(p), _ptr(mz), _ptr(inten), len(mz), prec_mz, z, tol,
                            _ptr(bins), _ptr(iq), _ptr(Mq), _ptr(valid))
    return bins[:n].copy(), iq[:n].copy(), float(Mq[0]), bool(valid[0])


def rank_key(nb, ny, S) -> int:
    return int(lib().or_rank_key(nb, ny, S))


def hyperscore(nb, ny, S) -> float:
    return float(lib().or_hyperscore(nb, ny, S))


def evalue(hist, keys, pids, evalue_mode=0) -> np.ndarray:
    hist = np.ascontiguousarray(hist, np.uint32)
    keys = np.ascontiguousarray(keys, np.int64)
    pids = np.ascontiguousarray(pids, np.uint32)
    out = np.zeros(len(keys), np.float64)
    lib().or_evalue(_ptr(hist), len(hist), _ptr(keys), _ptr(pids), len(keys), evalue_mode, _ptr(out))
    return out


def hist_sample(hist, s: int = 120):
    """R19: (lo, len, mean) of the bins kept when the score distribution is
    sampled down to at most s bins around its mean."""
    hist = np.ascontiguousarray(hist, np.uint32)
    lo = np.zeros(1, np.uint32)
    ln = np.zeros(1, np.uint32)
    m = lib().or_hist_sample(_ptr(hist), len(hist), s, _ptr(lo), _ptr(ln))
    return int(lo[0]), int(ln[0]), int(m)


def sampled(hist, s: int = 120) -> np.ndarray:
    """The histogram as the receiver of its sample sees it: the kept bins'
    counts, zero elsewhere."""
    hist = np.asarray(hist, np.uint32)
    lo, ln, _ = hist_sample(hist, s)
    out = np.zeros_like(hist)
    out[lo:lo + ln] = hist[lo:lo + ln]
    return out


def _seq_codes(pep):
    """(letters, codes) from a peptide written with '*' after modified residues."""
    letters, codes = [], []
    for ch in pep:
        if ch == "*":
            codes[-1] = 1
        else:
            letters.append(ch)
            codes.append(0)
    return "".join(letters).encode(), np.array(codes, np.uint8)


def edit_distance(x: str, y: str) -> int:
    """R18 edit distance of two peptides written with '*' after modified residues."""
    (xs, xc), (ys, yc) = _seq_codes(x), _seq_codes(y)
    return int(lib().or_edit_distance(xs, _ptr(xc), ys, _ptr(yc)))


def mod_distance(x: str, y: str) -> float:
    """R18 Mod Distance of two peptides written with '*' after modified residues."""
    (xs, xc), (ys, yc) = _seq_codes(x), _seq_codes(y)
    return float(lib().or_mod_distance(xs, _ptr(xc), ys, _ptr(yc)))
