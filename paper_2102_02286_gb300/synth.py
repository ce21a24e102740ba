"""Seeded synthetic proteomes and MS/MS query spectra.

The paper's datasets (PRIDE) and protein databases (UniProt) are not
available, so every input is generated here from a seed, shaped like the
paper's workloads (Experimental Setup): tryptic peptides of natural
amino-acid composition, b/y fragment peaks with mass-measurement jitter,
uniform noise peaks and lognormal intensities.

This module is an *instrument simulator*: it holds none of the search
method's arithmetic and neither the CUDA path nor the CPU oracle calls into
it; both only receive its arrays.  Its residue-mass table is its own
simulation constant, used only to place simulated peaks.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np

from .configs import Workload, SpectraRecipe

# UniProtKB/Swiss-Prot amino-acid composition (percent), the published
# release statistics; used as i.i.d. residue frequencies.
AA_COMPOSITION = {
    "A": 8.25, "R": 5.53, "N": 4.06, "D": 5.45, "C": 1.37, "Q": 3.93, "E": 6.75,
    "G": 7.07, "H": 2.27, "I": 5.96, "L": 9.66, "K": 5.84, "M": 2.42, "F": 3.86,
    "P": 4.70, "S": 6.56, "T": 5.34, "W": 1.08, "Y": 2.92, "V": 6.87,
}
_ALPHA = np.frombuffer("".join(AA_COMPOSITION).encode(), dtype=np.uint8)
_FREQ = np.array(list(AA_COMPOSITION.values()), dtype=np.float64)
_FREQ = _FREQ / _FREQ.sum()

# simulation constants (monoisotopic, Da)
_SIM_MASS = np.zeros(256, dtype=np.float64)
for _aa, _m in {"G": 57.021464, "A": 71.037114, "S": 87.032028, "P": 97.052764,
                "V": 99.068414, "T": 101.047679, "C": 103.009185, "L": 113.084064,
                "I": 113.084064, "N": 114.042927, "D": 115.026943, "Q": 128.058578,
                "K": 128.094963, "E": 129.042593, "M": 131.040485, "H": 137.058912,
                "F": 147.068414, "R": 156.101111, "Y": 163.063329, "W": 186.079313}.items():
    _SIM_MASS[ord(_aa)] = _m
_SIM_WATER = 18.010565
_SIM_PROTON = 1.007276466812


@dataclass
class Proteome:
    seq: np.ndarray   # uint8, all proteins concatenated (ASCII letters)
    off: np.ndarray   # uint64, n+1 offsets

    @property
    def n(self) -> int:
        return len(self.off) - 1

    def protein(self, i: int) -> str:
        return self.seq[self.off[i]:self.off[i + 1]].tobytes().decode()


@dataclass
class Spectra:
    """A batch in the search library's input layout (CSR peaks)."""
    peak_off: np.ndarray   # uint64 [n+1]
    mz: np.ndarray         # float32 [sum N]
    intensity: np.ndarray  # float32 [sum N]
    prec_mz: np.ndarray    # float64 [n]
    charge: np.ndarray     # uint8 [n]
    tol_da: np.ndarray     # float64 [n]
    # ground truth of the simulation (not used by the search)
    truth_protein: np.ndarray
    truth_start: np.ndarray
    truth_len: np.ndarray
    truth_modpos: np.ndarray  # uint64 bitmask of modified positions

    @property
    def n(self) -> int:
        return len(self.prec_mz)

    def subset(self, idx) -> "Spectra":
        idx = np.asarray(idx, dtype=np.int64)
        starts = self.peak_off[idx].astype(np.int64)
        ends = self.peak_off[idx + 1].astype(np.int64)
        counts = ends - starts
        off = np.zeros(len(idx) + 1, dtype=np.uint64)
        off[1:] = np.cumsum(counts)
        gather = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if len(idx) else np.zeros(0, np.int64)
        return Spectra(off, self.mz[gather], self.intensity[gather], self.prec_mz[idx],
                       self.charge[idx], self.tol_da[idx], self.truth_protein[idx],
                       self.truth_start[idx], self.truth_len[idx], self.truth_modpos[idx])


def make_proteome(n_proteins: int, seed: int, length=(100, 800)) -> Proteome:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    lens = rng.integers(length[0], length[1] + 1, size=n_proteins)
    off = np.zeros(n_proteins + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    seq = _ALPHA[rng.choice(len(_ALPHA), size=int(off[-1]), p=_FREQ)]
    return Proteome(seq=np.ascontiguousarray(seq), off=off)


def _pick_peptides(prot: Proteome, n: int, rng, min_len: int, max_len: int, mc: int):
    """Random tryptic peptides (cleave after K/R unless followed by P)."""
    seq = prot.seq
    total = len(seq)
    off = prot.off.astype(np.int64)
    is_kr = (seq == ord("K")) | (seq == ord("R"))
    nxt_p = np.zeros(total, dtype=bool)
    nxt_p[:-1] = seq[1:] == ord("P")
    cut = np.nonzero(is_kr & ~nxt_p)[0] + 1          # boundary after a cleavage site
    bounds = np.unique(np.concatenate([off, cut]))   # protein starts/ends are boundaries
    prot_of = lambda x: np.searchsorted(off, x, side="right") - 1   # noqa: E731
    out_s, out_l, out_p = [], [], []
    need = n
    while need > 0:
        m = max(4 * need, 1024)
        a = rng.integers(0, len(bounds) - 1, size=m)
        b = a + rng.integers(1, mc + 2, size=m)
        ok = b < len(bounds)
        a, b = a[ok], b[ok]
        start, stop = bounds[a], bounds[b]
        pa = prot_of(start)
        ok = (start < total) & (pa == prot_of(stop - 1))
        ln = stop - start
        ok &= (ln >= min_len) & (ln <= max_len)
        out_s.append(start[ok][:need]); out_l.append(ln[ok][:need]); out_p.append(pa[ok][:need])
        need -= len(out_s[-1])
    return np.concatenate(out_s)[:n], np.concatenate(out_l)[:n], np.concatenate(out_p)[:n]


def make_spectra(prot: Proteome, w: Workload, n: Optional[int] = None, seed: Optional[int] = None) -> Spectra:
    """Simulated query spectra for workload ``w`` (vectorised over spectra)."""
    rec: SpectraRecipe = w.spectra
    p = w.params
    n = rec.n_spectra if n is None else n
    rng = np.random.default_rng(np.random.SeedSequence([w.seed if seed is None else seed, 2]))
    L = p.max_len
    # draw extra peptides, drop the ones outside the mass range after mods
    starts, lens, prots, modmask, masses = [], [], [], [], []
    got = 0
    while got < n:
        m = int((n - got) * 1.3) + 64
        s, ln, pr = _pick_peptides(prot, m, rng, p.min_len, p.max_len, p.missed_cleavages)
        res = np.zeros((m, L), dtype=np.uint8)
        col = np.arange(L)
        valid = col[None, :] < ln[:, None]
        idx = np.where(valid, s[:, None] + col[None, :], 0)
        res[valid] = prot.seq[idx[valid]]
        mass = _SIM_MASS[res] * valid
        mm = np.zeros(m, dtype=np.uint64)
        for mod in w.mods:
            sites = np.isin(res, np.frombuffer(mod.residues.encode(), np.uint8)) & valid
            if mod.fixed:
                mass = mass + sites * mod.delta_da
                continue
            nsite = sites.sum(1)
            cap = np.minimum(nsite, mod.max_per_peptide)
            cnt = np.floor(rng.random(m) * (cap + 1)).astype(np.int64)
            key = np.where(sites, rng.random((m, L)), np.inf)
            rank = np.argsort(np.argsort(key, axis=1), axis=1)
            chosen = sites & (rank < cnt[:, None])
            mass = mass + chosen * mod.delta_da
            bits = (chosen.astype(np.uint64) << col.astype(np.uint64)[None, :]).sum(1, dtype=np.uint64)
            mm |= bits
        M = mass.sum(1) + _SIM_WATER
        ok = (M >= p.min_mass) & (M <= p.max_mass)
        starts.append(s[ok]); lens.append(ln[ok]); prots.append(pr[ok])
        modmask.append(mm[ok]); masses.append(mass[ok])
        got += int(ok.sum())
    start = np.concatenate(starts)[:n]
    ln = np.concatenate(lens)[:n]
    pr = np.concatenate(prots)[:n]
    mm = np.concatenate(modmask)[:n]
    mass = np.concatenate(masses)[:n]
    M = mass.sum(1) + _SIM_WATER

    # b_i = prefix_i + proton, y_i = suffix_i + water + proton, i = 1..len-1
    pre = np.cumsum(mass, axis=1)[:, :-1]
    suf = (mass.sum(1)[:, None] - np.cumsum(mass, axis=1))[:, :-1]
    b = pre + _SIM_PROTON
    y = suf + _SIM_WATER + _SIM_PROTON
    ion_ok = np.arange(L - 1)[None, :] < (ln - 1)[:, None]
    ions = np.concatenate([b, y], axis=1)
    ions_ok = np.concatenate([ion_ok, ion_ok], axis=1)
    nion = ions_ok.sum(1)
    nkeep = np.floor(rec.keep_frac * nion + 0.5).astype(np.int64)
    key = np.where(ions_ok, rng.random(ions.shape), np.inf)
    rank = np.argsort(np.argsort(key, axis=1), axis=1)
    keep = ions_ok & (rank < nkeep[:, None])
    sig_mz = ions + rng.normal(0.0, rec.jitter_da, size=ions.shape)
    sig_cnt = keep.sum(1)
    if rec.target_peaks is None:
        noise_cnt = rng.integers(rec.noise_lo, rec.noise_hi + 1, size=n)
    else:
        tgt = rng.integers(rec.target_peaks[0], rec.target_peaks[1] + 1, size=n)
        noise_cnt = np.maximum(tgt - sig_cnt, 0)
    tot = sig_cnt + noise_cnt
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum(tot)
    sig_vals = sig_mz[keep]
    sig_owner = np.repeat(np.arange(n), sig_cnt)
    noise_vals = rng.uniform(rec.mz_lo, rec.mz_hi, size=int(noise_cnt.sum()))
    noise_owner = np.repeat(np.arange(n), noise_cnt)
    all_mz = np.concatenate([sig_vals, noise_vals])
    owner = np.concatenate([sig_owner, noise_owner])
    order = np.lexsort((all_mz, owner))
    mz = all_mz[order].astype(np.float32)
    inten = (np.exp(rng.normal(0.0, 1.0, size=len(mz))) * 1000.0).astype(np.float32)
    z = rng.choice(np.array(rec.charges, dtype=np.int64), size=n)
    prec = (M + z * _SIM_PROTON) / z
    tol = rng.choice(np.array(rec.tol_da, dtype=np.float64), size=n)
    return Spectra(peak_off=off, mz=mz, intensity=inten, prec_mz=prec.astype(np.float64),
                   charge=z.astype(np.uint8), tol_da=tol, truth_protein=pr, truth_start=start,
                   truth_len=ln, truth_modpos=mm)


def make_workload_inputs(w: Workload, n_spectra: Optional[int] = None):
    prot = make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    spec = make_spectra(prot, w, n_spectra)
    return prot, spec


def write_ms2(spec: Spectra, path: str, sel=None, scan_base: int = 1) -> None:
    """Writes spectra ``sel`` (all when None) as an MS2 text file: every
    float32 peak and float64 precursor m/z written to round-trip exactly; a
    spectrum of charge 0 gets no Z line."""
    idx = range(spec.n) if sel is None else sel
    with open(path, "w") as f:
        f.write("H\tExtractor\tsynthetic\n")
        for j, q in enumerate(idx):
            a, e = int(spec.peak_off[q]), int(spec.peak_off[q + 1])
            pm = float(spec.prec_mz[q])
            z = int(spec.charge[q])
            f.write(f"S\t{scan_base + j}\t{scan_base + j}\t{pm!r}\n")
            if z:
                f.write(f"Z\t{z}\t{(pm - 1.007276466812) * z + 1.007276466812:.6f}\n")
            for m, i in zip(spec.mz[a:e], spec.intensity[a:e]):
                f.write(str(np.float32(m)) + " " + str(np.float32(i)) + "\n")   # shortest float32 round-trip


def spectra_from_lists(peaks, prec_mz, charge, tol) -> Spectra:
    """Hand-built batch (tests): ``peaks`` is a list of (mz list, intensity list)."""
    n = len(peaks)
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(m) for m, _ in peaks])
    mz = np.array([v for m, _ in peaks for v in m], dtype=np.float32)
    it = np.array([v for _, i in peaks for v in i], dtype=np.float32)
    z = np.zeros(n, dtype=np.int64)
    return Spectra(off, mz, it, np.asarray(prec_mz, np.float64), np.asarray(charge, np.uint8),
                   np.asarray(tol, np.float64), z, z, z, z.astype(np.uint64))
