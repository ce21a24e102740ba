"""Pins for the CPU oracle, against facts that do not come from the oracle.

* elemental-composition masses (a different arithmetic route than the
  residue-mass table) for the peptides printed in the paper (Supplementary
  Table 1, Supplementary Text 3) and the textbook y1 ions of K and R;
* hand-worked digestion cases (trypsin rule, missed cleavages, length and
  mass limits, the paper's Experimental Setup digestion);
* the closed-form variant count of the 2^m enumeration (Notation section);
* closed forms of the hyperscore, the rank key and the histogram bin;
* closed forms of the survival-tail fit (Superstep 4 e-value);
* hand-worked preprocessing cases;
* a brute-force re-implementation on tiny inputs (different digestion,
  enumeration, ordering and all-pairs matching code);
* invariants: shared counts <= min(query bins, peptide bins), window
  monotonicity, and the self-match of a noise-free spectrum;
* the e-value variants: the Savitzky-Golay smoothing (R16) against scipy's
  savgol_filter with the tail fit done by numpy's polyfit, the log-Weibull
  fit (R17) against numpy's polyfit and scipy's Gumbel survival function,
  and the recovery of a known Gumbel's location and scale from its binned
  counts;
* the LBE partition (R18): the paper's Mod Distance worked example, textbook
  edit distances, a Python brute force of the partition, and its balance
  (partition sizes and every cluster split evenly);
* the fragment tolerance of t bins (R15): a hand-worked spectrum with peaks
  one and two bins off the ions and two peaks covering one ion, the brute
  force above with every (ion, peak) pair compared by bin distance, the
  closed form when every peak covers every bin, and monotonicity in t.
"""
import dataclasses
import itertools
import math
import os

import numpy as np
import pytest

from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300.configs import Mod, SearchParams

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# monoisotopic atomic masses (IUPAC/AME) and the electron mass
ATOM = {"C": 12.0, "H": 1.00782503207, "N": 14.0030740048, "O": 15.99491461956,
        "S": 31.97207100, "P": 30.97376163}
ELECTRON = 0.00054857990946
# residue (amino acid minus water) elemental compositions
RESIDUE_FORMULA = {
    "G": "C2H3NO", "A": "C3H5NO", "S": "C3H5NO2", "P": "C5H7NO", "V": "C5H9NO",
    "T": "C4H7NO2", "C": "C3H5NOS", "L": "C6H11NO", "I": "C6H11NO", "N": "C4H6N2O2",
    "D": "C4H5NO3", "Q": "C5H8N2O2", "K": "C6H12N2O", "E": "C5H7NO3", "M": "C5H9NOS",
    "H": "C6H7N3O", "F": "C9H9NO", "R": "C6H12N4O", "Y": "C9H9NO2", "W": "C11H10N2O",
}
CAM = "C2H3NO"      # carbamidomethyl
OXID = "O"
PHOS = "HPO3"


def formula_mass(f: str) -> float:
    m, i = 0.0, 0
    while i < len(f):
        el = f[i]
        i += 1
        num = ""
        while i < len(f) and f[i].isdigit():
            num += f[i]
            i += 1
        m += ATOM[el] * (int(num) if num else 1)
    return m


WATER = 2 * ATOM["H"] + ATOM["O"]
PROTON = ATOM["H"] - ELECTRON


def paper_peptides():
    with open(os.path.join(GOLDEN, "paper_peptides.txt")) as f:
        return [l.strip() for l in f if l.strip() and not l.startswith("#")]


def single_peptide_db(oracle_lib, seq, mods=(configs.CARBAMIDOMETHYL_C,), **extra):
    """Database whose only protein is ``seq``; returns (db, pid of full seq)."""
    p = SearchParams(min_len=2, max_len=60, missed_cleavages=10, min_mass=0.0, max_mass=1e5, **extra)
    prot = np.frombuffer(seq.encode(), np.uint8)
    db = oracle_lib.OracleDb(prot, np.array([0, len(seq)], np.uint64), list(mods), p)
    hits = [i for i in range(db.n) if db.peptide(i)[0] == seq and not db.peptide(i)[2].any()]
    assert len(hits) == 1
    return db, hits[0]


# ---------------------------------------------------------------- masses


@pytest.mark.parametrize("seq", paper_peptides())
def test_by_ions_match_elemental_composition(oracle_lib, seq):
    db, pid = single_peptide_db(oracle_lib, seq)
    res = [formula_mass(RESIDUE_FORMULA[a]) + (formula_mass(CAM) if a == "C" else 0.0) for a in seq]
    M = sum(res) + WATER
    b_exp = [sum(res[:i]) + PROTON for i in range(1, len(seq))]
    y_exp = [sum(res[i:]) + WATER + PROTON for i in range(1, len(seq))]
    b, y = db.ions(pid)
    _, mass, _ = db.peptide(pid)
    assert abs(mass - M) < 2e-5
    np.testing.assert_allclose(b, b_exp, atol=2e-5, rtol=0)
    np.testing.assert_allclose(y, y_exp, atol=2e-5, rtol=0)


def test_y1_of_lys_and_arg(oracle_lib):
    # textbook y1 ions: K 147.112804, R 175.118952
    for seq, y1 in (("AAAAK", 147.112804), ("AAAAR", 175.118952)):
        db, pid = single_peptide_db(oracle_lib, seq)
        _, y = db.ions(pid)
        assert abs(y[-1] - y1) < 2e-6


def test_variable_mod_masses(oracle_lib):
    # MEGSYIRK of Supplementary Text 3 with oxidised M and phosphorylated S
    mods = [configs.CARBAMIDOMETHYL_C, configs.OX_M(1), configs.PHOSPHO_STY(1)]
    p = SearchParams(min_len=2, max_len=60, missed_cleavages=10, min_mass=0.0, max_mass=1e5)
    seq = "MEGSYIRK"
    db = oracle_lib.OracleDb(np.frombuffer(seq.encode(), np.uint8), np.array([0, 8], np.uint64), mods, p)
    base = [formula_mass(RESIDUE_FORMULA[a]) for a in seq]
    found = 0
    for pid in range(db.n):
        s, mass, codes = db.peptide(pid)
        if s != seq:
            continue
        res = list(base)
        for j, c in enumerate(codes):
            if c == 1:
                res[j] += formula_mass(OXID)
            elif c == 2:
                res[j] += formula_mass(PHOS)
        assert abs(mass - (sum(res) + WATER)) < 2e-5
        b, y = db.ions(pid)
        np.testing.assert_allclose(b, [sum(res[:i]) + PROTON for i in range(1, 8)], atol=2e-5, rtol=0)
        np.testing.assert_allclose(y, [sum(res[i:]) + WATER + PROTON for i in range(1, 8)], atol=2e-5, rtol=0)
        found += 1
    # M: 0/1 oxidation (2 states) x S/Y: none, S or Y (3 states)
    assert found == 6


# ---------------------------------------------------------------- digestion


def peptides_of(db):
    return sorted(db.peptide(i)[0] for i in range(db.n))


def test_digest_hand_case(oracle_lib):
    #   AAAAAAAK|PGGGGGGR  (K before P: no cut)   LLLLLLLK   VVVVVVV
    prot = "AAAAAAAKPGGGGGGR" + "LLLLLLLK" + "VVVVVVV"
    p = SearchParams(min_len=7, max_len=40, missed_cleavages=1, min_mass=500.0, max_mass=5000.0)
    db = oracle_lib.OracleDb(np.frombuffer(prot.encode(), np.uint8), np.array([0, len(prot)], np.uint64), [], p)
    exp = sorted(["AAAAAAAKPGGGGGGR", "LLLLLLLK", "VVVVVVV",
                  "AAAAAAAKPGGGGGGRLLLLLLLK", "LLLLLLLKVVVVVVV"])
    assert peptides_of(db) == exp
    p0 = SearchParams(min_len=7, max_len=40, missed_cleavages=0, min_mass=500.0, max_mass=5000.0)
    db0 = oracle_lib.OracleDb(np.frombuffer(prot.encode(), np.uint8), np.array([0, len(prot)], np.uint64), [], p0)
    assert peptides_of(db0) == sorted(["AAAAAAAKPGGGGGGR", "LLLLLLLK", "VVVVVVV"])


def test_digest_limits_and_dedup(oracle_lib):
    # GGGGGK: length 6 < 7 dropped; GGGGGGGK: 7 residues but mass 546.2 kept;
    # GGGGGGK (6) dropped; SSSSSSK mass 674 kept; two copies of a protein
    # give one entry per peptide; a peptide with 'X' is skipped.
    p = SearchParams(min_len=7, max_len=10, missed_cleavages=0, min_mass=540.0, max_mass=5000.0)
    prots = ["GGGGGKGGGGGGGKSSSSSSK", "GGGGGKGGGGGGGKSSSSSSK", "AAXAAAAK"]
    seq = "".join(prots)
    off = np.cumsum([0] + [len(x) for x in prots]).astype(np.uint64)
    db = oracle_lib.OracleDb(np.frombuffer(seq.encode(), np.uint8), off, [], p)
    assert peptides_of(db) == ["GGGGGGGK", "SSSSSSK"]
    # mass limit: 7 glycines + K = 7*57.021464+128.094963+18.010565 = 545.256 < 550
    p2 = SearchParams(min_len=7, max_len=10, missed_cleavages=0, min_mass=550.0, max_mass=5000.0)
    db2 = oracle_lib.OracleDb(np.frombuffer(seq.encode(), np.uint8), off, [], p2)
    assert peptides_of(db2) == ["SSSSSSK"]


def test_variant_count_closed_form(oracle_lib):
    # MSMSTYK: 2 M sites (<= 2 ox), 4 STY sites (<= 1 phospho):
    # (C(2,0)+C(2,1)+C(2,2)) * (C(4,0)+C(4,1)) = 4 * 5 = 20
    seq = "MSMSTYK"
    p = SearchParams(min_len=2, max_len=60, missed_cleavages=0, min_mass=0.0, max_mass=1e5)
    mods = [configs.OX_M(2), configs.PHOSPHO_STY(1)]
    db = oracle_lib.OracleDb(np.frombuffer(seq.encode(), np.uint8), np.array([0, 7], np.uint64), mods, p)
    assert db.n == 20
    # a global cap of 1 modification: 1 + 2 + 4 = 7
    p1 = SearchParams(min_len=2, max_len=60, missed_cleavages=0, min_mass=0.0, max_mass=1e5, max_total_mods=1)
    db1 = oracle_lib.OracleDb(np.frombuffer(seq.encode(), np.uint8), np.array([0, 7], np.uint64), mods, p1)
    assert db1.n == 7
    # pid order: masses ascending
    m = db.masses()
    assert np.all(np.diff(m) >= 0)


# ---------------------------------------------------------------- scoring


def test_hyperscore_closed_form(oracle_lib):
    # nb=3, ny=2, S=1000: log10(3! * 2! * 1000) = log10(12000)
    assert abs(oracle_lib.hyperscore(3, 2, 1000) - 4.079181246047625) < 1e-12
    assert oracle_lib.hyperscore(0, 1, 1) == 0.0
    for nb, ny, S in ((3, 2, 1000), (10, 7, 54321), (0, 4, 1), (39, 39, 780000)):
        K = oracle_lib.rank_key(nb, ny, S)
        hs = math.log10(math.factorial(nb) * math.factorial(ny) * S)
        assert abs(K / 2.0 ** 32 - hs) < 3 * 2.0 ** -32 + 1e-12 * hs
    # the key is monotone in each argument
    assert oracle_lib.rank_key(4, 2, 100) > oracle_lib.rank_key(3, 2, 100)
    assert oracle_lib.rank_key(3, 3, 100) > oracle_lib.rank_key(3, 2, 100)
    assert oracle_lib.rank_key(3, 2, 101) > oracle_lib.rank_key(3, 2, 100)


def test_evalue_geometric_tail(oracle_lib):
    # hist_j = 2^(30-j): survival s_j = 2^(31-j) - 1, a line of slope
    # log10(1/2) in log space; the fit at an integer x returns ~s_j / N * N
    hist = np.zeros(256, np.uint32)
    for j in range(31):
        hist[j] = 2 ** (30 - j)
    N = float(hist.sum())
    jtop = 20
    key = jtop * 2 ** 31
    ev = oracle_lib.evalue(hist, [key], [0])
    s = float(hist[jtop:].sum())
    assert abs(ev[0] - s) / s < 1e-3
    # at x = jtop + 0.5 the tail is sqrt(1/2) lower
    ev2 = oracle_lib.evalue(hist, [key + 2 ** 30], [0])
    assert abs(ev2[0] / ev[0] - 2 ** -0.5) < 1e-4
    assert N == 2 ** 31 - 1


def test_evalue_fallback_and_window(oracle_lib):
    # one populated bin: no fit points -> e = N
    hist = np.zeros(256, np.uint32)
    hist[5] = 17
    ev = oracle_lib.evalue(hist, [5 * 2 ** 31], [3])
    assert ev[0] == 17.0
    # padding rows keep +inf
    ev = oracle_lib.evalue(hist, [5 * 2 ** 31, -(2 ** 63)], [3, 0xFFFFFFFF])
    assert ev[1] == math.inf
    # counts at or below the mode only rescale N and the intercept together:
    # e = N * 10^(w x + b) is unchanged
    h = np.zeros(256, np.uint32)
    for j in range(2, 16):
        h[j] = 4 ** (15 - j)
    base = oracle_lib.evalue(h, [14 * 2 ** 31], [0])
    h2 = h.copy()
    h2[0] += 3
    h2[1] += 5
    h2[2] += 1000
    alt = oracle_lib.evalue(h2, [14 * 2 ** 31], [0])
    assert abs(alt[0] / base[0] - 1) < 1e-9
    # fit points are mode+1 .. jtop-1: mode 0 and jtop 3 give two points
    # (fallback e = N), jtop 4 gives three (a fit, e < N)
    g = np.zeros(256, np.uint32)
    g[:8] = [64, 32, 16, 8, 4, 2, 1, 1]
    assert oracle_lib.evalue(g, [3 * 2 ** 31], [0])[0] == float(g.sum())
    assert oracle_lib.evalue(g, [4 * 2 ** 31], [0])[0] < float(g.sum())


# ---------------------------------------------------------------- preprocessing


def test_preprocess_hand_cases(oracle_lib):
    p = SearchParams(top_n_peaks=3, bin_width_da=0.01, intensity_scale=10000)
    mz = [100.0, 150.004, 150.006, 200.0, 2000.0, 99.99, 300.0, 400.0, 500.0, float("nan")]
    it = [1000.0, 10.0, 20.0, 500.0, 9e9, 9e9, 0.0, -1.0, 500.0, 5.0]
    bins, iq, Mq, valid = oracle_lib.preprocess(p, mz, it, 500.0, 2, 10.0)
    # 150.004 and 150.006 share bin 15000 (max 20 kept); 2000.0 and 99.99
    # are out of range; 0 / negative intensity and NaN dropped; top-3 of
    # {10000:1000, 15000:20, 20000:500, 50000:500} -> 1000, 500 (bin 20000),
    # 500 (bin 50000), ties to the lower bin
    assert list(bins) == [10000, 20000, 50000]
    assert list(iq) == [10000, 5000, 5000]
    assert valid
    assert Mq == (500.0 - PROTON_CONST) * 2
    # iq floor and the minimum of 1
    bins, iq, _, _ = oracle_lib.preprocess(SearchParams(top_n_peaks=10), [100.0, 200.0, 300.0],
                                           [1000.0, 0.01, 333.5], 500.0, 2, 10.0)
    assert list(iq) == [10000, 1, 3335]
    # charge 0 or no peaks in range: invalid
    assert not oracle_lib.preprocess(p, [150.0], [1.0], 500.0, 0, 10.0)[3]
    assert not oracle_lib.preprocess(p, [50.0], [1.0], 500.0, 2, 10.0)[3]


PROTON_CONST = 1.007276466812


# ---------------------------------------------------------------- brute force

RES_MASS = {"G": 57.021464, "A": 71.037114, "S": 87.032028, "P": 97.052764, "V": 99.068414,
            "T": 101.047679, "C": 103.009185, "L": 113.084064, "I": 113.084064, "N": 114.042927,
            "D": 115.026943, "Q": 128.058578, "K": 128.094963, "E": 129.042593, "M": 131.040485,
            "H": 137.058912, "F": 147.068414, "R": 156.101111, "Y": 163.063329, "W": 186.079313}


def test_residue_table_matches_composition():
    for aa, f in RESIDUE_FORMULA.items():
        assert abs(RES_MASS[aa] - formula_mass(f)) < 1e-6


def brute_force_search(prot_seqs, mods, p: SearchParams, spec):
    """All-pairs re-implementation: substring digestion, itertools variants,
    Python sort, every (peak, ion) pair compared."""
    fixed = {}
    var = []
    for m in mods:
        if m.fixed:
            for r in m.residues:
                fixed[r] = m.delta_da
        else:
            var.append(m)

    def is_cut(s, k):  # boundary before position k
        return k == 0 or k == len(s) or (s[k - 1] in "KR" and s[k] != "P")

    peps = {}
    for s in prot_seqs:
        for i in range(len(s)):
            for j in range(i + p.min_len, min(len(s), i + p.max_len) + 1):
                if not (is_cut(s, i) and is_cut(s, j)):
                    continue
                if sum(1 for k in range(i + 1, j) if is_cut(s, k)) > p.missed_cleavages:
                    continue
                sub = s[i:j]
                if any(c not in RES_MASS for c in sub):
                    continue
                site_lists = [[k for k, c in enumerate(sub) if c in m.residues] for m in var]
                choices = []
                for t, sites in enumerate(site_lists):
                    opts = []
                    for c in range(0, min(len(sites), var[t].max_per_peptide) + 1):
                        opts.extend(itertools.combinations(sites, c))
                    choices.append(opts)
                for combo in itertools.product(*choices) if var else [()]:
                    code = [0] * len(sub)
                    for t, pos in enumerate(combo):
                        for k in pos:
                            code[k] = t + 1
                    if p.max_total_mods and sum(1 for c in code if c) > p.max_total_mods:
                        continue
                    ms = []
                    for k, c in enumerate(sub):
                        m = RES_MASS[c]
                        if c in fixed:
                            m = m + fixed[c]
                        if code[k]:
                            m = m + var[code[k] - 1].delta_da
                        ms.append(m)
                    tot = 0.0
                    for m in ms:
                        tot = tot + m
                    M = tot + 18.010565
                    if p.min_mass <= M <= p.max_mass:
                        peps[(sub, tuple(code))] = (M, ms)
    order = sorted(peps, key=lambda k: (peps[k][0], k[0], k[1]))
    masses = [peps[k][0] for k in order]
    w = p.bin_width_da
    out = []
    for q in range(spec.n):
        a, e = int(spec.peak_off[q]), int(spec.peak_off[q + 1])
        best = {}
        for mz, I in zip(spec.mz[a:e], spec.intensity[a:e]):
            mz, I = float(mz), float(I)
            if not (math.isfinite(mz) and math.isfinite(I) and I > 0 and p.frag_mz_min <= mz < p.frag_mz_max):
                continue
            bn = math.floor(mz / w)
            best[bn] = max(best.get(bn, 0.0), I)
        kept = sorted(best.items(), key=lambda t: (-t[1], t[0]))[:p.top_n_peaks]
        z = int(spec.charge[q])
        res = {"pids": [], "hist": [0] * 256, "nscored": 0}
        if not kept or z == 0:
            out.append(res)
            continue
        Imax = kept[0][1]
        qb = {bn: max(1, math.floor((I * p.intensity_scale) / Imax)) for bn, I in kept}
        Mq = (float(spec.prec_mz[q]) - 1.007276466812) * z
        tol = float(spec.tol_da[q])
        cands = []
        for pid, key in enumerate(order):
            if not (Mq - tol <= masses[pid] <= Mq + tol):
                continue
            ms = peps[key][1]
            L = len(ms)
            bset, yset = set(), set()
            for i in range(1, L):
                bm = 0.0
                for m in ms[:i]:
                    bm = bm + m
                bm = bm + 1.007276466812
                ym = 0.0
                for m in reversed(ms[i:]):
                    ym = ym + m
                ym = (ym + 18.010565) + 1.007276466812
                if p.frag_mz_min <= bm < p.frag_mz_max:
                    bset.add(math.floor(bm / w))
                if p.frag_mz_min <= ym < p.frag_mz_max:
                    yset.add(math.floor(ym / w))
            yset -= bset
            nb = ny = S = 0
            if p.tol_bins == 0:
                for bn, iqv in qb.items():
                    if bn in bset:
                        nb += 1
                        S += iqv
                    elif bn in yset:
                        ny += 1
                        S += iqv
            else:
                # every (ion bin, peak bin) pair; an ion bin counts once, with
                # the largest iq of the peaks within tol_bins of it
                for x in bset | yset:
                    cover = [iqv for bn, iqv in qb.items() if abs(bn - x) <= p.tol_bins]
                    if cover:
                        if x in bset:
                            nb += 1
                        else:
                            ny += 1
                        S += max(cover)
            if nb + ny >= p.min_shared:
                lfb = lfy = 0.0
                for i in range(2, nb + 1):
                    lfb = lfb + math.log10(i)
                for i in range(2, ny + 1):
                    lfy = lfy + math.log10(i)
                hs = lfb + lfy + math.log10(S)
                key = (int(np.rint(math.ldexp(lfb, 32))) + int(np.rint(math.ldexp(lfy, 32)))
                       + int(np.rint(math.ldexp(math.log10(S), 32))))
                cands.append((pid, nb, ny, S, hs, key))
        res["nscored"] = len(cands)
        res["cands"] = cands
        out.append(res)
    return order, masses, out


@pytest.mark.parametrize("min_shared,tol", [(4, 500.0), (3, 50.0)])
def test_oracle_matches_brute_force(oracle_lib, min_shared, tol):
    check_against_brute_force(oracle_lib, SearchParams(missed_cleavages=1, min_shared=min_shared, top_k=5,
                                                       top_n_peaks=60), tol)


@pytest.mark.parametrize("tol_bins,min_shared", [(1, 4), (2, 3), (3, 4)])
def test_tolerance_matches_brute_force(oracle_lib, tol_bins, min_shared):
    # a 0.005 Da grid: dF = tol_bins * 0.005 Da
    check_against_brute_force(oracle_lib, SearchParams(missed_cleavages=1, min_shared=min_shared, top_k=5,
                                                       top_n_peaks=60, bin_width_da=0.005,
                                                       tol_bins=tol_bins), 500.0)


def check_against_brute_force(oracle_lib, params, tol):
    w = configs.OPEN_MEDIUM
    prot = synth.make_proteome(12, seed=7, length=(60, 120))
    wl = configs.Workload("bf", 99, 12, w.mods, params,
                          configs.SpectraRecipe(n_spectra=12, noise_lo=30, noise_hi=60, tol_da=(tol,)))
    spec = synth.make_spectra(prot, wl)
    prots = [prot.protein(i) for i in range(prot.n)]
    order, masses, bf = brute_force_search(prots, w.mods, params, spec)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, params)
    assert db.n == len(order)
    np.testing.assert_array_equal(db.masses(), np.array(masses))
    for i in range(0, db.n, max(1, db.n // 50)):
        s, _, codes = db.peptide(i)
        assert (s, tuple(int(c) for c in codes)) == order[i]
    r = db.search(spec)
    n_any = 0
    for q in range(spec.n):
        assert r.n_scored[q] == bf[q]["nscored"]
        cands = bf[q].get("cands", [])
        n_any += len(cands)
        # histogram bin = K >> 31 = floor(2 * HS) (0.5 log10 units per bin)
        h = np.zeros(256, np.uint32)
        for c in cands:
            h[min(255, c[5] >> 31)] += 1
            assert (c[5] >> 31) == int(math.floor(2 * c[4]))
        np.testing.assert_array_equal(r.hist[q], h)
        top = sorted(cands, key=lambda c: (-c[5], c[0]))[:5]
        for k, c in enumerate(top):
            row = r.psm[q, k]
            assert (row["pid"], row["nb"], row["ny"], row["S"], row["key"]) == c[:4] + (c[5],)
            assert abs(row["hyperscore"] - c[4]) < 1e-9
        for k in range(len(top), 5):
            assert r.psm[q, k]["pid"] == 0xFFFFFFFF
    assert n_any > 0


# ---------------------------------------------------------------- invariants


@pytest.fixture(scope="module")
def tiny(oracle_lib):
    w = configs.TINY_CLOSED.with_proteins(120).with_spectra(80)
    prot, spec = synth.make_workload_inputs(w)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    return w, prot, spec, db


def test_counts_bounded(oracle_lib, tiny):
    w, prot, spec, db = tiny
    r = db.search(spec)
    for q in range(spec.n):
        a, e = int(spec.peak_off[q]), int(spec.peak_off[q + 1])
        qb, _, _, _ = oracle_lib.preprocess(w.params, spec.mz[a:e], spec.intensity[a:e],
                                            float(spec.prec_mz[q]), int(spec.charge[q]), float(spec.tol_da[q]))
        for row in r.psm[q]:
            if row["pid"] == 0xFFFFFFFF:
                continue
            nbins = len(db.bins(int(row["pid"]))[0])
            assert row["nb"] + row["ny"] <= min(len(qb), nbins)
            assert row["nb"] + row["ny"] >= w.params.min_shared


def test_window_monotone(oracle_lib, tiny):
    w, prot, spec, db = tiny
    r10 = db.search(spec)
    s5 = synth.Spectra(spec.peak_off, spec.mz, spec.intensity, spec.prec_mz, spec.charge,
                       spec.tol_da * 0.25, spec.truth_protein, spec.truth_start, spec.truth_len, spec.truth_modpos)
    r5 = db.search(s5)
    assert np.all(r5.lo >= r10.lo) and np.all(r5.hi <= r10.hi)
    assert np.all(r5.hist <= r10.hist)
    assert np.all(r5.n_scored <= r10.n_scored)


def test_self_match_is_top1(oracle_lib, tiny):
    w, prot, spec, db = tiny
    rng = np.random.default_rng(3)
    pids = rng.choice(db.n, size=25, replace=False)
    peaks, prec, z = [], [], []
    for pid in pids:
        # one peak at the centre of each ion bin (float32 m/z cannot cross a bin edge)
        bins, _ = db.bins(int(pid))
        mzs = [(float(bn) + 0.5) * w.params.bin_width_da for bn in bins]
        peaks.append((mzs, [100.0] * len(mzs)))
        _, mass, _ = db.peptide(int(pid))
        prec.append((mass + 2 * PROTON_CONST) / 2)
        z.append(2)
    sp = synth.spectra_from_lists(peaks, prec, z, [10.0] * len(pids))
    r = db.search(sp)
    for i, pid in enumerate(pids):
        nb = len(db.bins(int(pid))[0])
        top = r.psm[i, 0]
        if nb < w.params.min_shared:
            continue
        # the peptide itself, or an equal-key isobaric peptide with a lower pid
        if top["pid"] != pid:
            assert top["pid"] < pid
            row = [x for x in r.psm[i] if x["pid"] == pid]
            assert row and row[0]["key"] == top["key"]
        else:
            assert top["nb"] + top["ny"] == nb


# ---------------------------------------------------------------- R15: t bins


def test_tolerance_hand_case(oracle_lib):
    scale = 10000
    db, pid = single_peptide_db(oracle_lib, "SAMPLERTIDEK", tol_bins=0, min_shared=1, intensity_scale=scale)
    bins, is_y = db.bins(pid)
    bins = [int(b) for b in bins]
    bb = [b for b, y in zip(bins, is_y) if not y]
    yb = [b for b, y in zip(bins, is_y) if y]
    xb1, xb2, yb1, yb2 = bb[1], bb[3], yb[1], yb[3]
    # peak bin, intensity (iq = floor(I * scale / 1000))
    peaks = [(xb1 + 1, 1000.0),    # one bin above a b ion: iq 10000
             (yb1 - 1, 500.0),     # both sides of a y ion: iq 5000 ...
             (yb1 + 1, 250.0),     # ... and 2500 (the ion takes the larger)
             (xb2, 100.0),         # on a b ion: iq 1000
             (yb2 + 2, 800.0)]     # two bins above a y ion: iq 8000
    for b, _ in peaks:   # no other ion bin within 3 bins of a peak
        near = [x for x in bins if abs(x - b) <= 3]
        assert len(near) == 1
    w = 0.01
    _, mass, _ = db.peptide(pid)
    sp = synth.spectra_from_lists([([(b + 0.5) * w for b, _ in peaks], [I for _, I in peaks])],
                                  [(mass + 2 * PROTON_CONST) / 2], [2], [0.001])
    want = {0: (1, 0, 1000), 1: (2, 1, 10000 + 5000 + 1000), 2: (2, 2, 10000 + 5000 + 1000 + 8000),
            3: (2, 2, 24000)}
    for t, (nb, ny, S) in want.items():
        dbt, pt = single_peptide_db(oracle_lib, "SAMPLERTIDEK", tol_bins=t, min_shared=1, intensity_scale=scale)
        assert pt == pid
        r = dbt.search(sp)
        rows = [x for x in r.psm[0] if x["pid"] == pid]
        assert rows, t
        assert (int(rows[0]["nb"]), int(rows[0]["ny"]), int(rows[0]["S"])) == (nb, ny, S), t


def test_tolerance_covering_everything(oracle_lib, tiny):
    # every retained peak covers every bin: each in-range ion bin is shared,
    # each with the top peak's iq = intensity_scale
    w, prot, spec, _ = tiny
    p = dataclasses.replace(w.params, tol_bins=10 ** 7)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, p)
    r = db.search(spec)
    n_real = 0
    for q in range(spec.n):
        want = sum(1 for pid in range(int(r.lo[q]), int(r.hi[q]))
                   if len(db.bins(pid)[0]) >= p.min_shared)
        assert r.n_scored[q] == want
        for row in r.psm[q]:
            if row["pid"] == 0xFFFFFFFF:
                continue
            n_real += 1
            bins, is_y = db.bins(int(row["pid"]))
            assert (row["nb"], row["ny"]) == (int(np.sum(is_y == 0)), int(np.sum(is_y == 1)))
            assert row["S"] == len(bins) * p.intensity_scale
    assert n_real > 0


def test_tolerance_monotone(oracle_lib, tiny):
    # a larger t covers a superset of bins, each with a larger-or-equal iq
    w, prot, spec, _ = tiny
    prev = None
    for t in (0, 1, 2, 4):
        db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, dataclasses.replace(w.params, tol_bins=t))
        r = db.search(spec)
        if prev is not None:
            assert np.all(r.n_scored >= prev.n_scored)
            has = prev.psm["pid"][:, 0] != 0xFFFFFFFF
            assert np.all(r.psm["key"][has, 0] >= prev.psm["key"][has, 0])
        prev = r


# ---------------------------------------------------------------- R16, R17


def _keys(xs):
    return np.array([int(round(x * 2 ** 31)) for x in xs], np.int64)


def _binned_gumbel(mu, beta, m):
    from scipy.stats import gumbel_r
    f = gumbel_r.cdf(np.arange(257, dtype=float), loc=mu, scale=beta)
    return np.rint(m * np.diff(f)).astype(np.uint32)


def _fit_points(g, ev_mode, jtop):
    """(x, y) of the fit from the fit's histogram g (numpy)."""
    G = np.concatenate([np.cumsum(g[::-1])[::-1], [0]]).astype(np.float64)
    if ev_mode & 1:
        sel = (G[1:] > 0) & (G[1:] < G[0])
        return np.arange(1, 257)[sel].astype(float), -np.log(-np.log1p(-(G[1:][sel] / G[0])))
    mode = int(np.argmax(g))
    j = np.arange(256)
    sel = (j >= mode + 1) & (j <= jtop - 1) & (G[:256] > 0)
    return j[sel].astype(float), np.log10(G[:256][sel] / G[0])


@pytest.mark.parametrize("ev_mode", [1, 2, 3])
def test_evalue_variants_against_library_routines(oracle_lib, ev_mode):
    signal = pytest.importorskip("scipy.signal")
    from scipy.stats import gumbel_r
    rng = np.random.default_rng(ev_mode)
    for trial in range(4):
        h = _binned_gumbel(25.0 + 10 * trial, 3.0 + trial, 10 ** (5 + trial))
        h[int(rng.integers(5, 60))] += np.uint32(rng.integers(1000, 50000))   # a spike the smoothing spreads
        xs = [float(v) for v in np.sort(rng.uniform(30, 90, 5))[::-1]]
        keys = _keys(xs)
        pids = np.arange(5, dtype=np.uint32)
        got = oracle_lib.evalue(h, keys, pids, ev_mode)
        g = h.astype(np.float64)
        if ev_mode & 2:   # 35 x the 5-point quadratic smoothing, zero outside
            g = np.rint(35 * signal.savgol_filter(g, 5, 2, mode="constant", cval=0.0))
            assert np.allclose(signal.savgol_coeffs(5, 2) * 35, [-3, 12, 17, 12, -3])
        x, y = _fit_points(g, ev_mode, min(255, int(keys[0]) >> 31))
        N = float(h.sum())
        a, c = np.polyfit(x, y, 1)
        if ev_mode & 1:
            want = N * gumbel_r.sf(np.asarray(xs), loc=-c / a, scale=1 / a)
        else:
            want = N * 10 ** (a * np.asarray(xs) + c)
        np.testing.assert_allclose(got, want, rtol=1e-8)
    # mass in the first and last two bins: the histogram is 0 outside its bins
    h = _binned_gumbel(20.0, 4.0, 10 ** 5)
    h[0] += np.uint32(700)
    h[1] += np.uint32(90)
    h[254] += np.uint32(3)
    h[255] += np.uint32(11)
    keys = _keys([200.0, 60.0, 40.0])
    got = oracle_lib.evalue(h, keys, np.arange(3, dtype=np.uint32), ev_mode)
    g = h.astype(np.float64)
    if ev_mode & 2:
        g = np.rint(35 * signal.savgol_filter(g, 5, 2, mode="constant", cval=0.0))
    x, y = _fit_points(g, ev_mode, min(255, int(keys[0]) >> 31))
    a, c = np.polyfit(x, y, 1)
    xs = np.array([200.0, 60.0, 40.0])
    want = float(h.sum()) * (gumbel_r.sf(xs, loc=-c / a, scale=1 / a) if ev_mode & 1 else 10 ** (a * xs + c))
    np.testing.assert_allclose(got, want, rtol=1e-8)
    # the smoothing changes the answer
    h = _binned_gumbel(30.0, 3.0, 10 ** 6)
    h[20] += np.uint32(40000)
    k = _keys([60.0])
    one = np.zeros(1, np.uint32)
    assert oracle_lib.evalue(h, k, one, ev_mode)[0] != oracle_lib.evalue(h, k, one, ev_mode ^ 2)[0]


@pytest.mark.parametrize("mu,beta,m", [(40.0, 4.0, 4e9), (30.0, 2.5, 1e8), (60.0, 6.0, 1e6)])
def test_log_weibull_fit_recovers_a_binned_gumbel(oracle_lib, mu, beta, m):
    pytest.importorskip("scipy")
    h = _binned_gumbel(mu, beta, m)
    N = float(h.sum())
    xs = [mu + 3 * beta, mu]
    e = oracle_lib.evalue(h, _keys(xs), np.arange(2, dtype=np.uint32), 1)
    # e = N (1 - exp(-exp(-(x - mu) / beta))): -ln(-ln(1 - e / N)) is linear in x
    z = -np.log(-np.log1p(-e / N))
    a = (z[0] - z[1]) / (xs[0] - xs[1])
    c = z[0] - a * xs[0]
    assert abs(1 / a - beta) < 0.03 * beta
    assert abs(-c / a - mu) < 0.5


def test_evalue_variant_fallbacks(oracle_lib):
    # one occupied bin: no point with 0 < F < 1, so e = N; no top hit: +inf
    h = np.zeros(256, np.uint32)
    h[30] = 77
    for mode in (1, 3):
        assert oracle_lib.evalue(h, _keys([30.2]), np.zeros(1, np.uint32), mode)[0] == 77.0
        e = oracle_lib.evalue(h, np.array([np.iinfo(np.int64).min], np.int64), np.array([0xFFFFFFFF], np.uint32), mode)
        assert np.isinf(e[0])


# ---------------------------------------------------------------- R18: LBE


def test_mod_distance_worked_example(oracle_lib):
    with open(os.path.join(GOLDEN, "mod_distance_example.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for x, y, de, dm in rows:
        assert oracle_lib.edit_distance(x, y) == int(de)
        assert oracle_lib.mod_distance(x, y) == float(dm)
        assert oracle_lib.mod_distance(y, x) == float(dm)


def test_edit_distance_textbook(oracle_lib):
    assert oracle_lib.edit_distance("KITTEN", "SITTING") == 3
    assert oracle_lib.edit_distance("FLAW", "LAWN") == 2
    assert oracle_lib.edit_distance("PEPTIDE", "PEPTIDE") == 0
    assert oracle_lib.edit_distance("PEPTIDE", "PEPTIDEK") == 1
    assert oracle_lib.edit_distance("A", "A*") == 1            # a modified residue is another symbol
    assert oracle_lib.edit_distance("M*M*", "MM") == 2
    assert oracle_lib.mod_distance("PEPTIDE", "PEPTIDE") == 0.0
    assert oracle_lib.mod_distance("PEPTIDE", "P*EPTIDE") == 2 - 6 / 7


def _marked(seq, codes):
    return "".join(c + ("*" if int(m) else "") for c, m in zip(seq, codes))


def test_lbe_partition_hand_worked(oracle_lib):
    """The partition of a two-protein database worked out by hand
    (tests/golden/lbe_partition_hand.txt): the cluster order by lightest
    entry, the edit-distance tiers and the Mod Distance order inside a tier
    (which here runs against the mass order) all decide a position."""
    with open(os.path.join(GOLDEN, "lbe_partition_hand.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    prot_seqs = ["MSANAAKGGGGGGGGR", "HAAAAAAAKYAAAAAAAK"]
    seq = np.frombuffer("".join(prot_seqs).encode(), np.uint8).copy()
    off = np.array([0, len(prot_seqs[0]), len(prot_seqs[0]) + len(prot_seqs[1])], np.uint64)
    mods = (configs.OX_M(1), configs.PHOSPHO_STY(1), configs.DEAMID_NQ(1))
    params = configs.SearchParams(missed_cleavages=0)
    db = oracle_lib.OracleDb(seq, off, mods, params)
    names = [_marked(*[db.peptide(i)[j] for j in (0, 2)]) for i in range(db.n)]
    assert sorted(names) == sorted(r[0] for r in rows)
    pid = {n: i for i, n in enumerate(names)}
    for col, n_parts in enumerate((2, 3, 4)):
        part = db.partition_lbe(n_parts)
        for r in rows:
            assert part[pid[r[0]]] == int(r[1 + col]), (n_parts, r[0])


def test_lbe_partition_balance_invariants(oracle_lib):
    """Properties of any fine scatter of whole clusters, whatever the order
    inside them: parts differ by at most one entry, and so do the shares of
    every cluster (a cluster is one run of consecutive positions, so it
    gives ceil(|c|/P) entries to |c| mod P parts and floor(|c|/P) to the
    rest)."""
    w = configs.OPEN_MEDIUM.with_proteins(25)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    clusters = {}
    for pid in range(db.n):
        clusters.setdefault(db.peptide(pid)[0], []).append(pid)
    assert any(len(m) > 3 for m in clusters.values())
    for n_parts in (1, 3, 8):
        part = db.partition_lbe(n_parts)
        assert part.max() < n_parts
        sizes = np.bincount(part, minlength=n_parts)
        assert sizes.max() - sizes.min() <= 1
        for members in clusters.values():
            per = np.bincount(part[members], minlength=n_parts)
            c = len(members)
            assert sorted(per.tolist()) == sorted([c // n_parts + 1] * (c % n_parts) +
                                                  [c // n_parts] * (n_parts - c % n_parts))


# ---------------------------------------------------------------- R19: sampling


def _golden_samples():
    with open(os.path.join(GOLDEN, "sampling_hand.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for name, s, nbins, bins, mean, lo, ln in rows:
        h = np.zeros(int(nbins), np.uint32)
        if bins != "-":
            for jc in bins.split(","):
                j, c = jc.split(":")
                h[int(j)] = int(c)
        yield name, int(s), h, int(mean), int(lo), int(ln)


def test_sampling_hand_worked(oracle_lib):
    cases = list(_golden_samples())
    assert len(cases) == 7
    for name, s, h, mean, lo, ln in cases:
        got = oracle_lib.hist_sample(h, s)
        if ln:
            assert got == (lo, ln, mean), name
        else:
            assert got[1] == 0, name


def _window_by_definition(h, s):
    """The kept run stated without the pruning loop: among the runs of at
    most s bins inside the support that contain the mean, the shortest
    longest-side run (max distance from the mean to an end), ties to the
    lower run; the whole support when it has at most s bins."""
    nz = np.flatnonzero(h)
    if len(nz) == 0:
        return None
    order = np.lexsort((np.arange(len(h)), -h.astype(np.int64)))   # count desc, location asc
    m = int(order[:min(3, len(nz))].sum()) // min(3, len(nz))
    L, R = int(nz[0]), int(nz[-1])
    if R - L + 1 <= s:
        return L, R - L + 1, m
    best = None
    for a in range(L, R - s + 2):
        b = a + s - 1
        if a <= m <= b:
            key = (max(b - m, m - a), a)
            if best is None or key < best[0]:
                best = (key, a)
    return best[1], s, m


def test_sampling_against_its_definition(oracle_lib):
    rng = np.random.default_rng(19)
    for trial in range(400):
        nb = int(rng.integers(12, 80))
        h = np.zeros(nb, np.uint32)
        kind = trial % 4
        if kind == 0:      # a binned right-skewed (Gumbel) distribution, as the score histograms
            x = rng.gumbel(rng.uniform(5, nb - 5), rng.uniform(0.5, 6), size=int(rng.integers(1, 5000)))
            np.add.at(h, np.clip(x.astype(int), 0, nb - 1), 1)
        elif kind == 1:    # sparse bins with many equal counts (tie rules)
            h[rng.choice(nb, size=int(rng.integers(1, nb + 1)), replace=True)] = rng.integers(1, 4)
        elif kind == 2:    # long flat tails
            h[:] = rng.integers(0, 3, size=nb)
        else:              # one or two bins
            h[rng.integers(nb)] = int(rng.integers(1, 100))
            if rng.random() < 0.5:
                h[rng.integers(nb)] = int(rng.integers(1, 100))
        s = int(rng.integers(1, 40))
        want = _window_by_definition(h, s)
        got = oracle_lib.hist_sample(h, s)
        if want is None:
            assert got[1] == 0
        else:
            assert got == want, (trial, s, h.tolist())


def test_sampling_is_exact_within_s_bins(oracle_lib):
    """At most s non-zero bins from end to end: the sampled distribution is
    the distribution; and the score histograms of a real search (0.5 log10
    units a bin) never span 120 bins, so s = 120 keeps every count."""
    w = configs.OPEN_MEDIUM.with_proteins(120).with_spectra(40)
    w = dataclasses.replace(w, params=dataclasses.replace(w.params, min_shared=2))
    prot, spec = synth.make_workload_inputs(w)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    res = db.search(spec)
    assert res.n_scored.max() > 500
    for h in res.hist:
        np.testing.assert_array_equal(oracle_lib.sampled(h, 120), h)
        nz = np.flatnonzero(h)
        if len(nz):
            np.testing.assert_array_equal(oracle_lib.sampled(h, int(nz[-1] - nz[0] + 1)), h)
