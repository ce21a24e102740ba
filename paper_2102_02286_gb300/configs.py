"""The synthetic search workloads, as plain data (and as JSON).

Each workload names the proteome recipe, the digestion and modification
rules, the query-spectrum recipe and the search parameters.  The numbers
follow the paper's experimental setup (Experimental Setup: trypsin, up to
2 missed cleavages, peptide mass 500-5000 Da, fragment tolerance dF) and the
five workload descriptions this framework is measured on.  Nothing here
computes anything; both the CUDA path and the CPU oracle read these values.
"""
from __future__ import annotations

import json
from dataclasses import asdict, dataclass, field, replace
from typing import List, Optional, Tuple

# Base seed: the paper's arXiv number; workload i uses BASE_SEED + i.
BASE_SEED = 2102_02286


@dataclass(frozen=True)
class Mod:
    """One modification rule (fixed or variable) on a set of residues."""
    residues: str
    delta_da: float
    max_per_peptide: int = 0       # variable mods: cap per peptide
    fixed: bool = False
    name: str = ""


CARBAMIDOMETHYL_C = Mod("C", 57.021464, 0, True, "carbamidomethyl")
OX_M = lambda n: Mod("M", 15.994915, n, False, "oxidation")          # noqa: E731
PHOSPHO_STY = lambda n: Mod("STY", 79.966331, n, False, "phospho")   # noqa: E731
DEAMID_NQ = lambda n: Mod("NQ", 0.984016, n, False, "deamidation")   # noqa: E731


@dataclass(frozen=True)
class SearchParams:
    # digestion (Experimental Setup of the paper; lengths from the workloads)
    min_len: int = 7
    max_len: int = 40
    missed_cleavages: int = 2
    min_mass: float = 500.0
    max_mass: float = 5000.0
    # fragment index: b/y ions at charge 1 in [frag_mz_min, frag_mz_max),
    # binned at bin_width_da; a query peak and an ion are shared iff they
    # fall in the same bin (bin width = dF).
    frag_mz_min: float = 100.0
    frag_mz_max: float = 2000.0
    bin_width_da: float = 0.01
    # fragment tolerance in bins on that grid (dF = tol_bins * bin_width_da):
    # a peak in bin b covers bins b - tol_bins .. b + tol_bins; 0 = equal bins
    tol_bins: int = 0
    # scoring
    top_n_peaks: int = 100
    min_shared: int = 4
    top_k: int = 5
    hist_bins: int = 256
    intensity_scale: int = 10000
    # e-value: bit 0 = log-Weibull (Gumbel) fit instead of the linear tail
    # fit, bit 1 = Savitzky-Golay smoothing of the histogram before the fit.
    # Default 2: Superstep 4 smooths the assembled distribution first, then
    # fits its tail
    evalue_mode: int = 2
    max_total_mods: int = 0        # 0 = no global cap


@dataclass(frozen=True)
class SpectraRecipe:
    n_spectra: int
    keep_frac: float = 0.6           # fraction of the peptide's b/y ions kept
    jitter_da: float = 0.005         # N(0, jitter) on kept ion m/z
    noise_lo: int = 40               # noise peaks U{noise_lo..noise_hi} ...
    noise_hi: int = 100
    target_peaks: Optional[Tuple[int, int]] = None   # ... or fill to U{a..b} total peaks
    charges: Tuple[int, ...] = (2, 3)
    tol_da: Tuple[float, ...] = (10.0,)              # per spectrum, uniform over the tuple
    mz_lo: float = 100.0
    mz_hi: float = 2000.0


@dataclass(frozen=True)
class Workload:
    name: str
    index: int
    n_proteins: int
    mods: Tuple[Mod, ...]
    params: SearchParams
    spectra: SpectraRecipe
    protein_len: Tuple[int, int] = (100, 800)
    description: str = ""
    db_index: int = -1               # workload whose database this one searches (-1: its own)

    @property
    def seed(self) -> int:
        """Seed of the workload's spectra."""
        return BASE_SEED + self.index

    @property
    def db_seed(self) -> int:
        """Seed of the proteome (shared with the workload named by db_index)."""
        return BASE_SEED + (self.db_index if self.db_index >= 0 else self.index)

    def with_spectra(self, n: int) -> "Workload":
        return replace(self, spectra=replace(self.spectra, n_spectra=n))

    def with_proteins(self, n: int) -> "Workload":
        return replace(self, n_proteins=n)


TINY_CLOSED = Workload(
    name="tiny_closed", index=0, n_proteins=500,
    mods=(CARBAMIDOMETHYL_C,),
    params=SearchParams(missed_cleavages=1, bin_width_da=0.01, top_n_peaks=100, min_shared=4, top_k=5),
    spectra=SpectraRecipe(n_spectra=1000, noise_lo=40, noise_hi=100, charges=(2, 3), tol_da=(10.0,)),
    description="500 proteins, <=1 missed cleavage, fixed CAM-C; 1,000 spectra, +-10 Da, dF 0.01 Da, top-5",
)

OPEN_MEDIUM = Workload(
    name="open_medium", index=1, n_proteins=20_000,
    mods=(CARBAMIDOMETHYL_C, OX_M(2), PHOSPHO_STY(1)),
    params=SearchParams(missed_cleavages=2, bin_width_da=0.01, top_n_peaks=100, min_shared=4, top_k=5),
    spectra=SpectraRecipe(n_spectra=100_000, target_peaks=(100, 100), charges=(2, 3), tol_da=(500.0,)),
    description="20k proteins, <=2 missed cleavages, Met-ox<=2, STY-phospho<=1; 100k spectra x 100 peaks, +-500 Da, dF 0.01 Da, top-5",
)

OPEN_LARGE = Workload(
    name="open_large", index=2, n_proteins=50_000,
    mods=(CARBAMIDOMETHYL_C, OX_M(3), PHOSPHO_STY(2), DEAMID_NQ(1)),
    params=SearchParams(missed_cleavages=2, bin_width_da=0.02, top_n_peaks=150, min_shared=4, top_k=10),
    spectra=SpectraRecipe(n_spectra=1_000_000, target_peaks=(150, 150), charges=(2, 3, 4), tol_da=(500.0,)),
    description="50k proteins, Met-ox<=3, STY<=2, NQ-deam<=1; 1M spectra x 150 peaks, z 2-4, +-500 Da, dF 0.02 Da, top-10",
)

UNEVEN_BATCHED = Workload(
    name="uneven_batched", index=3, n_proteins=20_000, db_index=1,
    mods=(CARBAMIDOMETHYL_C, OX_M(2), PHOSPHO_STY(1)),
    params=SearchParams(missed_cleavages=2, bin_width_da=0.01, top_n_peaks=500, min_shared=4, top_k=5),
    spectra=SpectraRecipe(n_spectra=200_000, target_peaks=(50, 500), charges=(2, 3), tol_da=(10.0, 100.0, 500.0)),
    description="open_medium index; 200k spectra with 50-500 peaks and per-spectrum +-10/100/500 Da",
)

SERVING_STREAM = Workload(
    name="serving_stream", index=4, n_proteins=50_000, db_index=2,
    mods=(CARBAMIDOMETHYL_C, OX_M(3), PHOSPHO_STY(2), DEAMID_NQ(1)),
    params=SearchParams(missed_cleavages=2, bin_width_da=0.02, top_n_peaks=500, min_shared=4, top_k=10),
    spectra=SpectraRecipe(n_spectra=100_000, target_peaks=(50, 500), charges=(2, 3, 4), tol_da=(10.0, 500.0)),
    description="open_large index; Poisson batches of 1-4096 spectra, 50-500 peaks, +-10/500 Da",
)

# the fragment tolerance of t bins on a finer grid: open_medium's database
# binned at 0.005 Da, each retained peak covering its bin +-1 (dF = 0.005 Da,
# the paper's experiments' fragment tolerance)
OPEN_MEDIUM_TOL = Workload(
    name="open_medium_tol", index=5, n_proteins=20_000, db_index=1,
    mods=(CARBAMIDOMETHYL_C, OX_M(2), PHOSPHO_STY(1)),
    params=SearchParams(missed_cleavages=2, bin_width_da=0.005, tol_bins=1, top_n_peaks=100, min_shared=4,
                        top_k=5),
    spectra=SpectraRecipe(n_spectra=100_000, target_peaks=(100, 100), charges=(2, 3), tol_da=(500.0,)),
    description="open_medium database at a 0.005 Da grid, +-1 bin (dF 0.005 Da); 100k spectra x 100 peaks, +-500 Da, top-5",
)

WORKLOADS: List[Workload] = [TINY_CLOSED, OPEN_MEDIUM, OPEN_LARGE, UNEVEN_BATCHED, SERVING_STREAM, OPEN_MEDIUM_TOL]
BY_NAME = {w.name: w for w in WORKLOADS}



# ---- JSON form of a workload (a user's own workload for bench.py --config)


def workload_to_json(w: Workload) -> str:
    """The workload as a JSON object: every field of the workload, its
    modification rules, search parameters and spectrum recipe."""
    return json.dumps(asdict(w), indent=1)


def workload_from_json(text: str) -> Workload:
    """A workload from ``workload_to_json``'s form; fields left out take their
    defaults, unknown fields are an error."""
    d = json.loads(text)
    if not isinstance(d, dict):
        raise ValueError("a workload is a JSON object")
    d = dict(d)
    mods = tuple(Mod(**m) for m in d.pop("mods", []))
    params = SearchParams(**d.pop("params", {}))
    rec = dict(d.pop("spectra", {}))
    for k in ("target_peaks", "charges", "tol_da"):
        if rec.get(k) is not None:
            rec[k] = tuple(rec[k])
    spectra = SpectraRecipe(**rec)
    if "protein_len" in d:
        d["protein_len"] = tuple(d["protein_len"])
    return Workload(mods=mods, params=params, spectra=spectra, **d)


if __name__ == "__main__":
    import sys
    if len(sys.argv) != 2 or sys.argv[1] not in BY_NAME:
        raise SystemExit("usage: python -m paper_2102_02286_gb300.configs <workload name>  (prints its JSON)")
    print(workload_to_json(BY_NAME[sys.argv[1]]))
