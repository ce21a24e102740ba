"""Comparison of the CUDA path's results with the oracle's.

Bit-exact: window, candidate counts (n_scored), histogram, top-k peptide ids,
shared b/y counts and the integer rank key.  Floating point: the FP32
hyperscore within 1e-5 relative of the oracle's FP64 hyperscore; the FP64
e-value within 1e-9 relative (the fit sums run in a different order).
"""
import numpy as np

PAD = 0xFFFFFFFF
HS_RTOL = 1e-5
EV_RTOL = 1e-9


def assert_parity(got, ref, sel=None, label=""):
    """got: hicops.SearchResult for the whole batch; ref: oracle result for
    spectra ``sel`` (all when None)."""
    gp = got.psm if sel is None else got.psm[sel]
    gh = got.hist if sel is None else got.hist[sel]
    gn = got.n_scored if sel is None else got.n_scored[sel]
    np.testing.assert_array_equal(gn, ref.n_scored, err_msg=f"{label} n_scored")
    np.testing.assert_array_equal(gh, ref.hist, err_msg=f"{label} histogram")
    np.testing.assert_array_equal(gp["pid"], ref.psm["pid"], err_msg=f"{label} top-k pids")
    np.testing.assert_array_equal(gp["key"], ref.psm["key"], err_msg=f"{label} rank keys")
    np.testing.assert_array_equal(gp["nb"].astype(np.uint32), ref.psm["nb"], err_msg=f"{label} nb")
    np.testing.assert_array_equal(gp["ny"].astype(np.uint32), ref.psm["ny"], err_msg=f"{label} ny")
    real = ref.psm["pid"] != PAD
    np.testing.assert_allclose(gp["hyperscore"][real].astype(np.float64), ref.psm["hyperscore"][real],
                               rtol=HS_RTOL, atol=0, err_msg=f"{label} hyperscore")
    np.testing.assert_allclose(gp["evalue"][real], ref.psm["evalue"][real], rtol=EV_RTOL, atol=0,
                               err_msg=f"{label} e-value")
    assert np.all(np.isinf(gp["evalue"][~real])), f"{label} padding e-values"
    assert np.all(gp["hyperscore"][~real] == 0), f"{label} padding hyperscores"
    # n_scored is the histogram mass
    np.testing.assert_array_equal(gh.sum(axis=1), gn, err_msg=f"{label} n_scored vs histogram")
    return int(real.sum())
