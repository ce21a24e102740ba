"""Host-side checks (no GPU): the library loads and exports every entry point
that include/*.h declares, parameter validation, and the host half of
superstep 1 (digestion, variants, pid order) against the CPU oracle."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2102_02286_gb300 import build as pkg_build
from paper_2102_02286_gb300 import configs, synth
from paper_2102_02286_gb300 import hicops as hc
from paper_2102_02286_gb300.configs import SearchParams

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return hc.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(hicops_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "hicops_search" in names and "hicops_build_index" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_param_validation(lib):
    prot = synth.make_proteome(3, 1)
    bad = [SearchParams(max_len=65), SearchParams(top_k=0), SearchParams(top_k=33), SearchParams(hist_bins=128),
           SearchParams(bin_width_da=0.0), SearchParams(top_n_peaks=0), SearchParams(min_len=1),
           SearchParams(intensity_scale=20000)]
    for p in bad:
        with pytest.raises(hc.HicopsError) as e:
            hc.Index(prot.seq, prot.off, [], p, upload=False)
        assert e.value.status in (hc.EINVAL, hc.EOVERFLOW)
    # two variable rules on one residue are rejected
    with pytest.raises(hc.HicopsError):
        hc.Index(prot.seq, prot.off, [configs.OX_M(1), configs.Mod("M", 1.0, 1)], SearchParams(), upload=False)


def test_search_without_device_index_is_rejected(lib):
    prot = synth.make_proteome(3, 1)
    idx = hc.Index(prot.seq, prot.off, [configs.CARBAMIDOMETHYL_C], SearchParams(), upload=False)
    spec = synth.spectra_from_lists([([150.0, 250.0], [1.0, 2.0])], [500.0], [2], [10.0])
    with pytest.raises(hc.HicopsError) as e:
        idx.search(spec)
    assert e.value.status == hc.EINVAL


def _compare_tables(idx, db, mods):
    var = [m for m in mods if not m.fixed]
    n = db.n
    assert idx.n_peptides == n
    np.testing.assert_array_equal(db.masses(), np.array([idx.peptide(i)[1] for i in range(n)]))
    for pid in range(n):
        s, mass, mask = idx.peptide(pid)
        os_, om, codes = db.peptide(pid)
        assert s == os_
        exp_mask = 0
        for j, c in enumerate(codes):
            if c:
                assert s[j] in var[c - 1].residues
                exp_mask |= 1 << j
        assert mask == exp_mask


def test_digest_matches_oracle_closed(lib, oracle_lib):
    w = configs.TINY_CLOSED.with_proteins(150)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    _compare_tables(idx, db, w.mods)


def test_digest_matches_oracle_modified(lib, oracle_lib):
    w = configs.OPEN_LARGE.with_proteins(40)
    prot = synth.make_proteome(w.n_proteins, w.seed)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    _compare_tables(idx, db, w.mods)
    st = idx.stats()
    assert st.n_base_peptides <= st.n_peptides


def test_digest_global_cap_and_edges(lib, oracle_lib):
    p = SearchParams(min_len=2, max_len=64, missed_cleavages=3, min_mass=0.0, max_mass=1e6, max_total_mods=2)
    mods = [configs.CARBAMIDOMETHYL_C, configs.OX_M(3), configs.PHOSPHO_STY(2), configs.DEAMID_NQ(1)]
    seqs = ["MSMSTYKCNQMSK", "AAXAAK", "PPPPKPPPR", "K", "R", "MMMMMMMMK", "C" * 63 + "K"]
    s = "".join(seqs)
    off = np.cumsum([0] + [len(x) for x in seqs]).astype(np.uint64)
    arr = np.frombuffer(s.encode(), np.uint8)
    idx = hc.Index(arr, off, mods, p, upload=False)
    db = oracle_lib.OracleDb(arr, off, mods, p)
    _compare_tables(idx, db, mods)


# ---------------------------------------------------------------- LBE partition (host only)


@pytest.mark.parametrize("name,n_prot,n_parts", [("open_medium", 25, 3), ("open_medium", 40, 8),
                                                   ("open_large", 10, 5), ("tiny_closed", 60, 4)])
def test_lbe_partition_matches_oracle(lib, oracle_lib, name, n_prot, n_parts):
    w = configs.BY_NAME[name].with_proteins(n_prot)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    db = oracle_lib.OracleDb(prot.seq, prot.off, w.mods, w.params)
    assert idx.stats().n_peptides == db.n
    np.testing.assert_array_equal(idx.partition_lbe(n_parts), db.partition_lbe(n_parts))


def test_subset_indexes(lib):
    w = configs.OPEN_MEDIUM.with_proteins(20)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    P = idx.stats().n_peptides
    part = idx.partition_lbe(4)
    pids = np.flatnonzero(part == 2).astype(np.uint32)
    sub = idx.subset(pids, upload=False)
    assert sub.stats().n_peptides == len(pids)
    for g in pids[::max(1, len(pids) // 20)]:
        assert sub.peptide(int(g)) == idx.peptide(int(g))   # global pids on the subset
    other = int(np.flatnonzero(part == 1)[0])
    with pytest.raises(hc.HicopsError):
        sub.peptide(other)                                   # not in this part
    with pytest.raises(hc.HicopsError):
        sub.subset(pids[:3], upload=False)                   # a part is not split again
    with pytest.raises(hc.HicopsError):
        idx.subset(np.array([5, 5, 9], np.uint32), upload=False)   # not strictly ascending
    with pytest.raises(hc.HicopsError):
        idx.subset(np.array([1, P], np.uint32), upload=False)      # past the database
    with pytest.raises(hc.HicopsError):
        idx.partition_lbe(0)
    with pytest.raises(hc.HicopsError):
        sub.partition_lbe(2)
    empty = idx.subset(np.zeros(0, np.uint32), upload=False)
    assert empty.stats().n_peptides == 0
    for h in (sub, empty):
        h.close()


def test_lbe_parts_cover_the_database(lib):
    from paper_2102_02286_gb300 import shard
    w = configs.OPEN_MEDIUM.with_proteins(30)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    P = idx.stats().n_peptides
    parts = shard.lbe_parts(idx, 5, upload=False)
    sizes = [p.stats().n_peptides for p in parts]
    assert sum(sizes) == P and max(sizes) - min(sizes) <= 1
    part = idx.partition_lbe(5)
    for s, p in enumerate(parts):
        mine = np.flatnonzero(part == s)
        # every global pid of the part resolves on it, with the whole database's peptide
        for g in mine[:: max(1, len(mine) // 10)]:
            assert p.peptide(int(g)) == idx.peptide(int(g))
        p.close()


# ---------------------------------------------------------------- checkpoint (host only)


def test_index_save_load_round_trip(lib, tmp_path):
    w = configs.OPEN_MEDIUM.with_proteins(30)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    path = str(tmp_path / "db.hix")
    idx.save(path)
    back = hc.Index.load(path, upload=False)
    assert back.params == w.params
    a, b = idx.stats(), back.stats()
    assert (a.n_peptides, a.n_base_peptides, a.n_bins) == (b.n_peptides, b.n_base_peptides, b.n_bins)
    for pid in range(0, a.n_peptides, max(1, a.n_peptides // 40)):
        assert back.peptide(pid) == idx.peptide(pid)
    np.testing.assert_array_equal(back.partition_lbe(3), idx.partition_lbe(3))
    # a part keeps its global pids through a checkpoint
    pids = np.flatnonzero(idx.partition_lbe(4) == 1).astype(np.uint32)
    sub = idx.subset(pids, upload=False)
    sub.save(path)
    sub2 = hc.Index.load(path, upload=False)
    assert sub2.peptide(int(pids[3])) == idx.peptide(int(pids[3]))
    with pytest.raises(hc.HicopsError):
        sub2.subset(pids[:2], upload=False)       # still a part
    for h in (back, sub, sub2):
        h.close()


def test_index_load_rejects_bad_files(lib, tmp_path):
    w = configs.TINY_CLOSED.with_proteins(20)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    good = tmp_path / "db.hix"
    idx.save(str(good))
    data = good.read_bytes()
    cases = {"missing": None, "empty": b"", "magic": b"X" + data[1:], "truncated": data[:-9],
             "trailing": data + b"\0", "format": data[:8] + b"\x07" + data[9:]}
    for name, blob in cases.items():
        p = tmp_path / f"{name}.hix"
        if blob is not None:
            p.write_bytes(blob)
        with pytest.raises(hc.HicopsError):
            hc.Index.load(str(p), upload=False)
    with pytest.raises(hc.HicopsError):
        idx.save(str(tmp_path / "no_such_dir" / "x.hix"))


def test_index_load_rejects_tampered_fields(lib, tmp_path):
    # fields the device half trusts: the bin count and largest S (they size
    # the bucket tables and the LS table) and the residue bytes (they index
    # the 128-entry mass tables of the ion generator)
    import struct
    w = configs.TINY_CLOSED.with_proteins(20)
    prot = synth.make_proteome(w.n_proteins, w.db_seed, w.protein_len)
    idx = hc.Index(prot.seq, prot.off, w.mods, w.params, upload=False)
    good = tmp_path / "db.hix"
    idx.save(str(good))
    data = bytearray(good.read_bytes())
    hc.Index.load(str(good), upload=False).close()
    tail = C.sizeof(hc.IndexStats)
    at_sm, at_nb = len(data) - tail - 8, len(data) - tail - 12
    n_bins = struct.unpack_from("<I", data, at_nb)[0]
    s_max = struct.unpack_from("<Q", data, at_sm)[0]
    assert n_bins == idx.stats().n_bins
    # n_var = 0 for this workload: two empty vectors before the residue count
    at_res = 16 + C.sizeof(hc.Params) + 1024 + 1024 + 128 + 4 + 8 + 8 + 8
    assert chr(data[at_res]) in "ACDEFGHIKLMNPQRSTVWY"
    cases = {"n_bins_small": (at_nb, struct.pack("<I", n_bins // 2)),
             "n_bins_large": (at_nb, struct.pack("<I", n_bins + 1)),
             "s_max_small": (at_sm, struct.pack("<Q", s_max - 1)),
             "s_max_huge": (at_sm, struct.pack("<Q", 1 << 60)),
             "residue_high": (at_res, bytes([0xC1])),
             "residue_no_mass": (at_res, b"B")}
    for name, (at, blob) in cases.items():
        bad = bytearray(data)
        bad[at:at + len(blob)] = blob
        p = tmp_path / f"{name}.hix"
        p.write_bytes(bytes(bad))
        with pytest.raises(hc.HicopsError) as e:
            hc.Index.load(str(p), upload=False)
        assert e.value.status == hc.EINVAL, name
    idx.close()
