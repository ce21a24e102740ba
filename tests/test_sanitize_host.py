"""The host half of the library and the oracle under AddressSanitizer and
UndefinedBehaviorSanitizer (no GPU): tests/sanitize/host_sanitize.cpp drives
digestion, the LBE partition, shards and subsets, MS2 parsing, the
scheduler's forecast and rules, and the oracle's database, partition, search
and e-values, with the device half of the library stubbed out."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_root():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nv)))


def test_host_half_and_oracle_under_sanitizers(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    cu = cuda_root()
    libdirs = [d for d in (os.path.join(cu, "lib64"), os.path.join(cu, "lib")) if os.path.isdir(d)]
    exe = str(tmp_path / "host_sanitize")
    csrc = os.path.join(ROOT, "paper_2102_02286_gb300", "csrc")
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-pthread", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           "-I" + os.path.join(ROOT, "include"), "-I" + csrc, "-I" + os.path.join(cu, "include"),
           os.path.join(ROOT, "tests", "sanitize", "host_sanitize.cpp"), os.path.join(csrc, "host.cpp"),
           os.path.join(ROOT, "oracle", "hicops_oracle.cpp"), "-x", "c++", os.path.join(csrc, "pipeline.cu"),
           "-x", "none", *["-L" + d for d in libdirs], "-lcudart", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1",
               LD_LIBRARY_PATH=":".join(libdirs + [os.environ.get("LD_LIBRARY_PATH", "")]))
    r = subprocess.run([exe, os.path.join(ROOT, "tests", "golden", "example.ms2"), str(tmp_path)],
                       capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-6000:])
    assert "host sanitize ok" in r.stdout
