"""The serving loop's device-pool allocator (host bookkeeping of
csrc/pool_map.h) against a brute-force granule model: first fit, exact
merging of returned ranges, used and peak bytes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


@pytest.mark.parametrize("sanitize", [False, True], ids=["plain", "asan_ubsan"])
def test_pool_map_matches_the_granule_model(tmp_path, sanitize):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "pool_map_check"
    flags = ["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
             "-fno-omit-frame-pointer"] if sanitize else []
    subprocess.run([cxx, "-O1", "-std=c++17", "-Wall", "-Werror", *flags,
                    "-I", os.path.join(ROOT, "paper_2102_02286_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "pool_map_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe), "20000"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok 20000"
