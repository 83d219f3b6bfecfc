"""The serving loop's range allocator (csrc/arena.h), compiled with g++ and
run against a brute-force first-fit model (tests/cpp/arena_test.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_matches_first_fit_model(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "arena_test"
    subprocess.run([gxx, "-O1", "-std=c++17", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2204_01287_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "cpp", "arena_test.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "arena ok" in r.stdout
