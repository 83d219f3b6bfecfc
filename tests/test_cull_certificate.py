"""The culling kernel's binary32 fast test (decide a plane only outside a band
of 2^-16 times its magnitude, else fall back to binary64), checked on the CPU
against the oracle's binary64 test on boxes placed at controlled distances from
each clip plane, under matrices scaled over 2^-60 .. 2^60
(tests/cpp/cull_certificate_test.c)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fast_cull_decisions_match_the_definition(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    exe = tmp_path / "cull_certificate_test"
    subprocess.run([cc, "-O1", "-std=c11", "-Wall", "-Werror", "-ffp-contract=off", "-pthread",
                    "-I", os.path.join(ROOT, "oracle"),
                    os.path.join(ROOT, "tests", "cpp", "cull_certificate_test.c"),
                    os.path.join(ROOT, "oracle", "pcr_oracle.c"), "-o", str(exe), "-lm"],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert "cull certificate ok" in r.stdout
