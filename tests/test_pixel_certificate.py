"""The raster kernel's certified fast pixel stage (a reciprocal estimate, one
Newton step or none, and a bracket of the floor bits), checked adversarially on
the CPU against the definition with an IEEE divide: with the Newton step any
reciprocal within 2^-20 of 1/w, without it any within 2 ulps, flushed to zero
like the estimate, on random and pixel-edge inputs over depths from 2^-126 to
2^127 (tests/cpp/pixel_certificate_test.c)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_certified_bracket_matches_the_definition(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    exe = tmp_path / "pixel_certificate_test"
    subprocess.run([cc, "-O1", "-std=c11", "-Wall", "-Werror", "-ffp-contract=off",
                    "-frounding-math", os.path.join(ROOT, "tests", "cpp", "pixel_certificate_test.c"),
                    "-o", str(exe), "-lm"], check=True, capture_output=True, text=True)
    for mode in ("newton", "plain"):
        r = subprocess.run([str(exe), mode], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, mode + ": " + r.stdout[-3000:] + r.stderr[-2000:]
        assert "pixel certificate ok" in r.stdout
    # a margin of 2^-23 without the Newton step is too narrow, and the check sees it
    r = subprocess.run([str(exe), "plain-narrow"], capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "FAIL" in r.stdout
