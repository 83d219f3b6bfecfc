"""The raster kernels' fast-path certificate (per batch and view, computed by
the cull pass), checked on the CPU: for every certified box, the corners and
random points at k = 1 and 2, decoded and projected by the oracle, must be
accepted with a clip w in [2^-99, 2^99]; the fast path's decode by one fused
multiply-add must give the definition's bits (Sec. 3.3). The boxes sit at
controlled distances from each edge of the view and close to the eye plane,
under matrices scaled over 2^-60 .. 2^60. Without its margins the certificate
must fail on the same cases (tests/cpp/fast_certificate_test.c)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    out = tmp_path_factory.mktemp("fastcert") / "fast_certificate_test"
    subprocess.run([cc, "-O1", "-std=c11", "-Wall", "-Werror", "-ffp-contract=off", "-pthread",
                    "-I", os.path.join(ROOT, "oracle"),
                    os.path.join(ROOT, "tests", "cpp", "fast_certificate_test.c"),
                    os.path.join(ROOT, "oracle", "pcr_oracle.c"), "-o", str(out), "-lm"],
                   check=True, capture_output=True, text=True)
    return str(out)


def test_certified_batches_land_inside_the_view(exe):
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert "fast certificate ok" in r.stdout


def test_certificate_without_margins_is_unsound(exe):
    r = subprocess.run([exe, "narrow"], capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "FAIL box" in r.stdout
