"""The C-ABI library loads and exports every entry point include/pc.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2204_01287_gb300 as pcr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pc_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so():
    return pcr.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pc_create", "pc_destroy", "pc_upload_cloud", "pc_upload_encoded",
                     "pc_build_lod", "pc_render", "pc_submit", "pc_poll", "pc_encode"]:
        assert required in names


def test_library_exports_every_declared_symbol(so):
    out = subprocess.check_output(["nm", "-D", "--defined-only", so], text=True)
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(so)
    for n in declared_functions():
        getattr(L, n)


def test_binding_covers_every_symbol(so):
    bound = {s[0] for s in pcr.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_host_calls_without_gpu(so):
    L = pcr.lib()
    assert L.pc_strerror(pcr.PC_EINVAL) == b"invalid argument"
    cfg = pcr.pc_config_default()
    assert cfg.batch_size == 10240 and cfg.precision_px == 512.0
    assert cfg.max_views_per_launch == 32
    h = ctypes.c_void_p()
    assert L.pc_create(None, 0, None) == pcr.PC_EINVAL
    assert L.pc_render(None, 1, None, 0, None, None) == pcr.PC_EINVAL
    assert L.pc_encode(None, None, 5, 10240, 1, 0, None, None, None, None, None, None) == pcr.PC_EINVAL
