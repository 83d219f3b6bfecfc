"""Build libpcr.so (CUDA kernels for sm_103a + the host C++ runtime).

nvcc compiles the .cu translation units (-gencode arch=compute_103a,code=sm_103a,
--fmad=false so that no float multiply and add is contracted), g++ the .cpp
ones, all in parallel; nvcc links the shared library with the static CUDA
runtime. Outputs go to paper_2204_01287_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libpcr.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpcr.so")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = sorted(f for f in os.listdir(CSRC) if f.endswith(".h"))
    return cu, cpp, hdr


def _stamp() -> str:
    cu, cpp, hdr = _sources()
    h = hashlib.sha256((platform.machine() + ARCH).encode())
    for f in cu + cpp + hdr:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(INCLUDE, "pc.h"), "rb") as fh:
        h.update(fh.read())
    with open(__file__, "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "stamp")
    st = _stamp()
    if not force and os.path.exists(SO) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == st:
                return SO
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    cu, cpp, _ = _sources()
    jobs, objs = [], []
    for f in cu:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc, ARCH, "-O3", "-std=c++17", "--fmad=false", "-lineinfo",
                     "-Xptxas", "-v" if verbose else "-O3", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", o])
    for f in cpp:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off",
                     "-Wall", "-I", INCLUDE, "-I", os.path.join(cuda_home, "include"),
                     "-c", os.path.join(CSRC, f), "-o", o])
    procs = [(j, subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
             for j in jobs]
    failed = []
    for j, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(j))
    if failed:
        raise RuntimeError("libpcr build failed:\n" + "\n".join(failed))
    tmp = SO + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs +
                          ["-lpthread"])
    os.replace(tmp, SO)
    with open(stamp_file, "w") as f:
        f.write(st)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
