"""Seeded synthetic point clouds and camera matrices (inputs only).

Both the GPU library and the CPU oracle consume what this module produces; it
holds none of the rasterizer's arithmetic. The C source (``pcsynth.c``) is
compiled into ``_build/libpcsynth.so`` by :func:`build`.

Workload recipes (the synthetic stand-ins for the paper's scanned data sets):

* :func:`unit_cube` — uniform points in [0,1)^3 with random RGBA8 colours.
* :func:`terrain` — value-noise heightfield (6 octaves, 2 km base wavelength,
  300 m amplitude, persistence 0.5, lacunarity 2, 1 cm jitter), colours from a
  height ramp plus noise, optionally a fraction of points on box buildings.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpcsynth.so")
_SOURCES = ["pcsynth.c", "pcsynth.h"]
_lock = threading.Lock()
_lib = None


def _stamp() -> str:
    h = hashlib.sha256(platform.machine().encode())
    for s in _SOURCES:
        with open(os.path.join(_HERE, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile libpcsynth.so for this machine (skipped when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp_file = os.path.join(_BUILD, "stamp")
    st = _stamp()
    if not force and os.path.exists(_SO) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == st:
                return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp,
                           os.path.join(_HERE, "pcsynth.c"), "-lm"])
    os.replace(tmp, _SO)
    with open(stamp_file, "w") as f:
        f.write(st)
    return _SO


class TerrainParams(ctypes.Structure):
    _fields_ = [("extent_m", ctypes.c_double), ("wavelength_m", ctypes.c_double),
                ("amplitude_m", ctypes.c_double), ("persistence", ctypes.c_double),
                ("lacunarity", ctypes.c_double), ("octaves", ctypes.c_uint32),
                ("jitter_m", ctypes.c_double), ("buildings_frac", ctypes.c_double),
                ("n_buildings", ctypes.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64, i32, u32 = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
            vp = ctypes.c_void_p
            d = ctypes.c_double
            P = ctypes.POINTER(TerrainParams)
            L.pcs_terrain_defaults.argtypes = [P, d]
            L.pcs_unit_cube.argtypes = [u64, u64, u64, vp, vp, i32]
            L.pcs_terrain.argtypes = [u64, P, u64, u64, vp, vp, i32]
            L.pcs_terrain_scan.argtypes = [u64, P, d, d, d, u64, u64, u64, u64, vp, vp, i32]
            L.pcs_terrain_height.argtypes = [u64, P, d, d]
            L.pcs_terrain_height.restype = d
            L.pcs_look_at_perspective.argtypes = [vp, vp, vp, d, d, d, d, vp]
            L.pcs_flythrough.argtypes = [u64, P, u32, u32, u32, u32, vp, vp]
            L.pcs_overview.argtypes = [P, u32, u32, vp]
            L.pcs_stereo.argtypes = [P, u32, u32, d, i32, vp]
            L.pcs_random_view.argtypes = [u64, P, u64, u32, u32, vp]
            L.pcs_uniform.argtypes = [u64, u64, u64]
            L.pcs_uniform.restype = d
            _lib = L
    return _lib


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def terrain_params(extent_m: float, buildings_frac: float = 0.0,
                   n_buildings: int = 0) -> TerrainParams:
    p = TerrainParams()
    lib().pcs_terrain_defaults(ctypes.byref(p), float(extent_m))
    p.buildings_frac = float(buildings_frac)
    p.n_buildings = int(n_buildings)
    return p


def unit_cube(n: int, seed: int = 0, first: int = 0, threads: int = 0,
              out=None):
    """Return (xyz float32[n,3], rgba uint32[n]) of the unit-cube cloud."""
    if out is None:
        xyz = np.empty((n, 3), np.float32)
        rgba = np.empty(n, np.uint32)
    else:
        xyz, rgba = out
    lib().pcs_unit_cube(seed, first, n, _ptr(xyz), _ptr(rgba), _threads(threads))
    return xyz, rgba


def terrain(n: int, params: TerrainParams, seed: int = 0, first: int = 0,
            threads: int = 0, out=None):
    """Return (xyz float32[n,3], rgba uint32[n]) of the terrain cloud."""
    if out is None:
        xyz = np.empty((n, 3), np.float32)
        rgba = np.empty(n, np.uint32)
    else:
        xyz, rgba = out
    lib().pcs_terrain(seed, ctypes.byref(params), first, n, _ptr(xyz), _ptr(rgba),
                      _threads(threads))
    return xyz, rgba


def terrain_scan(n: int, params: TerrainParams, scanner=(0.0, 0.0), max_dist_m: float = 2000.0,
                 points_per_line: int = 20000, seed: int = 0, first: int = 0, total: int = 0,
                 threads: int = 0, out=None):
    """Scan-ordered terrain points (consecutive points along rays from the
    scanner): (xyz float32[n,3], rgba uint32[n])."""
    if out is None:
        xyz = np.empty((n, 3), np.float32)
        rgba = np.empty(n, np.uint32)
    else:
        xyz, rgba = out
    lib().pcs_terrain_scan(seed, ctypes.byref(params), float(scanner[0]), float(scanner[1]),
                           float(max_dist_m), total or n, points_per_line, first, n, _ptr(xyz),
                           _ptr(rgba), _threads(threads))
    return xyz, rgba


def terrain_height(params: TerrainParams, x: float, y: float, seed: int = 0) -> float:
    return lib().pcs_terrain_height(seed, ctypes.byref(params), float(x), float(y))


def look_at_perspective(eye, target, up, fovy_deg, aspect, znear, zfar) -> np.ndarray:
    out = np.empty(16, np.float32)
    e = np.asarray(eye, np.float64)
    t = np.asarray(target, np.float64)
    u = np.asarray(up, np.float64)
    lib().pcs_look_at_perspective(_ptr(e), _ptr(t), _ptr(u), float(fovy_deg),
                                  float(aspect), float(znear), float(zfar), _ptr(out))
    return out


def flythrough(params: TerrainParams, frame: int, nframes: int, width: int,
               height: int, seed: int = 0) -> np.ndarray:
    out = np.empty(16, np.float32)
    lib().pcs_flythrough(seed, ctypes.byref(params), frame, nframes, width, height,
                         _ptr(out), None)
    return out


def overview(params: TerrainParams, width: int, height: int) -> np.ndarray:
    out = np.empty(16, np.float32)
    lib().pcs_overview(ctypes.byref(params), width, height, _ptr(out))
    return out


def stereo(params: TerrainParams, width: int, height: int, eye: int,
           ipd_m: float = 0.065) -> np.ndarray:
    out = np.empty(16, np.float32)
    lib().pcs_stereo(ctypes.byref(params), width, height, float(ipd_m), int(eye),
                     _ptr(out))
    return out


def random_view(params: TerrainParams, index: int, width: int, height: int,
                seed: int = 0) -> np.ndarray:
    out = np.empty(16, np.float32)
    lib().pcs_random_view(seed, ctypes.byref(params), index, width, height, _ptr(out))
    return out


def cube_camera(width: int = 512, height: int = 512) -> np.ndarray:
    """Unit-cube camera: 60 deg vertical FOV, eye (0.5,0.5,2.5) looking at the
    cube centre, +Y up, near 0.1, far 100."""
    return look_at_perspective((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0,
                               width / height, 0.1, 100.0)
