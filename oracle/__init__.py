"""CPU oracle for the point rasterizer — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The GPU
library never calls it, and it shares no code with the library: it is a plain
restatement of the paper's method in C (``pcr_oracle.c``, compiled with
``-ffp-contract=off``) wrapped with ctypes.

Function map (paper sections):
  quantize30 / split_words / decode_words   Eq. 1, Listing 2, Sec. 3.3
  morton_code / encode                      Sec. 3.1
  project_position / project_point          Listing 1
  select_k                                  Sec. 3.3 (precision threshold)
  cull                                      Sec. 3.2 (batch frustum culling)
  render / render_threaded / brute_force    Sec. 3.2-3.3 geometry pass
  resolve                                   Sec. 3.3 visibility buffer
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
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["pcr_oracle.c", "pcr_oracle.h"]
_lock = threading.Lock()
_lib = None

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
BATCH_DTYPE = np.dtype([("min", "<f4", (3,)), ("size", "<f4", (3,)),
                        ("first", "<u4"), ("count", "<u4")])
assert BATCH_DTYPE.itemsize == 32


def _stamp() -> str:
    h = hashlib.sha256(platform.machine().encode())
    for s in _SOURCES:
        with open(os.path.join(_HERE, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp_file = os.path.join(_BUILD, "stamp")
    st = _stamp()
    if not force and os.path.exists(_SO) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == st:
                return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-fno-fast-math", "-o", tmp,
                           os.path.join(_HERE, "pcr_oracle.c"), "-lm"])
    os.replace(tmp, _SO)
    with open(stamp_file, "w") as f:
        f.write(st)
    return _SO


class View(ctypes.Structure):
    _fields_ = [("m", ctypes.c_float * 16), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32), ("cull", ctypes.c_int),
                ("force_k", ctypes.c_int), ("threshold_px", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [("batches_rendered", ctypes.c_uint64),
                ("points_processed", ctypes.c_uint64),
                ("batches_k", ctypes.c_uint64 * 4), ("points_k", ctypes.c_uint64 * 4),
                ("points_accepted", ctypes.c_uint64)]

    def as_dict(self):
        return {"batches_rendered": self.batches_rendered,
                "points_processed": self.points_processed,
                "batches_k": list(self.batches_k), "points_k": list(self.points_k),
                "points_accepted": self.points_accepted}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # PCR_ORACLE_SO lets the mutation test load a copy of the oracle
            # with a planted mistake; normally the in-tree build is used.
            path = os.environ.get("PCR_ORACLE_SO") or build()
            L = ctypes.CDLL(path)
            vp, u32, u64, f32, i32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                      ctypes.c_float, ctypes.c_int)
            VP = ctypes.POINTER(View)
            SP = ctypes.POINTER(Stats)
            L.or_quantize30.argtypes = [f32, f32, f32]
            L.or_quantize30.restype = u32
            L.or_split_words.argtypes = [u32, u32, u32, vp]
            L.or_decode_words.argtypes = [u32, u32, u32, i32, vp]
            L.or_morton_code.argtypes = [vp, vp, vp]
            L.or_morton_code.restype = u64
            L.or_num_batches.argtypes = [u64, u32]
            L.or_num_batches.restype = u64
            L.or_encode.argtypes = [vp, vp, u64, u32, vp, vp, vp, vp, vp, vp]
            L.or_encode.restype = i32
            L.or_encode_in_order.argtypes = [vp, vp, u64, u32, vp, vp, vp, vp, vp]
            L.or_encode_in_order.restype = i32
            L.or_project_position.argtypes = [vp, VP, u32, vp, vp, vp]
            L.or_project_position.restype = i32
            L.or_project_point.argtypes = [vp, i32, u32, u32, u32, u32, VP, vp, vp]
            L.or_project_point.restype = i32
            L.or_decode_position.argtypes = [vp, i32, u32, u32, u32, vp]
            L.or_select_k.argtypes = [vp, VP]
            L.or_select_k.restype = i32
            L.or_cull.argtypes = [vp, VP]
            L.or_cull.restype = i32
            L.or_render.argtypes = [vp, u64, vp, vp, vp, VP, vp, vp, SP]
            L.or_render_threaded.argtypes = [vp, u64, vp, vp, vp, VP, i32, vp, SP]
            L.or_render_positions.argtypes = [vp, u64, VP, vp]
            L.or_brute_force.argtypes = [vp, u64, vp, vp, vp, VP, vp]
            L.or_resolve.argtypes = [vp, u64, vp, vp]
            L.or_decode_cloud.argtypes = [vp, u64, vp, vp, vp, i32, vp]
            L.or_projected_extent.argtypes = [vp, VP, vp]
            L.or_projected_extent.restype = i32
            L.or_splitmix64.argtypes = [u64]
            L.or_splitmix64.restype = u64
            L.or_lod_count_nodes.argtypes = [vp, u64, u32, u32, u32]
            L.or_lod_count_nodes.restype = ctypes.c_int64
            L.or_lod_build.argtypes = [vp, vp, u64, u32, u32, u32, vp, vp, vp, vp, vp, vp, vp, vp]
            L.or_lod_build.restype = ctypes.c_int64
            L.or_lod_select.argtypes = [vp, vp, u64, VP, f32, f32, vp]
            L.or_lod_render.argtypes = [vp, vp, u64, vp, vp, vp, VP, f32, f32, vp, SP]
            L.or_ring.argtypes = [f32, f32, u32, u32]
            L.or_ring.restype = i32
            L.or_resolve_dilated.argtypes = [vp, u32, u32, vp, vp]
            L.or_render_hqs.argtypes = [vp, u64, vp, vp, vp, vp, VP, vp, vp]
            L.or_lod_render_hqs.argtypes = [vp, vp, u64, vp, vp, vp, vp, VP, f32, f32, vp, vp]
            L.or_hqs_resolve_dilated.argtypes = [vp, u32, u32, vp, vp]
            L.or_render_hqs_threaded.argtypes = [vp, u64, vp, vp, vp, vp, VP, vp, i32, vp]
            L.or_verify_lod.argtypes = [vp, vp, u64, u32, u32, u32, vp, vp, vp, u64, vp, vp, vp,
                                        vp, vp, i32, vp]
            L.or_verify_encoding.argtypes = [vp, vp, u64, u32, vp, u64, vp, vp, vp, vp, vp, i32, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


def make_view(m, width, height, cull=False, force_k=0, threshold_px=512.0) -> View:
    v = View()
    mm = np.asarray(m, np.float32).reshape(16)
    for i in range(16):
        v.m[i] = float(mm[i])
    v.width, v.height = int(width), int(height)
    v.cull, v.force_k, v.threshold_px = int(bool(cull)), int(force_k), float(threshold_px)
    return v


# ---- Eq. 1, Listing 2, Sec. 3.3 --------------------------------------------

def quantize30(v, box_min, box_size) -> int:
    return lib().or_quantize30(float(np.float32(v)), float(np.float32(box_min)),
                               float(np.float32(box_size)))


def split_words(X30, Y30, Z30):
    w = np.zeros(3, np.uint32)
    lib().or_split_words(int(X30), int(Y30), int(Z30), _p(w))
    return [int(x) for x in w]


def decode_words(w1, w2, w3, k):
    out = np.zeros(3, np.uint32)
    lib().or_decode_words(int(w1), int(w2), int(w3), int(k), _p(out))
    return [int(x) for x in out]


def morton_code(p, cmin, csize) -> int:
    pp = np.asarray(p, np.float32).reshape(3).copy()
    a = np.asarray(cmin, np.float64).reshape(3).copy()
    b = np.asarray(csize, np.float64).reshape(3).copy()
    return lib().or_morton_code(_p(pp), _p(a), _p(b))


# ---- Sec. 3.1 encode ---------------------------------------------------------

class Encoded:
    """Oracle-encoded cloud: batches, the three coordinate words and colours in
    Morton order, and perm (sorted position -> input index)."""

    def __init__(self, batches, w1, w2, w3, color, perm):
        self.batches, self.w1, self.w2, self.w3 = batches, w1, w2, w3
        self.color, self.perm = color, perm

    @property
    def n(self):
        return len(self.w1)


def encode(xyz: np.ndarray, rgba: np.ndarray, batch_size: int = 10240) -> Encoded:
    xyz = np.ascontiguousarray(xyz, np.float32)
    rgba = np.ascontiguousarray(rgba, np.uint32)
    n = len(rgba)
    nb = lib().or_num_batches(n, batch_size)
    batches = np.zeros(nb, BATCH_DTYPE)
    w1 = np.zeros(n, np.uint32)
    w2 = np.zeros(n, np.uint32)
    w3 = np.zeros(n, np.uint32)
    color = np.zeros(n, np.uint32)
    perm = np.zeros(n, np.uint32)
    rc = lib().or_encode(_p(xyz), _p(rgba), n, batch_size, _p(perm), _p(batches),
                         _p(w1), _p(w2), _p(w3), _p(color))
    if rc < 0:
        raise RuntimeError(f"or_encode failed: {rc}")
    return Encoded(batches, w1, w2, w3, color, perm)


def encode_in_order(xyz: np.ndarray, rgba: np.ndarray, batch_size: int = 10240) -> Encoded:
    """Batches of consecutive input points, no Morton sort (Sec. 4.2 baseline)."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    rgba = np.ascontiguousarray(rgba, np.uint32)
    n = len(rgba)
    nb = lib().or_num_batches(n, batch_size)
    batches = np.zeros(nb, BATCH_DTYPE)
    w = [np.zeros(n, np.uint32) for _ in range(4)]
    rc = lib().or_encode_in_order(_p(xyz), _p(rgba), n, batch_size, _p(batches),
                                  *(_p(a) for a in w))
    if rc < 0:
        raise RuntimeError(f"or_encode_in_order failed: {rc}")
    return Encoded(batches, w[0], w[1], w[2], w[3], np.arange(n, dtype=np.uint32))


# ---- Listing 1 and the geometry pass -----------------------------------------

def project_position(p, view: View, idx: int = 0):
    """(accepted, pixel, key, fx, fy) for one float position."""
    pp = np.asarray(p, np.float32).reshape(3).copy()
    pix = np.zeros(1, np.uint32)
    key = np.zeros(1, np.uint64)
    fxy = np.zeros(2, np.float32)
    ok = lib().or_project_position(_p(pp), ctypes.byref(view), idx, _p(pix), _p(key), _p(fxy))
    return bool(ok), int(pix[0]), int(key[0]), float(fxy[0]), float(fxy[1])


def _batch_arr(b):
    a = np.zeros(1, BATCH_DTYPE)
    a[0] = b
    return a


def decode_position(batch, k, w1, w2, w3):
    b = _batch_arr(batch)
    p = np.zeros(3, np.float32)
    lib().or_decode_position(_p(b), int(k), int(w1), int(w2), int(w3), _p(p))
    return p


def select_k(batch, view: View) -> int:
    return lib().or_select_k(_p(_batch_arr(batch)), ctypes.byref(view))


def cull(batch, view: View) -> bool:
    return bool(lib().or_cull(_p(_batch_arr(batch)), ctypes.byref(view)))


def render(enc: Encoded, view: View, order=None):
    """Visibility buffer (uint64[H*W]) and stats of one view."""
    vis = np.empty(view.width * view.height, np.uint64)
    st = Stats()
    o = None
    if order is not None:
        o = np.ascontiguousarray(order, np.uint64)
    lib().or_render(_p(enc.batches), len(enc.batches), _p(enc.w1), _p(enc.w2),
                    _p(enc.w3), ctypes.byref(view), _p(o) if o is not None else None,
                    _p(vis), ctypes.byref(st))
    return vis, st.as_dict()


def render_threaded(enc: Encoded, view: View, threads: int = 0):
    vis = np.empty(view.width * view.height, np.uint64)
    st = Stats()
    lib().or_render_threaded(_p(enc.batches), len(enc.batches), _p(enc.w1), _p(enc.w2),
                             _p(enc.w3), ctypes.byref(view),
                             int(threads) if threads else (os.cpu_count() or 1),
                             _p(vis), ctypes.byref(st))
    return vis, st.as_dict()


def render_positions(xyz: np.ndarray, view: View):
    xyz = np.ascontiguousarray(xyz, np.float32)
    vis = np.empty(view.width * view.height, np.uint64)
    lib().or_render_positions(_p(xyz), len(xyz), ctypes.byref(view), _p(vis))
    return vis


def brute_force(enc: Encoded, view: View):
    vis = np.empty(view.width * view.height, np.uint64)
    lib().or_brute_force(_p(enc.batches), len(enc.batches), _p(enc.w1), _p(enc.w2),
                         _p(enc.w3), ctypes.byref(view), _p(vis))
    return vis


def resolve(vis: np.ndarray, color: np.ndarray):
    vis = np.ascontiguousarray(vis, np.uint64)
    color = np.ascontiguousarray(color, np.uint32)
    out = np.empty(len(vis), np.uint32)
    lib().or_resolve(_p(vis), len(vis), _p(color), _p(out))
    return out


# ---- Sec. 3.5 level of detail --------------------------------------------------

def projected_extent(batch, view: View):
    """Projected extent in pixels, or None when a corner has w <= 0."""
    e = np.zeros(1, np.float32)
    ok = lib().or_projected_extent(_p(_batch_arr(batch)), ctypes.byref(view), _p(e))
    return float(e[0]) if ok else None


def splitmix64(z: int) -> int:
    return lib().or_splitmix64(int(z) & 0xFFFFFFFFFFFFFFFF)


class LodCloud:
    """Oracle layered octree: nodes (batches), parent, level, words, colours
    and perm (LOD point -> input index)."""

    def __init__(self, nodes, parent, level, w1, w2, w3, color, perm):
        self.nodes, self.parent, self.level = nodes, parent, level
        self.w1, self.w2, self.w3, self.color, self.perm = w1, w2, w3, color, perm


def lod_build(xyz, rgba, max_levels=12, max_node_points=10240, seed=0) -> LodCloud:
    xyz = np.ascontiguousarray(xyz, np.float32)
    rgba = np.ascontiguousarray(rgba, np.uint32)
    n = len(xyz)
    nn = lib().or_lod_count_nodes(_p(xyz), n, max_levels, max_node_points, seed)
    nodes = np.zeros(max(nn, 1), BATCH_DTYPE)
    parent = np.zeros(max(nn, 1), np.uint32)
    level = np.zeros(max(nn, 1), np.uint32)
    w = [np.zeros(max(n, 1), np.uint32) for _ in range(5)]
    got = lib().or_lod_build(_p(xyz), _p(rgba), n, max_levels, max_node_points, seed,
                             _p(nodes), _p(parent), _p(level), _p(w[4]), _p(w[0]), _p(w[1]),
                             _p(w[2]), _p(w[3]))
    assert got == nn
    return LodCloud(nodes[:nn], parent[:nn], level[:nn], w[0][:n], w[1][:n], w[2][:n],
                    w[3][:n], w[4][:n])


def lod_select(lod: LodCloud, view: View, lod_px: float, lod_px_periphery: float = 0.0):
    sel = np.zeros(max(len(lod.nodes), 1), np.uint8)
    lib().or_lod_select(_p(lod.nodes), _p(lod.parent), len(lod.nodes), ctypes.byref(view),
                        float(lod_px), float(lod_px_periphery), _p(sel))
    return sel[:len(lod.nodes)]


def lod_render(lod: LodCloud, view: View, lod_px: float, lod_px_periphery: float = 0.0):
    vis = np.empty(view.width * view.height, np.uint64)
    st = Stats()
    lib().or_lod_render(_p(lod.nodes), _p(lod.parent), len(lod.nodes), _p(lod.w1), _p(lod.w2),
                        _p(lod.w3), ctypes.byref(view), float(lod_px), float(lod_px_periphery),
                        _p(vis), ctypes.byref(st))
    return vis, st.as_dict()


def ring(x: float, y: float, width: int, height: int) -> int:
    return lib().or_ring(float(np.float32(x)), float(np.float32(y)), width, height)


def resolve_dilated(vis: np.ndarray, width: int, height: int, color: np.ndarray):
    vis = np.ascontiguousarray(vis, np.uint64)
    color = np.ascontiguousarray(color, np.uint32)
    out = np.empty(width * height, np.uint32)
    lib().or_resolve_dilated(_p(vis), width, height, _p(color), _p(out))
    return out


def decode_cloud(enc: Encoded, k: int = 3) -> np.ndarray:
    """Decoded positions of every point of an encoded cloud at precision k."""
    out = np.zeros((max(enc.n, 1), 3), np.float32)
    lib().or_decode_cloud(_p(enc.batches), len(enc.batches), _p(enc.w1), _p(enc.w2),
                          _p(enc.w3), int(k), _p(out))
    return out[:enc.n]


def render_hqs(enc: Encoded, view: View, vis: np.ndarray):
    """Sec. 3.6 high-quality shading image after the geometry pass `vis`."""
    vis = np.ascontiguousarray(vis, np.uint64)
    out = np.empty(view.width * view.height, np.uint32)
    lib().or_render_hqs(_p(enc.batches), len(enc.batches), _p(enc.w1), _p(enc.w2), _p(enc.w3),
                        _p(enc.color), ctypes.byref(view), _p(vis), _p(out))
    return out


def render_hqs_threaded(enc: Encoded, view: View, vis: np.ndarray, threads: int = 0):
    """render_hqs on `threads` host threads (the same image)."""
    import os
    vis = np.ascontiguousarray(vis, np.uint64)
    out = np.empty(view.width * view.height, np.uint32)
    lib().or_render_hqs_threaded(_p(enc.batches), len(enc.batches), _p(enc.w1), _p(enc.w2),
                                 _p(enc.w3), _p(enc.color), ctypes.byref(view), _p(vis),
                                 int(threads or os.cpu_count() or 1), _p(out))
    return out


def lod_render_hqs(lod: LodCloud, view: View, vis: np.ndarray, lod_px: float,
                   lod_px_periphery: float = 0.0):
    """Sec. 3.6 high-quality shading image of a LOD cloud after its geometry pass."""
    vis = np.ascontiguousarray(vis, np.uint64)
    out = np.empty(view.width * view.height, np.uint32)
    lib().or_lod_render_hqs(_p(lod.nodes), _p(lod.parent), len(lod.nodes), _p(lod.w1),
                            _p(lod.w2), _p(lod.w3), _p(lod.color), ctypes.byref(view),
                            float(lod_px), float(lod_px_periphery), _p(vis), _p(out))
    return out


def hqs_resolve_dilated(vis: np.ndarray, width: int, height: int, hqs: np.ndarray):
    """Depth-aware dilation (Sec. 3.7) of a high-quality shading image."""
    vis = np.ascontiguousarray(vis, np.uint64)
    hqs = np.ascontiguousarray(hqs, np.uint32)
    out = np.empty(width * height, np.uint32)
    lib().or_hqs_resolve_dilated(_p(vis), width, height, _p(hqs), _p(out))
    return out


def verify_encoding(xyz, rgba, batch_size, batches, w1, w2, w3, color, perm, threads=0):
    """(code, where): 0 when the arrays are the unique encoding of (xyz, rgba)
    defined by Sec. 3.1, Eq. 1 and Listing 2 (see or_verify_encoding)."""
    import os
    xyz = np.ascontiguousarray(xyz, np.float32)
    rgba = None if rgba is None else np.ascontiguousarray(rgba, np.uint32)
    arrs = [np.ascontiguousarray(a, np.uint32) for a in (w1, w2, w3, color, perm)]
    b = np.ascontiguousarray(batches, BATCH_DTYPE)
    where = np.zeros(1, np.uint64)
    code = lib().or_verify_encoding(_p(xyz), _p(rgba) if rgba is not None else None, len(xyz),
                                    int(batch_size), _p(b), len(b), *(_p(a) for a in arrs),
                                    int(threads or os.cpu_count() or 1), _p(where))
    return int(code), int(where[0])


def verify_lod(xyz, rgba, max_levels, max_node_points, seed, nodes, parent, level, perm, w1, w2,
               w3, color, threads=0):
    """(code, where): 0 when the arrays are the unique LOD tree of (xyz, rgba)
    that Sec. 3.5 defines (see or_verify_lod)."""
    import os
    xyz = np.ascontiguousarray(xyz, np.float32)
    rgba = None if rgba is None else np.ascontiguousarray(rgba, np.uint32)
    arrs = [np.ascontiguousarray(a, np.uint32) for a in (perm, w1, w2, w3, color)]
    nd = np.ascontiguousarray(nodes, BATCH_DTYPE)
    par = np.ascontiguousarray(parent, np.uint32)
    lev = np.ascontiguousarray(level, np.uint32)
    where = np.zeros(1, np.uint64)
    code = lib().or_verify_lod(_p(xyz), _p(rgba) if rgba is not None else None, len(xyz),
                               int(max_levels), int(max_node_points), int(seed), _p(nd), _p(par),
                               _p(lev), len(nd), *(_p(a) for a in arrs),
                               int(threads or os.cpu_count() or 1), _p(where))
    return int(code), int(where[0])
