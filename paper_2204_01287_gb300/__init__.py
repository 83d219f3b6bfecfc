"""Python binding of libpcr.so, the GB300 point-cloud rasterizer.

Thin ctypes marshalling over the C ABI in include/pc.h; the functions keep the
C names (pc_create, pc_upload_cloud, pc_render, ...). Every step of a frame runs
in the library's CUDA kernels; PyTorch only supplies device memory (tensors)
and streams. There is no CPU fallback: if libpcr.so is missing or fails to
load, the first call into the library raises.

Convenience layer: :class:`Context` wraps a pc_ctx with numpy/torch helpers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build_mod

_lib = None
_lock = threading.Lock()

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ENOTFOUND = 0, -1, -2, -3
PC_EBUSY, PC_ETIMEDOUT, PC_ECUDA, PC_ENOTSUP, PC_EDEVICE = -4, -5, -6, -7, -8
PC_CFG_TIMING = 1
PC_CFG_GRAPHS = 2
PC_CFG_KEEP_ORDER = 4
PC_ENCODE_KEEP_ORDER = 1
PC_VIEW_CULL = 1
PC_VIEW_NO_EARLY_DEPTH = 2
PC_VIEW_DILATE = 0x40
PC_VIEW_HQS = 0x80
PC_VIEW_HQS_PACKED = 0x100
PC_VIEW_SIGNED_EMPTY = 0x200
EMPTY_SIGNED = 0x7FFFFFFFFFFFFFFF
EMPTY = 0xFFFFFFFFFFFFFFFF


def PC_VIEW_FORCE_K(k: int) -> int:
    return (int(k) & 3) << 4


BATCH_DTYPE = np.dtype([("min", "<f4", (3,)), ("size", "<f4", (3,)),
                        ("first", "<u4"), ("count", "<u4")])


class pc_config(ctypes.Structure):
    _fields_ = [("batch_size", ctypes.c_uint32), ("precision_px", ctypes.c_float),
                ("encoder_threads", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("serve_pool_bytes", ctypes.c_uint64), ("serve_streams", ctypes.c_uint32),
                ("max_views_per_launch", ctypes.c_uint32),
                ("threads_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 4)]


class pc_view(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_float * 16), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("lod_px", ctypes.c_float), ("lod_px_periphery", ctypes.c_float),
                ("reserved", ctypes.c_uint32 * 3)]


class pc_framebuffer(ctypes.Structure):
    _fields_ = [("vis", ctypes.c_void_p), ("rgba", ctypes.c_void_p)]


class pc_cloud_info(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_uint64), ("n_batches", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("is_lod", ctypes.c_uint32),
                ("lod_levels", ctypes.c_uint32)]


class pc_view_stats(ctypes.Structure):
    _fields_ = [("batches_total", ctypes.c_uint64), ("batches_rendered", ctypes.c_uint64),
                ("batches_k", ctypes.c_uint64 * 4), ("points_k", ctypes.c_uint64 * 4),
                ("points_processed", ctypes.c_uint64),
                ("words_loaded_bytes", ctypes.c_uint64),
                ("points_atomic", ctypes.c_uint64),
                ("points_blended", ctypes.c_uint64), ("hqs_fallback_pixels", ctypes.c_uint64)]

    def as_dict(self):
        return {"batches_total": self.batches_total, "batches_rendered": self.batches_rendered,
                "batches_k": list(self.batches_k), "points_k": list(self.points_k),
                "points_processed": self.points_processed,
                "words_loaded_bytes": self.words_loaded_bytes,
                "points_atomic": self.points_atomic,
                "points_blended": self.points_blended,
                "hqs_fallback_pixels": self.hqs_fallback_pixels}


class pc_timing(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_uint32), ("launches", ctypes.c_uint32),
                ("ms_clear", ctypes.c_double), ("ms_cull", ctypes.c_double),
                ("ms_raster", ctypes.c_double), ("ms_shade", ctypes.c_double),
                ("ms_resolve", ctypes.c_double),
                ("raster_launches", ctypes.c_uint64)]


class pc_tune_result(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("points_per_warp", ctypes.c_uint32), ("views_per_launch", ctypes.c_uint32),
                ("ms_per_view", ctypes.c_double), ("ms_per_view_single", ctypes.c_double),
                ("candidates", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class pc_lod_opts(ctypes.Structure):
    _fields_ = [("max_levels", ctypes.c_uint32), ("max_node_points", ctypes.c_uint32),
                ("seed", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class pc_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("nviews", ctypes.c_uint32),
                ("rgba", ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))),
                ("widths", ctypes.POINTER(ctypes.c_uint32)),
                ("heights", ctypes.POINTER(ctypes.c_uint32)),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


# (name, restype, argtypes) of every entry point declared in include/pc.h
_vp, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
_P = ctypes.POINTER
SIGNATURES = [
    ("pc_config_default", None, [_P(pc_config)]),
    ("pc_strerror", ctypes.c_char_p, [_i32]),
    ("pc_create", _i32, [_P(_vp), ctypes.c_int, _P(pc_config)]),
    ("pc_destroy", None, [_vp]),
    ("pc_last_error", ctypes.c_char_p, [_vp]),
    ("pc_encode", _i32, [_vp, _vp, _u64, _u32, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("pc_upload_cloud", _i32, [_vp, _vp, _vp, _u64, _P(_u64)]),
    ("pc_upload_encoded", _i32, [_vp, _vp, _u64, _vp, _vp, _vp, _vp, _u64, _P(_u64)]),
    ("pc_cloud_get_info", _i32, [_vp, _u64, _P(pc_cloud_info)]),
    ("pc_cloud_download", _i32, [_vp, _u64, _vp, _vp, _vp, _vp, _vp]),
    ("pc_release_cloud", _i32, [_vp, _u64]),
    ("pc_build_lod", _i32, [_vp, _u64, _P(pc_lod_opts), _P(_u64)]),
    ("pc_lod_encode", _i32, [_vp, _vp, _u64, _P(pc_lod_opts), _u32, _u64, _vp, _vp, _vp,
                             _P(_u64), _vp, _vp, _vp, _vp, _vp]),
    ("pc_render", _i32, [_vp, _u64, _P(pc_view), _u32, _P(pc_framebuffer), _vp]),
    ("pc_render_range", _i32, [_vp, _u64, _u64, _u64, _P(pc_view), _u32, _P(pc_framebuffer),
                               _vp]),
    ("pc_resolve", _i32, [_vp, _u64, _P(pc_view), _u32, _P(pc_framebuffer), _vp]),
    ("pc_merge_min", _i32, [_vp, _vp, _u64, _vp]),
    ("pc_render_host", _i32, [_vp, _u64, _P(pc_view), _u32, _P(_vp), _vp]),
    ("pc_render_noalloc", _i32, [_vp, _u64, _vp, _vp, _vp, _vp, _u64, _P(pc_view), _vp, _vp,
                                 ctypes.c_float, _vp, _vp]),
    ("pc_get_view_stats", _i32, [_vp, _vp, _u32, _P(pc_view_stats)]),
    ("pc_autotune", _i32, [_vp, _u64, _P(pc_view), _u32, _vp, _P(pc_tune_result)]),
    ("pc_set_views_per_launch", _i32, [_vp, _u32]),
    ("pc_timing_begin", _i32, [_vp]),
    ("pc_timing_end", _i32, [_vp, _P(pc_timing)]),
    ("pc_submit", _i32, [_vp, _u64, _P(pc_view), _u32, _P(pc_framebuffer), _P(_u64)]),
    ("pc_poll", _i32, [_vp, _u64, _i32, _P(pc_result)]),
    ("pc_release_ticket", _i32, [_vp, _u64]),
]


def build(force: bool = False) -> str:
    """Compile libpcr.so for sm_103a (see build.py)."""
    return _build_mod.build(force=force)


def lib_path() -> str:
    return _build_mod.SO


def lib() -> ctypes.CDLL:
    """Load libpcr.so (raises if it has not been built for this machine)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build_mod.SO
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run paper_2204_01287_gb300.build() "
                                   "(the rasterizer has no CPU fallback)")
            L = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class PCError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{lib().pc_strerror(status).decode()} ({status}) {msg}".strip())


def _check(ctx, rc):
    if rc != PC_OK:
        msg = lib().pc_last_error(ctx).decode() if ctx else ""
        raise PCError(rc, msg)


# ---- thin wrappers keeping the C names ---------------------------------------

def pc_config_default() -> pc_config:
    c = pc_config()
    lib().pc_config_default(ctypes.byref(c))
    return c


def pc_create(device: int = 0, cfg: pc_config | None = None) -> int:
    h = ctypes.c_void_p()
    rc = lib().pc_create(ctypes.byref(h), device, ctypes.byref(cfg) if cfg else None)
    _check(None, rc)
    return h.value


def pc_destroy(ctx: int) -> None:
    lib().pc_destroy(ctx)


def _np_ptr(a):
    return None if a is None else a.ctypes.data


# The C ABI takes bare pointers and counts, so the sizes that make its reads
# and writes stay inside the caller's arrays are checked here.

class _Framebuffers(tuple):
    """(vis, rgba) tensor pairs made by Context.framebuffers, with the pixel
    count each pair holds; a tuple, so its tensors cannot be swapped."""

    def __new__(cls, pairs, npix, device):
        t = super().__new__(cls, pairs)
        t.npix = tuple(npix)
        t.device = device
        return t

    def fits(self, views, device) -> bool:
        return (device == self.device and len(views) == len(self.npix) and
                all(int(v.width) * int(v.height) <= n for v, n in zip(views, self.npix)))


def _as_xyz(xyz) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, np.float32)
    if xyz.ndim != 2 or xyz.shape[1] != 3:
        raise ValueError(f"xyz must have shape (n, 3), got {xyz.shape}")
    return xyz


def _as_rgba(rgba, n: int):
    if rgba is None:
        return None
    rgba = np.ascontiguousarray(rgba, np.uint32)
    if rgba.size != n:
        raise ValueError(f"rgba must hold one colour per point ({n}), got {rgba.size}")
    return rgba


def _check_framebuffers(views, fbs, device: int) -> None:
    """Each (vis, rgba) torch pair must hold the view's pixels (8 and 4 bytes
    each) contiguously on the context's CUDA device."""
    if len(fbs) != len(views):
        raise ValueError(f"{len(views)} views but {len(fbs)} framebuffers")
    for i, (v, (vis, rgba)) in enumerate(zip(views, fbs)):
        npix = int(v.width) * int(v.height)
        pairs = ((vis, 8, "vis"), (rgba, 4, "rgba"))
        for t, nb, name in pairs:
            if t.numel() * t.element_size() < npix * nb or not t.is_contiguous():
                raise ValueError(f"view {i}: {name} must be a contiguous tensor of at least "
                                 f"{npix * nb} bytes")
        for t, _, name in pairs:
            if t.device.type != "cuda" or t.device.index != device:
                raise ValueError(f"view {i}: {name} is on {t.device}, the context on cuda:{device}")


def pc_encode(xyz: np.ndarray, rgba: np.ndarray | None, batch_size: int = 10240,
              threads: int = 0, flags: int = 0):
    """Host encoder: returns (batches, w1, w2, w3, color, perm) numpy arrays."""
    xyz = _as_xyz(xyz)
    n = xyz.shape[0]
    rgba = _as_rgba(rgba, n)
    nb = (n + batch_size - 1) // batch_size
    batches = np.zeros(nb, BATCH_DTYPE)
    w = [np.zeros(n, np.uint32) for _ in range(4)]
    perm = np.zeros(n, np.uint32)
    rc = lib().pc_encode(_np_ptr(xyz), _np_ptr(rgba), n, batch_size, threads, flags,
                         _np_ptr(batches), *(x.ctypes.data for x in w), _np_ptr(perm))
    _check(None, rc)
    return batches, w[0], w[1], w[2], w[3], perm


def pc_upload_cloud(ctx: int, xyz: np.ndarray, rgba: np.ndarray | None) -> int:
    xyz = _as_xyz(xyz)
    rgba = _as_rgba(rgba, xyz.shape[0])
    out = ctypes.c_uint64()
    _check(ctx, lib().pc_upload_cloud(ctx, _np_ptr(xyz), _np_ptr(rgba), xyz.shape[0],
                                      ctypes.byref(out)))
    return out.value


def pc_upload_encoded(ctx: int, batches, w1, w2, w3, color) -> int:
    arrs = [np.ascontiguousarray(a, np.uint32).reshape(-1) for a in (w1, w2, w3, color)]
    if len({len(a) for a in arrs}) != 1:
        raise ValueError("w1, w2, w3 and color must have one entry per point each, got "
                         f"{[len(a) for a in arrs]}")
    b = np.ascontiguousarray(batches, BATCH_DTYPE)
    out = ctypes.c_uint64()
    _check(ctx, lib().pc_upload_encoded(ctx, _np_ptr(b), len(b), *(a.ctypes.data for a in arrs),
                                        len(arrs[0]), ctypes.byref(out)))
    return out.value


def pc_cloud_get_info(ctx: int, cloud: int) -> pc_cloud_info:
    info = pc_cloud_info()
    _check(ctx, lib().pc_cloud_get_info(ctx, cloud, ctypes.byref(info)))
    return info


def pc_cloud_download(ctx: int, cloud: int):
    info = pc_cloud_get_info(ctx, cloud)
    batches = np.zeros(info.n_batches, BATCH_DTYPE)
    w = [np.zeros(info.n_points, np.uint32) for _ in range(4)]
    _check(ctx, lib().pc_cloud_download(ctx, cloud, _np_ptr(batches), *(x.ctypes.data for x in w)))
    return batches, w[0], w[1], w[2], w[3]


def pc_release_cloud(ctx: int, cloud: int) -> None:
    _check(ctx, lib().pc_release_cloud(ctx, cloud))


def pc_build_lod(ctx: int, cloud: int, max_levels: int = 12, max_node_points: int = 10240,
                 seed: int = 0) -> int:
    o = pc_lod_opts(max_levels, max_node_points, seed, 0)
    out = ctypes.c_uint64()
    _check(ctx, lib().pc_build_lod(ctx, cloud, ctypes.byref(o), ctypes.byref(out)))
    return out.value


def pc_lod_encode(xyz: np.ndarray, rgba, max_levels: int = 12, max_node_points: int = 10240,
                  seed: int = 0, threads: int = 0, max_nodes: int | None = None):
    """Host LOD builder: (nodes, parent, level, perm, w1, w2, w3, color).
    max_nodes bounds the node arrays (default: one per point)."""
    xyz = _as_xyz(xyz)
    n = xyz.shape[0]
    rgba = _as_rgba(rgba, n)
    cap = max(int(max_nodes) if max_nodes else n, 1)
    nodes = np.zeros(cap, BATCH_DTYPE)
    parent = np.zeros(cap, np.uint32)
    level = np.zeros(cap, np.uint32)
    nn = ctypes.c_uint64()
    w = [np.zeros(max(n, 1), np.uint32) for _ in range(5)]
    o = pc_lod_opts(max_levels, max_node_points, seed, 0)
    _check(None, lib().pc_lod_encode(_np_ptr(xyz), _np_ptr(rgba), n, ctypes.byref(o), threads,
                                     cap, _np_ptr(nodes), _np_ptr(parent), _np_ptr(level),
                                     ctypes.byref(nn), *(x.ctypes.data for x in w)))
    k = nn.value
    return nodes[:k], parent[:k], level[:k], w[0][:n], w[1][:n], w[2][:n], w[3][:n], w[4][:n]


def make_view(m, width: int, height: int, flags: int = 0, lod_px: float = 0.0,
              lod_px_periphery: float = 0.0) -> pc_view:
    v = pc_view()
    mm = np.asarray(m, np.float32).reshape(16)
    for i in range(16):
        v.view_proj[i] = float(mm[i])
    v.width, v.height, v.flags, v.lod_px = int(width), int(height), int(flags), float(lod_px)
    v.lod_px_periphery = float(lod_px_periphery)
    return v


def _views_arr(views):
    arr = (pc_view * len(views))()
    for i, v in enumerate(views):
        arr[i] = v
    return arr


def pc_render(ctx: int, cloud: int, views, fbs, stream: int = 0) -> None:
    """fbs: list of (vis_ptr, rgba_ptr) device pointers (e.g. tensor.data_ptr())."""
    va = _views_arr(views)
    fa = (pc_framebuffer * len(views))()
    for i, (vis, rgba) in enumerate(fbs):
        fa[i] = pc_framebuffer(vis, rgba)
    _check(ctx, lib().pc_render(ctx, cloud, va, len(views), fa, stream))


def pc_render_range(ctx: int, cloud: int, first_batch: int, batch_count: int, views, fbs,
                    stream: int = 0) -> None:
    """One shard of a frame: batches [first_batch, first_batch + batch_count).
    fbs: (vis_ptr, rgba_ptr or None) device pointers per view."""
    va = _views_arr(views)
    fa = (pc_framebuffer * len(views))()
    for i, (vis, rgba) in enumerate(fbs):
        fa[i] = pc_framebuffer(vis, rgba)
    _check(ctx, lib().pc_render_range(ctx, cloud, first_batch, batch_count, va, len(views), fa,
                                      stream))


def pc_resolve(ctx: int, cloud: int, views, fbs, stream: int = 0) -> None:
    """Resolve merged visibility buffers into their images (fbs as for pc_render)."""
    va = _views_arr(views)
    fa = (pc_framebuffer * len(views))()
    for i, (vis, rgba) in enumerate(fbs):
        fa[i] = pc_framebuffer(vis, rgba)
    _check(ctx, lib().pc_resolve(ctx, cloud, va, len(views), fa, stream))


def pc_merge_min(dst: int, src: int, n: int, stream: int = 0) -> None:
    """dst[i] = min(dst[i], src[i]) over n keys (device pointers)."""
    _check(None, lib().pc_merge_min(dst, src, n, stream))


def batch_range(n_batches: int, rank: int, world: int):
    """(first, count): the contiguous batch range of one rank when a frame's
    batches are split over `world` ranks as evenly as possible (Sec. 3.2:
    batches are independent, so the shards merge by a minimum of keys)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    first = n_batches * rank // world
    return first, n_batches * (rank + 1) // world - first


def merge_shards(vis, group=None) -> None:
    """Element-wise minimum of one visibility buffer (int64 torch tensor,
    rendered with PC_VIEW_SIGNED_EMPTY) over the ranks of a process group, in
    place: the exchange step of a frame split by batch ranges."""
    import torch.distributed as dist
    dist.all_reduce(vis, op=dist.ReduceOp.MIN, group=group)


def pc_render_host(ctx: int, cloud: int, views, out_images, stream: int = 0) -> None:
    """out_images: list of writable numpy uint32 arrays (width*height each)."""
    if len(out_images) != len(views):
        raise ValueError(f"{len(views)} views but {len(out_images)} images")
    for i, (v, o) in enumerate(zip(views, out_images)):
        if (not isinstance(o, np.ndarray) or o.nbytes < 4 * int(v.width) * int(v.height)
                or not o.flags.c_contiguous or not o.flags.writeable):
            raise ValueError(f"view {i}: the image must be a writable contiguous array of "
                             f"{v.width}x{v.height} 32-bit pixels")
    va = _views_arr(views)
    ptrs = (ctypes.c_void_p * len(views))(*[o.ctypes.data for o in out_images])
    _check(ctx, lib().pc_render_host(ctx, cloud, va, len(views), ptrs, stream))


def pc_get_view_stats(ctx: int, view: int = 0, stream: int = 0) -> dict:
    st = pc_view_stats()
    _check(ctx, lib().pc_get_view_stats(ctx, stream, view, ctypes.byref(st)))
    return st.as_dict()


def pc_autotune(ctx: int, cloud: int, views, stream: int = 0) -> dict:
    va = _views_arr(views)
    r = pc_tune_result()
    _check(ctx, lib().pc_autotune(ctx, cloud, va, len(views), stream, ctypes.byref(r)))
    return r.as_dict()


def pc_set_views_per_launch(ctx: int, n: int) -> None:
    _check(ctx, lib().pc_set_views_per_launch(ctx, n))


def pc_timing_begin(ctx: int) -> None:
    _check(ctx, lib().pc_timing_begin(ctx))


def pc_timing_end(ctx: int) -> pc_timing:
    t = pc_timing()
    _check(ctx, lib().pc_timing_end(ctx, ctypes.byref(t)))
    return t


def pc_submit(ctx: int, cloud: int, views, fbs=None) -> int:
    """fbs: None (library-owned framebuffers, host images from pc_poll) or a
    list of (vis, rgba) device pointers, one per view."""
    va = _views_arr(views)
    fa = None
    if fbs is not None:
        fa = (pc_framebuffer * len(views))()
        for i, (vis, rgba) in enumerate(fbs):
            fa[i].vis, fa[i].rgba = vis, rgba
    out = ctypes.c_uint64()
    _check(ctx, lib().pc_submit(ctx, cloud, va, len(views), fa, ctypes.byref(out)))
    return out.value


def pc_poll(ctx: int, ticket: int, timeout_ms: int = 10000, copy_images: bool = True):
    """Returns (status, result) — status PC_OK or PC_ETIMEDOUT; result holds
    numpy copies of the images when PC_OK (none with copy_images=False).
    timeout_ms: 0..60000 (larger values wait 60 s; negative ones raise)."""
    r = pc_result()
    rc = lib().pc_poll(ctx, ticket, timeout_ms, ctypes.byref(r))
    if rc == PC_ETIMEDOUT:
        return rc, None
    _check(ctx, rc)
    imgs = []
    for v in range(r.nviews if (r.rgba and copy_images) else 0):
        n = r.widths[v] * r.heights[v]
        imgs.append(np.ctypeslib.as_array(r.rgba[v], shape=(n,)).copy())
    return rc, {"status": r.status, "images": imgs, "t_submit_ms": r.t_submit_ms,
                "t_start_ms": r.t_start_ms, "t_done_ms": r.t_done_ms}


def pc_release_ticket(ctx: int, ticket: int) -> None:
    _check(ctx, lib().pc_release_ticket(ctx, ticket))


# ---- convenience ------------------------------------------------------------------

class Context:
    """A pc_ctx on one CUDA device with torch-allocated framebuffers."""

    def __init__(self, device: int = 0, **cfg_fields):
        cfg = pc_config_default()
        for k, v in cfg_fields.items():
            setattr(cfg, k, v)
        self.device = device
        self.h = pc_create(device, cfg)

    def close(self):
        if self.h:
            pc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, xyz, rgba=None) -> int:
        return pc_upload_cloud(self.h, xyz, rgba)

    def upload_encoded(self, batches, w1, w2, w3, color) -> int:
        return pc_upload_encoded(self.h, batches, w1, w2, w3, color)

    def framebuffers(self, views):
        """torch (vis, rgba) tensors for each view, on this device: an
        immutable sequence that remembers the pixel counts it was made for."""
        import torch
        dev = torch.device("cuda", self.device)
        return _Framebuffers(
            [(torch.empty(v.height * v.width, dtype=torch.int64, device=dev),
              torch.empty(v.height * v.width, dtype=torch.int32, device=dev)) for v in views],
            [int(v.width) * int(v.height) for v in views], self.device)

    def render(self, cloud, views, fbs=None, stream=None):
        """Render views into torch framebuffers (allocated when fbs is None)
        on `stream` (a torch.cuda.Stream; default the current stream). fbs not
        made by framebuffers() for views at least this large is checked tensor
        by tensor (size, contiguity, device) before the launch."""
        import torch
        if fbs is None:
            fbs = self.framebuffers(views)
        elif not (isinstance(fbs, _Framebuffers) and fbs.fits(views, self.device)):
            _check_framebuffers(views, fbs, self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        pc_render(self.h, cloud, views, [(a.data_ptr(), b.data_ptr()) for a, b in fbs],
                  s.cuda_stream)
        return fbs

    def render_range(self, cloud, first_batch, batch_count, views, fbs=None, stream=None):
        """One shard (a batch range) of each view into torch framebuffers."""
        import torch
        if fbs is None:
            fbs = self.framebuffers(views)
        elif not (isinstance(fbs, _Framebuffers) and fbs.fits(views, self.device)):
            _check_framebuffers(views, fbs, self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        pc_render_range(self.h, cloud, first_batch, batch_count, views,
                        [(a.data_ptr(), b.data_ptr()) for a, b in fbs], s.cuda_stream)
        return fbs

    def resolve(self, cloud, views, fbs, stream=None):
        """The images of visibility buffers filled (and merged) earlier."""
        import torch
        if not (isinstance(fbs, _Framebuffers) and fbs.fits(views, self.device)):
            _check_framebuffers(views, fbs, self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        pc_resolve(self.h, cloud, views, [(a.data_ptr(), b.data_ptr()) for a, b in fbs],
                   s.cuda_stream)
        return fbs

    def merge_min(self, dst, src, stream=None):
        """dst <- min(dst, src) for two int64 visibility tensors of one size."""
        import torch
        if dst.numel() != src.numel() or dst.dtype != torch.int64 or src.dtype != torch.int64:
            raise ValueError("merge_min needs two int64 visibility buffers of one size")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        pc_merge_min(dst.data_ptr(), src.data_ptr(), dst.numel(), s.cuda_stream)
        return dst

    def stats(self, view=0, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return pc_get_view_stats(self.h, view, s.cuda_stream)


def vis_to_numpy(t) -> np.ndarray:
    """int64 torch visibility buffer -> uint64 numpy array."""
    return t.cpu().numpy().view(np.uint64)


def rgba_to_numpy(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)
