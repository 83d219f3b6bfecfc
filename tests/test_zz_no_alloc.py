"""pc_render_noalloc: the render path for callers that may not allocate device
memory (code running while another thread captures a CUDA graph, plug-ins whose
host owns every allocation), with its scratch in a static device array. Its
visibility buffer and image must equal the CPU oracle's, bit for bit, on two
calls in a row (the shared array must start clean every call), for a cloud
with ragged batches and for a view that culls most of them. This file is named
to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu


def _device_words(torch, a):
    n = len(a)
    t = torch.zeros(((n + 3) // 4) * 4 + 4, dtype=torch.int32, device="cuda")
    t[:n] = torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    return t


def _device_batches(torch, batches):
    return torch.from_numpy(np.ascontiguousarray(batches).view(np.uint8).copy()).cuda()


def _render(L, torch, dev_batches, nb, words, n, view, err):
    vis = torch.empty(view.width * view.height, dtype=torch.int64, device="cuda")
    img = torch.empty(view.width * view.height, dtype=torch.int32, device="cuda")
    rc = L.pc_render_noalloc(dev_batches.data_ptr(), nb, *(w.data_ptr() for w in words), n,
                             ctypes.byref(view), vis.data_ptr(), img.data_ptr(), 512.0,
                             err.ctypes.data, torch.cuda.current_stream().cuda_stream)
    assert rc == pcr.PC_OK
    torch.cuda.synchronize()
    return pcr.vis_to_numpy(vis), pcr.rgba_to_numpy(img)


def test_noalloc_matches_oracle(cuda_lib):
    import torch
    p = S.terrain_params(4000.0, 0.2, 150)
    xyz, rgba = S.terrain(300_003, p, seed=8)
    enc = O.encode(xyz, rgba, 10240)          # the last batch is ragged (3,043 points)
    # a second cloud of batches with ragged counts everywhere: the oracle's
    # batches cut again at uneven points (still consecutive runs with boxes
    # that hold their points, so every point keeps its decoded position)
    rag = []
    for b in enc.batches:
        first, count = int(b["first"]), int(b["count"])
        cut = 1 + (first * 7919) % (count - 1)
        for f, c in ((first, cut), (first + cut, count - cut)):
            nb = b.copy()
            nb["first"], nb["count"] = f, c
            rag.append(nb)
    ragged = np.array(rag, dtype=enc.batches.dtype)
    L = pcr.lib()
    words = [_device_words(torch, a) for a in (enc.w1, enc.w2, enc.w3, enc.color)]
    W1, H1, W2, H2 = 200, 120, 96, 160
    h = S.terrain_height(p, 500.0, -300.0)
    views = [(S.flythrough(p, 5, 120, W1, H1, seed=8), W1, H1),
             (S.random_view(p, 3, W2, H2, seed=8), W2, H2),
             # looking down on a small patch from 400 m: most batches are culled
             (S.look_at_perspective((500, -300, h + 400), (500, -300, h), (0, 1, 0), 40.0,
                                    W1 / H1, 0.5, 1e5), W1, H1)]
    err = np.full(2, 7, np.uint32)
    for batches in (enc.batches, ragged):
        dev_b = _device_batches(torch, batches)
        renc = O.Encoded(batches, enc.w1, enc.w2, enc.w3, enc.color, enc.perm)
        for m, W, H in views:
            v = pcr.make_view(m, W, H, pcr.PC_VIEW_CULL)
            ovis, st = O.render(renc, O.make_view(m, W, H, cull=True))
            oimg = O.resolve(ovis, enc.color)
            for _ in range(2):   # two calls in a row on the shared array
                vis, img = _render(L, torch, dev_b, len(batches), words, enc.n, v, err)
                assert np.array_equal(vis, ovis)
                assert np.array_equal(img, oimg)
                assert err[0] == 0
            assert (ovis != O.EMPTY).sum() > 50
    # the culling view leaves most batches out
    _, st = O.render(enc, O.make_view(views[2][0], W1, H1, cull=True))
    assert st["batches_rendered"] < len(enc.batches) // 2


def test_noalloc_reports_device_errors(cuda_lib):
    """Batches that overlap so that their segments overflow the static draw
    list: the error word says so, and the next good call is clean again."""
    import torch
    xyz, rgba = S.unit_cube(1 << 20, seed=2)
    enc = O.encode(xyz, rgba, 10240)
    L = pcr.lib()
    words = [_device_words(torch, a) for a in (enc.w1, enc.w2, enc.w3, enc.color)]
    whole = enc.batches[:1].copy()
    whole["min"] = xyz.min(axis=0)
    whole["size"] = xyz.max(axis=0) - xyz.min(axis=0)
    whole["first"], whole["count"] = 0, enc.n
    over = np.repeat(whole, 300)   # 300 x 512 segments > 131,072 draw-list entries
    v = pcr.make_view(S.cube_camera(64, 64), 64, 64)
    err = np.zeros(2, np.uint32)
    _render(L, torch, _device_batches(torch, over), len(over), words, enc.n, v, err)
    assert err[0] == 1   # draw-list overflow
    vis, img = _render(L, torch, _device_batches(torch, enc.batches), len(enc.batches), words,
                       enc.n, v, err)
    assert err[0] == 0
    ovis, _ = O.render(enc, O.make_view(S.cube_camera(64, 64), 64, 64))
    assert np.array_equal(vis, ovis)


def test_noalloc_rejects_oversize_and_misaligned(cuda_lib):
    import torch
    L = pcr.lib()
    v = pcr.make_view(S.cube_camera(8, 8), 8, 8)
    vis = torch.empty(64, dtype=torch.int64, device="cuda")
    w = torch.zeros(16, dtype=torch.int32, device="cuda")
    b = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    wp = w.data_ptr()

    def call(batches, nb, w1, w2, w3, col):
        return L.pc_render_noalloc(batches, nb, w1, w2, w3, col, 4, ctypes.byref(v),
                                   vis.data_ptr(), None, 512.0, None, st)

    assert call(b.data_ptr(), 1 << 17, wp, wp, wp, wp) == pcr.PC_EINVAL
    assert call(b.data_ptr(), 1, wp + 4, wp, wp, wp) == pcr.PC_EINVAL
    assert call(b.data_ptr(), 1, wp, wp, wp, wp + 4) == pcr.PC_EINVAL        # colours
    assert call(b.data_ptr() + 4, 1, wp, wp, wp, wp) == pcr.PC_EINVAL        # batches
