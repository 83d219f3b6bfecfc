"""pc_render_noalloc: the render path for callers that may not allocate device
memory, with its scratch in a static device array. Its output must equal
pc_render's (bit-exact, like every other parity test here) on two calls in a
row, so the shared scratch must start clean on every call. This file is named
to be collected last."""
import ctypes

import numpy as np
import pytest

import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu


def _device_words(torch, a):
    n = len(a)
    t = torch.zeros(((n + 3) // 4) * 4 + 4, dtype=torch.int32, device="cuda")
    t[:n] = torch.from_numpy(a.view(np.int32)).cuda()
    return t


def test_noalloc_matches_pc_render(cuda_lib):
    import torch
    p = S.terrain_params(4000.0, 0.2, 150)
    xyz, rgba = S.terrain(300_003, p, seed=8)
    batches, w1, w2, w3, col, _ = pcr.pc_encode(xyz, rgba, batch_size=10240)
    with pcr.Context(0) as ctx:
        cloud = ctx.upload_encoded(batches, w1, w2, w3, col)
        dev_batches = torch.from_numpy(batches.view(np.uint8).copy()).cuda()
        words = [_device_words(torch, a) for a in (w1, w2, w3, col)]
        L = pcr.lib()
        views = [pcr.make_view(S.flythrough(p, 5, 120, 200, 120, seed=8), 200, 120, pcr.PC_VIEW_CULL),
                 pcr.make_view(S.random_view(p, 3, 96, 160, seed=8), 96, 160, pcr.PC_VIEW_CULL)]
        for v in views:
            [(ref_vis, ref_img)] = ctx.render(cloud, [v])
            vis = torch.empty(v.width * v.height, dtype=torch.int64, device="cuda")
            img = torch.empty(v.width * v.height, dtype=torch.int32, device="cuda")
            rc = L.pc_render_noalloc(dev_batches.data_ptr(), len(batches),
                                     *(w.data_ptr() for w in words), len(col),
                                     ctypes.byref(v), vis.data_ptr(), img.data_ptr(), 512.0,
                                     torch.cuda.current_stream().cuda_stream)
            assert rc == pcr.PC_OK
            torch.cuda.synchronize()
            assert torch.equal(vis, ref_vis)
            assert torch.equal(img, ref_img)
            assert int((vis != -1).sum()) > 100


def test_noalloc_rejects_oversize_and_misaligned(cuda_lib):
    import torch
    L = pcr.lib()
    v = pcr.make_view(S.cube_camera(8, 8), 8, 8)
    vis = torch.empty(64, dtype=torch.int64, device="cuda")
    w = torch.zeros(16, dtype=torch.int32, device="cuda")
    b = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.pc_render_noalloc(b.data_ptr(), 1 << 17, *(w.data_ptr(),) * 4, 4, ctypes.byref(v),
                               vis.data_ptr(), None, 512.0, st) == pcr.PC_EINVAL
    assert L.pc_render_noalloc(b.data_ptr(), 1, w.data_ptr() + 4, w.data_ptr(), w.data_ptr(),
                               w.data_ptr(), 4, ctypes.byref(v), vis.data_ptr(), None, 512.0,
                               st) == pcr.PC_EINVAL
