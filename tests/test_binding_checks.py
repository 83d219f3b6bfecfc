"""The Python binding's argument checks (no GPU): the C ABI takes bare pointers
and counts, so arrays whose sizes would make it read or write past their ends
are refused before the call."""
import numpy as np
import pytest
import torch

import paper_2204_01287_gb300 as pcr


def _view(w, h):
    return pcr.make_view(np.eye(4, dtype=np.float32), w, h)


def test_xyz_must_be_n_by_3():
    flat = np.zeros(30, np.float32)                 # 10 points, flattened
    with pytest.raises(ValueError):
        pcr.pc_encode(flat, None, batch_size=8)
    with pytest.raises(ValueError):
        pcr.pc_lod_encode(flat, None)
    with pytest.raises(ValueError):
        pcr.pc_encode(np.zeros((10, 4), np.float32), None, batch_size=8)


def test_one_colour_per_point():
    xyz = np.zeros((10, 3), np.float32)
    for bad in (np.zeros(9, np.uint32), np.zeros(11, np.uint32)):
        with pytest.raises(ValueError):
            pcr.pc_encode(xyz, bad, batch_size=8)
        with pytest.raises(ValueError):
            pcr.pc_lod_encode(xyz, bad)
    b, *_ = pcr.pc_encode(xyz, np.arange(10, dtype=np.uint32), batch_size=8)
    assert len(b) == 2


def test_upload_encoded_needs_equal_lengths():
    b = np.zeros(1, pcr.BATCH_DTYPE)
    w = np.zeros(8, np.uint32)
    with pytest.raises(ValueError):   # refused before the context is touched
        pcr.pc_upload_encoded(0, b, w, w, w, np.zeros(7, np.uint32))


def test_render_host_images_must_hold_the_view():
    v = _view(8, 4)
    with pytest.raises(ValueError):
        pcr.pc_render_host(0, 1, [v], [np.zeros(31, np.uint32)])
    with pytest.raises(ValueError):
        pcr.pc_render_host(0, 1, [v], [np.zeros(64, np.uint32)[::2]])   # not contiguous
    ro = np.zeros(32, np.uint32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        pcr.pc_render_host(0, 1, [v], [ro])
    with pytest.raises(ValueError):
        pcr.pc_render_host(0, 1, [v, v], [np.zeros(32, np.uint32)])


def test_framebuffer_tensors_checked():
    v = _view(8, 4)
    good = (torch.zeros(32, dtype=torch.int64), torch.zeros(32, dtype=torch.int32))
    with pytest.raises(ValueError, match="at least 256 bytes"):
        pcr._check_framebuffers([v], [(torch.zeros(31, dtype=torch.int64), good[1])], 0)
    with pytest.raises(ValueError, match="at least 128 bytes"):
        pcr._check_framebuffers([v], [(good[0], torch.zeros(16, dtype=torch.int32))], 0)
    with pytest.raises(ValueError, match="contiguous"):
        pcr._check_framebuffers([v], [(torch.zeros(64, dtype=torch.int64)[::2], good[1])], 0)
    with pytest.raises(ValueError, match="is on cpu"):
        pcr._check_framebuffers([v], [good], 0)
    with pytest.raises(ValueError, match="2 views but 1"):
        pcr._check_framebuffers([v, v], [good], 0)


def test_framebuffers_remember_their_sizes():
    pairs = [(torch.zeros(32, dtype=torch.int64), torch.zeros(32, dtype=torch.int32))]
    fb = pcr._Framebuffers(pairs, [32], 0)
    assert isinstance(fb, tuple) and len(fb) == 1
    [(vis, rgba)] = fb
    assert vis.numel() == 32
    assert fb.fits([_view(8, 4)], 0) and fb.fits([_view(4, 4)], 0)
    assert not fb.fits([_view(8, 5)], 0)            # larger than it was made for
    assert not fb.fits([_view(8, 4)], 1)            # another device
    assert not fb.fits([_view(8, 4)] * 2, 0)


def test_context_render_flow(monkeypatch):
    """Context.render's marshalling with the library call and the CUDA
    allocations replaced by CPU stand-ins: framebuffers it made itself skip
    the tensor checks; others are checked before any launch."""
    calls = []
    monkeypatch.setattr(pcr, "pc_render",
                        lambda h, cloud, views, ptrs, stream: calls.append((h, cloud, ptrs)))

    class _Stream:
        cuda_stream = 0

    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: _Stream())
    ctx = object.__new__(pcr.Context)
    ctx.h, ctx.device = 0, 0

    def cpu_framebuffers(views):
        return pcr._Framebuffers(
            [(torch.zeros(v.width * v.height, dtype=torch.int64),
              torch.zeros(v.width * v.height, dtype=torch.int32)) for v in views],
            [v.width * v.height for v in views], 0)

    monkeypatch.setattr(ctx, "framebuffers", cpu_framebuffers, raising=False)
    views = [_view(8, 4), _view(2, 2)]
    fbs = ctx.render(7, views)
    assert isinstance(fbs, pcr._Framebuffers) and len(calls) == 1
    assert calls[0][1] == 7 and calls[0][2] == [(a.data_ptr(), b.data_ptr()) for a, b in fbs]
    assert ctx.render(7, views, fbs) is fbs and len(calls) == 2
    with pytest.raises(ValueError, match="is on cpu"):   # a plain list is checked
        ctx.render(7, views, list(fbs))
    with pytest.raises(ValueError, match="at least"):    # views larger than the buffers
        ctx.render(7, [_view(8, 5), _view(2, 2)], fbs)
    assert len(calls) == 2
    ctx.h = None                                          # nothing to destroy
