"""Frames split by batch ranges (the multi-GPU partition of the method: Sec.
3.2's batches are drawn independently, and Listing 1's minimum over keys is
associative), run as shards on one GPU through the C ABI: every shard renders
its range into its own visibility buffer, the shards merge by an element-wise
minimum (pc_merge_min, or a signed int64 minimum with PC_VIEW_SIGNED_EMPTY, as
a MIN reduction across GPUs would do it), and pc_resolve writes the image. The
merged buffer and image must equal the CPU oracle's whole-frame render."""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world(cuda_lib):
    p = S.terrain_params(5000.0, 0.2, 200)
    xyz, rgba = S.terrain(700_001, p, seed=21)
    enc = O.encode(xyz, rgba, 10240)
    ctx = pcr.Context(0)
    cloud = ctx.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
    yield ctx, cloud, p, enc
    ctx.close()


def _views(p, W, H, flags):
    return [pcr.make_view(S.flythrough(p, 30, 120, W, H, seed=21), W, H, flags),
            pcr.make_view(S.random_view(p, 9, W, H, seed=21), W, H, flags)]


@pytest.mark.parametrize("world_size", [2, 3, 5])
def test_shards_merge_to_the_whole_frame(world, world_size):
    import torch
    ctx, cloud, p, enc = world
    W, H = 240, 135
    views = _views(p, W, H, pcr.PC_VIEW_CULL)
    nb = len(enc.batches)
    merged = None
    for r in range(world_size):
        first, count = pcr.batch_range(nb, r, world_size)
        fbs = ctx.render_range(cloud, first, count, views)
        if merged is None:
            merged = fbs
        else:
            for (dst, _), (src, _) in zip(merged, fbs):
                ctx.merge_min(dst, src)
    ctx.resolve(cloud, views, merged)
    torch.cuda.synchronize()
    for v, (vis, img) in zip(views, merged):
        ov = O.make_view(np.frombuffer(bytes(v.view_proj), np.float32), W, H, cull=True)
        ovis, _ = O.render(enc, ov)
        assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
        assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve(ovis, enc.color))
        assert (ovis != O.EMPTY).sum() > 1000


def test_signed_empty_merges_with_a_signed_minimum(world):
    """With PC_VIEW_SIGNED_EMPTY the empty key is 2^63 - 1, so the signed int64
    minimum that torch.distributed and MPI reduce with gives the same merge."""
    import torch
    ctx, cloud, p, enc = world
    W, H = 200, 150
    views = _views(p, W, H, pcr.PC_VIEW_CULL | pcr.PC_VIEW_SIGNED_EMPTY)
    nb = len(enc.batches)
    a = ctx.render_range(cloud, 0, nb // 3, views)
    b = ctx.render_range(cloud, nb // 3, nb - nb // 3, views)
    for (va, _), (vb, _) in zip(a, b):
        torch.minimum(va, vb, out=va)
    ctx.resolve(cloud, views, a)
    torch.cuda.synchronize()
    for v, (vis, img) in zip(views, a):
        ov = O.make_view(np.frombuffer(bytes(v.view_proj), np.float32), W, H, cull=True)
        ovis, _ = O.render(enc, ov)
        got = pcr.vis_to_numpy(vis)
        empty = ovis == O.EMPTY
        assert (got[empty] == pcr.EMPTY_SIGNED).all()
        assert np.array_equal(got[~empty], ovis[~empty])
        assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve(ovis, enc.color))
        assert empty.any() and (~empty).any()


def test_ranges_are_checked(world):
    ctx, cloud, p, enc = world
    nb = len(enc.batches)
    v = _views(p, 32, 32, 0)[:1]
    for first, count in ((0, 0), (nb, 1), (nb - 1, 2)):
        with pytest.raises(pcr.PCError) as e:
            ctx.render_range(cloud, first, count, v)
        assert e.value.status == pcr.PC_EINVAL
