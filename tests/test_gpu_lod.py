"""LOD clouds on the GPU (Sec. 3.5) against the oracle: the tree uploaded by
pc_build_lod and every rendered frame must be bit-identical."""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu

M, L, SEED = 4096, 12, 7


@pytest.fixture(scope="module")
def lodworld(cuda_lib):
    ctx = pcr.Context(0)
    p = S.terrain_params(6000.0, 0.2, 200)
    xyz, rgba = S.terrain(800_000, p, seed=12)
    enc = O.encode(xyz, rgba, 10240)
    cloud = ctx.upload(xyz, rgba)
    lod = pcr.pc_build_lod(ctx.h, cloud, L, M, SEED)
    ref = O.lod_build(O.decode_cloud(enc, 3), enc.color, L, M, SEED)
    yield ctx, p, lod, ref
    ctx.close()


def test_uploaded_tree_matches_oracle(lodworld):
    ctx, p, lod, ref = lodworld
    info = pcr.pc_cloud_get_info(ctx.h, lod)
    assert info.is_lod == 1 and info.n_batches == len(ref.nodes)
    assert info.lod_levels == int(ref.level.max()) + 1
    nodes, w1, w2, w3, col = pcr.pc_cloud_download(ctx.h, lod)
    assert nodes.tobytes() == ref.nodes.tobytes()
    for a, b in ((w1, ref.w1), (w2, ref.w2), (w3, ref.w3), (col, ref.color)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("lod_px", [0.0, 100.0, 300.0])
@pytest.mark.parametrize("frame", [0, 30, 75])
def test_lod_frames_match_oracle(lodworld, frame, lod_px):
    import torch
    ctx, p, lod, ref = lodworld
    W, H = 320, 180
    m = S.flythrough(p, frame, 120, W, H, seed=12)
    [(vis, img)] = ctx.render(lod, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL, lod_px)])
    torch.cuda.synchronize()
    st = ctx.stats()
    ovis, ost = O.lod_render(ref, O.make_view(m, W, H), lod_px)
    assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
    assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve(ovis, ref.color))
    assert st["batches_rendered"] == ost["batches_rendered"]
    assert st["points_processed"] == ost["points_processed"]
    assert st["batches_k"] == ost["batches_k"]


def test_lod_multiview_mixed_thresholds(lodworld):
    """Views with different thresholds in one launch each match the oracle."""
    import torch
    ctx, p, lod, ref = lodworld
    views = [pcr.make_view(S.random_view(p, 60 + i, 160, 100, seed=12), 160, 100,
                           pcr.PC_VIEW_CULL, [0.0, 50.0, 300.0, 1000.0][i % 4]) for i in range(7)]
    out = ctx.render(lod, views)
    torch.cuda.synchronize()
    for v, (vis, img) in zip(views, out):
        ovis, _ = O.lod_render(ref, O.make_view(np.array(v.view_proj), v.width, v.height), v.lod_px)
        assert np.array_equal(pcr.vis_to_numpy(vis), ovis)


def test_lod_threshold_reduces_work(lodworld):
    import torch
    ctx, p, lod, ref = lodworld
    m = S.flythrough(p, 40, 120, 640, 360, seed=12)
    processed = []
    for px in (0.0, 300.0, 1000.0, 3000.0):
        ctx.render(lod, [pcr.make_view(m, 640, 360, pcr.PC_VIEW_CULL, px)])
        torch.cuda.synchronize()
        processed.append(ctx.stats()["points_processed"])
    assert all(a >= b for a, b in zip(processed, processed[1:])) and processed[-1] > 0
    assert processed[0] > processed[-1]


@pytest.mark.parametrize("frame", [10, 64])
def test_foveated_lod_and_dilation_match_oracle(lodworld, frame):
    """Sec. 3.7: thresholds of 100 px in the centre, 200 px between and 300 px in
    the periphery, and the depth-aware 3x3 .. 7x7 dilation in the resolve."""
    import torch
    ctx, p, lod, ref = lodworld
    W, H = 300, 200
    m = S.flythrough(p, frame, 120, W, H, seed=12)
    v = pcr.make_view(m, W, H, pcr.PC_VIEW_CULL | pcr.PC_VIEW_DILATE, 100.0, 300.0)
    [(vis, img)] = ctx.render(lod, [v])
    torch.cuda.synchronize()
    st = ctx.stats()
    ovis, ost = O.lod_render(ref, O.make_view(m, W, H), 100.0, 300.0)
    assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
    assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve_dilated(ovis, W, H, ref.color))
    assert st["batches_rendered"] == ost["batches_rendered"]
    _, flat = O.lod_render(ref, O.make_view(m, W, H), 100.0)
    assert ost["points_processed"] <= flat["points_processed"]


def test_dilation_on_plain_cloud(cuda_lib):
    import torch
    p = S.terrain_params(3000.0)
    xyz, rgba = S.terrain(200_000, p, seed=13)
    enc = O.encode(xyz, rgba, 10240)
    with pcr.Context(0) as ctx:
        cloud = ctx.upload(xyz, rgba)
        m = S.random_view(p, 4, 180, 120, seed=13)
        [(vis, img)] = ctx.render(cloud, [pcr.make_view(m, 180, 120, pcr.PC_VIEW_DILATE)])
        torch.cuda.synchronize()
        ovis, _ = O.render(enc, O.make_view(m, 180, 120))
        assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
        assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve_dilated(ovis, 180, 120, enc.color))
