"""GPU path (through the C ABI) against the CPU oracle, element by element.

Visibility buffers and images must be bit-identical: keys are integers and
every float that decides a pixel or a depth follows the same binary32 operation
order on both sides (no contraction, IEEE divides).
"""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = pcr.Context(0)
    yield c
    c.close()


def gpu_render(ctx, cloud, views, **kw):
    import torch
    fbs = ctx.render(cloud, views, **kw)
    torch.cuda.synchronize()
    return [(pcr.vis_to_numpy(a), pcr.rgba_to_numpy(b)) for a, b in fbs]


def oracle_view(m, W, H, cull=False, force_k=0, T=512.0):
    return O.make_view(m, W, H, cull=cull, force_k=force_k, threshold_px=T)


def assert_same(gvis, grgba, ovis, color, what=""):
    diff = np.nonzero(gvis != ovis)[0]
    assert len(diff) == 0, f"{what}: {len(diff)} pixels differ, first {diff[:5]}, " \
                           f"gpu {gvis[diff[:3]]} oracle {ovis[diff[:3]]}"
    assert np.array_equal(grgba, O.resolve(ovis, color)), what


# ---- config 1, small and full -------------------------------------------------------

@pytest.mark.parametrize("n,W,H", [(20000, 64, 48), (1000000, 512, 512)])
def test_unit_cube_forced_k3(ctx, n, W, H):
    """1M uniform points, Morton batches of 10,240, one 512x512 view, 30-bit
    precision, no culling: visibility buffer and image bit-exact."""
    xyz, rgba = S.unit_cube(n, seed=0)
    enc = O.encode(xyz, rgba, 10240)
    cloud = ctx.upload(xyz, rgba)
    m = S.cube_camera(W, H)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, W, H, pcr.PC_VIEW_FORCE_K(3))])
    ovis, st = O.render(enc, oracle_view(m, W, H, force_k=3))
    assert_same(vis, img, ovis, enc.color, "cube")
    assert (ovis != O.EMPTY).sum() > 0.1 * W * H
    gst = ctx.stats()
    assert gst["points_k"][3] == n and gst["batches_rendered"] == len(enc.batches)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_forced_precisions(ctx, k):
    xyz, rgba = S.unit_cube(60000, seed=1)
    enc = O.encode(xyz, rgba, 10240)
    cloud = ctx.upload(xyz, rgba)
    m = S.look_at_perspective((0.1, 0.3, 1.9), (0.5, 0.5, 0.5), (0, 1, 0), 40, 1.5, 0.1, 10)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, 96, 64, pcr.PC_VIEW_FORCE_K(k))])
    ovis, _ = O.render(enc, oracle_view(m, 96, 64, force_k=k))
    assert_same(vis, img, ovis, enc.color, f"k={k}")


# ---- config 2 style: terrain, adaptive precision, culling ---------------------------------

@pytest.fixture(scope="module")
def terrain_small(ctx):
    p = S.terrain_params(10000.0)
    xyz, rgba = S.terrain(2_000_000, p, seed=2)
    enc = O.encode(xyz, rgba, 10240)
    cloud = ctx.upload(xyz, rgba)
    return p, enc, cloud


@pytest.mark.parametrize("frame", [0, 17, 40, 77, 101])
def test_terrain_flythrough_adaptive_culled(ctx, terrain_small, frame):
    p, enc, cloud = terrain_small
    W, H = 320, 180
    m = S.flythrough(p, frame, 120, W, H, seed=2)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL)])
    gst = ctx.stats()
    ovis_off, _ = O.render(enc, oracle_view(m, W, H, cull=False))
    assert_same(vis, img, ovis_off, enc.color, f"frame {frame}")
    _, ost = O.render(enc, oracle_view(m, W, H, cull=True))
    assert gst["batches_rendered"] == ost["batches_rendered"]
    assert gst["batches_k"] == ost["batches_k"]
    assert gst["points_k"] == ost["points_k"]


def test_adaptive_uses_all_precisions(ctx, terrain_small):
    """Some view of the fly-through exercises k = 1, 2 and 3."""
    p, enc, cloud = terrain_small
    seen = set()
    for frame in range(0, 120, 7):
        m = S.flythrough(p, frame, 120, 640, 360, seed=2)
        gpu_render(ctx, cloud, [pcr.make_view(m, 640, 360, pcr.PC_VIEW_CULL)])
        st = ctx.stats()
        seen |= {k for k in (1, 2, 3) if st["batches_k"][k]}
    assert {1, 2} <= seen


def test_culling_and_early_depth_invariance(ctx, terrain_small):
    p, enc, cloud = terrain_small
    W, H = 256, 144
    for i in range(4):
        m = S.random_view(p, i, W, H, seed=2)
        outs = gpu_render(ctx, cloud, [
            pcr.make_view(m, W, H, 0),
            pcr.make_view(m, W, H, pcr.PC_VIEW_CULL),
            pcr.make_view(m, W, H, pcr.PC_VIEW_NO_EARLY_DEPTH),
            pcr.make_view(m, W, H, pcr.PC_VIEW_CULL | pcr.PC_VIEW_NO_EARLY_DEPTH)])
        for vis, img in outs[1:]:
            assert np.array_equal(vis, outs[0][0])
            assert np.array_equal(img, outs[0][1])


@pytest.mark.parametrize("tpb,bps", [(32, 1), (64, 3), (128, 2), (256, 1), (256, 0)])
def test_launch_shape_invariance(cuda_lib, terrain_small, tpb, bps):
    p, enc, _ = terrain_small
    c = pcr.Context(0, threads_per_block=tpb, blocks_per_sm=bps)
    try:
        cloud = c.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
        m = S.random_view(p, 5, 200, 120, seed=2)
        [(vis, img)] = gpu_render(c, cloud, [pcr.make_view(m, 200, 120, pcr.PC_VIEW_CULL)])
        ovis, _ = O.render(enc, oracle_view(m, 200, 120))
        assert_same(vis, img, ovis, enc.color, f"shape {tpb}x{bps}")
    finally:
        c.close()


# ---- multi-view (Sec. 3.7) ----------------------------------------------------------

@pytest.mark.parametrize("nv", [2, 5, 32, 33])
def test_multiview_equals_single(ctx, terrain_small, nv):
    p, enc, cloud = terrain_small
    sizes = [(160, 90), (97, 61), (128, 128), (33, 200)]
    views = []
    for i in range(nv):
        W, H = sizes[i % len(sizes)]
        flags = pcr.PC_VIEW_CULL if i % 3 else pcr.PC_VIEW_CULL | pcr.PC_VIEW_FORCE_K(1 + i % 3)
        views.append(pcr.make_view(S.random_view(p, 100 + i, W, H, seed=2), W, H, flags))
    multi = gpu_render(ctx, cloud, views)
    for i in (0, 1, nv - 1):
        [(vis, img)] = gpu_render(ctx, cloud, [views[i]])
        assert np.array_equal(multi[i][0], vis)
        assert np.array_equal(multi[i][1], img)
        v = views[i]
        fk = (v.flags >> 4) & 3
        ovis, _ = O.render(enc, oracle_view(np.array(v.view_proj), v.width, v.height, force_k=fk))
        assert_same(multi[i][0], multi[i][1], ovis, enc.color, f"view {i}/{nv}")


@pytest.mark.parametrize("ks", [(2, 2), (1, 2), (3, 1), (0, 3)])
def test_two_views_mixed_precision(ctx, terrain_small, ks):
    """Two-view launches (the stereo kernel): both views certified at one k
    share a decode, at different k each takes its own, and a view at k = 3
    or an uncertified one takes the general path; every image equals its
    single-view image and the oracle's."""
    p, enc, cloud = terrain_small
    views = []
    for i, k in enumerate(ks):
        flags = pcr.PC_VIEW_CULL | (pcr.PC_VIEW_FORCE_K(k) if k else 0)
        views.append(pcr.make_view(S.random_view(p, 300 + i, 150, 110, seed=4), 150, 110, flags))
    pair = gpu_render(ctx, cloud, views)
    for i, v in enumerate(views):
        [(vis, img)] = gpu_render(ctx, cloud, [v])
        assert np.array_equal(pair[i][0], vis)
        assert np.array_equal(pair[i][1], img)
        ovis, _ = O.render(enc, oracle_view(np.array(v.view_proj), v.width, v.height, force_k=ks[i]))
        assert_same(pair[i][0], pair[i][1], ovis, enc.color, f"view {i} of {ks}")


def test_stereo_pair_one_launch(ctx, terrain_small):
    p, enc, cloud = terrain_small
    W, H = 126, 140
    views = [pcr.make_view(S.stereo(p, W, H, e, 20.0), W, H, pcr.PC_VIEW_CULL) for e in (0, 1)]
    out = gpu_render(ctx, cloud, views)
    for e in (0, 1):
        ovis, _ = O.render(enc, oracle_view(np.array(views[e].view_proj), W, H))
        assert_same(out[e][0], out[e][1], ovis, enc.color, f"eye {e}")


# ---- edge cases ------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 3, 4, 5, 4095, 10241])
def test_tiny_and_ragged_clouds(ctx, n):
    xyz, rgba = S.unit_cube(n, seed=n + 7)
    enc = O.encode(xyz, rgba, 10240)
    cloud = ctx.upload(xyz, rgba)
    m = S.cube_camera(31, 17)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, 31, 17, pcr.PC_VIEW_CULL)])
    ovis, _ = O.render(enc, oracle_view(m, 31, 17))
    assert_same(vis, img, ovis, enc.color, f"n={n}")


def test_empty_cloud(ctx):
    cloud = ctx.upload(np.zeros((0, 3), np.float32), np.zeros(0, np.uint32))
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(S.cube_camera(8, 8), 8, 8)])
    assert (vis == O.EMPTY).all() and (img == 0).all()


def test_unaligned_variable_batches(ctx):
    """Batches with arbitrary first/count (not multiples of 4, with gaps)."""
    xyz, rgba = S.unit_cube(50000, seed=3)
    enc = O.encode(xyz, rgba, 10240)
    rng = np.random.default_rng(4)
    cuts = np.sort(rng.choice(np.arange(1, 50000), 37, replace=False))
    edges = np.concatenate([[0], cuts, [50000]])
    b = np.zeros(len(edges) - 1, O.BATCH_DTYPE)
    for i in range(len(b)):
        f, e = edges[i], edges[i + 1]
        if i % 5 == 4:
            e = f + (e - f) // 2      # leave a gap of points no batch draws
        pts = xyz[enc.perm[f:e]]
        b[i]["min"] = pts.min(0)
        b[i]["size"] = pts.max(0) - pts.min(0)
        b[i]["first"], b[i]["count"] = f, e - f
    # re-quantize against the new boxes with the oracle's Eq. 1 and Listing 2
    w = np.zeros((50000, 3), np.uint32)
    for i in range(len(b)):
        f, c = int(b[i]["first"]), int(b[i]["count"])
        for j in range(f, f + c):
            q = [O.quantize30(xyz[enc.perm[j], a], b[i]["min"][a], b[i]["size"][a]) for a in range(3)]
            w[j] = O.split_words(*q)
    enc2 = O.Encoded(b, w[:, 0].copy(), w[:, 1].copy(), w[:, 2].copy(), enc.color, enc.perm)
    cloud = ctx.upload_encoded(b, enc2.w1, enc2.w2, enc2.w3, enc2.color)
    m = S.cube_camera(80, 80)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, 80, 80, pcr.PC_VIEW_CULL)])
    ovis, _ = O.render(enc2, oracle_view(m, 80, 80))
    assert_same(vis, img, ovis, enc2.color, "variable batches")


def test_degenerate_views(ctx, terrain_small):
    p, enc, cloud = terrain_small
    # 1x1 view, a camera looking away from the terrain, a camera inside the cloud
    m1 = S.random_view(p, 9, 1, 1, seed=2)
    away = S.look_at_perspective((0, 0, 3000.0), (0, 0, 9000.0), (0, 1, 0), 60, 1.0, 1, 1e5)
    inside = S.look_at_perspective((0, 0, S.terrain_height(p, 0, 0, seed=2) + 1.0),
                                   (100, 0, S.terrain_height(p, 100, 0, seed=2)), (0, 0, 1),
                                   90, 1.0, 0.1, 1e5)
    for m, W, H in [(m1, 1, 1), (away, 64, 64), (inside, 120, 90)]:
        [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL)])
        ovis, _ = O.render(enc, oracle_view(m, W, H))
        assert_same(vis, img, ovis, enc.color, "degenerate")


def test_render_host_equals_device(ctx, terrain_small):
    p, enc, cloud = terrain_small
    views = [pcr.make_view(S.flythrough(p, f, 120, 192, 108, seed=2), 192, 108, pcr.PC_VIEW_CULL)
             for f in (3, 60)]
    dev = gpu_render(ctx, cloud, views)
    host = [np.zeros(192 * 108, np.uint32) for _ in views]
    pcr.pc_render_host(ctx.h, cloud, views, host)
    for (vis, img), h in zip(dev, host):
        assert np.array_equal(img, h)


def test_invalid_arguments(ctx):
    with pytest.raises(pcr.PCError):
        pcr.pc_render(ctx.h, 987654, [pcr.make_view(np.eye(4), 4, 4)], [(0, 0)])
    cloud = ctx.upload(*S.unit_cube(100))
    with pytest.raises(pcr.PCError):
        pcr.pc_render(ctx.h, cloud, [pcr.make_view(np.eye(4), 0, 4)], [(0, 0)])
    bad = np.zeros(1, pcr.BATCH_DTYPE)
    bad[0]["first"], bad[0]["count"] = 10, 100
    with pytest.raises(pcr.PCError):
        pcr.pc_upload_encoded(ctx.h, bad, *[np.zeros(50, np.uint32)] * 4)


def _manual_cloud(pos, bmin, bsize, color=None):
    """One batch encoded against a caller-given box (oracle Eq. 1 + Listing 2)."""
    n = len(pos)
    b = np.zeros(1, O.BATCH_DTYPE)
    b[0]["min"], b[0]["size"], b[0]["first"], b[0]["count"] = bmin, bsize, 0, n
    w = np.array([O.split_words(*(O.quantize30(p[a], bmin[a], bsize[a]) for a in range(3)))
                  for p in pos], np.uint32).reshape(n, 3)
    col = np.arange(n, dtype=np.uint32) + 1 if color is None else color
    return O.Encoded(b, w[:, 0].copy(), w[:, 1].copy(), w[:, 2].copy(), col,
                     np.arange(n, dtype=np.uint32))


def test_points_on_pixel_edges(ctx):
    """Orthographic camera (w = 1) and positions whose pixel coordinate is an
    exact integer or one ulp away from it: the certified fast pixel path must
    hand these to the IEEE-divide path and agree with the oracle."""
    W, H = 64, 32
    rng = np.random.default_rng(12)
    m = np.zeros(16, np.float32)
    m[0] = m[5] = m[10] = m[15] = 1.0
    i = rng.integers(0, W + 1, 3000)
    jx = (2.0 * i / W - 1.0).astype(np.float32)
    jy = (2.0 * rng.integers(0, H + 1, 3000) / H - 1.0).astype(np.float32)
    nudge = rng.integers(-1, 2, 3000)
    jx = np.nextafter(jx, np.where(nudge > 0, 2, -2).astype(np.float32)) * (nudge != 0) + jx * (nudge == 0)
    pos = np.stack([jx.astype(np.float32), jy, rng.uniform(-0.9, 0.9, 3000).astype(np.float32)], 1)
    enc = _manual_cloud(pos, (-1.0, -1.0, -1.0), (2.0, 2.0, 2.0))
    cloud = ctx.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
    for k in (1, 2, 3):
        [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, W, H, pcr.PC_VIEW_FORCE_K(k))])
        ovis, _ = O.render(enc, oracle_view(m, W, H, force_k=k))
        assert_same(vis, img, ovis, enc.color, f"edges k={k}")


@pytest.mark.parametrize("scale_exp", [-110, -60, 0, 60, 110])
def test_matrix_power_of_two_scale(ctx, terrain_small, scale_exp):
    """Scaling the whole matrix by 2^s scales every clip coordinate exactly, so
    pixels and images stay the same; |w| outside [2^-100, 2^100] forces the
    IEEE-divide path for every point."""
    p, enc, cloud = terrain_small
    W, H = 200, 110
    m = S.random_view(p, 21, W, H, seed=2).astype(np.float64)
    ms = (m * 2.0**scale_exp).astype(np.float32)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(ms, W, H, pcr.PC_VIEW_CULL)])
    ovis, _ = O.render(enc, oracle_view(ms, W, H))
    assert_same(vis, img, ovis, enc.color, f"scale 2^{scale_exp}")
    [(vis0, img0)] = gpu_render(ctx, cloud, [pcr.make_view(m.astype(np.float32), W, H,
                                                           pcr.PC_VIEW_CULL)])
    assert np.array_equal(img, img0)


def test_large_view(ctx, terrain_small):
    """16384 x 64 view: the certification margin scales with the width."""
    p, enc, cloud = terrain_small
    W, H = 16384, 64
    m = S.random_view(p, 31, W, H, seed=2)
    [(vis, img)] = gpu_render(ctx, cloud, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL)])
    ovis, _ = O.render(enc, oracle_view(m, W, H))
    assert_same(vis, img, ovis, enc.color, "wide view")


def test_scan_order_cloud_keep_order(cuda_lib):
    """Sec. 4.2 baseline: batches of consecutive scan-order points, no Morton
    sort; adaptive precision and culling still match the oracle bit for bit."""
    import torch
    p = S.terrain_params(6000.0)
    xyz, rgba = S.terrain_scan(400_000, p, (0.0, 0.0), 2000.0, 8000, seed=4)
    enc = O.encode_in_order(xyz, rgba, 10240)
    c = pcr.Context(0, flags=pcr.PC_CFG_KEEP_ORDER)
    try:
        cloud = c.upload(xyz, rgba)
        h = S.terrain_height(p, 0.0, 0.0)
        views = [S.look_at_perspective((0, -2500, 1800), (0, 0, 0), (0, 0, 1), 60, 16 / 9, 1, 1e5),
                 S.look_at_perspective((0, 0, h + 2.0), (300, 80, h), (0, 0, 1), 70, 16 / 9, 0.5, 1e5)]
        for m in views:
            [(vis, img)] = gpu_render(c, cloud, [pcr.make_view(m, 256, 144, pcr.PC_VIEW_CULL)])
            ovis, _ = O.render(enc, oracle_view(m, 256, 144))
            assert_same(vis, img, ovis, enc.color, "scan order")
    finally:
        c.close()
