"""High-quality shading (Sec. 3.6) on the GPU against the oracle: the colour
pass sums the colours of the points within 1% behind the closest one and the
resolve averages them. Integer sums do not depend on the order of the atomic
additions, so every image must be bit-identical to the oracle's."""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu

HQS_MODES = [pcr.PC_VIEW_HQS, pcr.PC_VIEW_HQS_PACKED, pcr.PC_VIEW_HQS | pcr.PC_VIEW_HQS_PACKED]


@pytest.fixture(scope="module")
def world(cuda_lib):
    ctx = pcr.Context(0)
    p = S.terrain_params(4000.0, 0.2, 120)
    xyz, rgba = S.terrain(300_000, p, seed=21)
    enc = O.encode(xyz, rgba, 10240)
    cloud = ctx.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
    yield ctx, p, enc, cloud
    ctx.close()


def _oracle_view(v, cull=True):
    return O.make_view(np.array(v.view_proj, np.float32), v.width, v.height, cull=cull)


def _check_view(enc, v, vis, img):
    ov = _oracle_view(v, cull=bool(v.flags & pcr.PC_VIEW_CULL))
    ovis, _ = O.render(enc, ov)
    assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
    ref = O.render_hqs(enc, ov, ovis)
    if v.flags & pcr.PC_VIEW_DILATE:
        ref = O.hqs_resolve_dilated(ovis, v.width, v.height, ref)
    got = pcr.rgba_to_numpy(img)
    assert np.array_equal(got, ref), f"{int((got != ref).sum())} pixels differ"
    return ovis, ref


@pytest.mark.parametrize("mode", HQS_MODES)
@pytest.mark.parametrize("frame", [0, 40, 90])
def test_terrain_frames_match_oracle(world, frame, mode):
    import torch
    ctx, p, enc, cloud = world
    W, H = 320, 180
    v = pcr.make_view(S.flythrough(p, frame, 120, W, H, seed=21), W, H, pcr.PC_VIEW_CULL | mode)
    [(vis, img)] = ctx.render(cloud, [v])
    torch.cuda.synchronize()
    ovis, ref = _check_view(enc, v, vis, img)
    st = ctx.stats()
    _, ost = O.render(enc, _oracle_view(v))
    nonempty = int((ovis != O.EMPTY).sum())
    # the closest point of a pixel always counts; points that count landed in the view
    assert nonempty <= st["points_blended"] <= ost["points_accepted"]
    assert nonempty > 1000


def test_blending_changes_the_image(world):
    """Dense overview: many pixels hold several points within the window, so the
    averaged image differs from the closest point's colour there."""
    import torch
    ctx, p, enc, cloud = world
    W, H = 200, 120
    v = pcr.make_view(S.overview(p, W, H), W, H, pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS)
    [(vis, img)] = ctx.render(cloud, [v])
    torch.cuda.synchronize()
    ovis, ref = _check_view(enc, v, vis, img)
    plain = O.resolve(ovis, enc.color)
    assert int((ref != plain).sum()) > 0.2 * int((ovis != O.EMPTY).sum())
    assert ctx.stats()["points_blended"] > 2 * int((ovis != O.EMPTY).sum())


@pytest.mark.parametrize("batch", [1000, 1003])
def test_unit_cube_ragged_batches(cuda_lib, batch):
    """Batches of 1000 points (a ragged tail) and of 1003 points (batches that
    start at any offset, not at a multiple of the 4- or 8-point groups), every
    precision forced in turn."""
    import torch
    n = 3 * 10240 + 77
    xyz, rgba = S.unit_cube(n, seed=9)
    enc = O.encode(xyz, rgba, batch)
    with pcr.Context(0) as ctx:
        cloud = ctx.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
        for k in (1, 2, 3):
            for mode in (pcr.PC_VIEW_HQS, pcr.PC_VIEW_HQS_PACKED):
                v = pcr.make_view(S.cube_camera(97, 61), 97, 61, pcr.PC_VIEW_FORCE_K(k) | mode)
                [(vis, img)] = ctx.render(cloud, [v])
                torch.cuda.synchronize()
                ov = O.make_view(S.cube_camera(97, 61), 97, 61, force_k=k)
                ovis, _ = O.render(enc, ov)
                assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
                assert np.array_equal(pcr.rgba_to_numpy(img), O.render_hqs(enc, ov, ovis))


def test_mixed_views_in_one_launch(world):
    """Plain, shaded, packed and dilated views share one multi-view launch; each
    must equal its own oracle image."""
    import torch
    ctx, p, enc, cloud = world
    flags = [pcr.PC_VIEW_CULL, pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS,
             pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS_PACKED,
             pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS | pcr.PC_VIEW_DILATE,
             pcr.PC_VIEW_CULL | pcr.PC_VIEW_DILATE, pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS]
    views = [pcr.make_view(S.random_view(p, 30 + i, 150 + 10 * i, 90, seed=21), 150 + 10 * i, 90,
                           f) for i, f in enumerate(flags)]
    out = ctx.render(cloud, views)
    torch.cuda.synchronize()
    for v, (vis, img) in zip(views, out):
        if v.flags & (pcr.PC_VIEW_HQS | pcr.PC_VIEW_HQS_PACKED):
            _check_view(enc, v, vis, img)
        else:
            ovis, _ = O.render(enc, _oracle_view(v))
            ref = (O.resolve_dilated(ovis, v.width, v.height, enc.color)
                   if v.flags & pcr.PC_VIEW_DILATE else O.resolve(ovis, enc.color))
            assert np.array_equal(pcr.rgba_to_numpy(img), ref)


def test_graph_replay_and_host_images(world):
    """A context that captures frames in CUDA graphs renders the shaded view the
    same on first capture and replay; pc_render_host returns the same image."""
    import torch
    _, p, enc, _ = world
    W, H = 256, 144
    v = pcr.make_view(S.flythrough(p, 10, 120, W, H, seed=21), W, H,
                      pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS)
    ov = _oracle_view(v)
    ovis, _ = O.render(enc, ov)
    ref = O.render_hqs(enc, ov, ovis)
    with pcr.Context(0, flags=pcr.PC_CFG_GRAPHS) as ctx:
        cloud = ctx.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
        s = torch.cuda.Stream()
        for _ in range(3):
            [(vis, img)] = ctx.render(cloud, [v], stream=s)
            s.synchronize()
            assert np.array_equal(pcr.rgba_to_numpy(img), ref)
        host = np.zeros(W * H, np.uint32)
        pcr.pc_render_host(ctx.h, cloud, [v], [host])
        assert np.array_equal(host, ref)


def _stack_cloud(n, colour):
    """n points at one position (w = 5) that all land on pixel (2, 2) of a 4x4
    view; a batch of size 0 decodes every point to its minimum corner."""
    nb = (n + 9999) // 10000
    b = np.zeros(nb, pcr.BATCH_DTYPE)
    for i in range(nb):
        b[i]["min"] = (0.0, 0.0, -5.0)
        b[i]["first"] = 10000 * i
        b[i]["count"] = min(10000, n - 10000 * i)
    z = np.zeros(n, np.uint32)
    col = np.full(n, colour, np.uint32)
    m = np.zeros(16, np.float32)
    m[0] = m[5] = 1.0
    m[11] = -1.0
    return b, z, col, m


def test_two_word_sum_limit(cuda_lib):
    """At the largest count the 32-bit sums hold, a pixel averages exactly; one
    point more raises the device error flag (PC_EDEVICE at the next
    synchronizing call), and the context keeps working."""
    import torch
    limit = 16_843_009
    with pcr.Context(0) as ctx:
        for n, ok in ((limit, True), (limit + 1, False), (3, True)):
            b, z, col, m = _stack_cloud(n, 0x00FFFFFF)
            cloud = ctx.upload_encoded(b, z, z, z, col)
            v = pcr.make_view(m, 4, 4, pcr.PC_VIEW_FORCE_K(1) | pcr.PC_VIEW_HQS)
            [(vis, img)] = ctx.render(cloud, [v])
            torch.cuda.synchronize()
            if ok:
                st = ctx.stats()
                assert st["points_blended"] == n
                out = pcr.rgba_to_numpy(img)
                assert out[2 * 4 + 2] == 0xFFFFFFFF
                assert (np.delete(out, 2 * 4 + 2) == 0).all()
            else:
                with pytest.raises(pcr.PCError) as e:
                    ctx.stats()
                assert e.value.status == pcr.PC_EDEVICE
            pcr.pc_release_cloud(ctx.h, cloud)


def test_packed_fallback_is_exact(cuda_lib):
    """The packed sums hold 1023 points; a pixel with more is summed again by
    the second pass, so every count gives the exact average. Above 256 points
    of the cloud per pixel of the view (here 4 x 4 pixels, so above 4,096
    points) the library takes two-word sums instead: no second pass, the same
    average."""
    import torch
    rng = np.random.default_rng(4)
    with pcr.Context(0) as ctx:
        for n in (1, 1023, 1024, 1027, 5000, 300_000):
            b, z, _, m = _stack_cloud(n, 0)
            col = rng.integers(0, 1 << 24, n, dtype=np.uint32)
            cloud = ctx.upload_encoded(b, z, z, z, col)
            v = pcr.make_view(m, 4, 4, pcr.PC_VIEW_FORCE_K(1) | pcr.PC_VIEW_HQS_PACKED)
            [(vis, img)] = ctx.render(cloud, [v])
            torch.cuda.synchronize()
            st = ctx.stats()
            assert st["points_blended"] == n
            assert st["hqs_fallback_pixels"] == (1 if 1023 < n <= 256 * 16 else 0)
            c = col.astype(np.uint64)
            expect = (int((c & 255).sum()) // n | (int((c >> 8 & 255).sum()) // n) << 8 |
                      (int((c >> 16 & 255).sum()) // n) << 16 | 0xFF000000)
            assert pcr.rgba_to_numpy(img)[2 * 4 + 2] == expect
            pcr.pc_release_cloud(ctx.h, cloud)


def test_lod_foveated_dilated(cuda_lib):
    """LOD cloud with foveated thresholds, packed sums and dilation: the case
    the single-atomic variant is meant for."""
    import torch
    with pcr.Context(0) as ctx:
        p = S.terrain_params(5000.0, 0.2, 150)
        xyz, rgba = S.terrain(400_000, p, seed=31)
        enc = O.encode(xyz, rgba, 10240)
        cloud = ctx.upload_encoded(enc.batches, enc.w1, enc.w2, enc.w3, enc.color)
        lod = pcr.pc_build_lod(ctx.h, cloud, 12, 2048, 5)
        ref = O.lod_build(O.decode_cloud(enc, 3), enc.color, 12, 2048, 5)
        W, H = 320, 200
        for frame, (lp, lpp) in ((20, (60.0, 240.0)), (70, (0.0, 0.0)), (100, (150.0, 0.0))):
            m = S.flythrough(p, frame, 120, W, H, seed=31)
            for flags in (pcr.PC_VIEW_HQS_PACKED | pcr.PC_VIEW_DILATE, pcr.PC_VIEW_HQS):
                v = pcr.make_view(m, W, H, pcr.PC_VIEW_CULL | flags, lp, lpp)
                [(vis, img)] = ctx.render(lod, [v])
                torch.cuda.synchronize()
                ov = O.make_view(m, W, H)
                ovis, _ = O.lod_render(ref, ov, lp, lpp)
                assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
                img_ref = O.lod_render_hqs(ref, ov, ovis, lp, lpp)
                if flags & pcr.PC_VIEW_DILATE:
                    img_ref = O.hqs_resolve_dilated(ovis, W, H, img_ref)
                assert np.array_equal(pcr.rgba_to_numpy(img), img_ref)


def test_empty_view_and_noalloc_refusal(world):
    import torch
    ctx, p, enc, cloud = world
    # looking away from the terrain: nothing lands, the image stays 0
    m = S.look_at_perspective((0, 0, 100), (0, 0, 1000), (0, 1, 0), 60.0, 1.0, 0.1, 100.0)
    v = pcr.make_view(m, 64, 64, pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS)
    [(vis, img)] = ctx.render(cloud, [v])
    torch.cuda.synchronize()
    assert (pcr.rgba_to_numpy(img) == 0).all()
    assert ctx.stats()["points_blended"] == 0
    # the allocation-free entry point has no room for the sums
    L = pcr.lib()
    dev = torch.device("cuda", 0)
    b = torch.zeros(32, dtype=torch.uint8, device=dev)
    w = torch.zeros(64, dtype=torch.int32, device=dev)
    vis2 = torch.empty(64 * 64, dtype=torch.int64, device=dev)
    img2 = torch.empty(64 * 64, dtype=torch.int32, device=dev)
    assert L.pc_render_noalloc(b.data_ptr(), 1, *(w.data_ptr(),) * 4, 4, ctypes.byref(v),
                               vis2.data_ptr(), img2.data_ptr(), 512.0, None,
                               torch.cuda.current_stream().cuda_stream) == pcr.PC_ENOTSUP
