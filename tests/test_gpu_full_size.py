"""The bench's workload at full size.

The cloud is 2,000,000,000 terrain+building points over 40 km. It is encoded by
the library's host encoder and rendered in the bench's launch configuration
(autotuned raster shape): the 1920x1080 overview frame, and the stereo pair of
2016x2240 per eye in one launch.

The oracle cannot sort 2B points in a test's time, but it checks the library's
encoding against Sec. 3.1, Eq. 1 and Listing 2 in O(n). That encoding is unique,
so an encoding that passes is the oracle's. The oracle then renders the same
frames itself on all host cores, and every pixel of every view must match;
so must the overview's high-quality shading and the overview served through
pc_submit. About 75 GB of host memory and a few minutes.
"""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu

N = 2_000_000_000
BATCH = 10240


def test_full_size_frames_bit_exact(cuda_lib):
    import torch
    params = S.terrain_params(40000.0, 0.2, 20000)
    xyz = np.empty((N, 3), np.float32)
    rgba = np.empty(N, np.uint32)
    S.terrain(N, params, seed=3, out=(xyz, rgba))
    batches, w1, w2, w3, color, perm = pcr.pc_encode(xyz, rgba, BATCH)
    code, where = O.verify_encoding(xyz, rgba, BATCH, batches, w1, w2, w3, color, perm)
    assert code == 0, f"encoding differs from the definition (code {code} at {where})"
    del xyz, rgba, perm
    enc = O.Encoded(batches, w1, w2, w3, color, None)

    W, H = 1920, 1080
    overview = S.overview(params, W, H)
    eyes = [S.stereo(params, 2016, 2240, e, 6.5) for e in (0, 1)]
    with pcr.Context(0) as ctx:
        cloud = ctx.upload_encoded(batches, w1, w2, w3, color)
        v0 = pcr.make_view(overview, W, H, pcr.PC_VIEW_CULL)
        pcr.pc_autotune(ctx.h, cloud, [v0])
        [(vis0, img0)] = ctx.render(cloud, [v0])
        pcr.pc_set_views_per_launch(ctx.h, 2)
        stereo = [pcr.make_view(m, 2016, 2240, pcr.PC_VIEW_CULL) for m in eyes]
        pair = ctx.render(cloud, stereo)
        torch.cuda.synchronize()
        stats = [ctx.stats(v) for v in range(2)]   # the stereo pair's counters
        got = [(overview, W, H, vis0, img0)] + [(m, 2016, 2240, v, i) for m, (v, i) in zip(eyes, pair)]
        for n, (m, w, h, vis, img) in enumerate(got):
            ovis, ost = O.render_threaded(enc, O.make_view(m, w, h, cull=True))
            assert (ovis != O.EMPTY).sum() > 0.2 * w * h
            assert np.array_equal(pcr.vis_to_numpy(vis), ovis)
            assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve(ovis, enc.color))
            if n > 0:
                st = stats[n - 1]
                assert st["batches_rendered"] == ost["batches_rendered"]
                assert st["points_processed"] == ost["points_processed"]
                assert st["batches_k"] == ost["batches_k"]
            if n == 0:
                overview_vis = ovis
        # high-quality shading (Sec. 3.6) of the overview frame
        pcr.pc_set_views_per_launch(ctx.h, 1)
        vh = pcr.make_view(overview, W, H, pcr.PC_VIEW_CULL | pcr.PC_VIEW_HQS)
        [(_, hq)] = ctx.render(cloud, [vh])
        torch.cuda.synchronize()
        ref = O.render_hqs_threaded(enc, O.make_view(overview, W, H, cull=True), overview_vis)
        assert np.array_equal(pcr.rgba_to_numpy(hq), ref)
        # the serving path: the overview through pc_submit, into library-owned
        # and caller-owned framebuffers, equals the checked frame
        t1 = pcr.pc_submit(ctx.h, cloud, [v0])
        own = ctx.framebuffers([v0])
        t2 = pcr.pc_submit(ctx.h, cloud, [v0], [(own[0][0].data_ptr(), own[0][1].data_ptr())])
        for t in (t1, t2):
            rc, res = pcr.pc_poll(ctx.h, t, 60_000)
            assert rc == pcr.PC_OK and res["status"] == pcr.PC_OK
        expect = O.resolve(overview_vis, enc.color)
        assert np.array_equal(pcr.pc_poll(ctx.h, t1, 0)[1]["images"][0], expect)
        assert np.array_equal(pcr.rgba_to_numpy(own[0][1]), expect)
        for t in (t1, t2):
            pcr.pc_release_ticket(ctx.h, t)


def test_config2_flythrough_100m(cuda_lib):
    """100,000,000 terrain points over 10 km, four frames of the seeded
    120-frame fly-through at 1920x1080 with adaptive precision and culling;
    the encoding is checked by the oracle, every frame and its counters match
    the oracle's."""
    import torch
    n = 100_000_000
    params = S.terrain_params(10000.0)
    xyz, rgba = S.terrain(n, params, seed=2)
    batches, w1, w2, w3, color, perm = pcr.pc_encode(xyz, rgba, BATCH)
    code, where = O.verify_encoding(xyz, rgba, BATCH, batches, w1, w2, w3, color, perm)
    assert code == 0, f"encoding differs from the definition (code {code} at {where})"
    del xyz, rgba, perm
    enc = O.Encoded(batches, w1, w2, w3, color, None)
    W, H = 1920, 1080
    with pcr.Context(0) as ctx:
        cloud = ctx.upload_encoded(batches, w1, w2, w3, color)
        for f in (0, 30, 60, 90):
            m = S.flythrough(params, f, 120, W, H, seed=2)
            [(vis, img)] = ctx.render(cloud, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL)])
            torch.cuda.synchronize()
            st = ctx.stats()
            ovis, ost = O.render_threaded(enc, O.make_view(m, W, H, cull=True))
            assert np.array_equal(pcr.vis_to_numpy(vis), ovis), f"frame {f}"
            assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve(ovis, enc.color)), f"frame {f}"
            assert st["batches_rendered"] == ost["batches_rendered"]
            assert st["points_processed"] == ost["points_processed"]
            assert st["batches_k"] == ost["batches_k"]
            assert ost["batches_rendered"] < len(batches)   # the fly-through culls


def test_config4_lod_1b(cuda_lib):
    """Config 4 at full size: 1,000,000,000 points of the 10 km terrain as a
    layered octree (12 levels, <= 10,240 points per node), built on the device
    by pc_build_lod. The oracle checks the source encoding and the tree against
    their definitions. The device tree must equal the host builder's, and LOD
    frames of the fly-through at 1080p, with thresholds of 300 and 100 px, must
    match the oracle's LOD renders with their counters."""
    import torch
    n = 1_000_000_000
    params = S.terrain_params(10000.0)
    xyz = np.empty((n, 3), np.float32)
    rgba = np.empty(n, np.uint32)
    S.terrain(n, params, seed=10, out=(xyz, rgba))
    batches, w1, w2, w3, color, perm = pcr.pc_encode(xyz, rgba, BATCH)
    code, where = O.verify_encoding(xyz, rgba, BATCH, batches, w1, w2, w3, color, perm)
    assert code == 0, f"encoding differs from the definition (code {code} at {where})"
    del xyz, rgba, perm
    enc = O.Encoded(batches, w1, w2, w3, color, None)
    # the LOD builder's input: the source decoded at k = 3 (Sec. 3.3)
    dec = O.decode_cloud(enc, 3)
    tree = pcr.pc_lod_encode(dec, color, 12, 10240, 0, max_nodes=n // 1000 + 65536)
    nodes, parent, level, lperm, l1, l2, l3, lc = tree
    code, where = O.verify_lod(dec, color, 12, 10240, 0, nodes, parent, level, lperm, l1, l2, l3, lc)
    assert code == 0, f"LOD tree differs from the definition (code {code} at {where})"
    del dec
    ref = O.LodCloud(nodes, parent, level, l1, l2, l3, lc, lperm)
    W, H = 1920, 1080
    with pcr.Context(0) as ctx:
        src = ctx.upload_encoded(batches, w1, w2, w3, color)
        lod = pcr.pc_build_lod(ctx.h, src, 12, 10240, 0)
        pcr.pc_release_cloud(ctx.h, src)
        d_nodes, d1, d2, d3, dc = pcr.pc_cloud_download(ctx.h, lod)
        assert d_nodes.tobytes() == nodes.tobytes()
        for a, b in ((d1, l1), (d2, l2), (d3, l3), (dc, lc)):
            assert np.array_equal(a, b)
        del d1, d2, d3, dc
        for f in (0, 45, 90):
            m = S.flythrough(params, f, 120, W, H, seed=3)
            for lod_px in (300.0, 100.0):
                [(vis, img)] = ctx.render(lod, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL, lod_px)])
                torch.cuda.synchronize()
                st = ctx.stats()
                ovis, ost = O.lod_render(ref, O.make_view(m, W, H), lod_px)
                assert np.array_equal(pcr.vis_to_numpy(vis), ovis), f"frame {f}, {lod_px} px"
                assert np.array_equal(pcr.rgba_to_numpy(img), O.resolve(ovis, lc))
                assert st["batches_rendered"] == ost["batches_rendered"]
                assert st["points_processed"] == ost["points_processed"]
                assert st["batches_k"] == ost["batches_k"]
                assert (ovis != O.EMPTY).sum() > 0.1 * W * H
