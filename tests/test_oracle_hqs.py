"""Pins of the oracle's high-quality shading (Sec. 3.6): colours of the points
within 1% behind the closest one are averaged per pixel (hand-computed)."""
import numpy as np

import oracle as O


def _one_pixel_cloud(depths, colors, zmin=-100.0, zsize=100.0):
    """Points on the optical axis of an orthographic-like camera with w = depth:
    all land on the centre pixel of a 4x4 view."""
    m = np.zeros(16, np.float32)
    m[0] = m[5] = 1.0
    m[11] = -1.0                      # w = -z
    n = len(depths)
    b = np.zeros(1, O.BATCH_DTYPE)
    b[0]["min"], b[0]["size"], b[0]["first"], b[0]["count"] = (0.0, 0.0, zmin), (0.0, 0.0, zsize), 0, n
    w = [O.split_words(0, 0, O.quantize30(-d, zmin, zsize)) for d in depths]
    enc = O.Encoded(b, np.array([x[0] for x in w], np.uint32), np.array([x[1] for x in w], np.uint32),
                    np.array([x[2] for x in w], np.uint32), np.array(colors, np.uint32),
                    np.arange(n, dtype=np.uint32))
    return enc, O.make_view(m, 4, 4, force_k=3)


def test_average_within_one_percent():
    # depths 10, 10.05 (0.5 % behind) and 10.2 (2 % behind): the first two average
    # R: (10 + 21) // 2 = 15, G: (200 + 101) // 2 = 150, B: (7 + 8) // 2 = 7
    enc, v = _one_pixel_cloud([10.0, 10.05, 10.2],
                              [10 | 200 << 8 | 7 << 16, 21 | 101 << 8 | 8 << 16, 255 | 255 << 8])
    vis, _ = O.render(enc, v)
    out = O.render_hqs(enc, v, vis)
    hit = np.nonzero(vis != O.EMPTY)[0]
    assert len(hit) == 1
    assert out[hit[0]] == 15 | 150 << 8 | 7 << 16 | 255 << 24
    assert (out[vis == O.EMPTY] == 0).all()


def test_single_point_keeps_its_colour():
    enc, v = _one_pixel_cloud([5.0], [0x00332211])
    vis, _ = O.render(enc, v)
    out = O.render_hqs(enc, v, vis)
    assert out[vis != O.EMPTY][0] == 0xFF332211


def test_far_points_do_not_contribute():
    enc, v = _one_pixel_cloud([5.0, 5.2, 6.0], [3, 200, 100])
    vis, _ = O.render(enc, v)
    assert O.render_hqs(enc, v, vis)[vis != O.EMPTY][0] == 0xFF000003


def test_boundary_of_the_depth_window():
    # a z box of side 2^30 from -1024 decodes to whole numbers at k = 3, and
    # w = -z exactly; fl(100 * fl(1.01)) = 101, so the window of the pixel whose
    # closest point is at w = 100 is closed at 101: of colours 0 (w = 100),
    # 100 (w = 101) and 200 (w = 102) the first two count, (0 + 100) // 2 = 50
    assert np.float32(np.float32(100.0) * np.float32(1.01)) == np.float32(101.0)
    enc, v = _one_pixel_cloud([100.0, 101.0, 102.0], [0, 100, 200], zmin=-1024.0, zsize=2.0 ** 30)
    for i in range(3):
        p = O.decode_position(enc.batches[0], 3, enc.w1[i], enc.w2[i], enc.w3[i])
        assert p[2] == -(100.0 + i)
    vis, _ = O.render(enc, v)
    assert O.render_hqs(enc, v, vis)[vis != O.EMPTY][0] == 0xFF000000 | 50


def _scene(n=20000, seed=3):
    import pcsynth as S
    xyz, rgba = S.unit_cube(n, seed=seed)
    enc = O.encode(xyz, rgba, 1024)
    v = O.make_view(S.cube_camera(96, 64), 96, 64, cull=True)
    return enc, v


def test_winner_always_counted():
    # the closest point of a pixel is always inside its own window, so the
    # image is non-zero exactly where a point landed, with alpha 255
    enc, v = _scene()
    vis, _ = O.render(enc, v)
    out = O.render_hqs(enc, v, vis)
    assert ((out != 0) == (vis != O.EMPTY)).all()
    assert (out[vis != O.EMPTY] >> 24 == 255).all()


def test_uniform_colour_is_kept():
    enc, v = _scene()
    enc.color[:] = 0xFF4080C0
    vis, _ = O.render(enc, v)
    out = O.render_hqs(enc, v, vis)
    assert (out[vis != O.EMPTY] == 0xFF4080C0).all()


def test_sparse_cloud_equals_plain_resolve():
    # with at most one point per pixel the average is that point's colour
    enc, v = _scene(n=300, seed=5)
    enc.color[:] |= np.uint32(0xFF000000)
    vis, _ = O.render(enc, v)
    hit = vis[vis != O.EMPTY]
    idx = (hit & np.uint64(0xFFFFFFFF)).astype(np.int64)
    pixels_of = {}
    for i in range(enc.n):
        b = next(b for b in enc.batches if b["first"] <= i < b["first"] + b["count"])
        ok, pix, _ = _project(enc, b, i, v)
        if ok:
            pixels_of.setdefault(pix, []).append(i)
    single = [p for p, pts in pixels_of.items() if len(pts) == 1]
    assert len(single) > 100
    out = O.render_hqs(enc, v, vis)
    ref = O.resolve(vis, enc.color)
    assert (out[single] == ref[single]).all()
    assert len(idx) == len(pixels_of)


def _project(enc, b, i, v):
    k = O.select_k(b, v)
    p = O.decode_position(b, k, enc.w1[i], enc.w2[i], enc.w3[i])
    r = O.project_position(p, v, i)
    return r[0], r[1], r[2]


def test_dilated_takes_the_winning_pixels_average():
    # 5x5 image: ring 0 radius 1 at the centre pixel (2, 2); the smallest key
    # within its 3x3 window is at (1, 3), so it shows that pixel's average
    W = H = 5
    vis = np.full(W * H, O.EMPTY, np.uint64)
    hqs = np.zeros(W * H, np.uint32)
    vis[3 * W + 1] = np.uint64(5 << 32 | 7)
    hqs[3 * W + 1] = 0xFF010203
    vis[2 * W + 2] = np.uint64(9 << 32 | 1)
    hqs[2 * W + 2] = 0xFF0A0B0C
    out = O.hqs_resolve_dilated(vis, W, H, hqs)
    assert out[2 * W + 2] == 0xFF010203
    # a pixel that sees neither point stays empty
    assert O.ring(4.5, 0.5, W, H) >= 1
    r = 1 + O.ring(4.5, 0.5, W, H)
    assert out[0 * W + 4] == (0xFF010203 if r >= 3 else (0xFF0A0B0C if r >= 2 else 0))
    # the same two pixels with the keys swapped: now the winner comes first in
    # the window's row order, and the centre shows its own average
    vis[3 * W + 1], vis[2 * W + 2] = np.uint64(9 << 32 | 7), np.uint64(5 << 32 | 1)
    out = O.hqs_resolve_dilated(vis, W, H, hqs)
    assert out[2 * W + 2] == 0xFF0A0B0C and out[3 * W + 1] == 0xFF0A0B0C


def test_lod_hqs_matches_its_geometry_pass():
    import pcsynth as S
    p = S.terrain_params(3000.0, 0.15, 80)
    xyz, rgba = S.terrain(30000, p, seed=11)
    lod = O.lod_build(xyz, rgba, 8, 1000, 7)
    v = O.make_view(S.overview(p, 80, 60), 80, 60)
    for lod_px in (0.0, 30.0, 1e9):
        vis, _ = O.lod_render(lod, v, lod_px)
        out = O.lod_render_hqs(lod, v, vis, lod_px)
        assert ((out != 0) == (vis != O.EMPTY)).all()


def test_lod_hqs_of_the_root_alone():
    # with a threshold no child reaches only the root is drawn: the image is
    # the plain one of a cloud made of the root node's points
    import pcsynth as S
    p = S.terrain_params(3000.0, 0.15, 80)
    xyz, rgba = S.terrain(30000, p, seed=11)
    lod = O.lod_build(xyz, rgba, 8, 1000, 7)
    v = O.make_view(S.overview(p, 80, 60), 80, 60)
    assert O.lod_select(lod, v, 1e9).sum() == 1
    root = O.Encoded(lod.nodes[:1].copy(), lod.w1, lod.w2, lod.w3, lod.color, lod.perm)
    vis, _ = O.lod_render(lod, v, 1e9)
    vis_root, _ = O.render(root, v)
    assert (vis == vis_root).all()
    assert (O.lod_render_hqs(lod, v, vis, 1e9) == O.render_hqs(root, v, vis)).all()


def test_threaded_equals_single_thread():
    enc, v = _scene(n=40000, seed=9)
    vis, _ = O.render(enc, v)
    ref = O.render_hqs(enc, v, vis)
    for t in (1, 3, 8):
        assert (O.render_hqs_threaded(enc, v, vis, threads=t) == ref).all()
