"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: hand-computed
values (tests/golden/, each file citing the paper), closed forms, brute force
on tiny inputs, exactness special cases and invariants. test_oracle_mutants.py
plants plausible mistakes in a copy of the oracle and checks that this file
catches every one of them.
"""
import os

import numpy as np
import pytest

import oracle as O
import pcsynth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


# ---- Eq. 1 -------------------------------------------------------------------

def test_eq1_golden():
    for line in _rows("eq1_quantize.txt"):
        x, mn, sz, want = line.split()
        assert O.quantize30(float(x), float(mn), float(sz)) == int(want), line


def test_eq1_monotone_and_range():
    rng = np.random.default_rng(1)
    mn, sz = np.float32(-3.25), np.float32(7.5)
    xs = np.sort(rng.uniform(mn, mn + sz, 2000).astype(np.float32))
    q = [O.quantize30(x, mn, sz) for x in xs]
    assert all(a <= b for a, b in zip(q, q[1:]))
    assert min(q) >= 0 and max(q) <= 2**30 - 1
    # exact definition in rational arithmetic agrees away from rounding ties
    for x, qq in zip(xs[::50], q[::50]):
        exact = (2**30 * (float(x) - float(mn))) / float(sz)
        assert abs(qq - min(int(np.floor(exact)), 2**30 - 1)) <= 1


# ---- Listing 2 ---------------------------------------------------------------

def test_listing2_golden():
    for line in _rows("listing2_words.txt"):
        X, Y, Z, w1, w2, w3 = map(int, line.split())
        assert O.split_words(X, Y, Z) == [w1, w2, w3], line
        assert O.decode_words(w1, w2, w3, 3) == [X, Y, Z]
        assert O.decode_words(w1, w2, w3, 2) == [X >> 10, Y >> 10, Z >> 10]
        assert O.decode_words(w1, w2, w3, 1) == [X >> 20, Y >> 20, Z >> 20]


def test_words_roundtrip_random():
    rng = np.random.default_rng(2)
    for X, Y, Z in rng.integers(0, 2**30, size=(500, 3)):
        w = O.split_words(X, Y, Z)
        assert all(x < 2**30 for x in w)      # two padding bits stay zero
        for k in (1, 2, 3):
            assert O.decode_words(*w, k) == [int(X) >> (30 - 10 * k),
                                             int(Y) >> (30 - 10 * k),
                                             int(Z) >> (30 - 10 * k)]


# ---- Sec. 3.1 Morton order ---------------------------------------------------

def test_morton_golden():
    for line in _rows("morton.txt"):
        px, py, pz, want = line.split()
        p = [float(v) * 2.0**-21 for v in (px, py, pz)]
        assert O.morton_code(p, (0, 0, 0), (1, 1, 1)) == int(want), line


def _interleave(qx, qy, qz):
    code = 0
    for b in range(21):
        code |= ((qx >> b) & 1) << (3 * b) | ((qy >> b) & 1) << (3 * b + 1) | \
                ((qz >> b) & 1) << (3 * b + 2)
    return code


def test_morton_order_is_z_order():
    """The code of q = floor(2^21 p) is the bit interleave of the three
    21-bit integers (checked against an independent interleave)."""
    rng = np.random.default_rng(3)
    q = rng.integers(0, 2**21, size=(300, 3))
    codes = [O.morton_code([(v + 0.5) * 2.0**-21 for v in qq], (0, 0, 0), (1, 1, 1))
             for qq in q]
    assert codes == [_interleave(*map(int, qq)) for qq in q]


def test_encode_hand_cloud():
    """8 points of a 2x2x2 grid in scrambled order, plus duplicates: Morton
    order is x fastest, then y, then z; duplicates keep input order; batches of
    3 consecutive points get their own boxes."""
    grid = [(x, y, z) for z in (0.0, 1.0) for y in (0.0, 1.0) for x in (0.0, 1.0)]
    order_in = [5, 2, 7, 0, 3, 6, 1, 4]
    pts = [grid[i] for i in order_in] + [grid[3], grid[0]]
    xyz = np.array(pts, np.float32)
    rgba = np.arange(len(pts), dtype=np.uint32) + 100
    enc = O.encode(xyz, rgba, batch_size=3)
    # sorted by Morton code: grid index 0,0(dup),1,2,3,3(dup),4,5,6,7
    want_grid = [0, 0, 1, 2, 3, 3, 4, 5, 6, 7]
    got_grid = [grid.index(tuple(xyz[i])) for i in enc.perm]
    assert got_grid == want_grid
    # stable: the duplicate of grid 0 (input index 9) comes after input index 3
    assert list(enc.perm[:2]) == [3, 9]
    assert list(enc.perm[4:6]) == [4, 8]
    assert list(enc.color) == list(rgba[enc.perm])
    assert len(enc.batches) == 4
    assert [int(b["count"]) for b in enc.batches] == [3, 3, 3, 1]
    assert [int(b["first"]) for b in enc.batches] == [0, 3, 6, 9]
    # batch 1 holds grid points 2, 3, 3: x in {0,1}, y = 1, z = 0
    b1 = enc.batches[1]
    assert list(b1["min"]) == [0, 1, 0] and list(b1["size"]) == [1, 0, 0]
    # words: grid point 3 = (1,1,0) in batch 1: X30 clamps to 2^30-1, Y, Z sizes 0
    assert enc.w1[4] == 1023 and enc.w2[4] == 1023 and enc.w3[4] == 1023


# ---- Listing 1 projection -----------------------------------------------------

def test_listing1_golden():
    for line in _rows("listing1_project.txt"):
        name, ents, wh, p, want = [s.strip() for s in line.split("|")]
        m = np.zeros(16, np.float32)
        for e in ents.split():
            i, v = e.split(":")
            m[int(i)] = float(v)
        W, H = map(int, wh.split())
        pt = [float(v) for v in p.split()]
        acc, pix, khi = want.split()
        view = O.make_view(m, W, H)
        ok, gpix, key, _, _ = O.project_position(pt, view, idx=77)
        assert ok == bool(int(acc)), name
        if ok:
            assert gpix == int(pix), name
            assert key >> 32 == int(khi, 16), name
            assert key & 0xFFFFFFFF == 77, name


def test_projection_matches_rational_arithmetic():
    """Away from rounding boundaries the pixel is floor of the exact ratio."""
    from fractions import Fraction as F
    rng = np.random.default_rng(4)
    m = S.cube_camera(97, 61)
    view = O.make_view(m, 97, 61)
    checked = 0
    for p in rng.uniform(-0.2, 1.2, size=(400, 3)).astype(np.float32):
        ok, pix, key, fx, fy = O.project_position(p, view)
        M = [F(float(v)) for v in m]
        x, y, z = (F(float(v)) for v in p)
        cx = M[0] * x + M[4] * y + M[8] * z + M[12]
        cy = M[1] * x + M[5] * y + M[9] * z + M[13]
        cw = M[3] * x + M[7] * y + M[11] * z + M[15]
        if cw <= 0:
            assert not ok
            continue
        ex = (cx / cw + 1) / 2 * 97
        ey = (cy / cw + 1) / 2 * 61
        if min(abs(ex - round(ex)), abs(ey - round(ey))) < F(1, 1000):
            continue  # too close to a pixel edge for a rounding-free claim
        inside = 0 <= ex < 97 and 0 <= ey < 61
        assert ok == inside
        assert abs(float(ex) - fx) < 1e-3 and abs(float(ey) - fy) < 1e-3
        if ok:
            import math
            assert pix == math.floor(ey) * 97 + math.floor(ex)
            assert abs(float(cw) - float(np.uint32(key >> 32).view(np.float32))) <= 1e-5 * float(cw)
            checked += 1
    assert checked > 100


def test_depth_then_index_tiebreak():
    m = np.zeros(16, np.float32)
    m[0] = m[5] = 1.0
    m[11] = -1.0                       # w = -z: a GL camera looking down -z
    v = O.make_view(m, 4, 4)
    # batch box [0,1]^2 x [-4,-1]: points at the centre pixel with depths 3, 2, 2
    batch = np.zeros(1, O.BATCH_DTYPE)
    batch[0]["min"] = (0.0, 0.0, -4.0)
    batch[0]["size"] = (1.0, 1.0, 3.0)
    batch[0]["first"], batch[0]["count"] = 0, 3
    zs = [-3.0, -2.0, -2.0]
    words = [O.split_words(0, 0, O.quantize30(z, -4.0, 3.0)) for z in zs]
    enc = O.Encoded(batch, np.array([w[0] for w in words], np.uint32),
                    np.array([w[1] for w in words], np.uint32),
                    np.array([w[2] for w in words], np.uint32),
                    np.array([10, 11, 12], np.uint32), np.arange(3, dtype=np.uint32))
    vis, _ = O.render(enc, O.make_view(m, 4, 4, force_k=3))
    hit = vis[vis != O.EMPTY]
    assert len(hit) == 1
    assert int(hit[0]) & 0xFFFFFFFF == 1          # depth 2 beats 3; index 1 beats 2
    assert O.resolve(vis, enc.color)[vis != O.EMPTY][0] == 11


# ---- the geometry pass against brute force -------------------------------------

def _tiny_clouds():
    rng = np.random.default_rng(5)
    xyz, rgba = S.unit_cube(3000, seed=11)
    yield "cube", xyz, rgba, S.cube_camera(16, 12), 16, 12
    # adversarial: duplicates (equal depth), exact pixel edges, behind camera
    m = S.look_at_perspective((0.5, 0.5, 1.5), (0.5, 0.5, 0.5), (0, 1, 0), 90.0, 1.0, 0.1, 10)
    pts = rng.uniform(-0.5, 1.5, size=(1500, 3)).astype(np.float32)
    pts[:200] = pts[200:400]                              # exact duplicates
    pts[400:500, 2] = 2.0                                 # behind the eye plane
    grid = (np.arange(16) / 16.0).astype(np.float32)      # pixel-edge x values
    pts[500:600, 0] = rng.choice(grid, 100)
    col = rng.integers(0, 2**32, len(pts), dtype=np.uint64).astype(np.uint32)
    yield "adversarial", pts, col, m, 16, 16


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_render_equals_brute_force(k):
    for name, xyz, rgba, m, W, H in _tiny_clouds():
        enc = O.encode(xyz, rgba, batch_size=256)
        v = O.make_view(m, W, H, cull=False, force_k=k)
        vis, st = O.render(enc, v)
        bf = O.brute_force(enc, v)
        assert np.array_equal(vis, bf), name
        assert st["points_processed"] == len(xyz)
        assert (vis != O.EMPTY).sum() > 10, name


# ---- Sec. 3.3 decode: exact special cases ---------------------------------------

def _manual_batch(positions, bmin, bsize):
    """Encode positions against a caller-given box (Eq. 1 + Listing 2)."""
    n = len(positions)
    b = np.zeros(1, O.BATCH_DTYPE)
    b[0]["min"], b[0]["size"], b[0]["first"], b[0]["count"] = bmin, bsize, 0, n
    w = np.array([O.split_words(*(O.quantize30(p[a], bmin[a], bsize[a]) for a in range(3)))
                  for p in positions], np.uint32).reshape(n, 3)
    return O.Encoded(b, w[:, 0].copy(), w[:, 1].copy(), w[:, 2].copy(),
                     np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32))


def _grid_camera():
    return S.look_at_perspective((300.0, 700.0, 2500.0), (512.0, 512.0, 512.0),
                                 (0, 1, 0), 50.0, 1.0, 10.0, 10000.0)


@pytest.mark.parametrize("k,res_bits", [(1, 0), (2, 10), (3, 20)])
def test_dyadic_grid_exact(k, res_bits):
    """Positions on the 2^-res grid of a box [0,1024)^3 decode exactly at
    precision k, so the quantized image equals the unquantized one; one
    precision lower the positions decode to the truncated grid."""
    rng = np.random.default_rng(6 + k)
    n = 4000
    bmin, bsize = (0.0, 0.0, 0.0), (1024.0, 1024.0, 1024.0)
    if k == 3:   # keep 24 significant bits so float(X30) is exact
        X = (rng.integers(0, 2**24, size=(n, 3)) << 6).astype(np.float64)
    else:
        X = (rng.integers(0, 2**(10 + res_bits), size=(n, 3)) << (20 - res_bits)).astype(np.float64)
    pos = (X * 2.0**-20).astype(np.float32)          # X30 * cell_3, exact
    enc = _manual_batch(pos, bmin, bsize)
    m = _grid_camera()
    raw = O.render_positions(pos, O.make_view(m, 96, 96))
    vis, _ = O.render(enc, O.make_view(m, 96, 96, force_k=k))
    assert np.array_equal(vis, raw)
    for j in range(0, n, 97):
        p = O.decode_position(enc.batches[0], k, enc.w1[j], enc.w2[j], enc.w3[j])
        assert np.array_equal(p, pos[j])
        if k > 1:
            lower = O.decode_position(enc.batches[0], k - 1, enc.w1[j], enc.w2[j], enc.w3[j])
            trunc = np.floor(pos[j].astype(np.float64) * 2.0**(10 * (k - 1) - 10)) \
                * 2.0**(10 - 10 * (k - 1))
            assert np.array_equal(lower.astype(np.float64), trunc)


def test_decode_offset_box():
    """Integer positions in a box with a nonzero, non-dyadic minimum decode
    exactly at k = 1 (min + X * size/1024 with size = 1024)."""
    rng = np.random.default_rng(9)
    bmin = (-512.0, 3.0, 100.0)
    q = rng.integers(0, 1024, size=(2000, 3))
    pos = (q + np.array(bmin)).astype(np.float32)
    enc = _manual_batch(pos, bmin, (1024.0, 1024.0, 1024.0))
    for j in range(0, 2000, 37):
        for k in (1, 2, 3):
            p = O.decode_position(enc.batches[0], k, enc.w1[j], enc.w2[j], enc.w3[j])
            assert np.array_equal(p, pos[j]), (j, k)


def test_quantization_error_bound():
    """|decoded - raw| per axis is below one cell of the chosen precision plus
    binary32 rounding of the decode (Sec. 3.3)."""
    xyz, rgba = S.terrain(20000, S.terrain_params(2000.0), seed=3)
    enc = O.encode(xyz, rgba, batch_size=1024)
    raw = xyz[enc.perm]
    for b in enc.batches[::3]:
        f, c = int(b["first"]), int(b["count"])
        size = b["size"].astype(np.float64)
        mag = np.maximum(np.abs(b["min"]), np.abs(b["min"] + b["size"])).astype(np.float64)
        for k in (1, 2, 3):
            cell = size * 2.0**(-10 * k)
            for j in range(f, f + c, 41):
                p = O.decode_position(b, k, enc.w1[j], enc.w2[j], enc.w3[j]).astype(np.float64)
                err = raw[j].astype(np.float64) - p
                tol = 2.0**-22 * mag
                assert np.all(err >= -tol - 2.0**-22 * size), (k, j)
                assert np.all(err < cell + tol + 2.0**-22 * size), (k, j)


def test_k3_image_close_to_unquantized():
    """At k = 3 almost every pixel keeps the same winner as the unquantized
    image (differences need a point within the quantization bound of a pixel
    edge or a depth tie)."""
    xyz, rgba = S.unit_cube(60000, seed=4)
    enc = O.encode(xyz, rgba, batch_size=2048)
    m = S.cube_camera(128, 128)
    vis, _ = O.render(enc, O.make_view(m, 128, 128, force_k=3))
    raw = O.render_positions(xyz[enc.perm], O.make_view(m, 128, 128))
    covered = raw != O.EMPTY
    assert np.array_equal(covered, vis != O.EMPTY) or \
        (covered != (vis != O.EMPTY)).sum() < 0.001 * covered.sum()
    same = (vis == raw).sum()
    assert same > 0.99 * covered.sum()


# ---- Sec. 3.3 precision choice ---------------------------------------------------

def _ortho(scale=1.0):
    m = np.zeros(16, np.float32)
    m[0] = m[5] = scale
    m[10] = m[15] = 1.0
    return m


@pytest.mark.parametrize("s,T,want", [(0.99, 512.0, 1), (1.01, 512.0, 2),
                                      (0.99, 500.0, 2), (0.97, 500.0, 1),
                                      (1023.0, 512.0, 2), (1025.0, 512.0, 3),
                                      (1.0, 512.0, 2), (1024.0, 512.0, 3)])
def test_select_k_thresholds(s, T, want):
    """Orthographic camera (c = x, w = 1) on a 1024 px wide view: a box of
    width s in x projects to an extent of s * 0.5 * 1024 px (hand-computed:
    506.88, 517.12, 496.64, 523776, 524800, and exactly 512 and 524288, where
    the strict comparison of Sec. 3.3's threshold picks the larger k)."""
    b = np.zeros(1, O.BATCH_DTYPE)[0]
    b["min"] = (-s / 2, 0.0, 0.0)
    b["size"] = (s, 0.001, 0.001)
    v = O.make_view(_ortho(), 1024, 16, threshold_px=T)
    assert O.select_k(b, v) == want


def test_select_k_behind_camera_is_3():
    m = np.zeros(16, np.float32)
    m[0] = m[5] = 1.0
    m[11] = -1.0
    b = np.zeros(1, O.BATCH_DTYPE)[0]
    b["min"] = (-0.01, -0.01, -1.0)
    b["size"] = (0.02, 0.02, 2.0)     # straddles the eye plane z = 0
    assert O.select_k(b, O.make_view(m, 64, 64)) == 3
    b["size"] = (0.02, 0.02, 0.5)
    assert O.select_k(b, O.make_view(m, 64, 64)) == 1


# ---- Sec. 3.2 culling ---------------------------------------------------------------

def _terrain_encoded(n=60000, extent=4000.0, bs=1024, seed=7):
    xyz, rgba = S.terrain(n, S.terrain_params(extent), seed=seed)
    return O.encode(xyz, rgba, batch_size=bs)


def test_culling_is_conservative_per_batch():
    """A culled batch has no point that any precision would draw."""
    enc = _terrain_encoded()
    p = S.terrain_params(4000.0)
    culled = 0
    for vi in range(6):
        v = O.make_view(S.random_view(p, vi, 64, 48, seed=7), 64, 48, cull=True)
        for b in enc.batches:
            if not O.cull(b, v):
                continue
            culled += 1
            f, c = int(b["first"]), int(b["count"])
            for k in (1, 2, 3):
                for j in range(f, f + c, 7):
                    p3 = O.decode_position(b, k, enc.w1[j], enc.w2[j], enc.w3[j])
                    assert not O.project_position(p3, v)[0]
    assert culled > 20


def test_culling_on_equals_off():
    enc = _terrain_encoded()
    p = S.terrain_params(4000.0)
    total_culled = 0
    for vi in range(8):
        m = S.random_view(p, vi, 80, 60, seed=7)
        on, st_on = O.render(enc, O.make_view(m, 80, 60, cull=True))
        off, st_off = O.render(enc, O.make_view(m, 80, 60, cull=False))
        assert np.array_equal(on, off)
        total_culled += st_off["batches_rendered"] - st_on["batches_rendered"]
    assert total_culled > 0


def test_culling_plane_cases():
    """Hand-placed boxes: fully left/right/below/above/behind are culled,
    boxes touching the frustum are kept."""
    m = np.zeros(16, np.float32)
    m[0] = m[5] = 1.0
    m[11] = -1.0            # w = -z, ndc = (x, y) / -z
    v = O.make_view(m, 64, 64, cull=True)

    def box(mn, sz):
        b = np.zeros(1, O.BATCH_DTYPE)[0]
        b["min"], b["size"] = mn, sz
        return b
    assert O.cull(box((2.0, -0.5, -1.5), (1.0, 1.0, 1.0)), v)       # right of x = w
    assert O.cull(box((-3.0, -0.5, -1.5), (1.0, 1.0, 1.0)), v)      # left
    assert O.cull(box((-0.5, 2.0, -1.5), (1.0, 1.0, 1.0)), v)       # above
    assert O.cull(box((-0.5, -3.0, -1.5), (1.0, 1.0, 1.0)), v)      # below
    assert O.cull(box((-0.5, -0.5, 1.0), (1.0, 1.0, 1.0)), v)       # behind
    assert not O.cull(box((-0.5, -0.5, -1.5), (1.0, 1.0, 1.0)), v)  # inside
    assert not O.cull(box((0.9, -0.5, -1.0), (1.0, 1.0, 0.5)), v)   # straddles x = w
    assert not O.cull(box((-0.5, -0.5, -0.5), (1.0, 1.0, 1.0)), v)  # straddles the eye plane


# ---- order independence ------------------------------------------------------------

def test_order_and_thread_independence():
    enc = _terrain_encoded(n=40000, bs=512)
    p = S.terrain_params(4000.0)
    m = S.random_view(p, 3, 64, 64, seed=7)
    v = O.make_view(m, 64, 64, cull=True)
    ref, _ = O.render(enc, v)
    rng = np.random.default_rng(8)
    perm = rng.permutation(len(enc.batches)).astype(np.uint64)
    shuf, _ = O.render(enc, v, order=perm)
    assert np.array_equal(ref, shuf)
    for t in (1, 3, 8):
        thr, _ = O.render_threaded(enc, v, threads=t)
        assert np.array_equal(ref, thr)


# ---- resolve -------------------------------------------------------------------

def test_resolve():
    color = np.array([7, 8, 9, 10], np.uint32)
    vis = np.array([O.EMPTY, (5 << 32) | 2, (1 << 32) | 0, O.EMPTY, (3 << 32) | 3], np.uint64)
    assert list(O.resolve(vis, color)) == [0, 9, 7, 0, 10]


# ---- per-frame counters (Table 2) on a hand-built cloud ------------------------------

def _hand_stats_cloud():
    """Four batches under the orthographic camera (c = x, w = 1) of a 64x64
    view, where f = 32 x + 32 and a point is inside iff -1 <= x, y < 1:
      A  x in [-0.5, 0], 16 px wide: k = 1, 4 points, all inside;
      B  x in [-20, 20], 1280 px: k = 2, x = -20, -10, 0, 10, 20: one inside;
      C  x in [5, 6], right of the view: culled, 3 points;
      D  x in [-20000, 20000], 1,280,000 px: k = 3, x = -20000 + 10000 j: one inside.
    Every coordinate is a dyadic grid point of its box, so it decodes exactly
    at its batch's k."""
    boxes = [((-0.5, -0.5, 0.0), (0.5, 0.5, 0.0), [(-0.5 + 0.125 * i, -0.5, 0.0) for i in range(4)]),
             ((-20.0, -0.25, 0.0), (40.0, 0.5, 0.0), [(-20.0 + 10.0 * j, -0.25, 0.0) for j in range(5)]),
             ((5.0, 0.0, 0.0), (1.0, 0.0, 0.0), [(5.0, 0.0, 0.0), (5.5, 0.0, 0.0), (6.0, 0.0, 0.0)]),
             ((-20000.0, 0.0, 0.0), (40000.0, 0.0, 0.0),
              [(-20000.0 + 10000.0 * j, 0.0, 0.0) for j in range(5)])]
    batches = np.zeros(len(boxes), O.BATCH_DTYPE)
    words, first = [], 0
    for i, (mn, sz, pts) in enumerate(boxes):
        batches[i]["min"], batches[i]["size"] = mn, sz
        batches[i]["first"], batches[i]["count"] = first, len(pts)
        first += len(pts)
        for p in pts:
            words.append(O.split_words(*[O.quantize30(p[a], mn[a], sz[a]) for a in range(3)]))
    w = np.array(words, np.uint32)
    n = len(w)
    return O.Encoded(batches, w[:, 0].copy(), w[:, 1].copy(), w[:, 2].copy(),
                     np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32))


def test_frame_counters_hand_built():
    enc = _hand_stats_cloud()
    m = _ortho()
    on = O.make_view(m, 64, 64, cull=True)
    off = O.make_view(m, 64, 64, cull=False)
    assert [O.select_k(b, on) for b in enc.batches] == [1, 2, 1, 3]
    want_on = {"batches_rendered": 3, "points_processed": 14, "batches_k": [0, 1, 1, 1],
               "points_k": [0, 4, 5, 5], "points_accepted": 6}
    want_off = {"batches_rendered": 4, "points_processed": 17, "batches_k": [0, 2, 1, 1],
                "points_k": [0, 7, 5, 5], "points_accepted": 6}
    for v, want in ((on, want_on), (off, want_off)):
        vis, st = O.render(enc, v)
        assert {k: st[k] for k in want} == want
        assert int((vis != O.EMPTY).sum()) == 6
        for t in (1, 2, 3, 4):          # the threaded merge adds every counter
            tvis, tst = O.render_threaded(enc, v, threads=t)
            assert np.array_equal(tvis, vis) and {k: tst[k] for k in want} == want


# ---- Sec. 3.2 culling under binary32 rounding -----------------------------------------

def test_culling_covers_binary32_rounding():
    """One point whose exact clip x is 0.75 % left of -w, but whose binary32
    row value fl(fl(m0 x) + m12) rounds to exactly -1 = -w, so it lands on
    pixel column 0 (found by a search, checked here with exact rationals).
    Culling must keep its batch: the rounding bound of the test, not the
    plane margin 1 + 2^-10, is what covers it."""
    from fractions import Fraction
    m0, x, m12 = 1.5094573497772217, 88018.546875, -132861.25
    assert np.float32(m0) == m0 and np.float32(x) == x and np.float32(m12) == m12
    exact = Fraction(m0) * Fraction(x) + Fraction(m12)
    assert exact < -(1 + Fraction(1, 1024))
    m = np.zeros(16, np.float32)
    m[0], m[12], m[5], m[15] = m0, m12, 1.0, 1.0
    v = O.make_view(m, 64, 64, cull=True)
    ok, pix, _, fx, _ = O.project_position((x, 0.0, 0.0), v)
    assert ok and fx == 0.0 and pix == 32 * 64
    b = np.zeros(1, O.BATCH_DTYPE)[0]
    b["min"], b["size"], b["count"] = (x, 0.0, 0.0), (0.0, 0.0, 0.0), 1
    assert not O.cull(b, v)


# ---- Sec. 4.2 batches in input order ----------------------------------------------------

def test_encode_in_order_hand_cloud():
    """Batches of 3 consecutive input points in input order; each box is the
    per-axis min and max of its own points (none of them the first point's),
    and the words are Eq. 1 against that box."""
    pts = [(4, 1, 2), (0, 3, 1), (2, 0, 0),       # box min (0,0,0), size (4,3,2)
           (1, 5, 7), (-1, 6, 5), (0, 5, 6),      # box min (-1,5,5), size (2,1,2)
           (9, 9, 9)]                             # a box of size 0
    xyz = np.array(pts, np.float32)
    rgba = np.arange(7, dtype=np.uint32) + 50
    enc = O.encode_in_order(xyz, rgba, batch_size=3)
    assert [list(b["min"]) for b in enc.batches] == [[0, 0, 0], [-1, 5, 5], [9, 9, 9]]
    assert [list(b["size"]) for b in enc.batches] == [[4, 3, 2], [2, 1, 2], [0, 0, 0]]
    assert [int(b["first"]) for b in enc.batches] == [0, 3, 6]
    assert [int(b["count"]) for b in enc.batches] == [3, 3, 1]
    assert list(enc.color) == list(rgba)
    # (0, 3, 1) in the first box: X = 0, Y clamps to 2^30 - 1, Z = 2^29
    assert O.split_words(0, (1 << 30) - 1, 1 << 29) == [int(enc.w1[1]), int(enc.w2[1]), int(enc.w3[1])]
    # (-1, 6, 5) in the second box: X = 0, Y = 2^30 - 1, Z = 0
    assert O.split_words(0, (1 << 30) - 1, 0) == [int(enc.w1[4]), int(enc.w2[4]), int(enc.w3[4])]
    assert [int(enc.w1[6]), int(enc.w2[6]), int(enc.w3[6])] == [0, 0, 0]
