"""Pins of the oracle's level-of-detail structure and node selection (Sec. 3.5)
against properties that define them: an additive layered octree holds every
point exactly once, nodes are cubic octants of their parent, a parent keeps the
max_node_points points of smallest priority among its subtree, points are
quantized with Eq. 1 against their node's cube, and selection draws a node
only when it is in the frustum, big enough on screen and its parent is drawn.
"""
import numpy as np
import pytest

import oracle as O
import pcsynth as S

M, L, SEED = 1024, 12, 7


@pytest.fixture(scope="module")
def lod():
    p = S.terrain_params(3000.0, 0.15, 80)
    xyz, rgba = S.terrain(60000, p, seed=11)
    return p, xyz, rgba, O.lod_build(xyz, rgba, L, M, SEED)


def _children(lod):
    ch = {i: [] for i in range(len(lod.nodes))}
    for i in range(1, len(lod.nodes)):
        ch[int(lod.parent[i])].append(i)
    return ch


def test_every_point_exactly_once(lod):
    _, xyz, rgba, t = lod
    assert np.array_equal(np.sort(t.perm), np.arange(len(xyz), dtype=np.uint32))
    assert np.array_equal(t.color, rgba[t.perm])
    firsts = t.nodes["first"].astype(np.int64)
    counts = t.nodes["count"].astype(np.int64)
    assert firsts[0] == 0 and np.array_equal(firsts[1:], np.cumsum(counts)[:-1])
    assert counts.sum() == len(xyz)


def test_tree_shape(lod):
    _, xyz, _, t = lod
    ch = _children(t)
    assert t.level[0] == 0 and t.parent[0] == 0
    for i in range(1, len(t.nodes)):
        par = int(t.parent[i])
        assert par < i and t.level[i] == t.level[par] + 1          # breadth first
        assert t.level[i] >= t.level[i - 1]
        half = np.float32(t.nodes[par]["size"][0] * np.float32(0.5))
        assert np.all(t.nodes[i]["size"] == half)
        lo_p = t.nodes[par]["min"]
        mid = (lo_p + half).astype(np.float32)
        lo_c = t.nodes[i]["min"]
        assert all(lo_c[a] in (lo_p[a], mid[a]) for a in range(3))
    for i, cs in ch.items():
        octs = [int(sum((t.nodes[c]["min"][a] != t.nodes[i]["min"][a]) << a for a in range(3)))
                for c in cs]
        assert octs == sorted(octs) and len(set(octs)) == len(octs)
        if cs:
            assert t.nodes[i]["count"] == M                     # full parents
        else:
            assert t.nodes[i]["count"] <= M or t.level[i] == L - 1
    assert len(t.nodes) > 20 and t.level.max() >= 3


def test_points_in_their_octants(lod):
    _, xyz, _, t = lod
    for i in range(len(t.nodes)):
        f, c = int(t.nodes[i]["first"]), int(t.nodes[i]["count"])
        pts = xyz[t.perm[f:f + c]]
        lo = t.nodes[i]["min"]
        # every ancestor split puts the point on its node's side of the midpoint
        node = i
        while node != 0:
            par = int(t.parent[node])
            half = np.float32(t.nodes[par]["size"][0] * np.float32(0.5))
            mid = (t.nodes[par]["min"] + half).astype(np.float32)
            for a in range(3):
                upper = t.nodes[node]["min"][a] != t.nodes[par]["min"][a]
                assert np.all((pts[:, a] >= mid[a]) == upper)
            node = par
        assert np.all(pts >= lo)


def test_parent_keeps_lowest_priorities_of_subtree(lod):
    _, xyz, _, t = lod
    ch = _children(t)

    def subtree(i):
        f, c = int(t.nodes[i]["first"]), int(t.nodes[i]["count"])
        out = list(t.perm[f:f + c])
        for cc in ch[i]:
            out += subtree(cc)
        return out

    pri = lambda idx: (O.splitmix64((SEED << 32) + int(idx)), int(idx))
    for i in [0] + ch[0][:3]:
        if not ch[i]:
            continue
        allpts = subtree(i)
        want = sorted(sorted(allpts, key=pri)[:M])
        f, c = int(t.nodes[i]["first"]), int(t.nodes[i]["count"])
        assert list(t.perm[f:f + c]) == want          # kept in input order


def test_subset_is_spatially_uniform(lod):
    """The root's subset covers the area like the whole cloud (uniform draw)."""
    _, xyz, _, t = lod
    root = xyz[t.perm[:M]]
    h_all, _ = np.histogram(xyz[:, 0], bins=8, range=(xyz[:, 0].min(), xyz[:, 0].max()))
    h_root, _ = np.histogram(root[:, 0], bins=8, range=(xyz[:, 0].min(), xyz[:, 0].max()))
    assert np.abs(h_root / M - h_all / len(xyz)).max() < 0.03


def test_words_are_eq1_against_node_cube(lod):
    _, xyz, _, t = lod
    for i in range(0, len(t.nodes), 5):
        b = t.nodes[i]
        f, c = int(b["first"]), int(b["count"])
        for j in range(f, f + c, 97):
            p = xyz[t.perm[j]]
            q = [O.quantize30(p[a], b["min"][a], b["size"][a]) for a in range(3)]
            assert O.split_words(*q) == [int(t.w1[j]), int(t.w2[j]), int(t.w3[j])]


def test_selection_rules(lod):
    p, xyz, _, t = lod
    for vi in range(5):
        m = S.random_view(p, vi, 160, 120, seed=11)
        v = O.make_view(m, 160, 120)
        sel_all = O.lod_select(t, v, 0.0)
        sel_300 = O.lod_select(t, v, 300.0)
        sel_big = O.lod_select(t, v, 1e9)
        for i in range(len(t.nodes)):
            in_frustum = not O.cull(t.nodes[i], v)
            par_ok = i == 0 or sel_all[int(t.parent[i])]
            assert sel_all[i] == (in_frustum and par_ok)
            if sel_300[i]:
                assert sel_all[i]
                if i:
                    e = O.projected_extent(t.nodes[i], v)
                    assert e is None or not (e < 300.0)
                    assert sel_300[int(t.parent[i])]
        # with a huge threshold only the root and nodes reaching behind the
        # eye (a corner with w <= 0 counts as large) remain
        for i in np.nonzero(sel_big)[0][1:]:
            assert O.projected_extent(t.nodes[i], v) is None
        assert sel_300.sum() <= sel_all.sum()


def test_lod_render_all_nodes_equals_plain_render(lod):
    """With no size threshold, the LOD pass draws exactly the in-frustum nodes,
    which (culling being conservative) equals a plain render of all nodes."""
    p, xyz, _, t = lod
    m = S.random_view(p, 2, 120, 90, seed=11)
    v = O.make_view(m, 120, 90)
    lvis, lst = O.lod_render(t, v, 0.0)
    enc = O.Encoded(t.nodes, t.w1, t.w2, t.w3, t.color, t.perm)
    pvis, _ = O.render(enc, v)
    assert np.array_equal(lvis, pvis)
    svis, sst = O.lod_render(t, v, 200.0)
    assert sst["points_processed"] < lst["points_processed"]


# ---- Sec. 3.7 foveated thresholds and depth-aware dilation --------------------------

@pytest.mark.parametrize("x,y,want", [(45, 45, 0), (66, 45, 0), (67, 45, 1), (87, 45, 1),
                                      (88, 45, 2), (45, 24, 0), (0, 0, 2), (45, 3, 1)])
def test_ring_boundaries(x, y, want):
    """90x90 view: R2 = 45^2 + 45^2 = 4050; ring 0 iff 9 d2 < 4050 (d2 < 450,
    d <= 21), ring 1 iff 9 d2 < 16200 (d2 < 1800, d <= 42); hand-computed."""
    assert O.ring(x, y, 90, 90) == want


def test_dilation_window_grows_with_ring():
    W = H = 90
    color = np.array([0xAA, 0xBB], np.uint32)
    vis = np.full(W * H, O.EMPTY, np.uint64)
    vis[45 * W + 45] = (5 << 32) | 0          # centre point: 3x3
    vis[2 * W + 2] = (5 << 32) | 1            # corner point: 7x7 (ring 2 pixels)
    out = O.resolve_dilated(vis, W, H, color).reshape(H, W)
    assert (out[44:47, 44:47] == 0xAA).all() and out[43, 45] == 0 and out[45, 47] == 0
    assert (out[0:6, 0:6] == 0xBB).all() and out[6, 2] == 0
    assert (out == 0xAA).sum() == 9


def test_dilation_is_depth_aware():
    W, H = 90, 90
    color = np.array([1, 2], np.uint32)
    vis = np.full(W * H, O.EMPTY, np.uint64)
    vis[45 * W + 45] = (9 << 32) | 0          # farther
    vis[45 * W + 46] = (3 << 32) | 1          # nearer: wins wherever both are in reach
    out = O.resolve_dilated(vis, W, H, color).reshape(H, W)
    assert out[45, 45] == 2 and out[45, 44] == 1 and out[44, 46] == 2


def test_foveated_selection(lod):
    p, xyz, _, t = lod
    for vi in range(4):
        v = O.make_view(S.random_view(p, 10 + vi, 160, 120, seed=11), 160, 120)
        flat = O.lod_select(t, v, 100.0)
        fov = O.lod_select(t, v, 100.0, 300.0)
        same = O.lod_select(t, v, 100.0, 100.0)
        assert np.array_equal(flat, same)
        assert np.all(fov <= flat) and fov.sum() >= 1
        for i in np.nonzero(fov)[0][1:]:
            e = O.projected_extent(t.nodes[i], v)
            if e is not None:
                assert e >= 100.0


# ---- rules pinned on hand-made inputs ----------------------------------------------

def _boxes(boxes, parents):
    """A node list from (min, size) boxes, for selection only."""
    nodes = np.zeros(len(boxes), O.BATCH_DTYPE)
    for i, (lo, size) in enumerate(boxes):
        nodes[i]["min"], nodes[i]["size"] = lo, size
    return O.LodCloud(nodes, np.asarray(parents, np.uint32), np.zeros(len(boxes), np.uint32),
                      None, None, None, None, None)


# identity view of 100x100 pixels: w = 1 everywhere and pixel f = 50 x + 50, so a
# box of side s in x and y projects to 50 s pixels around 50 + 50 x_centre
IDENTITY = np.eye(4, dtype=np.float32)


def test_selection_root_and_parent_rules():
    """The root needs only the frustum (even when tiny); any other node also
    needs its parent drawn, even when it is in view and large itself."""
    v = O.make_view(IDENTITY, 100, 100)
    t = _boxes([((-0.01, -0.01, 0), (0.02, 0.02, 0)),     # 0: root, 1 px
                ((2.0, 2.0, 0), (1.0, 1.0, 0)),           # 1: outside the frustum
                ((-0.5, -0.5, 0), (1.0, 1.0, 0)),         # 2: 50 px, parent culled
                ((-0.5, -0.5, 0), (1.0, 1.0, 0))],        # 3: 50 px, parent the root
               [0, 0, 1, 0])
    assert O.cull(t.nodes[1], v) and not O.cull(t.nodes[2], v)
    assert list(O.lod_select(t, v, 10.0)) == [1, 0, 0, 1]


def test_foveated_threshold_by_ring():
    """lod_px = 10 in ring 0, (10 + 30) / 2 = 20 in ring 1, 30 in ring 2 (the
    ring of the projected box's centre; 100x100: R2 = 5000, ring 0 iff
    9 d2 < 5000, ring 1 iff 9 d2 < 20000). Centres: (85, 50) is d = 35, ring 1;
    (95, 95) is d2 = 4050, ring 2; (50, 50) is ring 0."""
    v = O.make_view(IDENTITY, 100, 100)
    t = _boxes([((-1, -1, 0), (2, 2, 0)),                 # root
                ((0.55, -0.15, 0), (0.3, 0.3, 0)),        # ring 1, 15 px: below 20
                ((0.45, -0.25, 0), (0.5, 0.5, 0)),        # ring 1, 25 px
                ((0.7, 0.7, 0), (0.4, 0.4, 0)),           # ring 2, 20 px: below 30
                ((0.55, 0.55, 0), (0.7, 0.7, 0)),         # ring 2, 35 px
                ((-0.12, -0.12, 0), (0.24, 0.24, 0)),     # ring 0, 12 px
                ((-0.08, -0.08, 0), (0.16, 0.16, 0))],    # ring 0, 8 px: below 10
               [0] * 7)
    assert [O.ring(85, 50, 100, 100), O.ring(95, 95, 100, 100)] == [1, 2]
    assert list(O.lod_select(t, v, 10.0, 30.0)) == [1, 0, 1, 0, 1, 1, 0]
    assert list(O.lod_select(t, v, 10.0)) == [1, 1, 1, 1, 1, 1, 0]


def test_root_is_the_cubic_box():
    """Corner = per-axis minimum, side = the largest extent (here y's)."""
    rng = np.random.default_rng(3)
    xyz = (rng.random((50, 3)) * [1.0, 3.0, 2.0] + [5.0, -1.0, 2.0]).astype(np.float32)
    xyz[0] = (5.0, -1.0, 2.0)
    xyz[1] = (6.0, 2.0, 4.0)
    t = O.lod_build(xyz, np.zeros(50, np.uint32), L, 1000, SEED)
    assert len(t.nodes) == 1
    assert list(t.nodes[0]["min"]) == [5.0, -1.0, 2.0]
    assert list(t.nodes[0]["size"]) == [3.0, 3.0, 3.0]


def test_split_only_above_max_node_points():
    rng = np.random.default_rng(4)
    xyz = rng.random((101, 3)).astype(np.float32)
    rgba = np.zeros(101, np.uint32)
    assert len(O.lod_build(xyz[:100], rgba[:100], L, 100, SEED).nodes) == 1   # exactly M: a leaf
    t = O.lod_build(xyz, rgba, L, 100, SEED)
    assert len(t.nodes) == 2 and list(t.nodes["count"]) == [100, 1]


def test_depth_limit_keeps_every_point_in_the_last_level():
    """max_levels = 2: the root splits, its children are at the last level and
    keep all their points however many."""
    rng = np.random.default_rng(5)
    xyz = rng.random((5000, 3)).astype(np.float32)
    t = O.lod_build(xyz, np.zeros(5000, np.uint32), 2, 100, SEED)
    assert int(t.level.max()) == 1 and len(t.nodes) == 9
    assert t.nodes["count"][0] == 100 and t.nodes["count"][1:].min() > 100
    assert t.nodes["count"].sum() == 5000


def test_dilation_window_is_set_by_the_pixel_centre_ring():
    """One point at q shows in pixel p exactly when q is within Chebyshev
    distance 1 + ring(p's centre) of p: a sweep of q across the ring
    boundaries of a 64x64 view."""
    W = H = 64
    color = np.array([0x5A], np.uint32)
    py, px = np.mgrid[0:H, 0:W]
    radius = np.array([[1 + O.ring(x + 0.5, y + 0.5, W, H) for x in range(W)] for y in range(H)])
    for qx, qy in [(x, 32) for x in range(0, 64, 3)] + [(x, x) for x in range(1, 64, 4)]:
        vis = np.full(W * H, O.EMPTY, np.uint64)
        vis[qy * W + qx] = (7 << 32) | 0
        out = O.resolve_dilated(vis, W, H, color).reshape(H, W)
        reach = np.maximum(abs(px - qx), abs(py - qy)) <= radius
        assert np.array_equal(out == 0x5A, reach), (qx, qy)
