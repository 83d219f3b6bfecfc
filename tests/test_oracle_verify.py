"""Pins of the oracle's encoding checker (Sec. 3.1, Eq. 1, Listing 2): it
accepts the oracle's own encoding and rejects each kind of planted mistake
with the matching code (1 header, 2 permutation, 3 order, 4 box, 5 words,
6 colour)."""
import numpy as np
import pytest

import oracle as O
import pcsynth as S

BS = 1000


@pytest.fixture(scope="module")
def cloud():
    xyz, rgba = S.unit_cube(20000, seed=8)
    # a block of duplicated positions, so that equal Morton codes occur
    xyz[100:140] = xyz[100]
    enc = O.encode(xyz, rgba, BS)
    return xyz, rgba, enc


def _check(xyz, rgba, enc, **over):
    a = dict(batches=enc.batches.copy(), w1=enc.w1.copy(), w2=enc.w2.copy(), w3=enc.w3.copy(),
             color=enc.color.copy(), perm=enc.perm.copy())
    a.update(over)
    return O.verify_encoding(xyz, rgba, BS, a["batches"], a["w1"], a["w2"], a["w3"], a["color"],
                             a["perm"], threads=3)


def test_accepts_the_oracle_encoding(cloud):
    xyz, rgba, enc = cloud
    assert _check(xyz, rgba, enc) == (0, 0)
    assert O.verify_encoding(xyz, rgba, BS, enc.batches, enc.w1, enc.w2, enc.w3, enc.color,
                             enc.perm, threads=1) == (0, 0)


def test_rejects_order_and_permutation_mistakes(cloud):
    xyz, rgba, enc = cloud
    p = enc.perm.copy()
    p[[10, 15000]] = p[[15000, 10]]
    assert _check(xyz, rgba, enc, perm=p)[0] == 3
    # equal codes must keep input order
    pos = np.nonzero(np.isin(enc.perm, np.arange(100, 140)))[0]
    p = enc.perm.copy()
    p[[pos[0], pos[1]]] = p[[pos[1], pos[0]]]
    assert _check(xyz, rgba, enc, perm=p) == (3, int(pos[1]))
    p = enc.perm.copy()
    p[5] = p[6]
    assert _check(xyz, rgba, enc, perm=p)[0] in (2, 3)
    p = enc.perm.copy()
    p[7] = 20000
    assert _check(xyz, rgba, enc, perm=p)[0] == 2


def test_rejects_header_box_word_and_colour_mistakes(cloud):
    xyz, rgba, enc = cloud
    b = enc.batches.copy()
    b[3]["count"] -= 1
    assert _check(xyz, rgba, enc, batches=b) == (1, 3)
    assert O.verify_encoding(xyz, rgba, BS, enc.batches[:-1], enc.w1, enc.w2, enc.w3, enc.color,
                             enc.perm)[0] == 1
    b = enc.batches.copy()
    b[4]["min"][1] = np.nextafter(b[4]["min"][1], np.float32(-1))
    assert _check(xyz, rgba, enc, batches=b) == (4, 4)
    for name, code in (("w1", 5), ("w2", 5), ("w3", 5), ("color", 6)):
        w = getattr(enc, name).copy()
        w[12345] ^= 1 << 10
        assert _check(xyz, rgba, enc, **{name: w}) == (code, 12345)


def test_rejects_an_unsorted_encoding(cloud):
    xyz, rgba, _ = cloud
    enc = O.encode_in_order(xyz, rgba, BS)
    perm = np.arange(len(xyz), dtype=np.uint32)
    assert O.verify_encoding(xyz, rgba, BS, enc.batches, enc.w1, enc.w2, enc.w3, enc.color,
                             perm)[0] == 3


# ---- the LOD tree checker (Sec. 3.5) ------------------------------------------------

L, M, SEED = 12, 700, 5


@pytest.fixture(scope="module")
def tree():
    p = S.terrain_params(3000.0, 0.15, 80)
    xyz, rgba = S.terrain(50000, p, seed=13)
    return xyz, rgba, O.lod_build(xyz, rgba, L, M, SEED)


def _lod(xyz, rgba, t, levels=L, m=M, seed=SEED, **over):
    a = dict(nodes=t.nodes.copy(), parent=t.parent.copy(), level=t.level.copy(), perm=t.perm.copy(),
             w1=t.w1.copy(), w2=t.w2.copy(), w3=t.w3.copy(), color=t.color.copy())
    a.update(over)
    return O.verify_lod(xyz, rgba, levels, m, seed, a["nodes"], a["parent"], a["level"], a["perm"],
                        a["w1"], a["w2"], a["w3"], a["color"], threads=3)


def test_lod_accepts_the_oracle_tree(tree):
    xyz, rgba, t = tree
    assert len(t.nodes) > 20 and t.level.max() >= 2
    assert _lod(xyz, rgba, t) == (0, 0)


def test_lod_rejects_wrong_parameters(tree):
    xyz, rgba, t = tree
    assert _lod(xyz, rgba, t, seed=SEED + 1)[0] == 5      # another priority order
    assert _lod(xyz, rgba, t, m=M + 1)[0] == 5            # another split size
    assert _lod(xyz, rgba, t, levels=int(t.level.max()))[0] == 2


def test_lod_rejects_structure_mistakes(tree):
    xyz, rgba, t = tree
    nd = t.nodes.copy()
    nd[0]["size"][0] *= np.float32(1.5)
    assert _lod(xyz, rgba, t, nodes=nd)[0] == 1
    b = int(np.nonzero(t.level == 2)[0][0])
    par = t.parent.copy()
    par[b] = 0
    assert _lod(xyz, rgba, t, parent=par)[0] == 2
    nd = t.nodes.copy()
    nd[b]["min"][0] = np.nextafter(nd[b]["min"][0], np.float32(np.inf))
    assert _lod(xyz, rgba, t, nodes=nd) == (2, b)
    # the first points of two sibling nodes exchanged (with their words and
    # colours): each now sits in the wrong octant of the root
    kids = np.nonzero(t.parent == 0)[0][1:]
    i, j = int(t.nodes[kids[0]]["first"]), int(t.nodes[kids[1]]["first"])
    sw = {k: getattr(t, k).copy() for k in ("perm", "w1", "w2", "w3", "color")}
    for a in sw.values():
        a[[i, j]] = a[[j, i]]
    assert _lod(xyz, rgba, t, **sw) == (4, i)


def test_lod_rejects_order_word_and_colour_mistakes(tree):
    xyz, rgba, t = tree
    f = int(t.nodes[3]["first"])
    # two points of a node exchanged with their words and colours: only the
    # input order within the node is broken
    sw = {k: getattr(t, k).copy() for k in ("perm", "w1", "w2", "w3", "color")}
    for a in sw.values():
        a[[f, f + 1]] = a[[f + 1, f]]
    assert _lod(xyz, rgba, t, **sw) == (3, f + 1)
    for name, code in (("w1", 6), ("w3", 6), ("color", 7)):
        w = getattr(t, name).copy()
        w[f + 2] ^= 1 << 12
        assert _lod(xyz, rgba, t, **{name: w}) == (code, f + 2)


def test_lod_rejects_a_leaf_that_should_have_split(tree):
    """A tree cut at 3 levels keeps more than M points in its deepest leaves;
    under a 12-level rule those leaves should have split."""
    xyz, rgba, _ = tree
    t3 = O.lod_build(xyz, rgba, 3, M, SEED)
    assert _lod(xyz, rgba, t3, levels=3) == (0, 0)
    assert (t3.nodes["count"][t3.level == 2] > M).any()
    code, b = _lod(xyz, rgba, t3, levels=L)
    assert code == 5 and t3.level[b] == 2 and t3.nodes[b]["count"] > M


def test_lod_rejects_header_cube_sibling_order_and_count_mistakes(tree):
    xyz, rgba, t = tree
    b = int(np.nonzero(t.level == 2)[0][1])
    # a node whose points do not start where the previous node's end
    nd = t.nodes.copy()
    nd[b]["first"] += 1
    assert _lod(xyz, rgba, t, nodes=nd) == (1, b)
    # a child cube that is not half of its parent's on one axis
    nd = t.nodes.copy()
    nd[b]["size"][1] = np.nextafter(nd[b]["size"][1], np.float32(np.inf))
    assert _lod(xyz, rgba, t, nodes=nd) == (2, b)
    # two leaf siblings exchanged (records and point blocks), so that every
    # node still holds its own cube's points: only the octant order breaks
    leaves = set(range(len(t.nodes))) - set(int(p) for p in t.parent[1:])
    s = next(i for i in range(1, len(t.nodes) - 1)
             if i in leaves and i + 1 in leaves and t.parent[i] == t.parent[i + 1])
    fa, ca = int(t.nodes[s]["first"]), int(t.nodes[s]["count"])
    cb = int(t.nodes[s + 1]["count"])
    nd = t.nodes.copy()
    nd[s], nd[s + 1] = t.nodes[s + 1], t.nodes[s]
    nd[s]["first"], nd[s + 1]["first"] = fa, fa + cb
    order = np.r_[0:fa, fa + ca:fa + ca + cb, fa:fa + ca, fa + ca + cb:len(t.perm)]
    sw = {k: getattr(t, k)[order].copy() for k in ("perm", "w1", "w2", "w3", "color")}
    assert _lod(xyz, rgba, t, nodes=nd, **sw) == (2, s + 1)
    # the last node dropped: its points are missing from the tree
    k = len(t.nodes) - 1
    assert _lod(xyz, rgba, t, nodes=t.nodes[:k].copy(), parent=t.parent[:k].copy(),
                level=t.level[:k].copy()) == (1, k)
