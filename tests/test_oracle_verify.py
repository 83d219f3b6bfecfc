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
