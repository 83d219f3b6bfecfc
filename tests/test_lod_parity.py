"""Host LOD builder of the library (Sec. 3.5) against the oracle's, bit-exact
on the same decoded positions (runs without a GPU)."""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S


@pytest.mark.parametrize("n,M,L,seed,threads", [(1, 16, 12, 0, 1), (5000, 256, 12, 3, 4),
                                                (120000, 2048, 12, 9, 0), (80000, 1000, 4, 1, 3),
                                                (70000, 10240, 12, 5, 0)])
def test_lod_builder_matches_oracle(n, M, L, seed, threads):
    p = S.terrain_params(5000.0, 0.2, 100)
    xyz, rgba = S.terrain(n, p, seed=n)
    enc = O.encode(xyz, rgba, 10240)
    pos = O.decode_cloud(enc, 3)
    ref = O.lod_build(pos, enc.color, L, M, seed)
    nodes, parent, level, perm, w1, w2, w3, col = pcr.pc_lod_encode(pos, enc.color, L, M, seed,
                                                                     threads)
    assert nodes.tobytes() == ref.nodes.tobytes()
    assert np.array_equal(parent, ref.parent) and np.array_equal(level, ref.level)
    assert np.array_equal(perm, ref.perm)
    for a, b in ((w1, ref.w1), (w2, ref.w2), (w3, ref.w3), (col, ref.color)):
        assert np.array_equal(a, b)


def test_lod_builder_degenerate():
    xyz = np.zeros((3000, 3), np.float32)          # all points equal: depth limit stops it
    rgba = np.arange(3000, dtype=np.uint32)
    ref = O.lod_build(xyz, rgba, 6, 100, 0)
    nodes, parent, level, perm, *_ = pcr.pc_lod_encode(xyz, rgba, 6, 100, 0)
    assert nodes.tobytes() == ref.nodes.tobytes() and np.array_equal(perm, ref.perm)
    assert level.max() == 5
