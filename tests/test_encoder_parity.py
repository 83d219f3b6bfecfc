"""Host encoder of the library (Sec. 3.1, Eq. 1, Listing 2) against the oracle's
encoder: bit-exact permutation, batches and words on the same seeded inputs.
The encoder is host C++, so this runs without a GPU."""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S


def _compare(xyz, rgba, bs, threads=0):
    enc = O.encode(xyz, rgba, batch_size=bs)
    b, w1, w2, w3, col, perm = pcr.pc_encode(xyz, rgba, batch_size=bs, threads=threads)
    assert np.array_equal(perm, enc.perm)
    assert b.tobytes() == enc.batches.tobytes()
    assert np.array_equal(w1, enc.w1)
    assert np.array_equal(w2, enc.w2)
    assert np.array_equal(w3, enc.w3)
    assert np.array_equal(col, enc.color)


@pytest.mark.parametrize("n,bs", [(1, 4), (3, 4), (5, 4), (10240, 10240), (100003, 10240),
                                  (70000, 2048)])
def test_unit_cube(n, bs):
    xyz, rgba = S.unit_cube(n, seed=n)
    _compare(xyz, rgba, bs)


def test_terrain_with_buildings():
    xyz, rgba = S.terrain(300000, S.terrain_params(40000.0, 0.2, 2000), seed=5)
    _compare(xyz, rgba, 10240)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_thread_count_does_not_matter(threads):
    xyz, rgba = S.terrain(150000, S.terrain_params(10000.0), seed=9)
    _compare(xyz, rgba, 10240, threads=threads)


def test_duplicates_and_degenerate_boxes():
    rng = np.random.default_rng(0)
    base = rng.uniform(-1, 1, size=(50, 3)).astype(np.float32)
    xyz = base[rng.integers(0, 50, 20000)]          # many exact duplicates
    xyz[:5000, 2] = 0.25                            # a flat slab: zero-size z boxes
    rgba = np.arange(len(xyz), dtype=np.uint32)
    _compare(xyz, rgba, 1024)


def test_empty_and_invalid():
    xyz = np.zeros((0, 3), np.float32)
    b, *_ = pcr.pc_encode(xyz, None, batch_size=10240)
    assert len(b) == 0
    with pytest.raises(pcr.PCError):
        pcr.pc_encode(np.zeros((4, 3), np.float32), None, batch_size=10)   # not a multiple of 4


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("flags", [0, pcr.PC_ENCODE_KEEP_ORDER])
def test_non_finite_coordinates_refused(bad, flags):
    """Eq. 1 divides by a batch box that a NaN or an infinity would make
    undefined: the encoder and the LOD builder refuse such clouds."""
    xyz = np.random.default_rng(1).uniform(0, 1, size=(30000, 3)).astype(np.float32)
    xyz[29999 - 7, 1] = bad                        # one coordinate, late in the input
    with pytest.raises(pcr.PCError) as e:
        pcr.pc_encode(xyz, None, batch_size=1024, threads=4, flags=flags)
    assert e.value.status == pcr.PC_EINVAL
    with pytest.raises(pcr.PCError) as e:
        pcr.pc_lod_encode(xyz, None, max_node_points=1000, threads=4)
    assert e.value.status == pcr.PC_EINVAL


@pytest.mark.parametrize("n", [7, 30000, 104000])
def test_keep_order_matches_oracle(n):
    """Batches of consecutive input points, no Morton sort (Sec. 4.2 baseline)."""
    xyz, rgba = S.terrain_scan(n, S.terrain_params(4000.0), (0.0, 0.0), 1500.0, 5000, seed=n)
    enc = O.encode_in_order(xyz, rgba, 10240)
    b, w1, w2, w3, col, perm = pcr.pc_encode(xyz, rgba, 10240, 0, pcr.PC_ENCODE_KEEP_ORDER)
    assert np.array_equal(perm, np.arange(n))
    assert b.tobytes() == enc.batches.tobytes()
    for a, r in ((w1, enc.w1), (w2, enc.w2), (w3, enc.w3), (col, enc.color)):
        assert np.array_equal(a, r)
