"""The seeded input generators (pcsynth): every point is a function of (seed,
index) alone, so a workload generated in chunks, on any number of threads,
equals the workload generated at once. The full-size tests and the bench
generate their 2B-point clouds in chunks and rely on this."""
import numpy as np
import pytest

import pcsynth as S


@pytest.mark.parametrize("gen", ["cube", "terrain", "terrain_buildings"])
def test_chunks_and_threads_do_not_matter(gen):
    n = 50_000
    p = S.terrain_params(3000.0, 0.15, 80)

    def make(count, first, threads):
        if gen == "cube":
            return S.unit_cube(count, seed=4, first=first, threads=threads)
        q = p if gen == "terrain_buildings" else S.terrain_params(3000.0)
        return S.terrain(count, q, seed=4, first=first, threads=threads)

    xyz, rgba = make(n, 0, 1)
    for threads in (2, 7):
        x2, r2 = make(n, 0, threads)
        assert np.array_equal(x2, xyz) and np.array_equal(r2, rgba)
    cuts = [0, 1, 999, 20_000, 33_333, n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        xc, rc = make(b - a, a, 3)
        assert np.array_equal(xc, xyz[a:b]) and np.array_equal(rc, rgba[a:b])


def test_seeds_differ_and_values_are_finite():
    a, _ = S.unit_cube(10_000, seed=1)
    b, _ = S.unit_cube(10_000, seed=2)
    assert not np.array_equal(a, b)
    assert np.isfinite(a).all() and (a >= 0).all() and (a < 1).all()
    t, _ = S.terrain(10_000, S.terrain_params(10_000.0), seed=3)
    assert np.isfinite(t).all()


def test_scan_order_chunks():
    p = S.terrain_params(3000.0)
    n = 30_000
    xyz, rgba = S.terrain_scan(n, p, seed=5, threads=1)
    xc, rc = S.terrain_scan(10_000, p, seed=5, first=12_345, total=n, threads=4)
    assert np.array_equal(xc, xyz[12_345:22_345]) and np.array_equal(rc, rgba[12_345:22_345])
