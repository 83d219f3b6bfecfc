"""Batch culling (Sec. 3.2) on the GPU decides exactly as the oracle's
binary64 test, also for boxes that touch a clip plane: the kernels evaluate the
test in binary32 first and defer to binary64 near the decision boundary, so
the count of drawn batches must equal the oracle's for every view."""
import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu


def _boxes_on_planes(m, n, rng, rel):
    """n boxes near the frustum's side, near and far planes: points of the NDC
    boundary pushed outward by 2^-10 (the culling margin) plus a random offset
    of size `rel` (a quarter of them well inside or well outside), mapped back
    to world space, with random small sizes (some zero)."""
    M = np.asarray(m, np.float64).reshape(4, 4, order="F")
    inv = np.linalg.inv(M)
    ndc = rng.uniform(-1.0, 1.0, (n, 3))
    axis = rng.integers(0, 3, n)
    side = rng.choice([-1.0, 1.0], n)
    eps = 2.0 ** -10 + rel * rng.normal(size=n)
    far = rng.random(n) < 0.25
    eps[far] = rng.choice([-0.05, 0.05], int(far.sum()))
    ndc[np.arange(n), axis] = side * (1.0 + eps)
    h = np.c_[ndc, np.ones(n)] @ inv.T
    p = h[:, :3] / h[:, 3:4]
    scale = np.abs(p).max(axis=1, keepdims=True) + 1.0
    size = np.abs(rng.normal(size=(n, 3))) * scale * rng.choice([0.0, 1e-7, 1e-5], (n, 1))
    b = np.zeros(n, pcr.BATCH_DTYPE)
    b["min"] = (p - size / 2).astype(np.float32)
    b["size"] = size.astype(np.float32)
    b["first"] = np.arange(n, dtype=np.uint32) * 4
    b["count"] = 4
    return b


@pytest.mark.parametrize("rel", [0.0, 1e-8, 1e-6, 1e-4])
def test_culling_decisions_near_planes(cuda_lib, rel):
    import torch
    rng = np.random.default_rng(int(rel * 1e9) + 3)
    views = [S.cube_camera(64, 48), S.look_at_perspective((3, -2, 1), (0, 0.5, 0.2), (0, 0, 1),
                                                          40.0, 1.5, 0.5, 50.0)]
    with pcr.Context(0) as ctx:
        for m in views:
            b = _boxes_on_planes(m, 20000, rng, rel)
            n = 4 * len(b)
            words = rng.integers(0, 1 << 30, n, dtype=np.uint32)
            cloud = ctx.upload_encoded(b, words, words, words, np.zeros(n, np.uint32))
            v = pcr.make_view(m, 64, 48, pcr.PC_VIEW_CULL)
            ctx.render(cloud, [v])
            torch.cuda.synchronize()
            got = ctx.stats()["batches_rendered"]
            ov = O.make_view(m, 64, 48, cull=True)
            expect = sum(not O.cull(bt, ov) for bt in b)
            assert 0 < expect < len(b)
            assert got == expect
            pcr.pc_release_cloud(ctx.h, cloud)
