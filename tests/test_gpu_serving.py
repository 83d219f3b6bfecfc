"""Serving loop, autotuner and CUDA-graph replay through the C ABI.

Every result must be bit-identical to rendering the same view alone with
pc_render (and therefore to the CPU oracle, which test_gpu_parity checks).
"""
import threading
import time

import numpy as np
import pytest

import oracle as O
import paper_2204_01287_gb300 as pcr
import pcsynth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world(cuda_lib):
    ctx = pcr.Context(0, serve_pool_bytes=1 << 30, serve_streams=3)
    p1 = S.terrain_params(6000.0, 0.1, 300)
    xyz1, rgba1 = S.terrain(1_500_000, p1, seed=4)
    p2 = S.terrain_params(2000.0)
    xyz2, rgba2 = S.terrain(400_000, p2, seed=5)
    c1 = ctx.upload(xyz1, rgba1)
    c2 = ctx.upload(xyz2, rgba2)
    yield ctx, (c1, p1), (c2, p2)
    ctx.close()


def alone(ctx, cloud, view):
    import torch
    [(vis, img)] = ctx.render(cloud, [view])
    torch.cuda.synchronize()
    return pcr.rgba_to_numpy(img)


def _requests(c1, p1, c2, p2, n, seed=0):
    rng = np.random.default_rng(seed)
    sizes = [(128, 72), (192, 108), (256, 144), (64, 64)]
    reqs = []
    for i in range(n):
        cloud, p = (c1, p1) if rng.random() < 0.6 else (c2, p2)
        if rng.random() < 0.25:   # stereo pair, one request of two views
            W, H = 96, 108
            views = [pcr.make_view(S.stereo(p, W, H, e, 30.0), W, H, pcr.PC_VIEW_CULL) for e in (0, 1)]
        else:
            W, H = sizes[int(rng.integers(len(sizes)))]
            views = [pcr.make_view(S.random_view(p, 1000 + i, W, H, seed=seed), W, H, pcr.PC_VIEW_CULL)]
        reqs.append((cloud, views))
    return reqs


def test_each_result_same_alone_and_in_the_mix(world):
    ctx, (c1, p1), (c2, p2) = world
    reqs = _requests(c1, p1, c2, p2, 60, seed=1)
    # submit from two host threads at once, interleaved with polling
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for i in range(lo, hi):
            tickets[i] = pcr.pc_submit(ctx.h, reqs[i][0], reqs[i][1])

    th = [threading.Thread(target=submit, args=(0, 30)), threading.Thread(target=submit, args=(30, 60))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    starts = set()
    for i, t in enumerate(tickets):
        rc, res = pcr.pc_poll(ctx.h, t, 30000)
        assert rc == pcr.PC_OK and res["status"] == pcr.PC_OK
        starts.add(res["t_start_ms"])
        cloud, views = reqs[i]
        assert len(res["images"]) == len(views)
        for v, img in zip(views, res["images"]):
            assert np.array_equal(img, alone(ctx, cloud, v)), f"request {i}"
        assert res["t_submit_ms"] <= res["t_start_ms"] <= res["t_done_ms"]
        pcr.pc_release_ticket(ctx.h, t)
    # continuous batching: several requests shared a launch group
    assert len(starts) < len(tickets)


def test_serving_matches_oracle(world):
    ctx, (c1, p1), _ = world
    xyz, rgba = S.terrain(1_500_000, p1, seed=4)
    enc = O.encode(xyz, rgba, 10240)
    W, H = 160, 90
    m = S.random_view(p1, 7, W, H, seed=4)
    t = pcr.pc_submit(ctx.h, c1, [pcr.make_view(m, W, H, pcr.PC_VIEW_CULL)])
    rc, res = pcr.pc_poll(ctx.h, t, 10000)
    assert rc == pcr.PC_OK
    ovis, _ = O.render(enc, O.make_view(m, W, H))
    assert np.array_equal(res["images"][0], O.resolve(ovis, enc.color))
    pcr.pc_release_ticket(ctx.h, t)


def test_poll_never_hangs_and_times_out(world):
    ctx, (c1, p1), _ = world
    views = [pcr.make_view(S.random_view(p1, 50 + i, 1024, 1024, seed=4), 1024, 1024,
                           pcr.PC_VIEW_CULL) for i in range(8)]
    tickets = [pcr.pc_submit(ctx.h, c1, views) for _ in range(6)]
    t0 = time.time()
    rc, _ = pcr.pc_poll(ctx.h, tickets[-1], 0)
    assert rc in (pcr.PC_OK, pcr.PC_ETIMEDOUT)
    assert time.time() - t0 < 1.0
    for t in tickets:
        rc, res = pcr.pc_poll(ctx.h, t, 20000)
        assert rc == pcr.PC_OK and res["status"] == pcr.PC_OK
        pcr.pc_release_ticket(ctx.h, t)
    with pytest.raises(pcr.PCError):
        pcr.pc_poll(ctx.h, 987654321, 0)
    with pytest.raises(pcr.PCError):
        pcr.pc_release_ticket(ctx.h, 987654321)


def test_poll_wait_is_bounded(world):
    """pc_poll has no unbounded wait: a negative timeout is refused, and a
    request still queued behind others answers PC_ETIMEDOUT after about the
    timeout it was given."""
    import torch
    ctx, (c1, p1), _ = world
    W = H = 1024
    views = [pcr.make_view(S.random_view(p1, 80 + i, W, H, seed=4), W, H,
                           pcr.PC_VIEW_CULL | pcr.PC_VIEW_NO_EARLY_DEPTH) for i in range(8)]
    # caller-owned framebuffers: a long queue without pool admission or host images
    fbs = [[(torch.empty(W * H, dtype=torch.int64, device="cuda"),
             torch.empty(W * H, dtype=torch.int32, device="cuda")) for _ in views]
           for _ in range(12)]
    tickets = [pcr.pc_submit(ctx.h, c1, views, [(a.data_ptr(), b.data_ptr()) for a, b in fb])
               for fb in fbs]
    with pytest.raises(pcr.PCError) as e:
        pcr.pc_poll(ctx.h, tickets[-1], -1)
    assert e.value.status == pcr.PC_EINVAL
    t0 = time.perf_counter()
    rc, _ = pcr.pc_poll(ctx.h, tickets[-1], 25)
    dt = time.perf_counter() - t0
    if rc == pcr.PC_ETIMEDOUT:
        assert 0.02 <= dt < 0.5
    for t in tickets:
        rc, res = pcr.pc_poll(ctx.h, t, 20000)
        assert rc == pcr.PC_OK and res["status"] == pcr.PC_OK
        pcr.pc_release_ticket(ctx.h, t)


def test_admission_refused_when_it_can_never_fit(cuda_lib):
    ctx = pcr.Context(0, serve_pool_bytes=8 << 20)
    try:
        cloud = ctx.upload(*S.unit_cube(10000))
        big = [pcr.make_view(S.cube_camera(2048, 2048), 2048, 2048)]
        with pytest.raises(pcr.PCError) as e:
            pcr.pc_submit(ctx.h, cloud, big)
        assert e.value.status == pcr.PC_EBUSY
        small = [pcr.make_view(S.cube_camera(64, 64), 64, 64)]
        t = pcr.pc_submit(ctx.h, cloud, small)
        rc, res = pcr.pc_poll(ctx.h, t, 10000)
        assert rc == pcr.PC_OK
        assert np.array_equal(res["images"][0], alone(ctx, cloud, small[0]))
    finally:
        ctx.close()


def test_memory_pressure_queues_instead_of_failing(cuda_lib):
    """A pool that holds only a few requests at once still serves many: device
    framebuffers are admitted as they free up, and a full pinned image pool
    answers PC_EBUSY until finished tickets are released."""
    ctx = pcr.Context(0, serve_pool_bytes=3 * 512 * 512 * 12 + 4096, serve_streams=4)
    try:
        cloud = ctx.upload(*S.unit_cube(200000, seed=2))
        views = [pcr.make_view(S.look_at_perspective((0.5 + 0.1 * i, 0.5, 2.5), (0.5, 0.5, 0.5),
                                                      (0, 1, 0), 60, 1, 0.1, 10), 512, 512)
                 for i in range(12)]
        pending, busy_seen = [], 0

        def collect_oldest():
            v, t = pending.pop(0)
            rc, res = pcr.pc_poll(ctx.h, t, 20000)
            assert rc == pcr.PC_OK
            assert np.array_equal(res["images"][0], alone(ctx, cloud, v))
            pcr.pc_release_ticket(ctx.h, t)

        for v in views:
            while True:
                try:
                    pending.append((v, pcr.pc_submit(ctx.h, cloud, [v])))
                    break
                except pcr.PCError as e:
                    assert e.status == pcr.PC_EBUSY and pending
                    busy_seen += 1
                    collect_oldest()
        while pending:
            collect_oldest()
        assert busy_seen > 0
    finally:
        ctx.close()


def test_release_cloud_while_requests_queued(cuda_lib):
    ctx = pcr.Context(0)
    try:
        xyz, rgba = S.unit_cube(300000, seed=3)
        cloud = ctx.upload(xyz, rgba)
        v = pcr.make_view(S.cube_camera(256, 256), 256, 256)
        ref = alone(ctx, cloud, v)
        tickets = [pcr.pc_submit(ctx.h, cloud, [v]) for _ in range(5)]
        pcr.pc_release_cloud(ctx.h, cloud)
        for t in tickets:
            rc, res = pcr.pc_poll(ctx.h, t, 20000)
            assert rc == pcr.PC_OK and np.array_equal(res["images"][0], ref)
    finally:
        ctx.close()


def test_autotune_keeps_bits(world):
    ctx, (c1, p1), _ = world
    views = [pcr.make_view(S.random_view(p1, 300 + i, 200, 120, seed=4), 200, 120, pcr.PC_VIEW_CULL)
             for i in range(6)]
    before = [alone(ctx, c1, v) for v in views]
    r = pcr.pc_autotune(ctx.h, c1, views)
    assert r["threads_per_block"] in (128, 256) and r["points_per_warp"] in (1024, 2048, 4096)
    assert 1 <= r["views_per_launch"] <= 32 and r["candidates"] > 10
    after = [alone(ctx, c1, v) for v in views]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    import torch
    multi = ctx.render(c1, views)
    torch.cuda.synchronize()
    for (vis, img), b in zip(multi, before):
        assert np.array_equal(pcr.rgba_to_numpy(img), b)


def test_graph_replay_keeps_bits(world):
    import torch
    ctx, (c1, p1), _ = world
    g = pcr.Context(0, flags=pcr.PC_CFG_GRAPHS)
    try:
        xyz, rgba = S.terrain(1_500_000, p1, seed=4)
        cloud = g.upload(xyz, rgba)
        stream = torch.cuda.Stream()
        for i in range(5):
            views = [pcr.make_view(S.random_view(p1, 400 + i * 3 + j, 160, 96, seed=4), 160, 96,
                                   pcr.PC_VIEW_CULL) for j in range(1 + i % 3)]
            with torch.cuda.stream(stream):
                fbs = g.render(cloud, views, stream=stream)
            stream.synchronize()
            for (vis, img), v in zip(fbs, views):
                assert np.array_equal(pcr.rgba_to_numpy(img), alone(ctx, c1, v))
    finally:
        g.close()


def test_caller_owned_framebuffers(world):
    """Requests that bring their own device framebuffers: nothing is admitted
    or copied to the host, and the images in the caller's buffers equal the
    same views rendered alone; they batch with library-owned requests."""
    import torch
    ctx, (c1, p1), (c2, p2) = world
    reqs = _requests(c1, p1, c2, p2, 12, seed=7)
    owned = []
    tickets = []
    for i, (cloud, views) in enumerate(reqs):
        if i % 2 == 0:
            fbs = ctx.framebuffers(views)
            owned.append(fbs)
            tickets.append(pcr.pc_submit(ctx.h, cloud, views,
                                         [(a.data_ptr(), b.data_ptr()) for a, b in fbs]))
        else:
            owned.append(None)
            tickets.append(pcr.pc_submit(ctx.h, cloud, views))
    for i, t in enumerate(tickets):
        rc, res = pcr.pc_poll(ctx.h, t, 60_000)
        assert rc == pcr.PC_OK and res["status"] == pcr.PC_OK
        cloud, views = reqs[i]
        if owned[i] is not None:
            assert res["images"] == []
            got = [pcr.rgba_to_numpy(img) for _, img in owned[i]]
        else:
            got = res["images"]
        for v, img in zip(views, got):
            assert np.array_equal(img, alone(ctx, cloud, v))
        pcr.pc_release_ticket(ctx.h, t)
    # misaligned caller framebuffers are refused
    v = reqs[0][1][:1]
    buf = torch.empty(v[0].width * v[0].height + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(pcr.PCError) as e:
        pcr.pc_submit(ctx.h, reqs[0][0], v, [(buf.data_ptr() + 8, 0)])
    assert e.value.status == pcr.PC_EINVAL
