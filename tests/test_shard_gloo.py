"""The batch-range partition of a frame across ranks and its exchange step,
on CPU with two and three gloo ranks: each rank renders its shard with the
oracle, the empty key is taken as 2^63 - 1 (what PC_VIEW_SIGNED_EMPTY clears
to), the library's merge_shards reduces the buffers with a signed int64 MIN,
and every rank must then hold the oracle's whole-frame visibility buffer."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cloud():
    import oracle as O
    import pcsynth as S
    p = S.terrain_params(3000.0, 0.2, 100)
    xyz, rgba = S.terrain(250_003, p, seed=31)
    enc = O.encode(xyz, rgba, 10240)
    view = O.make_view(S.flythrough(p, 40, 120, 160, 90, seed=31), 160, 90, cull=True)
    return enc, view


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle as O
    import paper_2204_01287_gb300 as pcr
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    enc, view = _cloud()
    first, count = pcr.batch_range(len(enc.batches), rank, world)
    shard = O.Encoded(enc.batches[first:first + count], enc.w1, enc.w2, enc.w3, enc.color,
                      enc.perm)
    vis, _ = O.render(shard, view)
    signed = vis.view(np.int64).copy()
    signed[vis == O.EMPTY] = pcr.EMPTY_SIGNED
    t = torch.from_numpy(signed)
    pcr.merge_shards(t)
    merged = t.numpy().view(np.uint64).copy()
    merged[merged == pcr.EMPTY_SIGNED] = O.EMPTY
    out.put((rank, first, count, merged.tobytes()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partition_and_min_reduce_give_the_whole_frame(world):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    enc, view = _cloud()
    whole, _ = O.render(enc, view)
    # the ranges cover every batch once, in order
    assert [r[1] for r in res] == sorted(r[1] for r in res)
    assert sum(r[2] for r in res) == len(enc.batches)
    assert all(a[1] + a[2] == b[1] for a, b in zip(res, res[1:]))
    for _, _, _, buf in res:
        assert np.array_equal(np.frombuffer(buf, np.uint64), whole)
    assert (whole != O.EMPTY).sum() > 500


def test_batch_range_edges():
    sys.path.insert(0, ROOT)
    import paper_2204_01287_gb300 as pcr
    for nb in (1, 7, 195_313):
        for world in (1, 2, 3, 8):
            parts = [pcr.batch_range(nb, r, world) for r in range(world)]
            assert parts[0][0] == 0 and sum(c for _, c in parts) == nb
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        pcr.batch_range(10, 2, 2)
