"""The N > 1 path on CPU: two gloo ranks shard frames with no overlap and no
gap, and time/work are combined with max/sum over ranks (the only
collectives; the data path has none)."""
import os
import socket

import pytest

from paper_1604_03498_gb300.multigpu import frame_shard, reduce_over_ranks


def test_frame_shards_partition_the_frames():
    for n in (0, 1, 7, 256, 1001):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in frame_shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(frame_shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        frame_shard(10, 2, 2)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shard = frame_shard(256, rank, world)
    frames_done = len(shard)
    elapsed = 1.0 + rank           # rank 1 is the slower one
    t = reduce_over_ranks(elapsed, "max")
    n = reduce_over_ranks(frames_done, "sum")
    q.put((rank, t, n, shard.start, shard.stop))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_time_and_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]        # max over ranks
    assert [r[2] for r in res] == [256.0, 256.0]    # sum over ranks
    assert res[0][3:] == (0, 128) and res[1][3:] == (128, 256)
