"""World-size-2 check of the multi-rank host logic on CPU (gloo): channel
ownership is a disjoint cover and the job time is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_2607_16629_gb300.sharding import channels_for_rank, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = channels_for_rank(3, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = max_over_ranks(10.0 + rank)
        out[rank] = (gathered, t)
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_channels_and_take_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        gathered, t = res[rank]
        flat = sorted(c for chans in gathered for c in chans)
        assert flat == list(range(3 * world))
        assert t == 10.0 + world - 1


def test_bad_arguments():
    from paper_2607_16629_gb300.sharding import channels_for_rank
    with pytest.raises(ValueError):
        channels_for_rank(0, 2, 0)
    with pytest.raises(ValueError):
        channels_for_rank(1, 2, 2)
