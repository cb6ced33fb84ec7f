"""Host logic of the z-slab partition of one volume over ranks (no GPU): the
ranges tile [0, nz) in order, start on the backprojection's 16-slice grid and
differ by at most one tile; world-size-2 gloo ranks each take their own range
and together cover the volume once."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2201_02309_b300 import slab_partition


@pytest.mark.parametrize("nz,world", [(256, 1), (256, 2), (256, 3), (150, 4), (48, 8), (1, 2), (17, 2), (70, 5)])
def test_partition_properties(nz, world):
    parts = slab_partition(nz, world)
    assert len(parts) == world
    assert parts[0][0] == 0 and parts[-1][1] == nz
    for (a0, a1), (b0, b1) in zip(parts, parts[1:]):
        assert a1 == b0
    tiles = []
    for s0, s1 in parts:
        assert 0 <= s0 <= s1 <= nz
        if s0 < s1:
            assert s0 % 16 == 0
        tiles.append(-(-(s1 - s0) // 16))
    assert max(tiles) - min(tiles) <= 1
    assert sum(tiles) == -(-nz // 16)


def test_partition_rejects_bad_arguments():
    for args in ((0, 1), (16, 0), (16, 1, 0)):
        with pytest.raises(ValueError):
            slab_partition(*args)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, nz, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = slab_partition(nz, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_two_ranks_cover_the_volume_once():
    nz = 256
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, nz, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    covered = sorted(s for a, b in res[0] for s in range(a, b))
    assert covered == list(range(nz))
