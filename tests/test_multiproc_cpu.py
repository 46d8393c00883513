"""The multi-rank path on CPU (gloo, world size 2): realisation sharding and
the max-over-ranks step time.  Each rank computes its own realisations of a
small Eq. 3 case with the FP64 oracle through real_offset; gathered, they are
bit-identical to one process computing all of them (the stream continues
across realisations, so no exchange is needed on the data path)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2404_02978_gb300.shard import max_over_ranks, realisation_slice

N_F, PER_RANK = 64, 3


def _xy():
    rng = np.random.default_rng(3)
    return rng.uniform(-2, 2, size=(40, 2)).astype(np.float32)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, cnt = realisation_slice(rank, world, PER_RANK)
        mine = torch.from_numpy(oracle.synthesize(oracle.params(seed=9), N_F, cnt, _xy(), real_offset=off))
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        t = max_over_ranks(1.5 + rank, world)
        if rank == 0:
            q.put((torch.cat(parts).numpy(), t))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_reproduce_one_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, PORT, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle.synthesize(oracle.params(seed=9), N_F, world * PER_RANK, _xy())
    assert np.array_equal(got, ref)
    assert t == 2.5


def test_slices_partition_and_reject_bad_ranks():
    s = [realisation_slice(r, 4, 250, base=10) for r in range(4)]
    assert s == [(10, 250), (260, 250), (510, 250), (760, 250)]
    assert max_over_ranks(3.0, 1) == 3.0
    for bad in ((4, 4, 1), (-1, 2, 1), (0, 0, 1), (0, 2, -1)):
        with pytest.raises(ValueError):
            realisation_slice(*bad)


PORT = _free_port()
