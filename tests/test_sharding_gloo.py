"""The multi-rank path of bench.py on CPU with gloo, world size 2: ranks run
independent workloads (weak scaling, no data-path collective) and the
timing is the maximum over ranks, the work the sum."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2509_15377_gb300 import workloads as W

    seed = bench.shard_seed(rank)
    w = W.plate_batched(n_avalanches=64, seed=seed)
    t = 1.0 + rank  # stand-in step times
    out[rank] = (bench.max_over_ranks(t), bench.sum_over_ranks(float(w.primaries.n)),
                 int(w.primaries.aval_field[0] * 1000))
    bench.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    from paper_2509_15377_gb300 import workloads as W
    n0 = W.plate_batched(n_avalanches=64, seed=0).primaries.n
    n1 = W.plate_batched(n_avalanches=64, seed=1).primaries.n
    for r in range(2):
        tmax, total, _ = out[r]
        assert tmax == 2.0
        assert total == float(n0 + n1)
    # the two ranks transport different avalanches
    assert out[0][2] != out[1][2]
