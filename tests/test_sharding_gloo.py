"""The multi-process path on CPU with gloo, world size 2.

A workload's avalanches are split into contiguous ranges, one per rank
(`shard.partition`); each rank runs its range alone with aval_base = its
first avalanche and the workload's electron ids, and rank 0 gathers the
parts (`shard.gather`).  The oracle stands in for the GPU of each rank: the
gathered result must equal one oracle run of the whole workload, electron for
electron and bit for bit.  The bench's timing reductions (maximum of the
ranks' times, sum of their work) are checked on the same ranks.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2509_15377_gb300 import shard
from paper_2509_15377_gb300 import workloads as W

N_AVAL = 30
SEED = 11
T_MAX = 0.4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload():
    return W.plate_batched(n_avalanches=N_AVAL, seed=5)


def _run_oracle(w, prim, aval_base):
    import oracle
    return oracle.run(w.gas, w.field, prim, seed=SEED, t_max=T_MAX, n_threads=2, majorant=1,
                      aval_base=aval_base)


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w = _workload()
    a0, a1 = shard.partition(N_AVAL, world, rank)
    part = shard.part_primaries(w.primaries, a0, a1)
    res = _run_oracle(w, part, a0)
    merged = shard.gather(res, a0, N_AVAL)
    t = 1.0 + rank  # stand-in step times
    out[rank] = {"tmax": bench.max_over_ranks(t),
                 "total": bench.sum_over_ranks(float(part.n)),
                 "merged": None if merged is None else {k: v for k, v in merged.items()}}
    bench.barrier()
    dist.destroy_process_group()


def _by_uid(res):
    order = np.argsort(res["uid"], kind="stable")
    return {k: (v[order] if k not in shard.PER_AVALANCHE else v) for k, v in res.items()}


def test_two_ranks_gather_equals_the_whole_run():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    w = _workload()
    for r in range(2):
        assert out[r]["tmax"] == 2.0
        assert out[r]["total"] == float(w.primaries.n)
    assert out[1]["merged"] is None
    merged = _by_uid(out[0]["merged"])
    whole = _by_uid(_run_oracle(w, w.primaries, 0))
    assert set(merged) == set(whole)
    assert len(whole["uid"]) > 3 * w.primaries.n        # the avalanches multiplied
    for k in whole:
        assert np.array_equal(merged[k], whole[k]), k


def test_aval_base_keys_the_random_streams():
    """A part run with aval_base = 0 instead of its first avalanche draws
    other random numbers: the offset is what makes the parts add up."""
    w = _workload()
    a0, a1 = shard.partition(N_AVAL, 2, 1)
    part = shard.part_primaries(w.primaries, a0, a1)
    right = _by_uid(_run_oracle(w, part, a0))
    wrong = _by_uid(_run_oracle(w, part, 0))
    assert not (np.array_equal(right["uid"], wrong["uid"]) and
                np.array_equal(right["z1"], wrong["z1"]))


@pytest.mark.parametrize("n,world", [(30, 2), (4096, 8), (7, 3), (2, 4), (0, 2)])
def test_partition_tiles_the_avalanches(n, world):
    ranges = [shard.partition(n, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (_, b), (c, _) in zip(ranges, ranges[1:]):
        assert b == c
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_part_primaries_and_merge():
    w = _workload()
    p = w.primaries
    a0, a1 = 7, 19
    part = shard.part_primaries(p, a0, a1)
    keep = (p.aval >= a0) & (p.aval < a1)
    assert part.n_avalanches == a1 - a0
    assert np.array_equal(part.aval, p.aval[keep] - a0)
    assert np.array_equal(part.uid, p.uid[keep])
    assert np.array_equal(part.aval_field, p.aval_field[a0:a1])
    # merge places per-avalanche arrays and shifts endpoint avalanche numbers
    r0 = {"uid": np.array([1, 2], np.uint64), "aval": np.array([0, 1], np.int32),
          "electrons": np.array([1, 1], np.uint64), "tallies": np.ones((2, 3), np.uint64)}
    r1 = {"uid": np.array([3], np.uint64), "aval": np.array([0], np.int32),
          "electrons": np.array([5], np.uint64), "tallies": 2 * np.ones((1, 3), np.uint64)}
    m = shard.merge([(2, r1), (0, r0)], 3)
    assert m["aval"].tolist() == [0, 1, 2]
    assert m["electrons"].tolist() == [1, 1, 5]
    assert m["tallies"][2].tolist() == [2, 2, 2]
    with pytest.raises(ValueError):
        shard.merge([(0, r0)], 3)          # avalanche 2 missing
    with pytest.raises(ValueError):
        shard.merge([(0, r0), (1, r1)], 3)  # overlap
