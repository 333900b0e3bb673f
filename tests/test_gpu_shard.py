"""A workload split into avalanche ranges and gathered equals the whole run.

Each part runs alone through the C ABI with aval_base = its first avalanche
(the random streams stay keyed by the workload's avalanche numbers) and the
workload's electron ids; `shard.merge` concatenates the endpoints and places
the per-avalanche arrays.  Electron by electron, sorted by id, the merged
result must be bit-identical to one run of the whole workload: in FP64, and
in mixed precision with the same launch shape (an electron's step sequence,
including its FP32-to-FP64 folds every K collision rounds, does not depend
on which lane or CTA runs it).  This is the multi-GPU split, run here as
consecutive calls on one GPU.
"""
import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import shard
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import by_uid, run_gpu

pytestmark = pytest.mark.gpu

KEYS = ("uid", "aval", "status", "n_flight", "x0", "y0", "z0", "t0", "e0", "x1", "y1", "z1", "t1",
        "e1")


@pytest.fixture(scope="module")
def av():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    a = A.Avalanche(0)
    yield a
    a.close()


def _split_and_gather(av, w, world, **kw):
    parts = []
    for rank in range(world):
        a0, a1 = shard.partition(w.primaries.n_avalanches, world, rank)
        part = shard.part_primaries(w.primaries, a0, a1)
        _, out = run_gpu(av, w, prim=part, aval_base=a0, **kw)
        parts.append((a0, out))
    return shard.merge(parts, w.primaries.n_avalanches)


def _assert_identical(a, b):
    ga, gb = by_uid(a), by_uid(b)
    for k in KEYS:
        assert np.array_equal(ga[k], gb[k]), k
    assert np.array_equal(a["electrons"], b["electrons"])
    assert np.array_equal(a["tallies"], b["tallies"])


@pytest.mark.parametrize("world", [2, 3])
def test_fp64_parts_equal_the_whole_run(av, world):
    w = W.plate_batched(n_avalanches=96, seed=3)
    av.set_gas(w.gas)
    av.set_field(w.field)
    kw = dict(seed=17, t_max=0.6, precision=A.GT_FP64, capacity=2_000_000,
              majorant=A.GT_MAJORANT_BANDED)
    _, whole = run_gpu(av, w, **kw)
    merged = _split_and_gather(av, w, world, **kw)
    assert len(whole["uid"]) > 4 * w.primaries.n
    _assert_identical(merged, whole)
    # and the whole run is the oracle's, electron by electron (1e-9)
    ref = oracle.run(w.gas, w.field, w.primaries.subset(range(8)), seed=17, t_max=0.6, majorant=1)
    g = by_uid({k: v[np.isin(whole["aval"], range(8))] for k, v in whole.items()
                if k not in shard.PER_AVALANCHE})
    r = by_uid(ref)
    assert np.array_equal(g["uid"], r["uid"])
    assert np.allclose(g["z1"], r["z1"], rtol=1e-9, atol=1e-12)


def test_mixed_parts_equal_the_whole_run(av):
    w = W.plate_batched(n_avalanches=128, seed=4)
    av.set_gas(w.gas)
    av.set_field(w.field)
    kw = dict(seed=23, precision=A.GT_MIXED, capacity=8_000_000, majorant=A.GT_MAJORANT_BANDED,
              block=512, refill_period=16, flights_per_phase=1)
    _, whole = run_gpu(av, w, **kw)
    merged = _split_and_gather(av, w, 2, **kw)
    _assert_identical(merged, whole)


def test_aval_base_out_of_range_is_refused(av):
    w = W.plate_batched(n_avalanches=8, seed=5)
    av.set_gas(w.gas)
    av.set_field(w.field)
    with pytest.raises(A.GtError):
        run_gpu(av, w, seed=1, t_max=0.1, aval_base=-1)
    with pytest.raises(A.GtError):
        run_gpu(av, w, seed=1, t_max=0.1, aval_base=2**31 - 4)
