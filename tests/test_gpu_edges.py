"""GPU edge cases through the C ABI: empty inputs, empty avalanches,
primaries outside the volume, capacity overflow, the per-avalanche size cap,
a bounded wait that gives up (fault injected on the host side: a queue slot
that nothing fills), invalid device-side inputs, and argument errors."""
import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import assert_same_electrons, by_uid, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def av():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    a = A.Avalanche(0)
    w = W.plate(n_avalanches=8, seed=0)
    a.set_gas(w.gas)
    a.set_field(w.field)
    yield a
    a.close()


def test_empty_run(av):
    w = W.plate(n_avalanches=4, seed=0)
    empty = w.primaries.subset([])
    for mode in (A.GT_BATCHED, A.GT_PLAIN):
        st, out = run_gpu(av, w, seed=0, prim=empty, mode=mode, capacity=64)
        assert st["n_endpoints"] == 0
        assert np.all(out["electrons"] == 0) and np.all(out["tallies"] == 0)


def test_empty_avalanches_and_ragged_counts(av):
    """Poisson primary counts include zeros; those avalanches stay empty."""
    w = W.plate_batched(n_avalanches=300, seed=2)
    counts = np.bincount(w.primaries.aval, minlength=300)
    assert (counts == 0).any()
    st, out = run_gpu(av, w, seed=2, t_max=0.2, capacity=200000)
    assert np.all(out["electrons"][counts == 0] == 0)
    L = w.gas.n_levels
    assert np.array_equal(out["electrons"], counts + out["tallies"][:, L - 1])


def test_primary_outside_volume_retires_at_once(av):
    w = W.plate(n_avalanches=6, seed=4)
    w.primaries.z[:] = [-1e-6, 0.0, 0.0128, 0.02, 0.0, 0.005]
    st, out = run_gpu(av, w, seed=4, t_max=0.05, capacity=1000)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=4, t_max=0.05)
    assert_same_electrons(out, ref, scale_pos=0.0128, scale_t=0.05)
    first = out["status"][:6]
    assert first[0] == W.CATHODE and first[2] == W.ANODE and first[3] == W.ANODE
    assert np.all(out["n_flight"][[0, 2, 3]] == 0)


@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
def test_capacity_overflow_is_reported_and_consistent(av, mode):
    w = W.plate(n_avalanches=8, e_field=45_000.0, seed=6)
    st, out = run_gpu(av, w, seed=6, capacity=200, mode=mode,
                      allow=(A.GT_ERR_QUEUE_OVERFLOW,))
    assert st["status"] == A.GT_ERR_QUEUE_OVERFLOW
    assert st["n_endpoints"] == 200 and st["n_dropped"] > 0
    assert np.all(out["status"] != 0)  # every stored electron finished
    # the context is still usable
    st2, _ = run_gpu(av, w, seed=6, t_max=0.05, capacity=10000)
    assert st2["status"] == A.GT_OK


def test_size_limit_caps_avalanches(av):
    w = W.plate(n_avalanches=16, e_field=45_000.0, seed=7)
    st, out = run_gpu(av, w, seed=7, capacity=2_000_000, size_limit=50)
    assert out["electrons"].max() <= 50
    assert st["n_dropped"] > 0


def test_bounded_wait_gives_up_and_context_survives(av):
    """A queue slot that is reserved but never filled: every worker waits on
    it, gives up after spin_limit_ms and the run returns GT_ERR_TIMEOUT."""
    w = W.plate(n_avalanches=4, seed=8)
    st, out = run_gpu(av, w, seed=8, t_max=0.05, capacity=1000, spin_limit_ms=200.0,
                      debug_flags=A.GT_DEBUG_UNFILLED_SLOT, allow=(A.GT_ERR_TIMEOUT,))
    assert st["status"] == A.GT_ERR_TIMEOUT
    st2, out2 = run_gpu(av, w, seed=8, t_max=0.05, capacity=1000)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=8, t_max=0.05)
    assert_same_electrons(out2, ref, scale_pos=0.0128, scale_t=0.05)


def test_run_time_budget(av):
    w = W.plate(n_avalanches=64, e_field=50_000.0, seed=9)
    st, _ = run_gpu(av, w, seed=9, capacity=4_000_000, time_limit_ms=1.0,
                    allow=(A.GT_ERR_TIMEOUT, A.GT_OK))
    assert st["status"] in (A.GT_ERR_TIMEOUT, A.GT_OK)


def test_invalid_device_avalanche_id_is_rejected(av):
    w = W.plate(n_avalanches=4, seed=10)
    bad = w.primaries.subset([0, 1, 2, 3])
    bad.aval = bad.aval.copy()
    bad.aval[1] = 7
    with pytest.raises(A.GtError) as e:
        run_gpu(av, w, seed=10, prim=bad, t_max=0.05, capacity=100)
    assert e.value.code == A.GT_ERR_ARG


def test_autotune_picks_and_remembers_a_shape(av):
    w = W.plate_batched(n_avalanches=128, seed=11)
    av.set_gas(w.gas)
    av.set_field(w.field)
    p = av.primaries_device(w.primaries)
    opt = A.RunOptions(seed=11, t_max=w.t_max, precision=A.GT_MIXED)
    best, pts = av.autotune(p, opt, capacity=2_000_000)
    # coordinate descent: no shape measured twice, far fewer than the 64 of
    # the full grid, and the best is the fastest shape measured
    shapes = [(q["block"], q["refill_period"], q["flights_per_phase"]) for q in pts]
    assert len(set(shapes)) == len(shapes) and 8 <= len(pts) <= 40
    assert best["real_per_ms"] == max(q["real_per_ms"] for q in pts)
    assert best["block"] in (512, 768, 896, 1024) and best["refill_period"] in (4, 8, 16, 32)
    assert best["flights_per_phase"] in (1, 2, 4, 6)
    # a dimension set in the run stays fixed
    fixed, fpts = av.autotune(p, A.RunOptions(seed=11, t_max=w.t_max, precision=A.GT_MIXED,
                                              block=768), capacity=2_000_000)
    assert fixed["block"] == 768 and all(q["block"] == 768 for q in fpts)
    best, pts = av.autotune(p, opt, capacity=2_000_000)
    st = av.run(p, opt, capacity=2_000_000)
    assert st["block"] == best["block"] and st["refill_period"] == best["refill_period"]
    assert st["flights_per_phase"] == best["flights_per_phase"]
    # the shape does not change the physics: same electrons, same tallies
    _, a = run_gpu(av, w, seed=11, precision=A.GT_FP64, capacity=2_000_000, block=128,
                   refill_period=8, t_max=0.3)
    _, b = run_gpu(av, w, seed=11, precision=A.GT_FP64, capacity=2_000_000, block=512,
                   refill_period=64, t_max=0.3)
    assert np.array_equal(np.sort(a["uid"]), np.sort(b["uid"]))
    assert np.array_equal(a["tallies"], b["tallies"])
    w = W.plate(n_avalanches=8, seed=0)
    av.set_gas(w.gas)
    av.set_field(w.field)


def test_argument_errors(av):
    import ctypes as C
    lib = A.load()
    assert lib.gas_table_upload(av.ctx, None) == A.GT_ERR_ARG
    g = W.argon_like_gas()
    bad = W.Gas(g.level_type, g.threshold, -g.rate, g.d_eps, g.recoil)
    with pytest.raises(A.GtError):
        A.gas_table_upload(av.ctx, bad)
    with pytest.raises(A.GtError):
        A.gas_table_upload(av.ctx, W.Gas(g.level_type, g.threshold, g.rate, g.d_eps, g.recoil,
                                         nu_max=1.0))
    with pytest.raises(A.GtError):
        A.field_setup(av.ctx, W.Field(W.COAX, wire_r=0.5, tube_r=0.1, voltage=1.0))
    # the uniform field needs a time or collision limit
    A.field_setup(av.ctx, W.Field(W.UNIFORM, e0=100.0))
    w = W.drift_model(n_electrons=4, n_coll=0)
    with pytest.raises(A.GtError) as e:
        run_gpu(av, w, seed=0, coll_limit=0, t_max=0.0, capacity=16)
    assert e.value.code == A.GT_ERR_ARG
    # undersized work space
    p = av.primaries_device(w.primaries)
    r = av.make_run(p, A.RunOptions(coll_limit=10))
    av.alloc(16, 4, r)
    o = av.endpoints_struct(16)
    st = A.gt_stats()
    rc = lib.avalanche_run(av.ctx, C.byref(r), C.byref(o), av.ws.data_ptr(), 64, None, C.byref(st))
    assert rc == A.GT_ERR_WORKSPACE
    # restore the plate set-up for the other tests
    w = W.plate(n_avalanches=8, seed=0)
    av.set_gas(w.gas)
    av.set_field(w.field)


def test_graph_replays_equal_runs(av):
    """A captured graph replays the batched run: with the run's seed it
    gives the same electrons and tallies as avalanche_run (FP64, bitwise
    by id), a new seed gives the run with that seed, and the summary and
    status come back through gt_graph_stats."""
    w = W.plate(n_avalanches=64, e_field=40_000.0, seed=111)
    av.set_gas(w.gas)
    av.set_field(w.field)
    p = av.primaries_device(w.primaries)
    cap = 400_000
    opt = A.RunOptions(seed=5, t_max=w.t_max, precision=A.GT_FP64, mode=A.GT_BATCHED)
    ref5 = av.run(p, opt, cap)
    a5 = av.fetch(ref5["n_endpoints"])
    ref6 = av.run(p, A.RunOptions(**{**opt.__dict__, "seed": 6}), cap)
    a6 = av.fetch(ref6["n_endpoints"])
    g = av.graph(p, opt, cap)
    try:
        for seed, st_ref, ref in ((5, ref5, a5), (6, ref6, a6), (5, ref5, a5)):
            g.launch(seed)
            st = g.stats()
            assert st["n_endpoints"] == st_ref["n_endpoints"]
            assert st["real_collisions"] == st_ref["real_collisions"]
            out = av.fetch(st["n_endpoints"])
            assert np.array_equal(out["tallies"], ref["tallies"])
            assert np.array_equal(out["electrons"], ref["electrons"])
            o, r = by_uid(out), by_uid(ref)
            for k in ("x1", "y1", "z1", "t1", "e1", "status"):
                assert np.array_equal(o[k], r[k]), k
    finally:
        g.close()
    with pytest.raises(A.GtError) as e:
        av.graph(av.primaries_pinned(w.primaries), opt, cap)
    assert e.value.code == A.GT_ERR_UNSUPPORTED


def test_graph_refuses_a_replaced_setup(av):
    """A graph holds the gas table and field of the setup it was recorded
    with: after field_setup (or gas_table_upload) replaces them, a replay is
    refused with GT_ERR_STATE instead of reading freed tables; a new graph
    runs."""
    w = W.plate(n_avalanches=8, e_field=40_000.0, seed=113)
    av.set_gas(w.gas)
    av.set_field(w.field)
    p = av.primaries_device(w.primaries)
    opt = A.RunOptions(seed=7, t_max=w.t_max, precision=A.GT_MIXED, mode=A.GT_BATCHED)
    g = av.graph(p, opt, 100_000)
    try:
        g.launch(7)
        g.stats()
        av.set_field(w.field)
        with pytest.raises(A.GtError) as e:
            g.launch(8)
        assert e.value.code == A.GT_ERR_STATE
    finally:
        g.close()
    g = av.graph(p, opt, 100_000)
    try:
        g.launch(8)
        assert g.stats()["n_endpoints"] > 0
    finally:
        g.close()
