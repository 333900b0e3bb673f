"""The configurations at their full sizes, in the launch configuration the
benchmark times (batched, mixed precision, banded majorant, autotuned
shape, captured-graph replay): invariants that hold at any size on every
electron, FP64 electron-by-electron parity on sampled whole avalanches, and
the mixed-precision gain of sampled avalanches against the oracle's."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import assert_same_electrons, two_sample_ks

pytestmark = pytest.mark.gpu

BANDED = dict(majorant=A.GT_MAJORANT_BANDED, majorant_window=2.0)


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


def _invariants(out, w, boundary_ok):
    """Charge (electrons = primaries + ionisations, per avalanche), unique
    ids, statuses, times and energies of every electron."""
    n_aval = w.primaries.n_avalanches
    L = w.gas.n_levels
    ion = [j for j in range(L) if w.gas.level_type[j] == W.IONISATION][0]
    n_prim = np.bincount(w.primaries.aval, minlength=n_aval)
    assert np.array_equal(out["electrons"], n_prim + out["tallies"][:, ion])
    assert np.array_equal(np.bincount(out["aval"], minlength=n_aval), out["electrons"])
    assert len(np.unique(out["uid"])) == len(out["uid"])
    assert np.all(out["status"] > 0)
    assert np.all(out["t1"] >= out["t0"]) and np.all(out["t1"] <= w.t_max * (1 + 1e-12))
    assert np.all(out["e1"] >= 0.0) and np.all(np.isfinite(out["e1"]))
    assert boundary_ok(out)


def _run_graph(av, w, seed, capacity, precision=A.GT_MIXED, tune=True):
    av.set_gas(w.gas)
    av.set_field(w.field)
    p = av.primaries_device(w.primaries)
    opt = A.RunOptions(seed=seed, t_max=w.t_max, precision=precision, mode=A.GT_BATCHED,
                       **BANDED)
    if tune and precision == A.GT_MIXED:
        sample = w.primaries.subset(list(range(min(512, w.primaries.n_avalanches))))
        av.autotune(av.primaries_device(sample), opt, capacity)
    g = av.graph(p, opt, capacity)
    try:
        g.launch(seed)
        st = g.stats(allow=(A.GT_OK,))
    finally:
        g.close()
    return st, av.fetch(st["n_endpoints"])


def _gain_vs_oracle(out, w, sample, status, seed_ref):
    ref = oracle.run(w.gas, w.field, w.primaries.subset(sample), seed=seed_ref, t_max=w.t_max,
                     majorant=1, window=2.0)
    n = len(sample)
    g_ref = np.bincount(ref["aval"][ref["status"] == status], minlength=w.primaries.n_avalanches)
    g_gpu = np.bincount(out["aval"][out["status"] == status], minlength=w.primaries.n_avalanches)
    n_prim = np.bincount(w.primaries.aval, minlength=w.primaries.n_avalanches)
    keep = np.array([a for a in sample if n_prim[a] > 0])
    a, b = g_ref[keep].astype(float), g_gpu[keep].astype(float)
    se = math.sqrt(a.var() / len(keep) + b.var() / len(keep))
    assert abs(a.mean() - b.mean()) < 3 * se, (a.mean(), b.mean(), se)
    assert two_sample_ks(np.log1p(a), np.log1p(b)).pvalue > 0.01
    return n


def test_plate_batched_4096_full_size(av):
    """The benchmark's workload itself: 4096 avalanches, per-avalanche field
    U(30, 50) kV/cm, Poisson(3) primaries."""
    w = W.plate_batched(n_avalanches=4096, seed=0)
    gap = w.field.gap
    st, out = _run_graph(av, w, seed=0, capacity=100_000_000)
    assert st["n_endpoints"] > 1e7
    _invariants(out, w, lambda o: np.all(o["z1"][o["status"] == W.ANODE] >= gap) and
                np.all(o["z1"][o["status"] == W.CATHODE] < 0.0))
    sample = list(range(0, 4096, 32))  # 128 avalanches
    _gain_vs_oracle(out, w, sample, W.ANODE, seed_ref=7)


def test_plate_batched_4096_fp64_sampled_per_electron(av):
    w = W.plate_batched(n_avalanches=4096, seed=0)
    _, out = _run_graph(av, w, seed=3, capacity=100_000_000, precision=A.GT_FP64)
    sample = [0, 1000, 2047, 4095]
    ref = oracle.run(w.gas, w.field, w.primaries.subset(sample), seed=3, t_max=w.t_max,
                     majorant=1, window=2.0)
    keep = np.isin(out["aval"], sample)
    sub = {k: v[keep] for k, v in out.items() if k not in ("electrons", "tallies")}
    assert_same_electrons(sub, ref, scale_pos=w.field.gap, scale_t=1.0)
    assert np.array_equal(out["tallies"][sample], ref["tallies"][sample])


def test_coax_b_2048_full_size(av):
    w = W.coax(n_avalanches=2048, seed=0)
    a2, b2 = w.field.wire_r ** 2, w.field.tube_r ** 2
    # each primary drifts ~1e6 flights in one thread before it multiplies: a
    # run lasts as long as its longest chain, so the autotuner is skipped
    _, out = _run_graph(av, w, seed=0, capacity=60_000_000, tune=False)

    def ok(o):
        r2 = o["x1"] ** 2 + o["y1"] ** 2
        return (np.all(r2[o["status"] == W.WIRE] <= a2) and
                np.all(r2[o["status"] == W.TUBE] >= b2))
    _invariants(out, w, ok)
    # (the coax's long drift makes the oracle slow: a sample of 24 avalanches)
    _gain_vs_oracle(out, w, list(range(0, 2048, 86)), W.WIRE, seed_ref=11)


def test_grid_stress_256_full_size(av):
    """The 256^3 coax-sampled map at the gain-1e5 voltage, 256 avalanches."""
    w = W.grid_stress(n_avalanches=256, seed=0)
    st, out = _run_graph(av, w, seed=0, capacity=60_000_000)
    assert st["n_endpoints"] > 5e6
    a2 = w.field.wire_r ** 2
    _invariants(out, w, lambda o: np.all((o["x1"] ** 2 + o["y1"] ** 2)[o["status"] == W.WIRE]
                                         <= a2))
    g = np.bincount(out["aval"][out["status"] == W.WIRE], minlength=256)
    assert 4e4 < g.mean() < 2.5e5  # the map's voltage gives a mean gain near 1e5
    _gain_vs_oracle(out, w, list(range(0, 256, 8)), W.WIRE, seed_ref=13)
