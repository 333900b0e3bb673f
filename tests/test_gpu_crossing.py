"""GPU parity for exact boundary crossings and field re-evaluation in
sub-steps: FP64 electron by electron against the oracle; mixed precision
against the closed forms the oracle is pinned to and against the oracle's
distributions."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests import physics as P
from tests.gpu_helpers import assert_same_electrons, by_uid, run_gpu, two_sample_ks
from tests.test_oracle_pins import _coax_potential, _collisionless

pytestmark = pytest.mark.gpu


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


def _setup(av, w):
    av.set_gas(w.gas)
    av.set_field(w.field)


def _exit_return_workload(n=400):
    w = _collisionless(n, 30_000.0, 69)
    w.primaries.z[:] = 1e-4
    w.primaries.dz[:] = -np.abs(w.primaries.dz)
    w.primaries.e[:] = np.random.default_rng(5).uniform(1.0, 20.0, n)
    return w


@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
def test_fp64_crossings_collisionless(av, mode):
    for w in (_collisionless(200, 30_000.0, 67), _exit_return_workload()):
        _setup(av, w)
        ref = oracle.run(w.gas, w.field, w.primaries, seed=w.seed, t_max=100.0, crossing=True)
        _, out = run_gpu(av, w, seed=w.seed, t_max=100.0, mode=mode, crossing=1,
                         capacity=len(ref["uid"]))
        assert_same_electrons(out, ref, scale_pos=w.field.gap, scale_t=1.0)


@pytest.mark.parametrize("majorant", [A.GT_MAJORANT_GLOBAL, A.GT_MAJORANT_BANDED])
def test_fp64_coax_substeps_and_crossing(av, majorant):
    w = W.coax(n_avalanches=100, r_lo=0.004, r_hi=0.02, b_axial=0.0, seed=71)
    w.gas = W.model_gas(1e-9)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=71, t_max=0.05, substeps=128,
                     crossing=True, majorant=int(majorant == A.GT_MAJORANT_BANDED))
    _, out = run_gpu(av, w, seed=71, t_max=0.05, substeps=128, crossing=1, majorant=majorant,
                     majorant_window=2.0, capacity=100)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=0.05)


@pytest.mark.parametrize("case", ["plate", "coax_b"])
def test_fp64_collisional_with_crossing_and_substeps(av, case):
    if case == "plate":
        w = W.plate(n_avalanches=40, e_field=45_000.0, seed=81)
        kw, t_max, scale = dict(crossing=True), 0.3, w.field.gap
    else:
        w = W.coax(n_avalanches=24, r_lo=0.004, r_hi=0.02, seed=83)
        kw, t_max, scale = dict(crossing=True, substeps=4), 0.2, 0.01
    _setup(av, w)
    for mj in (0, 1):
        ref = oracle.run(w.gas, w.field, w.primaries, seed=w.seed, t_max=t_max, majorant=mj,
                         window=2.0, **kw)
        _, out = run_gpu(av, w, seed=w.seed, t_max=t_max, majorant=mj, majorant_window=2.0,
                         capacity=4 * len(ref["uid"]) + 64,
                         crossing=1, substeps=kw.get("substeps", 0))
        assert_same_electrons(out, ref, scale_pos=scale, scale_t=t_max)
        assert np.array_equal(out["tallies"], ref["tallies"])


def test_mixed_crossing_closed_forms(av):
    """Mixed precision: the anode arrival time of the collisionless plate
    and the cathode touches decided by vz^2 > 2 a z0 (away from the
    threshold), at the analytic times."""
    w = _collisionless(200, 30_000.0, 67)
    _setup(av, w)
    a = P.ACCEL_PER_VCM * 30_000.0
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    ts = (np.sqrt(vz * vz + 2 * a * w.field.gap) - vz) / a
    _, o = run_gpu(av, w, seed=67, t_max=100.0, precision=A.GT_MIXED, crossing=1, capacity=200)
    o = by_uid(o)
    assert np.all(o["status"] == W.ANODE)
    assert np.allclose(o["t1"] - o["t0"], ts, rtol=1e-5)
    # the crossing is searched in FP32 offsets: on the anode to FP32 rounding
    # of the flight's displacement (1e-6 of 0.0128 cm and the time resolution)
    assert np.all(np.abs(o["z1"] - w.field.gap) < 1e-7)
    w = _exit_return_workload()
    _setup(av, w)
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    margin = vz * vz / (2 * a * 1e-4) - 1.0
    clear = np.abs(margin) > 1e-3
    _, o = run_gpu(av, w, seed=69, t_max=100.0, precision=A.GT_MIXED, crossing=1, capacity=400)
    o = by_uid(o)
    hits = margin > 0
    assert np.array_equal((o["status"] == W.CATHODE)[clear], hits[clear])
    h = hits & clear
    tsc = (-vz[h] - np.sqrt(vz[h] ** 2 - 2 * a * 1e-4)) / a
    assert np.allclose(o["t1"][h] - o["t0"][h], tsc, rtol=1e-4)


def test_mixed_substeps_converge(av):
    w = W.coax(n_avalanches=100, r_lo=0.004, r_hi=0.02, b_axial=0.0, seed=71)
    w.gas = W.model_gas(1e-9)
    _setup(av, w)
    errs = []
    for n in (32, 128, 512):
        _, o = run_gpu(av, w, seed=71, t_max=0.05, substeps=n, crossing=1,
                       precision=A.GT_MIXED, capacity=100)
        assert np.all(o["status"] == W.WIRE)
        r0, r1 = np.hypot(o["x0"], o["y0"]), np.hypot(o["x1"], o["y1"])
        gain = _coax_potential(w.field, r1) - _coax_potential(w.field, r0)
        errs.append(np.abs((o["e1"] - o["e0"]) - gain).max() / gain.max())
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 2.5, errs
    assert errs[2] < 2e-2


def test_mixed_plate_with_crossing_matches_oracle(av):
    n = 300
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=85)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=85, t_max=w.t_max, crossing=True)
    _, out = run_gpu(av, w, seed=86, precision=A.GT_MIXED, crossing=1, capacity=4_000_000,
                     majorant=A.GT_MAJORANT_BANDED, majorant_window=2.0)
    ga = np.bincount(ref["aval"][ref["status"] == W.ANODE], minlength=n).astype(float)
    gb = np.bincount(out["aval"][out["status"] == W.ANODE], minlength=n).astype(float)
    se = math.sqrt(ga.var() / n + gb.var() / n)
    assert abs(ga.mean() - gb.mean()) < 3 * se
    assert two_sample_ks(np.log1p(ga), np.log1p(gb)).pvalue > 0.01
    an = out["status"] == W.ANODE
    assert np.all(np.abs(out["z1"][an] - w.field.gap) < 1e-7)
