"""GPU parity for induced signals (Shockley-Ramo): FP64 per avalanche and
bin against the oracle; mixed precision against the closed forms the
oracle is pinned to."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests import physics as P
from tests.gpu_helpers import run_gpu
from tests.test_oracle_pins import _collisionless

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


def _sig(kind, bins, t0, dt):
    return dict(signal_kind=kind, signal_bins=bins, signal_t0=t0, signal_dt=dt)


@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
@pytest.mark.parametrize("crossing", [0, 1])
def test_fp64_plate_signal_per_bin(av, mode, crossing):
    n = 40
    w = W.plate(n_avalanches=n, e_field=45_000.0, seed=101)
    _setup(av, w)
    t_max, sig = 0.4, (W.W_PLATE, 200, 0.0, 0.002)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=101, t_max=t_max, crossing=bool(crossing),
                     signal=sig)
    _, out = run_gpu(av, w, seed=101, t_max=t_max, mode=mode, crossing=crossing,
                     capacity=4 * len(ref["uid"]) + 64, **_sig(*sig))
    scale = np.abs(ref["signal"]).max()
    assert np.allclose(out["signal"], ref["signal"], rtol=1e-9, atol=1e-9 * scale)


@pytest.mark.parametrize("case", ["coax_b", "grid_map"])
def test_fp64_wire_signal_per_bin(av, case):
    if case == "coax_b":
        w = W.coax(n_avalanches=24, r_lo=0.004, r_hi=0.02, seed=103)
        sig, kw = (W.W_COAX, 100, 0.0, 0.003), dict(substeps=2, crossing=True)
    else:
        f = W.coax_grid_map(n=48, half_width=0.02, length=0.05, voltage=1500.0)
        w = W.grid_stress(n_avalanches=16, n=48, seed=105)
        w.field = f
        ph = np.random.default_rng(3).uniform(0, 2 * math.pi, 16)
        w.primaries.x[:] = 0.008 * np.cos(ph)
        w.primaries.y[:] = 0.008 * np.sin(ph)
        w.primaries.z[:] = 0.025
        sig, kw = (W.W_MAP, 100, 0.0, 0.003), dict()
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=w.seed, t_max=0.3, signal=sig, **kw)
    _, out = run_gpu(av, w, seed=w.seed, t_max=0.3, capacity=4 * len(ref["uid"]) + 64,
                     substeps=kw.get("substeps", 0), crossing=int(kw.get("crossing", False)),
                     **_sig(*sig))
    scale = np.abs(ref["signal"]).max()
    assert np.allclose(out["signal"], ref["signal"], rtol=1e-9, atol=1e-9 * scale)


def test_mixed_signal_telescopes(av):
    n = 200
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=107)
    _setup(av, w)
    _, o = run_gpu(av, w, seed=107, precision=A.GT_MIXED, t_max=w.t_max, capacity=4_000_000,
                   majorant=A.GT_MAJORANT_BANDED, majorant_window=2.0,
                   **_sig(W.W_PLATE, 400, 0.0, 0.005))
    per_e = (o["z1"] - o["z0"]) / w.field.gap
    expect = np.bincount(o["aval"], weights=per_e, minlength=n)
    assert np.allclose(o["signal"].sum(axis=1), expect, rtol=1e-5, atol=1e-3)


def test_mixed_signal_bins_of_a_uniform_acceleration(av):
    w = _collisionless(50, 30_000.0, 93)
    a = P.ACCEL_PER_VCM * 30_000.0
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    tr = 0.0052
    w.primaries.t[:] = tr
    ts = tr + (np.sqrt(vz * vz + 2 * a * w.field.gap) - vz) / a
    t0, dt, nb = 0.001, 0.003, 9
    _setup(av, w)
    _, o = run_gpu(av, w, seed=93, precision=A.GT_MIXED, t_max=100.0, crossing=1, capacity=50,
                   **_sig(W.W_PLATE, nb, t0, dt))
    edges = t0 + dt * np.arange(nb + 1)
    for i in range(50):  # avalanche i is primary i
        te = np.clip(edges, tr, ts[i]) - tr
        z = np.where(edges < ts[i], vz[i] * te + 0.5 * a * te * te, w.field.gap)
        assert np.allclose(o["signal"][i], np.diff(z) / w.field.gap, rtol=1e-4, atol=1e-5), i


def test_mixed_signal_drift_current(av):
    n, nu, e_field, gap = 20000, 1000.0, 1000.0, 100.0
    w = W.drift_model(n_electrons=n, n_coll=0, e_field=e_field, seed=95)
    w.field = W.Field(W.PLATE, e0=e_field, gap=gap)
    w.primaries.z[:] = 1.0
    dt, nb = 0.5, 10
    _setup(av, w)
    _, o = run_gpu(av, w, seed=95, precision=A.GT_MIXED, t_max=nb * dt, capacity=n,
                   **_sig(W.W_PLATE, nb, 0.0, dt))
    s = o["signal"][:, 1:]
    vd = P.drift_velocity(e_field, nu)
    for k in range(s.shape[1]):
        assert abs(s[:, k].mean() - vd * dt / gap) < 3 * s[:, k].std() / math.sqrt(n)
