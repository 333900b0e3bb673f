"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64: per electron, every start/end coordinate, time and energy within 1e-9
relative, identical status, flight count, electron ids, per-avalanche counts
and collision tallies.  Mixed precision: distributional agreement (mean gain
within 3 sigma, two-sample KS at p > 0.01) with independent seeds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import assert_same_electrons, by_uid, run_gpu, two_sample_ks

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


def _charge(out, L):
    assert np.array_equal(out["electrons"], np.bincount(out["aval"], minlength=len(out["electrons"])))


# --------------------------------------------------------------- FP64 parity
@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
def test_fp64_plate_per_collision(av, mode):
    """Argon-like gas, plate gap, short time limit: identical avalanches."""
    w = W.plate(n_avalanches=48, e_field=45_000.0, seed=21)
    _setup(av, w)
    t_max = 0.35
    ref = oracle.run(w.gas, w.field, w.primaries, seed=21, t_max=t_max)
    st, out = run_gpu(av, w, seed=21, t_max=t_max, mode=mode, capacity=4 * len(ref["uid"]) + 64)
    assert st["n_endpoints"] == len(ref["uid"])
    assert_same_electrons(out, ref, scale_pos=w.field.gap, scale_t=t_max)
    assert np.array_equal(out["electrons"], ref["electrons"])
    assert np.array_equal(out["tallies"], ref["tallies"])
    L = w.gas.n_levels
    assert np.array_equal(out["electrons"], 1 + out["tallies"][:, L - 1])
    assert st["real_collisions"] == int(ref["tallies"][:, :L].sum())
    assert st["null_collisions"] == int(ref["tallies"][:, L].sum())
    assert st["flights"] == int(ref["n_flight"].astype(np.int64).sum())


def test_fp64_drift_model_per_collision(av):
    w = W.drift_model(n_electrons=256, n_coll=3000, seed=4)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=4, coll_limit=w.coll_limit)
    st, out = run_gpu(av, w, seed=4)
    assert_same_electrons(out, ref, scale_pos=1e-3, scale_t=3.0, scale_e=1.0)
    assert np.array_equal(out["tallies"], ref["tallies"])


def test_fp64_crossed_fields_per_collision(av):
    """Uniform E with a transverse B: the exact Lorentz flight on both sides."""
    w = W.drift_model(n_electrons=256, n_coll=3000, b=(3.0, 0.5, 0.0), seed=6)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=6, coll_limit=w.coll_limit)
    st, out = run_gpu(av, w, seed=6)
    assert_same_electrons(out, ref, scale_pos=1e-3, scale_t=3.0)


def test_fp64_coax_axial_b_per_collision(av):
    w = W.coax(n_avalanches=32, r_lo=0.004, r_hi=0.02, seed=8)
    _setup(av, w)
    t_max = 0.4
    ref = oracle.run(w.gas, w.field, w.primaries, seed=8, t_max=t_max)
    st, out = run_gpu(av, w, seed=8, t_max=t_max, capacity=4 * len(ref["uid"]) + 64)
    assert set(np.unique(out["status"])) <= {W.WIRE, W.TUBE, W.TIME}
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=t_max)
    assert np.array_equal(out["tallies"], ref["tallies"])


def test_fp64_grid_map_per_collision(av):
    """Coax-sampled regular map read by trilinear interpolation."""
    f = W.coax_grid_map(n=48, half_width=0.02, length=0.05, voltage=1500.0)
    w = W.grid_stress(n_avalanches=24, n=48, seed=10)
    w.field = f
    rng = np.random.default_rng(1)
    ph = rng.uniform(0, 2 * math.pi, 24)
    w.primaries.x[:] = 0.008 * np.cos(ph)
    w.primaries.y[:] = 0.008 * np.sin(ph)
    w.primaries.z[:] = 0.025
    _setup(av, w)
    t_max = 0.3
    ref = oracle.run(w.gas, w.field, w.primaries, seed=10, t_max=t_max)
    st, out = run_gpu(av, w, seed=10, t_max=t_max, capacity=4 * len(ref["uid"]) + 64)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=t_max)


def test_fp64_batched_equals_plain_bitwise(av):
    """The same device step in both schedules: identical per electron."""
    w = W.plate_batched(n_avalanches=40, seed=12)
    _setup(av, w)
    _, a = run_gpu(av, w, seed=12, t_max=0.3, mode=A.GT_BATCHED, capacity=20000)
    _, b = run_gpu(av, w, seed=12, t_max=0.3, mode=A.GT_PLAIN, capacity=20000)
    ga, gb = by_uid(a), by_uid(b)
    for k in ("uid", "status", "n_flight", "x1", "y1", "z1", "t1", "e1"):
        assert np.array_equal(ga[k], gb[k]), k
    assert np.array_equal(a["tallies"], b["tallies"])


def test_batched_runs_are_reproducible(av):
    w = W.plate_batched(n_avalanches=64, seed=13)
    _setup(av, w)
    _, a = run_gpu(av, w, seed=13, precision=A.GT_MIXED, capacity=4_000_000)
    _, b = run_gpu(av, w, seed=13, precision=A.GT_MIXED, capacity=4_000_000)
    ga, gb = by_uid(a), by_uid(b)
    for k in ("uid", "status", "n_flight", "x1", "z1", "t1", "e1"):
        assert np.array_equal(ga[k], gb[k]), k


def test_fp64_full_avalanches_sampled(av):
    """The 1000-avalanche argon plate at 40 kV/cm (gain ~1e3), FP64 batched
    in one launch; a sample of whole avalanches matches the oracle electron
    by electron."""
    w = W.plate(n_avalanches=1000, e_field=40_000.0, seed=0)
    _setup(av, w)
    st, out = run_gpu(av, w, seed=0, capacity=8_000_000)
    L = w.gas.n_levels
    assert np.array_equal(out["electrons"], 1 + out["tallies"][:, L - 1])
    sample = [0, 17, 256, 511, 998]
    ref = oracle.run(w.gas, w.field, w.primaries.subset(sample), seed=0, t_max=w.t_max)
    keep = np.isin(out["aval"], sample)
    sub = {k: v[keep] for k, v in out.items() if k not in ("electrons", "tallies")}
    assert_same_electrons(sub, ref, scale_pos=w.field.gap, scale_t=1.0)
    assert np.array_equal(out["tallies"][sample], ref["tallies"][sample])


# ----------------------------------------------------- mixed precision: distributions
def test_mixed_plate_distribution(av):
    """Mixed precision (GPU, seed 1) vs the FP64 oracle (seed 0), independent
    samples: mean gain within 3 sigma, KS p > 0.01 on log gain and on the
    transverse position and arrival time of anode electrons."""
    n = 300
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=0)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, t_max=w.t_max)
    st, out = run_gpu(av, w, seed=1, precision=A.GT_MIXED, capacity=4_000_000)
    g_ref = np.bincount(ref["aval"][ref["status"] == W.ANODE], minlength=n).astype(float)
    g_gpu = np.bincount(out["aval"][out["status"] == W.ANODE], minlength=n).astype(float)
    se = math.sqrt(g_ref.var() / n + g_gpu.var() / n)
    assert abs(g_ref.mean() - g_gpu.mean()) < 3 * se, (g_ref.mean(), g_gpu.mean(), se)
    assert two_sample_ks(np.log1p(g_ref), np.log1p(g_gpu)).pvalue > 0.01
    # Electrons of one avalanche are correlated, so the KS tests on endpoint
    # distributions use one value per avalanche: the mean arrival time and the
    # rms transverse spread of its anode electrons.
    for k, f in (("t1", np.mean), ("x1", lambda v: np.sqrt(np.mean(v * v)))):
        ma = np.array([f(ref[k][(ref["aval"] == i) & (ref["status"] == W.ANODE)])
                       for i in range(n) if g_ref[i] > 0])
        mb = np.array([f(out[k][(out["aval"] == i) & (out["status"] == W.ANODE)])
                       for i in range(n) if g_gpu[i] > 0])
        assert two_sample_ks(ma, mb).pvalue > 0.01, k


def test_mixed_drift_model_closed_form_and_oracle(av):
    """Mixed precision on the constant-rate gas: drift velocity and
    transverse spread against the closed forms and against the oracle."""
    from tests import physics as P
    w = W.drift_model(n_electrons=20000, n_coll=10000, seed=31)
    _setup(av, w)
    st, out = run_gpu(av, w, seed=31, precision=A.GT_MIXED, capacity=20000)
    dz, dt = out["z1"] - out["z0"], out["t1"] - out["t0"]
    vd = P.drift_velocity(1000.0, 1000.0)
    se = np.std(dz - vd * dt) / math.sqrt(len(dz)) / dt.mean()
    assert abs(dz.mean() / dt.mean() - vd) < 3 * se
    xs = np.concatenate([out["x1"] - out["x0"], out["y1"] - out["y0"]]) ** 2
    ex = P.transverse_msd(1000.0, 1000.0, 10000, 0.1)
    assert abs(xs.mean() - ex) < 3 * xs.std() / math.sqrt(len(xs) / 2)
    # energy = field work per electron (no loss), to FP32 accumulation accuracy
    assert np.allclose(out["e1"], out["e0"] + 1000.0 * dz, rtol=1e-4, atol=1e-3)


def test_mixed_coax_b_distribution(av):
    """Coax with axial B, mixed vs FP64 oracle: gain and arrival times."""
    n = 96
    w = W.coax(n_avalanches=n, r_lo=0.02, r_hi=0.05, seed=0)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, t_max=w.t_max)
    st, out = run_gpu(av, w, seed=1, precision=A.GT_MIXED, capacity=4_000_000)
    g_ref = np.bincount(ref["aval"][ref["status"] == W.WIRE], minlength=n).astype(float)
    g_gpu = np.bincount(out["aval"][out["status"] == W.WIRE], minlength=n).astype(float)
    se = math.sqrt(g_ref.var() / n + g_gpu.var() / n)
    assert abs(g_ref.mean() - g_gpu.mean()) < 3 * se, (g_ref.mean(), g_gpu.mean(), se)
    assert two_sample_ks(np.log1p(g_ref), np.log1p(g_gpu)).pvalue > 0.01
    tr = np.array([ref["t1"][(ref["aval"] == i) & (ref["status"] == W.WIRE)].min()
                   for i in range(n) if g_ref[i] > 0])
    tg = np.array([out["t1"][(out["aval"] == i) & (out["status"] == W.WIRE)].min()
                   for i in range(n) if g_gpu[i] > 0])
    assert two_sample_ks(tr, tg).pvalue > 0.01


# ------------------------------------------------------------- observables
def test_observables_kernel_matches_numpy(av):
    w = W.plate(n_avalanches=200, e_field=40_000.0, seed=5)
    _setup(av, w)
    st, out = run_gpu(av, w, seed=5, precision=A.GT_MIXED, capacity=2_000_000)
    obs = av.observables(st["n_endpoints"], w.primaries, collect_status=W.ANODE,
                         drift_status=W.ANODE, gap=w.field.gap)
    g = np.bincount(out["aval"][out["status"] == W.ANODE], minlength=200).astype(float)
    assert obs[0] == pytest.approx(g.mean(), rel=1e-12)
    assert obs[1] == pytest.approx(g.std(ddof=1) / math.sqrt(200), rel=1e-9)
    m = out["status"] == W.ANODE
    dz, dt = (out["z1"] - out["z0"])[m], (out["t1"] - out["t0"])[m]
    tr = ((out["x1"] - out["x0"]) ** 2 + (out["y1"] - out["y0"]) ** 2)[m]
    assert obs[3] == pytest.approx(dz.sum() / dt.sum(), rel=1e-9)
    assert obs[4] == pytest.approx(tr.mean() / (4 * dt.mean()), rel=1e-9)
    assert obs[5] == pytest.approx(dz.var(ddof=1) / (2 * dt.mean()), rel=1e-6)
    assert obs[6] == m.sum()
    assert obs[7] == pytest.approx(math.log(g.mean()) / w.field.gap, rel=1e-12)


# ------------------------------------------------ banded majorant (next row f1)
BANDED = dict(majorant=A.GT_MAJORANT_BANDED, majorant_window=2.0)


@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
def test_fp64_banded_plate_per_collision(av, mode):
    """Banded majorant, FP64: identical to the oracle's banded transport."""
    w = W.plate(n_avalanches=48, e_field=45_000.0, seed=41)
    _setup(av, w)
    t_max = 0.35
    ref = oracle.run(w.gas, w.field, w.primaries, seed=41, t_max=t_max, majorant=1, window=2.0,
                     band_width=1.0)
    st, out = run_gpu(av, w, seed=41, t_max=t_max, mode=mode, capacity=4 * len(ref["uid"]) + 64,
                      **BANDED)
    assert_same_electrons(out, ref, scale_pos=w.field.gap, scale_t=t_max)
    assert np.array_equal(out["tallies"], ref["tallies"])
    assert st["flights"] == int(ref["n_flight"].astype(np.int64).sum())


def test_fp64_banded_coax_b_and_grid_per_collision(av):
    w = W.coax(n_avalanches=24, r_lo=0.004, r_hi=0.02, seed=43)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=43, t_max=0.4, majorant=1, window=2.0)
    _, out = run_gpu(av, w, seed=43, t_max=0.4, capacity=4 * len(ref["uid"]) + 64, **BANDED)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=0.4)
    f = W.coax_grid_map(n=48, half_width=0.02, length=0.05, voltage=1500.0)
    w = W.grid_stress(n_avalanches=16, n=48, seed=44)
    w.field = f
    ph = np.random.default_rng(2).uniform(0, 2 * math.pi, 16)
    w.primaries.x[:] = 0.008 * np.cos(ph)
    w.primaries.y[:] = 0.008 * np.sin(ph)
    w.primaries.z[:] = 0.025
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=44, t_max=0.3, majorant=1, window=2.0)
    _, out = run_gpu(av, w, seed=44, t_max=0.3, capacity=4 * len(ref["uid"]) + 64, **BANDED)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=0.3)


def test_mixed_banded_matches_global_oracle(av):
    """Exactness across methods: GPU mixed precision with the banded
    majorant against the FP64 oracle with the global nu_max (independent
    seeds): gain (3 sigma, KS), arrival times (KS), collision mix."""
    n = 300
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=0)
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, t_max=w.t_max)
    st, out = run_gpu(av, w, seed=5, precision=A.GT_MIXED, capacity=4_000_000, **BANDED)
    g_ref = np.bincount(ref["aval"][ref["status"] == W.ANODE], minlength=n).astype(float)
    g_gpu = np.bincount(out["aval"][out["status"] == W.ANODE], minlength=n).astype(float)
    se = math.sqrt(g_ref.var() / n + g_gpu.var() / n)
    assert abs(g_ref.mean() - g_gpu.mean()) < 3 * se, (g_ref.mean(), g_gpu.mean(), se)
    assert two_sample_ks(np.log1p(g_ref), np.log1p(g_gpu)).pvalue > 0.01
    ma = np.array([ref["t1"][(ref["aval"] == i) & (ref["status"] == W.ANODE)].mean()
                   for i in range(n) if g_ref[i] > 0])
    mb = np.array([out["t1"][(out["aval"] == i) & (out["status"] == W.ANODE)].mean()
                   for i in range(n) if g_gpu[i] > 0])
    assert two_sample_ks(ma, mb).pvalue > 0.01
    L = w.gas.n_levels
    fa = ref["tallies"][:, :L].sum(0) / ref["tallies"][:, :L].sum()
    fb = out["tallies"][:, :L].sum(0) / out["tallies"][:, :L].sum()
    assert np.allclose(fa, fb, atol=0.005)
    # far fewer flights per real collision than the global majorant
    assert st["real_collisions"] / st["flights"] > 0.4


def test_mixed_banded_drift_closed_form(av):
    from tests import physics as P
    w = W.drift_model(n_electrons=20000, n_coll=10000, seed=33)
    w.gas = W.model_gas(1000.0, exact_nu_max=False)
    _setup(av, w)
    st, out = run_gpu(av, w, seed=33, precision=A.GT_MIXED, capacity=20000, **BANDED)
    dz, dt = out["z1"] - out["z0"], out["t1"] - out["t0"]
    vd = P.drift_velocity(1000.0, 1000.0)
    se = np.std(dz - vd * dt) / math.sqrt(len(dz)) / dt.mean()
    assert abs(dz.mean() / dt.mean() - vd) < 3 * se
    assert np.allclose(out["e1"], out["e0"] + 1000.0 * dz, rtol=1e-4, atol=1e-3)


@pytest.mark.parametrize("precision", [A.GT_FP64, A.GT_MIXED])
@pytest.mark.parametrize("majorant,band_width,window",
                         [(A.GT_MAJORANT_GLOBAL, 1.0, 2.0), (A.GT_MAJORANT_BANDED, 1.0, 2.0),
                          (A.GT_MAJORANT_BANDED, 0.1, 0.5)])
def test_ramp_first_collision_closed_form(av, precision, majorant, band_width, window):
    """Rate linear in energy (a rising rate is where an unsafe majorant
    shows): the first real collision times follow the closed-form survival
    (KS of the probability integral transform); in FP64 the run is also
    identical to the oracle's electron by electron."""
    from scipy import stats
    from tests.test_oracle_pins import ramp_pit, ramp_workload
    w, c = ramp_workload(40000, 37, band_width)
    _setup(av, w)
    st, out = run_gpu(av, w, seed=37, precision=precision, capacity=40000, majorant=majorant,
                      majorant_window=window)
    assert np.all(out["status"] == W.COLL_LIMIT)
    assert stats.kstest(ramp_pit(out, w, c), "uniform").pvalue > 0.01
    if precision == A.GT_FP64:
        ref = oracle.run(w.gas, w.field, w.primaries, seed=37, coll_limit=1,
                         majorant=int(majorant == A.GT_MAJORANT_BANDED), window=window,
                         band_width=band_width)
        assert_same_electrons(out, ref, scale_pos=1e-3, scale_t=0.05, scale_e=1.0)


def test_banded_zero_rate_bands(av):
    """Bands whose rates are all zero (no collisions below 5 eV) take the
    tiny positive bound, so windows stay finite: FP64 identical to the
    oracle, mixed precision finite and complete."""
    from tests.test_oracle_pins import ramp_workload
    w, _ = ramp_workload(4000, 39, 1.0)
    eps = np.arange(w.gas.n_nodes, dtype=np.float64) * w.gas.d_eps
    w.gas.rate[:, 0] = 34.0 * np.maximum(eps - 5.0, 0.0)
    w.coll_limit = 3
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=39, coll_limit=3, majorant=1, window=2.0,
                     band_width=1.0)
    _, out = run_gpu(av, w, seed=39, capacity=4000, **BANDED)
    assert_same_electrons(out, ref, scale_pos=1e-3, scale_t=0.05)
    _, out = run_gpu(av, w, seed=39, precision=A.GT_MIXED, capacity=4000, **BANDED)
    assert np.all(out["status"] == W.COLL_LIMIT)
    for k in ("x1", "y1", "z1", "t1", "e1"):
        assert np.all(np.isfinite(out[k]))
