"""GPU parity for attachment, screened-Coulomb anisotropic scattering and
Opal-Peterson-Beaty ionisation sharing: FP64 electron by electron against
the oracle, mixed precision against the oracle's distributions and the
closed forms of the model gases."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests import physics as P
from tests.gpu_helpers import assert_same_electrons, run_gpu, two_sample_ks

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


@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
@pytest.mark.parametrize("majorant", [A.GT_MAJORANT_GLOBAL, A.GT_MAJORANT_BANDED])
def test_fp64_physical_gas_per_collision(av, mode, majorant):
    """With anisotropic scattering the direction after a collision depends on
    the one before, so rounding differences grow from collision to collision
    (about 3 % per collision between two builds of the oracle); the
    electron-by-electron comparison therefore covers short trajectories
    (0.05 ns, up to ~1100 flights), started at 15.3 eV (off the band edges)
    so that ionisation and attachment happen within them."""
    w = W.plate(n_avalanches=400, e_field=45_000.0, seed=71)
    w.gas = W.argon_like_physical_gas()
    w.primaries.e[:] = 15.3
    _setup(av, w)
    t_max = 0.05
    ref = oracle.run(w.gas, w.field, w.primaries, seed=71, t_max=t_max,
                     majorant=int(majorant == A.GT_MAJORANT_BANDED), window=2.0)
    st, out = run_gpu(av, w, seed=71, t_max=t_max, mode=mode, capacity=4 * len(ref["uid"]) + 64,
                      majorant=majorant, majorant_window=2.0)
    assert_same_electrons(out, ref, scale_pos=w.field.gap, scale_t=t_max)
    assert np.array_equal(out["tallies"], ref["tallies"])
    assert (ref["status"] == W.ATTACHED).any()


def test_fp64_physical_gas_coax_b(av):
    w = W.coax(n_avalanches=64, r_lo=0.004, r_hi=0.02, seed=73)
    w.gas = W.argon_like_physical_gas()
    w.primaries.e[:] = 15.3
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=73, t_max=0.05, majorant=1, window=2.0)
    _, out = run_gpu(av, w, seed=73, t_max=0.05, capacity=4 * len(ref["uid"]) + 64,
                     majorant=A.GT_MAJORANT_BANDED, majorant_window=2.0)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=0.05)
    assert (ref["status"] == W.ATTACHED).any()


def test_mixed_physical_gas_distributions(av):
    """Mixed precision, banded majorant, against the FP64 oracle with the
    global nu_max (independent seeds): gain (3 sigma, KS), attached electrons
    per avalanche (3 sigma), arrival times (KS), collision mix."""
    n = 300
    w = W.plate(n_avalanches=n, e_field=45_000.0, seed=1)
    w.gas = W.argon_like_physical_gas()
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=1, t_max=w.t_max)
    _, out = run_gpu(av, w, seed=9, precision=A.GT_MIXED, capacity=4_000_000,
                     majorant=A.GT_MAJORANT_BANDED, majorant_window=2.0)
    for status in (W.ANODE, W.ATTACHED):
        a = np.bincount(ref["aval"][ref["status"] == status], minlength=n).astype(float)
        b = np.bincount(out["aval"][out["status"] == status], minlength=n).astype(float)
        se = math.sqrt(a.var() / n + b.var() / n)
        assert abs(a.mean() - b.mean()) < 3 * se, (status, a.mean(), b.mean(), se)
        if status == W.ANODE:
            assert two_sample_ks(np.log1p(a), np.log1p(b)).pvalue > 0.01
    L = w.gas.n_levels
    fa = ref["tallies"][:, :L].sum(0) / ref["tallies"][:, :L].sum()
    fb = out["tallies"][:, :L].sum(0) / out["tallies"][:, :L].sum()
    assert np.allclose(fa, fb, atol=0.005)
    # arrival times: one mean per avalanche (electrons of an avalanche are
    # correlated, avalanches are independent)
    ga = np.bincount(ref["aval"][ref["status"] == W.ANODE], minlength=n)
    gb = np.bincount(out["aval"][out["status"] == W.ANODE], minlength=n)
    ta = np.bincount(ref["aval"][ref["status"] == W.ANODE],
                     weights=ref["t1"][ref["status"] == W.ANODE], minlength=n)
    tb = np.bincount(out["aval"][out["status"] == W.ANODE],
                     weights=out["t1"][out["status"] == W.ANODE], minlength=n)
    assert two_sample_ks(ta[ga > 0] / ga[ga > 0], tb[gb > 0] / gb[gb > 0]).pvalue > 0.01


@pytest.mark.parametrize("precision", [A.GT_FP64, A.GT_MIXED])
def test_anisotropic_drift_closed_form(av, precision):
    xi = 0.6
    w = W.drift_model(n_electrons=20000, n_coll=3000, seed=53)
    w.gas = W.model_gas(1000.0, xi_elastic=xi)
    _setup(av, w)
    _, out = run_gpu(av, w, seed=53, precision=precision, capacity=20000)
    g = P.screened_coulomb_mean_cos(xi)
    dz, dt = out["z1"] - out["z0"], out["t1"] - out["t0"]
    vd = P.drift_velocity(1000.0, 1000.0 * (1.0 - g))
    se = np.std(dz - vd * dt) / math.sqrt(len(dz)) / dt.mean()
    assert abs(dz.mean() / dt.mean() - vd) < 3 * se
    rtol, atol = (1e-9, 1e-9) if precision == A.GT_FP64 else (1e-4, 1e-3)
    assert np.allclose(out["e1"], out["e0"] + 1000.0 * dz, rtol=rtol, atol=atol)


@pytest.mark.parametrize("precision", [A.GT_FP64, A.GT_MIXED])
def test_screened_diffusion_closed_form(av, precision):
    eps0, screen, N, n = 10.0, 5.0, 40, 20000
    w = W.drift_model(n_electrons=n, n_coll=N, e_field=0.0, seed=65)
    w.gas = W.model_gas(1000.0)
    w.gas.screen = np.array([screen])
    w.primaries.e[:] = eps0
    _setup(av, w)
    _, out = run_gpu(av, w, seed=65, precision=precision, capacity=n)
    r2 = (out["x1"] - out["x0"]) ** 2 + (out["y1"] - out["y0"]) ** 2 + (out["z1"] - out["z0"]) ** 2
    g = P.screened_coulomb_mean_cos(eps0 / (eps0 + screen))
    k = np.arange(1, N)
    expect = P.speed_sq(eps0) / 1000.0 ** 2 * (2 * N + 2 * np.sum((N - k) * g ** k))
    assert abs(r2.mean() - expect) < 3 * r2.std() / math.sqrt(n)
    assert np.allclose(out["e1"], eps0, rtol=1e-9 if precision == A.GT_FP64 else 1e-5)


@pytest.mark.parametrize("precision", [A.GT_FP64, A.GT_MIXED])
def test_birth_death_and_capture(av, precision):
    from scipy import stats
    lam, mu, T, n = 10.0, 4.0, 0.4, 3000
    w = W.drift_model(n_electrons=n, n_coll=0, e_field=100.0, seed=59)
    w.gas = W.model_gas(1000.0, nu_ion=lam, ion_threshold=0.0, nu_att=mu)
    _setup(av, w)
    _, out = run_gpu(av, w, seed=59, precision=precision, t_max=T, capacity=400_000)
    alive = np.bincount(out["aval"][out["status"] == W.TIME], minlength=n).astype(float)
    mean, p0 = P.birth_death(lam, mu, T)
    assert abs(alive.mean() - mean) < 3 * alive.std() / math.sqrt(n)
    assert abs((alive == 0).mean() - p0) < 3 * math.sqrt(p0 * (1 - p0) / n)
    assert set(np.unique(out["status"])) <= {W.TIME, W.ATTACHED}
    # capture times of the primaries (ids < n) that were captured: Exp(mu)
    # truncated at T
    prim = (out["uid"] < n) & (out["status"] == W.ATTACHED)
    tc = out["t1"][prim] - out["t0"][prim]
    cdf = lambda x: (1 - np.exp(-mu * x)) / (1 - math.exp(-mu * T))  # noqa: E731
    assert stats.kstest(tc, cdf).pvalue > 0.01


def test_opb_sharing_on_gpu(av):
    """New electrons of the physical gas never take more than half the
    remainder, and in FP64 their energies equal the oracle's (covered
    electron by electron above); here the mixed path's shares follow the
    same law: the share of the first generation against the oracle's (KS)."""
    w = W.plate(n_avalanches=200, e_field=45_000.0, seed=75)
    w.gas = W.argon_like_physical_gas()
    _setup(av, w)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=75, t_max=0.2)
    _, out = run_gpu(av, w, seed=77, precision=A.GT_MIXED, t_max=0.2, capacity=2_000_000)
    ea = ref["e0"][ref["uid"] >= 200]
    eb = out["e0"][out["uid"] >= 200]
    assert len(ea) > 500 and len(eb) > 500
    assert np.all(eb <= (100.0 - 15.7) / 2 + 1e-3)
    assert two_sample_ks(ea, eb).pvalue > 0.01
