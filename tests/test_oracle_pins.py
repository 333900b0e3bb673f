"""Pins of the CPU oracle against facts that do not come from the oracle:
published known-answer vectors, closed forms of model gases, textbook
integrators, brute-force frequencies and conservation laws.

A plausible slip anywhere in the oracle's step (a dropped term of the flight,
a sign of E or B, cumulative vs per-level rates, the threshold guard, the
recoil factor, the ionisation bookkeeping, the RNG keying) fails one of
these.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import workloads as W
from tests import physics as P
from tests.conftest import golden_path


def _read_hex_table(name):
    rows = []
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(tok, 16) for tok in line.split()])
    return rows


# ----------------------------------------------------------- random numbers
def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors."""
    for row in _read_hex_table("philox4x32_10_kat.txt"):
        ctr, key, expect = row[0:4], row[4:6], row[6:10]
        assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_splitmix64_reference_sequence():
    """The uid mixer is SplitMix64's output function: its sequence from state
    0 matches the published reference output."""
    state = 0
    for (expect,) in _read_hex_table("splitmix64_seed0.txt"):
        state = (state + 0x9E3779B97F4A7C15) % 2**64
        assert oracle.splitmix64_mix(state) == expect


def test_child_uid_distinct():
    uids = {oracle.child_uid(p, f) for p in range(64) for f in range(256)}
    assert len(uids) == 64 * 256
    assert not (uids & set(range(64)))


# ------------------------------------------------------------------ flight
def _rk4(r, v, a, w, dt, n=4000):
    """Textbook RK4 for dr/dt = v, dv/dt = a + v x w."""
    y = np.concatenate([r, v]).astype(float)

    def f(y):
        return np.concatenate([y[3:], a + np.cross(y[3:], w)])

    h = dt / n
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return y[:3], y[3:]


@pytest.mark.parametrize("case", range(6))
def test_flight_matches_rk4(case):
    """The closed-form flight equals a numerical integration of the Lorentz
    force (E only, B only, E and B at arbitrary angles)."""
    rng = np.random.default_rng(100 + case)
    r = rng.normal(size=3) * 1e-3
    v = rng.normal(size=3) * 0.05
    a = rng.normal(size=3) * 50.0 if case != 1 else np.zeros(3)
    w = rng.normal(size=3) * 200.0 if case not in (0, 5) else np.zeros(3)
    dt = 0.02 * (1 + case)
    r1, v1 = oracle.flight(r, v, a, w, dt)
    r2, v2 = _rk4(r, v, a, w, dt)
    assert np.allclose(r1, r2, rtol=1e-9, atol=1e-12)
    assert np.allclose(v1, v2, rtol=1e-9, atol=1e-10)


def test_flight_crossed_fields_guiding_centre():
    """Collisionless motion in E perpendicular to B drifts at E x B / B^2 on
    average (textbook guiding-centre drift)."""
    e_vcm, b_t = np.array([0.0, 0.0, -1000.0]), np.array([1.0, 0.0, 0.0])
    a = -P.ACCEL_PER_VCM * e_vcm
    w = -P.OMEGA_PER_T * b_t
    period = 2 * math.pi / np.linalg.norm(w)
    r, v = oracle.flight(np.zeros(3), np.zeros(3), a, w, 50 * period)
    drift = np.cross(e_vcm * 100.0, b_t) / 1.0  # m/s, from SI E [V/m] x B [T] / B^2
    drift_cm_ns = drift * 1e-7
    assert np.allclose(r / (50 * period), drift_cm_ns, rtol=1e-9, atol=1e-15)
    # speed unchanged by B alone
    v0 = np.array([0.01, 0.02, -0.03])
    _, v1 = oracle.flight(np.zeros(3), v0, np.zeros(3), w, 0.37)
    assert np.isclose(np.linalg.norm(v1), np.linalg.norm(v0), rtol=1e-14)


# ---------------------------------------------------------------- collisions
def test_elastic_matches_two_body_kinematics():
    """Lab-frame elastic scattering on a target at rest (textbook two-body
    kinematics): E'/E = ((m cos chi + sqrt(M^2 - m^2 sin^2 chi)) / (m + M))^2.
    The oracle's first-order form must agree to O((m/M)^2) at every angle,
    and the new direction is the isotropic one drawn from the uniforms."""
    for mass_ratio in (W.ELECTRON_MASS_U / W.ARGON_MASS_U, 1e-3):
        recoil = 2.0 * mass_ratio
        rng = np.random.default_rng(8)
        for _ in range(500):
            v = rng.normal(size=3) * 0.3
            uc, up = rng.uniform(size=2)
            v1 = oracle.elastic(recoil, v, uc, up)
            n = v1 / np.linalg.norm(v1)
            assert n[2] == pytest.approx(1.0 - 2.0 * uc, abs=1e-12)
            assert math.atan2(n[1], n[0]) % (2 * math.pi) == pytest.approx(
                2 * math.pi * up, abs=1e-9)
            c = np.dot(n, v) / np.linalg.norm(v)
            mu = mass_ratio
            exact = ((mu * c + math.sqrt(1.0 - mu * mu * (1 - c * c))) / (1.0 + mu)) ** 2
            ratio = np.dot(v1, v1) / np.dot(v, v)
            # second-order term of the expansion is 2 mu^2 (1 - cos chi)^2 <= 8 mu^2
            assert abs(ratio - exact) <= 8.0 * mu * mu * (1 + 1e-6) + 1e-13


def test_ionisation_split_and_secondary_identity():
    """E = 0 and a pure ionisation gas (threshold I): after its single
    collision the primary keeps (eps0 - I)(1 - u) and the new electron
    starts with (eps0 - I) u, u uniform; the new electron's id is the
    documented function of the parent id and flight index."""
    e0, I, n = 10.0, 2.0, 4000
    w = W.drift_model(n_electrons=n, n_coll=1, e_field=0.0, seed=13)
    g = W.model_gas(0.0, nu_ion=1000.0, ion_threshold=I)
    w.primaries.e[:] = e0
    o = oracle.run(g, w.field, w.primaries, seed=13, coll_limit=1, t_max=0.02)
    prim = o["uid"] < n
    pu = o["uid"][prim]
    by_uid = {int(u): i for i, u in enumerate(o["uid"])}
    frac = []
    for i in np.nonzero(prim)[0]:
        if o["status"][i] != W.COLL_LIMIT:
            continue
        child = oracle.child_uid(int(o["uid"][i]), int(o["n_flight"][i]) - 1)
        j = by_uid[child]
        assert o["e0"][j] + o["e1"][i] == pytest.approx(e0 - I, rel=1e-12)
        assert o["t0"][j] == o["t1"][i]
        frac.append(o["e1"][i] / (e0 - I))
    frac = np.sort(frac)
    assert len(frac) > 0.9 * len(pu)
    d = np.max(np.abs(np.arange(1, len(frac) + 1) / len(frac) - frac))
    assert d < 1.63 / math.sqrt(len(frac))


# ------------------------------------------------------------------- fields
def test_coax_field_integrates_to_voltage():
    """The line integral of the coaxial field from the wire to the tube
    equals the applied voltage, and the field points away from a positive
    wire."""
    f = W.Field(W.COAX, wire_r=25e-4, tube_r=0.5, voltage=1500.0)
    rs = np.geomspace(f.wire_r, f.tube_r, 20001)
    phi = 0.7
    er = [np.dot(oracle.field_eval(f, [r * math.cos(phi), r * math.sin(phi), 0.3]),
                 [math.cos(phi), math.sin(phi), 0.0]) for r in rs]
    assert np.all(np.asarray(er) > 0)
    integral = np.trapezoid(er, rs)
    assert abs(integral - 1500.0) < 1e-3


def test_grid_trilinear_exact_on_affine_field():
    """Trilinear interpolation reproduces an affine field exactly."""
    n = (5, 6, 7)
    origin, spacing = (-0.1, 0.2, 0.0), (0.05, 0.04, 0.03)
    A = np.array([[1.0, 2.0, -3.0], [0.5, -1.0, 2.0], [4.0, 0.0, 1.0]])
    c = np.array([10.0, -20.0, 5.0])
    g = np.zeros((n[2], n[1], n[0], 4), np.float32)
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                p = np.array(origin) + np.array(spacing) * (i, j, k)
                g[k, j, i, :3] = A @ p + c
    f = W.Field(W.GRID, grid=g, origin=origin, spacing=spacing)
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = np.array(origin) + rng.uniform(0, 1, 3) * np.array(spacing) * (np.array(n) - 1)
        e = oracle.field_eval(f, p)
        # node values were rounded to float32; interpolation adds no error of its own
        assert np.allclose(e, A @ p + c, rtol=0, atol=2e-5)


def test_grid_converges_to_coax_away_from_wire():
    f = W.coax_grid_map(n=64, half_width=0.15, length=1.0)
    fc = W.Field(W.COAX, wire_r=f.wire_r, tube_r=f.tube_r, voltage=f.voltage)
    rng = np.random.default_rng(4)
    for _ in range(100):
        r = rng.uniform(0.05, 0.1)
        ph = rng.uniform(0, 2 * math.pi)
        p = [r * math.cos(ph), r * math.sin(ph), rng.uniform(0.1, 0.9)]
        eg, ec = oracle.field_eval(f, p), oracle.field_eval(fc, p)
        assert np.linalg.norm(eg - ec) < 0.02 * np.linalg.norm(ec)


def test_boundaries():
    plate = W.Field(W.PLATE, e0=1.0, gap=0.0128)
    assert oracle.boundary(plate, [0, 0, 0.0]) == 0
    assert oracle.boundary(plate, [0, 0, 0.0128]) == W.ANODE
    assert oracle.boundary(plate, [0, 0, -1e-12]) == W.CATHODE
    cx = W.Field(W.COAX, wire_r=25e-4, tube_r=0.5, voltage=1.0)
    assert oracle.boundary(cx, [0.002, 0.0, 5.0]) == W.WIRE
    assert oracle.boundary(cx, [0.3, 0.4, 0.0]) == W.TUBE
    assert oracle.boundary(cx, [0.1, 0.1, -3.0]) == 0
    g = W.coax_grid_map(n=8, half_width=0.15, length=1.0)
    assert oracle.boundary(g, [0.0, 0.0, 0.5]) == W.WIRE
    assert oracle.boundary(g, [0.16, 0.0, 0.5]) == W.OUT_OF_MAP
    assert oracle.boundary(g, [0.1, 0.0, 1.01]) == W.OUT_OF_MAP
    assert oracle.boundary(g, [0.1, 0.0, 0.5]) == 0


# ---------------------------------------------------------------- selection
@pytest.mark.parametrize("eps", [0.0, 0.73, 11.62, 12.0, 15.69, 15.71, 33.3, 99.99, 140.0])
def test_selection_frequencies_brute_force(eps):
    """Over a fine uniform grid of u1 the fraction choosing level j equals
    nu_j(eps)/nu_max, with nu_j linearly interpolated from the per-level
    input rates (np.interp, not cumulative sums) and zero below the level's
    threshold; the remainder is null."""
    gas = W.argon_like_gas()
    n = 40000
    us = (np.arange(n) + 0.5) / n
    counts = np.zeros(gas.n_levels + 1)
    nu_max = None
    for u in us:
        j, nu_max = oracle.select(gas, eps, u)
        counts[j if j >= 0 else -1] += 1
    nodes = np.arange(gas.n_nodes) * gas.d_eps
    expect = np.array([np.interp(eps, nodes, gas.rate[:, j]) for j in range(gas.n_levels)])
    expect[(gas.level_type != W.ELASTIC) & (eps < gas.threshold)] = 0.0
    assert nu_max == pytest.approx(gas.rate.sum(1).max() * (1 + 1e-6), rel=1e-15)
    frac = counts[:-1] / n
    assert np.allclose(frac, expect / nu_max, atol=2.0 / n)


# ---------------------------------------------------------------- transport
@pytest.fixture(scope="module")
def drift_run():
    w = W.drift_model(n_electrons=20000, n_coll=10000, seed=11)
    return w, oracle.run(w.gas, w.field, w.primaries, seed=11, coll_limit=w.coll_limit)


def test_drift_velocity_closed_form(drift_run):
    """Constant nu, isotropic elastic, no loss: v_d = eE/(m nu) exactly in
    the mean; E[t] = N/nu."""
    w, o = drift_run
    assert np.all(o["status"] == W.COLL_LIMIT)
    dz, dt = o["z1"] - o["z0"], o["t1"] - o["t0"]
    n = len(dz)
    vd = P.drift_velocity(1000.0, 1000.0)
    # ratio estimator; its standard error from the sample
    se = np.std(dz - vd * dt) / math.sqrt(n) / dt.mean()
    assert P.within_sigma(dz.mean() / dt.mean(), vd, se)
    assert P.within_sigma(dt.mean(), 10000 / 1000.0, dt.std() / math.sqrt(n))


def test_transverse_spread_closed_form(drift_run):
    w, o = drift_run
    xs = np.concatenate([o["x1"] - o["x0"], o["y1"] - o["y0"]]) ** 2
    expect = P.transverse_msd(1000.0, 1000.0, 10000, 0.1)
    assert P.within_sigma(xs.mean(), expect, xs.std() / math.sqrt(len(xs) / 2))


def test_energy_is_field_work_without_loss(drift_run):
    """Per electron: final energy = initial energy + E * dz (exact up to
    rounding) when collisions conserve energy."""
    w, o = drift_run
    gain = 1000.0 * (o["z1"] - o["z0"])
    assert np.allclose(o["e1"], o["e0"] + gain, rtol=1e-9, atol=1e-9)


def test_recoil_cooling_closed_form():
    """E = 0, elastic scattering on a target with 2m/M = r: each isotropic
    collision multiplies the energy by 1 - r (1 - cos chi), E[cos chi] = 0, so
    E[eps_N] = eps_0 (1 - r)^N."""
    r, N = 0.02, 60
    w = W.drift_model(n_electrons=20000, n_coll=N, e_field=0.0, seed=5)
    w.gas = W.model_gas(1000.0, recoil=r)
    w.primaries.e[:] = 2.0
    o = oracle.run(w.gas, w.field, w.primaries, seed=5, coll_limit=N)
    expect = 2.0 * (1.0 - r) ** N
    assert P.within_sigma(o["e1"].mean(), expect, o["e1"].std() / math.sqrt(len(o["e1"])))
    # with E = 0 no work is done: the ledger is all recoil
    assert np.allclose(o["e0"] - o["ledger"][:, 2], o["e1"], rtol=1e-12, atol=1e-12)


def test_langevin_crossed_field_drift():
    """Constant nu with E perpendicular to B: the mean velocity obeys
    d<v>/dt = a + <v> x w - nu <v> exactly, so the drift solves a 3x3 linear
    system (magnitude and Lorentz angle)."""
    b = (3.0, 0.0, 0.0)
    w = W.drift_model(n_electrons=20000, n_coll=10000, b=b, seed=7)
    o = oracle.run(w.gas, w.field, w.primaries, seed=7, coll_limit=w.coll_limit)
    vd = P.langevin_drift([0.0, 0.0, -1000.0], b, 1000.0)
    dt = o["t1"] - o["t0"]
    for k, c in enumerate("xyz"):
        d = o[c + "1"] - o[c + "0"]
        se = np.std(d - vd[k] * dt) / math.sqrt(len(d)) / dt.mean()
        assert P.within_sigma(d.mean() / dt.mean(), vd[k], se), (c, d.mean() / dt.mean(), vd[k], se)
    # the drift has a sizeable E x B component (Lorentz angle ~ 28 degrees)
    assert abs(vd[1]) > 0.4 * abs(vd[2])
    # magnetic force does no work
    assert np.allclose(o["e1"], o["e0"] + 1000.0 * (o["z1"] - o["z0"]), rtol=1e-9, atol=1e-9)


def test_yule_gain_distribution():
    """Constant ionisation rate nu_i with zero threshold and time limit T:
    the number of electrons at T is geometric with p = exp(-nu_i T), mean
    exp(nu_i T) (Yule-Furry pure birth)."""
    nu_i, T, n_av = 10.0, 0.5, 1500
    w = W.drift_model(n_electrons=n_av, n_coll=0, e_field=100.0, seed=9)
    w.gas = W.model_gas(1000.0, nu_ion=nu_i, ion_threshold=0.0)
    o = oracle.run(w.gas, w.field, w.primaries, seed=9, t_max=T)
    n = o["electrons"].astype(float)
    assert np.all(o["status"] == W.TIME)
    assert np.allclose(o["t1"], T)
    mean = math.exp(nu_i * T)
    assert P.within_sigma(n.mean(), mean, n.std() / math.sqrt(n_av))
    # KS distance against the geometric law
    ks = np.sort(n)
    emp = np.arange(1, n_av + 1) / n_av
    d = np.max(np.abs(emp - P.geometric_cdf(ks, math.exp(-nu_i * T))))
    assert d < 1.63 / math.sqrt(n_av)  # KS critical value, alpha = 0.01
    # charge: every electron beyond the primary came from one ionisation
    assert np.array_equal(o["electrons"], 1 + o["tallies"][:, 1])


@pytest.fixture(scope="module")
def plate_run():
    w = W.plate(n_avalanches=24, e_field=40_000.0, seed=2)
    return w, oracle.run(w.gas, w.field, w.primaries, seed=2, t_max=w.t_max)


def test_plate_charge_and_ids(plate_run):
    w, o = plate_run
    L = w.gas.n_levels
    ion = o["tallies"][:, L - 1]
    assert np.array_equal(o["electrons"], 1 + ion)
    assert len(np.unique(o["uid"])) == len(o["uid"])
    assert set(np.unique(o["status"])) <= {W.ANODE, W.CATHODE, W.TIME}
    an = o["status"] == W.ANODE
    assert np.all(o["z1"][an] >= 0.0128) and np.all(o["z1"][~an] < 0.0128)
    assert np.all(o["e1"] >= 0.0) and np.all(o["t1"] <= w.t_max)


def test_plate_energy_ledger(plate_run):
    """Per electron: e_end = e_start + field work - inelastic thresholds -
    recoil losses - energy handed to secondaries."""
    w, o = plate_run
    L = o["ledger"]
    bal = o["e0"] + L[:, 0] - L[:, 1] - L[:, 2] - L[:, 3]
    scale = 1.0 + np.abs(L).sum(1)
    assert np.all(np.abs(bal - o["e1"]) <= 1e-12 * scale + 1e-12)
    # ionisation and excitation losses are whole multiples of thresholds
    assert np.all(L[:, 1] >= 0) and np.all(L[:, 2] >= 0) and np.all(L[:, 3] >= 0)


def test_plate_subset_reproduces_avalanches(plate_run):
    """Keying by (seed, avalanche, electron id) makes any subset of
    avalanches reproduce exactly."""
    w, o = plate_run
    sub = w.primaries.subset([3, 17])
    s = oracle.run(w.gas, w.field, sub, seed=2, t_max=w.t_max, n_threads=1)
    for k in (3, 17):
        a, b = o["aval"] == k, s["aval"] == k
        ia, ib = np.argsort(o["uid"][a]), np.argsort(s["uid"][b])
        for c in ("x1", "y1", "z1", "t1", "e1", "status", "uid"):
            assert np.array_equal(o[c][a][ia], s[c][b][ib])


# ------------------------------------------------------- banded majorant
def test_banded_majorant_drift_closed_form():
    """The banded majorant is exact: on the constant-rate gas the drift
    velocity and the energy ledger are unchanged."""
    w = W.drift_model(n_electrons=20000, n_coll=3000, seed=21)
    w.gas = W.model_gas(1000.0, exact_nu_max=False)  # nu_max above the rate: nulls exist
    o = oracle.run(w.gas, w.field, w.primaries, seed=21, coll_limit=3000, majorant=1,
                   window=2.0, band_width=50.0)
    dz, dt = o["z1"] - o["z0"], o["t1"] - o["t0"]
    vd = P.drift_velocity(1000.0, 1000.0)
    se = np.std(dz - vd * dt) / math.sqrt(len(dz)) / dt.mean()
    assert P.within_sigma(dz.mean() / dt.mean(), vd, se)
    assert np.allclose(o["e1"], o["e0"] + 1000.0 * dz, rtol=1e-9, atol=1e-9)


def test_banded_majorant_yule():
    nu_i, T, n_av = 10.0, 0.5, 1500
    w = W.drift_model(n_electrons=n_av, n_coll=0, e_field=100.0, seed=23)
    w.gas = W.model_gas(1000.0, nu_ion=nu_i, ion_threshold=0.0, exact_nu_max=False)
    o = oracle.run(w.gas, w.field, w.primaries, seed=23, t_max=T, majorant=1, window=1.5,
                   band_width=100.0)
    n = o["electrons"].astype(float)
    assert P.within_sigma(n.mean(), math.exp(nu_i * T), n.std() / math.sqrt(n_av))


def test_banded_majorant_matches_global_in_distribution():
    """Same physics, different random-number use: the argon plate with the
    banded majorant has the same gain distribution, arrival times and
    collision mix as with the global nu_max (two-sample KS, 3 sigma), in far
    fewer flights."""
    from scipy import stats
    n = 160
    w = W.plate(n_avalanches=n, e_field=35_000.0, seed=3)
    g = oracle.run(w.gas, w.field, w.primaries, seed=3, t_max=w.t_max)
    b = oracle.run(w.gas, w.field, w.primaries, seed=4, t_max=w.t_max, majorant=1,
                   window=2.0, band_width=1.0)
    ga = np.bincount(g["aval"][g["status"] == W.ANODE], minlength=n).astype(float)
    gb = np.bincount(b["aval"][b["status"] == W.ANODE], minlength=n).astype(float)
    se = math.sqrt(ga.var() / n + gb.var() / n)
    assert abs(ga.mean() - gb.mean()) < 3 * se
    assert stats.ks_2samp(np.log1p(ga), np.log1p(gb)).pvalue > 0.01
    L = w.gas.n_levels
    fa = g["tallies"][:, :L].sum(0) / g["tallies"][:, :L].sum()
    fb = b["tallies"][:, :L].sum(0) / b["tallies"][:, :L].sum()
    assert np.allclose(fa, fb, atol=0.01)  # share of each level among real collisions
    ta = np.array([g["t1"][(g["aval"] == i) & (g["status"] == W.ANODE)].mean()
                   for i in range(n) if ga[i] > 0])
    tb = np.array([b["t1"][(b["aval"] == i) & (b["status"] == W.ANODE)].mean()
                   for i in range(n) if gb[i] > 0])
    assert stats.ks_2samp(ta, tb).pvalue > 0.01
    # real collisions per flight rise several-fold
    ra = g["tallies"][:, :L].sum() / g["n_flight"].astype(np.int64).sum()
    rb = b["tallies"][:, :L].sum() / b["n_flight"].astype(np.int64).sum()
    assert rb > 3 * ra


@pytest.mark.parametrize("gas_name", ["argon_like", "ramp", "ramp_above_5eV", "v_shape"])
def test_banded_majorant_bounds_the_rate_along_every_flight(gas_name):
    """Thinning is exact only if the majorant is never below the true rate
    on the flight.  For random starts (energy, angle to the acceleration,
    field, window, band width) the exact no-B trajectory v0 + a t gives the
    energy range reached over [0, tau]; the largest tabulated total rate on
    that range (its ends and every node inside, since the table is linear
    between nodes) must not exceed the majorant.  The window itself is
    window / (largest node rate of the start band)."""
    if gas_name == "argon_like":
        gas = W.argon_like_gas()
    else:
        eps = np.arange(1001, dtype=np.float64) * 0.1
        if gas_name == "ramp_above_5eV":  # zero-rate bands below 5 eV
            eps = np.maximum(eps - 5.0, 0.0)
        if gas_name == "v_shape":  # falling below 20 eV: the lower end of the range counts
            eps = np.abs(eps - 20.0)
        gas = W.Gas(np.array([W.ELASTIC], np.int32), np.zeros(1), (34.0 * eps)[:, None], 0.1)
    nodes = np.arange(gas.n_nodes) * gas.d_eps
    total = gas.rate.sum(axis=1)
    rng = np.random.default_rng(41)
    worst = 0.0
    for _ in range(3000):
        bw = rng.choice([0.05, 0.25, 1.0, 5.0])
        window = rng.choice([0.5, 2.0, 4.0])
        eps0 = rng.choice([0.0, rng.uniform(0.0, 5.0), rng.uniform(0.0, 60.0)])
        e_mag = rng.choice([0.0, rng.uniform(0.0, 6.0e4)], p=[0.05, 0.95])
        s0 = math.sqrt(P.speed_sq(eps0))
        n_v, n_e = rng.normal(size=3), rng.normal(size=3)
        v = s0 * n_v / np.linalg.norm(n_v)
        e_vec = e_mag * n_e / np.linalg.norm(n_e)
        # angle between the velocity and the acceleration -(e/m) E
        cos_a = -float(np.dot(n_v, n_e)) / (np.linalg.norm(n_v) * np.linalg.norm(n_e))
        nu_w, tau = oracle.majorant(gas, bw, v, e_vec, False, window)
        n = max(1, int(math.floor(bw / gas.d_eps + 0.5)))
        b0 = min(int(eps0 / (n * gas.d_eps)), (gas.n_nodes - 2) // n)
        bound = total[b0 * n:(b0 + 1) * n + 1].max()
        bound = bound if bound > 0.0 else total.max() * 2.0 ** -40
        assert tau == pytest.approx(window / bound, rel=1e-12)
        assert math.isfinite(nu_w) and nu_w > 0.0
        a = P.ACCEL_PER_VCM * e_mag
        # |v(t)|^2 = s0^2 + 2 s0 a cos t + a^2 t^2 is convex in t
        ends = [0.0, tau]
        if a > 0.0 and 0.0 < -s0 * cos_a / a < tau:
            ends.append(-s0 * cos_a / a)
        v2 = [s0 * s0 + 2.0 * s0 * a * cos_a * t + a * a * t * t for t in ends]
        e_lo = min(v2) / (2.0 * P.ACCEL_PER_VCM)
        e_hi = max(v2) / (2.0 * P.ACCEL_PER_VCM)
        inside = total[(nodes >= e_lo) & (nodes <= e_hi)]
        true_max = max(np.interp(e_lo, nodes, total), np.interp(e_hi, nodes, total),
                       inside.max() if inside.size else 0.0)
        assert true_max <= nu_w * (1.0 + 1e-12), (gas_name, bw, window, eps0, cos_a, e_mag)
        worst = max(worst, true_max / nu_w)
    assert worst > 0.9  # the bound is attained closely somewhere (not vacuous)


def test_banded_majorant_bounds_the_rate_with_magnetic_field():
    """With B the flight turns; the majorant must still cover the tabulated
    rate at every point of the trajectory within the window, here sampled
    50 times along an RK4 integration of the Lorentz force."""
    gas = W.argon_like_gas()
    nodes = np.arange(gas.n_nodes) * gas.d_eps
    total = gas.rate.sum(axis=1)
    rng = np.random.default_rng(43)
    for _ in range(60):
        eps0 = rng.uniform(0.0, 30.0)
        e_vec = rng.normal(size=3)
        e_vec *= rng.uniform(1.0e3, 6.0e4) / np.linalg.norm(e_vec)
        b_vec = rng.normal(size=3)
        b_vec *= rng.uniform(0.1, 4.0) / np.linalg.norm(b_vec)
        n_v = rng.normal(size=3)
        v = math.sqrt(P.speed_sq(eps0)) * n_v / np.linalg.norm(n_v)
        nu_w, tau = oracle.majorant(gas, 1.0, v, e_vec, True, 2.0)
        a = -P.ACCEL_PER_VCM * e_vec
        w = -P.OMEGA_PER_T * b_vec
        r, u = np.zeros(3), v.copy()
        for _ in range(50):
            r, u = _rk4(r, u, a, w, tau / 50, n=20)
            eps = float(np.dot(u, u)) / (2.0 * P.ACCEL_PER_VCM)
            assert np.interp(eps, nodes, total) <= nu_w * (1.0 + 1e-12)


def ramp_workload(n, seed, band_width):
    """Rate linear in energy, nu = c * eps, 0-100 eV (exact under linear
    interpolation), E = 10 kV/cm, one real collision per electron, isotropic
    directions; a quarter of the electrons start at rest (the energy reach
    of a flight is then the acceleration term alone), the rest with
    U(0, 20) eV."""
    c, n_nodes, d_eps = 34.0, 1001, 0.1
    eps = np.arange(n_nodes, dtype=np.float64) * d_eps
    gas = W.Gas(np.array([W.ELASTIC], np.int32), np.zeros(1), (c * eps)[:, None], d_eps,
                0.0, 0.0, band_width)
    w = W.drift_model(n_electrons=n, n_coll=1, e_field=1.0e4, seed=seed)
    w.gas = gas
    e0 = np.random.default_rng(seed + 1).uniform(0.0, 20.0, n)
    e0[: n // 4] = 0.0
    w.primaries.e[:] = e0
    return w, c


def ramp_pit(o, w, c):
    """Probability integral transform of each electron's first-collision
    time under the closed-form survival: uniform on (0, 1) when exact."""
    p = w.primaries
    cos_a = p.dz[o["uid"].astype(np.int64)]  # acceleration is along +z (E along -z)
    s = P.ramp_first_collision_survival(o["t1"] - o["t0"], o["e0"], cos_a,
                                        w.field.e0, c)
    return 1.0 - s


@pytest.mark.parametrize("majorant,band_width,window",
                         [(0, 1.0, 2.0), (1, 1.0, 2.0), (1, 5.0, 2.0), (1, 0.1, 0.5)])
def test_ramp_first_collision_closed_form(majorant, band_width, window):
    """A rising rate is where a majorant can fail: the electron gains energy
    during the flight, so a bound taken at the start energy, or without
    the drift or the acceleration term of the energy reach, falls below
    the rate along the path and delays the collisions.  The first real
    collision times follow the closed-form survival exactly (KS of the
    probability integral transform against the uniform law)."""
    from scipy import stats
    w, c = ramp_workload(40000, 31, band_width)
    o = oracle.run(w.gas, w.field, w.primaries, seed=31, coll_limit=1, majorant=majorant,
                   window=window, band_width=band_width)
    assert np.all(o["status"] == W.COLL_LIMIT)
    u = ramp_pit(o, w, c)
    assert stats.kstest(u, "uniform").pvalue > 0.01


# ------------------------------------------ attachment, anisotropy, sharing
@pytest.mark.parametrize("xi", [0.3, 0.8, 0.97, -0.5])
def test_screened_coulomb_deflection(xi):
    """Deflection cosines follow the screened-Coulomb law (KS against its
    distribution function), measured from the geometry of the returned
    direction; the azimuth about the incident direction is uniform; the
    direction is a unit vector."""
    from scipy import stats
    rng = np.random.default_rng(51)
    v = rng.normal(size=3) * 0.1
    d = v / np.linalg.norm(v)
    # a frame of the test's own: e1 from Gram-Schmidt on the x axis
    e1 = np.array([1.0, 0.0, 0.0]) - d[0] * d
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    mus, phis = [], []
    for u, w in rng.uniform(size=(6000, 2)):
        n, mu = oracle.scatter(xi, v, u, w)
        assert abs(np.linalg.norm(n) - 1.0) < 1e-12
        assert abs(mu - float(np.dot(n, d))) < 1e-12
        mus.append(float(np.dot(n, d)))
        phis.append(math.atan2(float(np.dot(n, e2)), float(np.dot(n, e1))))
    assert stats.kstest(mus, lambda m: P.screened_coulomb_cdf(m, xi)).pvalue > 0.01
    assert stats.kstest(np.mod(phis, 2 * math.pi) / (2 * math.pi), "uniform").pvalue > 0.01


def test_screened_coulomb_from_rest_and_isotropic_limit():
    n, mu = oracle.scatter(0.6, np.zeros(3), 0.3, 0.7)  # a resting electron: d = +z
    assert abs(n[2] - mu) < 1e-15 and abs(np.linalg.norm(n) - 1.0) < 1e-12
    n0, _ = oracle.scatter(0.0, np.array([0.1, 0.0, 0.0]), 0.3, 0.7)
    assert np.allclose(n0[2], 1.0 - 2.0 * 0.3)  # lab-frame isotropic sampling


def test_anisotropic_drift_closed_form():
    """Constant rate nu, energy-independent anisotropy: each collision keeps
    the mean velocity fraction g = <cos chi>, so the drift velocity is
    eE / (m nu (1 - g)) exactly (momentum-transfer rate)."""
    xi = 0.6
    w = W.drift_model(n_electrons=20000, n_coll=3000, seed=53)
    w.gas = W.model_gas(1000.0, xi_elastic=xi)
    o = oracle.run(w.gas, w.field, w.primaries, seed=53, coll_limit=3000)
    g = P.screened_coulomb_mean_cos(xi)
    dz, dt = o["z1"] - o["z0"], o["t1"] - o["t0"]
    vd = P.drift_velocity(1000.0, 1000.0 * (1.0 - g))
    se = np.std(dz - vd * dt) / math.sqrt(len(dz)) / dt.mean()
    assert P.within_sigma(dz.mean() / dt.mean(), vd, se)
    assert np.allclose(o["e1"], o["e0"] + 1000.0 * dz, rtol=1e-9, atol=1e-9)


def test_elastic_recoil_uses_the_deflection_with_anisotropy():
    rng = np.random.default_rng(55)
    r = 0.02
    for _ in range(200):
        v = rng.normal(size=3) * 0.1
        u, ph, xi = rng.uniform(), rng.uniform(), rng.uniform(-0.9, 0.99)
        v1 = oracle.elastic(r, v, u, ph, xi)
        n, mu = oracle.scatter(xi, v, u, ph)
        assert np.allclose(v1 / np.linalg.norm(v1), n, atol=1e-12)
        assert np.dot(v1, v1) == pytest.approx(np.dot(v, v) * (1.0 - r * (1.0 - mu)), rel=1e-12)


def test_attachment_time_is_exponential():
    """Constant attachment rate nu_a: the capture time is Exp(nu_a); the
    electron ends where it was captured with its energy unchanged (the
    energy ledger still closes)."""
    from scipy import stats
    nu_a = 5.0
    w = W.drift_model(n_electrons=5000, n_coll=0, seed=57)
    w.gas = W.model_gas(1000.0, nu_att=nu_a)
    # ~200 collisions before capture; the limit only bounds a broken capture
    o = oracle.run(w.gas, w.field, w.primaries, seed=57, coll_limit=200_000)
    assert np.all(o["status"] == W.ATTACHED)
    assert stats.kstest((o["t1"] - o["t0"]) * nu_a, "expon").pvalue > 0.01
    led = o["ledger"]
    assert np.allclose(o["e1"], o["e0"] + led[:, 0] - led[:, 1] - led[:, 2] - led[:, 3],
                       rtol=1e-10, atol=1e-9)
    assert np.all(o["tallies"][:, 1] == 1)  # one attachment per avalanche


def test_birth_death_process():
    """Constant ionisation (lam) and attachment (mu) rates: the number of
    electrons alive at T has mean exp((lam - mu) T) and the avalanche is
    extinct by T with Kendall's probability."""
    lam, mu, T, n = 10.0, 4.0, 0.4, 3000
    w = W.drift_model(n_electrons=n, n_coll=0, e_field=100.0, seed=59)
    w.gas = W.model_gas(1000.0, nu_ion=lam, ion_threshold=0.0, nu_att=mu)
    o = oracle.run(w.gas, w.field, w.primaries, seed=59, t_max=T)
    alive = np.bincount(o["aval"][o["status"] == W.TIME], minlength=n).astype(float)
    mean, p0 = P.birth_death(lam, mu, T)
    assert P.within_sigma(alive.mean(), mean, alive.std() / math.sqrt(n))
    ext = float((alive == 0).mean())
    assert P.within_sigma(ext, p0, math.sqrt(p0 * (1 - p0) / n))
    # every electron ends either alive at T or attached
    assert set(np.unique(o["status"])) <= {W.TIME, W.ATTACHED}


@pytest.mark.parametrize("w_opb,rest", [(10.0, 30.0), (2.0, 80.0), (50.0, 5.0)])
def test_ionisation_sharing_opb(w_opb, rest):
    from scipy import stats
    rng = np.random.default_rng(61)
    x = np.array([oracle.ionisation_share(w_opb, rest, u) for u in rng.uniform(size=8000)])
    assert np.all((x >= 0.0) & (x <= rest / 2 * (1 + 1e-12)))
    assert stats.kstest(x, lambda q: P.opb_cdf(q, w_opb, rest)).pvalue > 0.01
    assert oracle.ionisation_share(0.0, rest, 0.25) == 0.25 * rest  # uniform split


def test_physical_gas_ledger_and_charge():
    """The argon-like gas with anisotropy, OPB sharing and attachment: the
    energy ledger closes per electron, charge is conserved per avalanche,
    attached electrons end with status ATTACHED, and new electrons never
    take more than half the remainder (shares <= (eps - I) / 2)."""
    w = W.plate(n_avalanches=40, e_field=45_000.0, seed=63)
    w.gas = W.argon_like_physical_gas()
    o = oracle.run(w.gas, w.field, w.primaries, seed=63, t_max=w.t_max)
    led = o["ledger"]
    assert np.allclose(o["e1"], o["e0"] + led[:, 0] - led[:, 1] - led[:, 2] - led[:, 3],
                       rtol=1e-9, atol=1e-8)
    L = w.gas.n_levels
    ion = o["tallies"][:, L - 2]  # ionisation is the level before attachment
    assert np.array_equal(o["electrons"], 1 + ion)
    att = o["tallies"][:, L - 1]
    assert np.array_equal(np.bincount(o["aval"][o["status"] == W.ATTACHED], minlength=40), att)
    assert att.sum() > 0 and ion.sum() > 0
    child = o["uid"] >= 40
    assert np.all(o["e0"][child] <= (100.0 - 15.7) / 2)


def test_screened_anisotropy_diffusion_closed_form():
    """No field, constant rate nu and fixed energy eps0 (nothing changes the
    speed): with the energy-dependent anisotropy xi = eps0 / (eps0 + screen)
    successive directions have <n_i . n_j> = g^|i-j| (g = <cos chi>), so after
    N flights <|r|^2> = (v/nu)^2 (2N + 2 sum_k (N - k) g^k)."""
    eps0, screen, N, n = 10.0, 5.0, 40, 20000
    w = W.drift_model(n_electrons=n, n_coll=N, e_field=0.0, seed=65)
    w.gas = W.model_gas(1000.0)
    w.gas.screen = np.array([screen])
    w.primaries.e[:] = eps0
    o = oracle.run(w.gas, w.field, w.primaries, seed=65, coll_limit=N)
    r2 = (o["x1"] - o["x0"]) ** 2 + (o["y1"] - o["y0"]) ** 2 + (o["z1"] - o["z0"]) ** 2
    g = P.screened_coulomb_mean_cos(eps0 / (eps0 + screen))
    k = np.arange(1, N)
    expect = P.speed_sq(eps0) / 1000.0 ** 2 * (2 * N + 2 * np.sum((N - k) * g ** k))
    assert P.within_sigma(r2.mean(), expect, r2.std() / math.sqrt(n))
    assert np.allclose(o["e1"], eps0, rtol=1e-12)


# --------------------------------------- boundary crossings and sub-steps
def by_uid(o):
    """Per-electron arrays of a run ordered by electron id (primaries: input order)."""
    idx = np.argsort(o["uid"], kind="stable")
    n = len(o["uid"])
    return {k: (v[idx] if hasattr(v, "__len__") and len(v) == n and k not in
                ("electrons", "tallies") else v) for k, v in o.items()}


def _collisionless(n, e_field, seed):
    """Plate electrons in a gas with a negligible rate: each flight runs to
    the 100 ns time limit unless the electron leaves first."""
    w = W.plate(n_avalanches=n, e_field=e_field, seed=seed)
    w.gas = W.model_gas(1e-9)
    return w


def test_crossing_at_the_anode_closed_form():
    """Uniform acceleration a from z = 0: the anode (z = d) is reached at
    t* = (sqrt(vz^2 + 2 a d) - vz) / a; with exact crossings the endpoint is
    the crossing point at t*, without them the post-flight point."""
    w = _collisionless(200, 30_000.0, 67)
    a = P.ACCEL_PER_VCM * 30_000.0
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    ts = (np.sqrt(vz * vz + 2 * a * w.field.gap) - vz) / a
    o = by_uid(oracle.run(w.gas, w.field, w.primaries, seed=67, t_max=100.0, crossing=True))
    assert np.all(o["status"] == W.ANODE)
    # (1e-10: e/m is quoted to 12 digits; the test derives it from e and m_e)
    assert np.allclose(o["t1"] - o["t0"], ts, rtol=1e-10, atol=0)
    assert np.all((o["z1"] >= w.field.gap) & (o["z1"] - w.field.gap < 1e-12))
    led = o["ledger"]
    assert np.allclose(o["e1"], o["e0"] + led[:, 0], rtol=1e-12, atol=1e-12)
    p = oracle.run(w.gas, w.field, w.primaries, seed=67, t_max=100.0)
    assert np.all(p["z1"] > 1.0)  # the post-flight point is far beyond the anode


def test_crossing_catches_an_exit_and_return():
    """An electron started 1 um from the cathode towards it, in a field
    that turns it back: it touches the cathode iff vz^2 > 2 a z0, at the
    smaller root of z0 + vz t + a t^2 / 2 = 0.  A post-flight test misses it
    (the flight ends at the anode)."""
    n = 400
    w = _collisionless(n, 30_000.0, 69)
    a = P.ACCEL_PER_VCM * 30_000.0
    z0 = 1e-4
    w.primaries.z[:] = z0
    w.primaries.dz[:] = -np.abs(w.primaries.dz)
    w.primaries.e[:] = np.random.default_rng(5).uniform(1.0, 20.0, n)
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    hits = vz * vz > 2 * a * z0
    assert 0.2 < hits.mean() < 0.8
    o = by_uid(oracle.run(w.gas, w.field, w.primaries, seed=69, t_max=100.0, crossing=True))
    assert np.array_equal(o["status"] == W.CATHODE, hits)
    ts = (-vz[hits] - np.sqrt(vz[hits] ** 2 - 2 * a * z0)) / a
    assert np.allclose(o["t1"][hits] - o["t0"][hits], ts, rtol=1e-9, atol=0)
    assert np.all((o["z1"][hits] < 0.0) & (o["z1"][hits] > -1e-12))
    p = oracle.run(w.gas, w.field, w.primaries, seed=69, t_max=100.0)
    assert np.all(p["status"] == W.ANODE)


def _coax_potential(field, r):
    """Potential of the coax (V): V at the wire, 0 at the tube."""
    return field.voltage * np.log(r / field.tube_r) / math.log(field.wire_r / field.tube_r)


def test_substeps_converge_to_energy_conservation():
    """Collisionless electrons in the coax field drift to the wire: the
    energy gained must equal e (V(r1) - V(r0)).  With the field held over a
    flight it does not; re-evaluating it over n sub-steps the error falls
    like 1/n.  With exact crossings the electrons end on the wire."""
    w = W.coax(n_avalanches=100, r_lo=0.004, r_hi=0.02, b_axial=0.0, seed=71)
    w.gas = W.model_gas(1e-9)
    errs, times = [], []
    for n in (32, 128, 512):  # one flight of 0.05 ns (the fall takes ~0.02 ns)
        o = oracle.run(w.gas, w.field, w.primaries, seed=71, t_max=0.05, substeps=n,
                       crossing=True)
        assert np.all(o["status"] == W.WIRE)
        r0 = np.hypot(o["x0"], o["y0"])
        r1 = np.hypot(o["x1"], o["y1"])
        assert np.all(r1 <= w.field.wire_r) and np.all(r1 > w.field.wire_r * (1 - 1e-9))
        gain = _coax_potential(w.field, r1) - _coax_potential(w.field, r0)
        errs.append(np.abs((o["e1"] - o["e0"]) - gain).max() / gain.max())
        times.append(by_uid(o)["t1"] - by_uid(o)["t0"])
        led = o["ledger"]
        assert np.allclose(o["e1"], o["e0"] + led[:, 0], rtol=1e-12, atol=1e-9)
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs
    assert errs[2] < 2e-2
    # the fall times converge too
    assert np.allclose(times[2], times[1], rtol=0.05) and times[2].min() > 1e-3


def test_crossing_keeps_the_physics_of_the_plate():
    """With collisions, exact crossings change only where electrons end:
    the gain distribution is the same (KS), every anode endpoint lies on
    the anode, and the ledger closes."""
    from scipy import stats
    n = 200
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=73)
    a = oracle.run(w.gas, w.field, w.primaries, seed=73, t_max=w.t_max)
    b = oracle.run(w.gas, w.field, w.primaries, seed=73, t_max=w.t_max, crossing=True)
    ga = np.bincount(a["aval"][a["status"] == W.ANODE], minlength=n)
    gb = np.bincount(b["aval"][b["status"] == W.ANODE], minlength=n)
    assert stats.ks_2samp(np.log1p(ga), np.log1p(gb), method="asymp").pvalue > 0.01
    an = b["status"] == W.ANODE
    assert np.all((b["z1"][an] >= w.field.gap) & (b["z1"][an] - w.field.gap < 1e-12))
    led = b["ledger"]
    assert np.allclose(b["e1"], b["e0"] + led[:, 0] - led[:, 1] - led[:, 2] - led[:, 3],
                       rtol=1e-9, atol=1e-9)


# --------------------------------------------------------- induced signals
def test_signal_telescopes_to_the_weighting_potential():
    """Shockley-Ramo: summed over a window that covers every electron's life,
    an avalanche's signal equals the sum over its electrons of
    phi_w(end) - phi_w(start) (phi_w = z / d for the plate anode): no piece
    of any path is lost or counted twice, with or without crossings and
    sub-steps."""
    n = 40
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=91)
    for kw in (dict(), dict(crossing=True, substeps=3)):
        o = oracle.run(w.gas, w.field, w.primaries, seed=91, t_max=w.t_max,
                       signal=(W.W_PLATE, 400, 0.0, 0.005), **kw)
        per_e = (o["z1"] - o["z0"]) / w.field.gap
        expect = np.bincount(o["aval"], weights=per_e, minlength=n)
        assert np.allclose(o["signal"].sum(axis=1), expect, rtol=1e-12, atol=1e-12)


def test_signal_bins_of_a_uniform_acceleration():
    """Collisionless plate electrons released at t_r inside a bin: in bin
    [b_k, b_k+1) the signal is (z(b_k+1) - z(b_k)) / d with
    z(t) = vz (t - t_r) + a (t - t_r)^2 / 2, counted from the release in its
    own bin and up to the arrival at the anode (crossing mode), where it is
    (d - z(b_k)) / d; the bin before the release holds nothing."""
    w = _collisionless(50, 30_000.0, 93)
    a = P.ACCEL_PER_VCM * 30_000.0
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    tr = 0.0052  # released inside the first bin [0.004, 0.007)
    w.primaries.t[:] = tr
    ts = tr + (np.sqrt(vz * vz + 2 * a * w.field.gap) - vz) / a
    t0, dt, nb = 0.001, 0.003, 9
    o = oracle.run(w.gas, w.field, w.primaries, seed=93, t_max=100.0, crossing=True,
                   signal=(W.W_PLATE, nb, t0, dt))
    edges = t0 + dt * np.arange(nb + 1)
    for i in range(50):
        te = np.clip(edges, tr, ts[i]) - tr
        z = np.where(edges < ts[i], vz[i] * te + 0.5 * a * te * te, w.field.gap)
        expect = np.diff(z) / w.field.gap
        # (atol: e/m is quoted to 12 digits, the test derives it from e and m_e)
        assert np.allclose(o["signal"][i], expect, rtol=1e-9, atol=1e-10), i


def test_signal_drift_current_closed_form():
    """Constant rate nu in a uniform field, far from the electrodes: each
    electron carries the mean current e v_d / d, so after the first
    collisions a bin of width dt holds v_d dt / d per electron (3 sigma)."""
    n, nu, e_field, gap = 20000, 1000.0, 1000.0, 100.0
    w = W.drift_model(n_electrons=n, n_coll=0, e_field=e_field, seed=95)
    w.field = W.Field(W.PLATE, e0=e_field, gap=gap)
    w.primaries.z[:] = 1.0
    dt, nb = 0.5, 10
    o = oracle.run(w.gas, w.field, w.primaries, seed=95, t_max=nb * dt,
                   signal=(W.W_PLATE, nb, 0.0, dt))
    s = o["signal"][:, 1:]  # per electron (one per avalanche), bins after the transient
    vd = P.drift_velocity(e_field, nu)
    assert np.all(o["status"] == W.TIME)
    for k in range(s.shape[1]):
        assert P.within_sigma(s[:, k].mean(), vd * dt / gap, s[:, k].std() / math.sqrt(n))


def test_signal_of_a_fall_onto_the_wire():
    """Collisionless fall onto the coax wire (crossing mode): every
    electron induces 1 - phi_w(r0) on the wire, phi_w = ln(r/b) / ln(a/b);
    the grid map's 4th component gives the same within its interpolation."""
    w = W.coax(n_avalanches=60, r_lo=0.004, r_hi=0.02, b_axial=0.0, seed=97)
    w.gas = W.model_gas(1e-9)
    o = oracle.run(w.gas, w.field, w.primaries, seed=97, t_max=0.05, substeps=256,
                   crossing=True, signal=(W.W_COAX, 5, 0.0, 0.01))
    r0 = np.hypot(o["x0"], o["y0"])
    phi0 = np.log(r0 / w.field.tube_r) / math.log(w.field.wire_r / w.field.tube_r)
    assert np.all(o["status"] == W.WIRE)
    assert np.allclose(o["signal"].sum(axis=1), 1.0 - phi0, rtol=1e-9)
    f = W.coax_grid_map(n=64, half_width=0.03, length=0.05)
    for r in ([0.004, 0.0, 0.02], [0.01, 0.013, 0.03], [-0.02, 0.005, 0.001]):
        rr = math.hypot(r[0], r[1])
        exact = math.log(rr / f.tube_r) / math.log(f.wire_r / f.tube_r)
        assert abs(oracle.weighting_potential(f, W.W_MAP, r) - exact) < 2e-3
