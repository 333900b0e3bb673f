"""The host observables (paper_2509_15377_gb300/observables.py) on endpoint
sets built by hand, against their definitions computed directly from the
electrons (no GPU, no oracle)."""
import math

import numpy as np
import pytest

from paper_2509_15377_gb300 import observables as O

ANODE, CATHODE, WIRE = 1, 2, 3


def _endpoints(rows):
    """rows: (aval, status, x0, y0, z0, t0, x1, y1, z1, t1)."""
    a = np.array(rows, dtype=np.float64)
    keys = ("aval", "status", "x0", "y0", "z0", "t0", "x1", "y1", "z1", "t1")
    out = {k: a[:, i] for i, k in enumerate(keys)}
    out["aval"] = out["aval"].astype(np.int64)
    out["status"] = out["status"].astype(np.int64)
    return out


def test_plate_observables_follow_their_definitions():
    rng = np.random.default_rng(5)
    rows = []
    n_aval = 4
    for av in range(n_aval):
        for _ in range(rng.integers(3, 9)):
            st = ANODE if rng.random() < 0.8 else CATHODE
            x0, y0, z0, t0 = rng.normal(size=3).tolist() + [rng.random()]
            dx, dy, dz, dt = rng.normal(size=3).tolist() + [1.0 + rng.random()]
            rows.append((av, st, x0, y0, z0, t0, x0 + dx, y0 + dy, z0 + dz, t0 + dt))
    out = _endpoints(rows)
    prim = np.array([1, 2, 0, 3])  # avalanche 2 has no primaries: not in the gain
    gap = 0.0128
    est = O.estimates(O.per_avalanche(out, n_aval, ANODE, prim), gap)

    m = out["status"] == ANODE
    dx, dy = (out["x1"] - out["x0"])[m], (out["y1"] - out["y0"])[m]
    dz, dt = (out["z1"] - out["z0"])[m], (out["t1"] - out["t0"])[m]
    counts = np.array([np.sum(out["aval"][m] == i) for i in range(n_aval)])
    gain = np.mean([counts[i] / prim[i] for i in range(n_aval) if prim[i] > 0])
    assert est["gain"] == pytest.approx(gain, rel=1e-12)
    assert est["alpha"] == pytest.approx(math.log(gain) / gap, rel=1e-12)
    assert est["vd"] == pytest.approx(dz.sum() / dt.sum(), rel=1e-12)
    assert est["DT"] == pytest.approx(np.mean(dx * dx + dy * dy) / (4 * dt.mean()), rel=1e-12)
    assert est["DL"] == pytest.approx(np.var(dz, ddof=1) / (2 * dt.mean()), rel=1e-10)


def test_coax_turn_is_taken_the_short_way_round():
    """An electron that crosses the -pi/pi cut turns by a small angle, not
    by nearly 2 pi; the radial velocity is the drop in radius over time."""
    eps = 0.05

    def pt(r, th):
        return r * math.cos(th), r * math.sin(th)

    # electron 0: from angle pi - eps at r = 1 to -pi + eps at r = 0.5 (turn +2 eps)
    # electron 1: from angle 0 at r = 1 to 0.1 at r = 0.5 (turn +0.1)
    (a0, b0), (a1, b1) = pt(1.0, math.pi - eps), pt(0.5, -math.pi + eps)
    (c0, d0), (c1, d1) = pt(1.0, 0.0), pt(0.5, 0.1)
    rows = [(0, WIRE, a0, b0, 0.0, 0.0, a1, b1, 0.0, 2.0),
            (0, WIRE, c0, d0, 0.0, 0.0, c1, d1, 0.0, 2.0)]
    out = _endpoints(rows)
    est = O.estimates(O.per_avalanche(out, 1, WIRE, np.array([2]), "coax"), 0.0, "coax")
    assert est["turn"] == pytest.approx((2 * eps + 0.1) / 2, rel=1e-12)
    assert est["vr"] == pytest.approx((0.5 + 0.5) / 4.0, rel=1e-12)
    assert est["gain"] == pytest.approx(1.0)


def test_bootstrap_error_of_the_gain_matches_its_spread():
    """Independent avalanches with their own gains: the bootstrap error of
    the mean gain agrees with the spread of the mean over repeats."""
    rng = np.random.default_rng(7)
    n = 200

    def sample():
        g = rng.geometric(1.0 / 50.0, size=n).astype(np.float64)
        return {"n": g, "prim": np.ones(n), "dt": g * 2.0, "dz": g * 1e-3, "dz2": g * 1e-6,
                "tr": g * 1e-6}

    means, ses = [], []
    for k in range(60):
        s = sample()
        means.append(O.estimates(s, 0.0128)["gain"])
        if k < 10:
            ses.append(O.with_errors(s, 0.0128, n_boot=400, seed=k)["gain"][1])
    spread = float(np.std(means, ddof=1))
    assert 0.7 < np.mean(ses) / spread < 1.4, (np.mean(ses), spread)


def test_compare_flags_a_shift_beyond_three_sigma():
    a = {"gain": (100.0, 2.0)}
    assert O.compare(a, {"gain": (104.0, 2.0)})["gain"]["within_3sigma"]
    r = O.compare(a, {"gain": (110.0, 2.0)})["gain"]
    assert not r["within_3sigma"]
    assert r["sigma"] == pytest.approx(10.0 / math.hypot(2.0, 2.0))
    assert r["rel_diff"] == pytest.approx(0.1)
