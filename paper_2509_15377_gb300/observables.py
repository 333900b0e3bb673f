"""Transport observables of a set of avalanches with standard errors.

Host analysis of endpoint records (numpy), used to compare two samples of
the same process, e.g. the mixed-precision GPU path against the FP64
oracle.  The electrons of one avalanche are correlated (they descend from
the same primaries), so the independent units are avalanches: every
observable is formed from per-avalanche sums and its standard error comes
from a bootstrap over avalanches.

The definitions are those of the library's avalanche_observables.
Plate geometry (collected = reached the anode):
  gain  G = mean over avalanches with primaries of collected electrons /
        primaries (Sec. 2);
  alpha = ln G / gap (Townsend coefficient of the mean gain);
  vd    = sum dz / sum dt over collected electrons (drift velocity);
  DT    = <dx^2 + dy^2> / (4 <dt>);  DL = var(dz) / (2 <dt>), the variance
        with n - 1.
Coaxial geometry (collected = reached the wire): G; the radial drift
velocity vr = sum (r0 - r1) / sum dt; the mean turn about the wire of the
collected electrons (rad, from the Lorentz force in an axial B); DL along the
wire, var(dz) / (2 <dt>).
"""
from __future__ import annotations

import math

import numpy as np


def per_avalanche(out: dict, n_avalanches: int, collect: int, n_primaries,
                  geometry: str = "plate") -> dict:
    """Per-avalanche sums over the electrons that end with status `collect`."""
    m = out["status"] == collect
    a = np.asarray(out["aval"])[m].astype(np.int64)

    def s(v):
        return np.bincount(a, weights=v, minlength=n_avalanches)[:n_avalanches]

    dt = (out["t1"] - out["t0"])[m]
    dz = (out["z1"] - out["z0"])[m]
    sums = {"n": s(np.ones_like(dt)), "prim": np.asarray(n_primaries, np.float64)[:n_avalanches],
            "dt": s(dt), "dz": s(dz), "dz2": s(dz * dz)}
    if geometry == "plate":
        dx, dy = (out["x1"] - out["x0"])[m], (out["y1"] - out["y0"])[m]
        sums["tr"] = s(dx * dx + dy * dy)
    else:
        x0, y0, x1, y1 = (out[k][m] for k in ("x0", "y0", "x1", "y1"))
        sums["dr"] = s(np.hypot(x0, y0) - np.hypot(x1, y1))
        sums["turn"] = s(np.angle(np.exp(1j * (np.arctan2(y1, x1) - np.arctan2(y0, x0)))))
    return sums


def estimates(sums: dict, gap: float, geometry: str = "plate") -> dict:
    """Observables from per-avalanche sums (arrays [..., n_avalanches]; the
    sums run over the last axis)."""
    tot = {k: np.asarray(v).sum(axis=-1) for k, v in sums.items()}
    n = tot["n"]
    prim = np.asarray(sums["prim"])
    with np.errstate(divide="ignore", invalid="ignore"):
        has = prim > 0
        gain = (np.where(has, np.asarray(sums["n"]) / np.where(has, prim, 1.0), 0.0).sum(axis=-1)
                / has.sum(axis=-1))
        mdt = tot["dt"] / n
        var_z = (tot["dz2"] - tot["dz"] * tot["dz"] / n) / (n - 1.0)
        out = {"gain": gain}
        if geometry == "plate":
            out["alpha"] = np.log(gain) / gap
            out["vd"] = tot["dz"] / tot["dt"]
            out["DT"] = tot["tr"] / n / (4.0 * mdt)
            out["DL"] = var_z / (2.0 * mdt)
        else:
            out["vr"] = tot["dr"] / tot["dt"]
            out["turn"] = tot["turn"] / n
            out["DL"] = var_z / (2.0 * mdt)
    return out


def with_errors(sums: dict, gap: float, geometry: str = "plate", n_boot: int = 1000,
                seed: int = 0) -> dict:
    """{name: (estimate, bootstrap standard error)} over the avalanches with
    at least one primary."""
    keep = np.asarray(sums["prim"]) > 0
    S = {k: np.asarray(v)[keep] for k, v in sums.items()}
    est = estimates(S, gap, geometry)
    na = int(keep.sum())
    idx = np.random.default_rng(seed).integers(0, na, size=(n_boot, na))
    boot = estimates({k: v[idx] for k, v in S.items()}, gap, geometry)
    return {k: (float(est[k]), float(np.std(boot[k], ddof=1))) for k in est}


def compare(a: dict, b: dict) -> dict:
    """Two independent samples' observables (from with_errors): per
    observable the values, their errors, the relative difference of b from a
    and the difference in units of the combined error."""
    rows = {}
    for k in a:
        (va, sa), (vb, sb) = a[k], b[k]
        sig = math.hypot(sa, sb)
        rows[k] = {"a": va, "se_a": sa, "b": vb, "se_b": sb,
                   "rel_diff": (vb - va) / va if va else float("nan"),
                   "sigma": (vb - va) / sig if sig > 0 else float("nan"),
                   "within_3sigma": bool(abs(vb - va) <= 3.0 * sig)}
    return rows
