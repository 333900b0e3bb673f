"""Pins of the banded majorant when the field changes along a flight.

With sub-steps the field is re-evaluated during a flight, so the energy
reach of the window can no longer come from the field held at the flight's
start.  The oracle then bounds |E| along the flight by the largest field
magnitude of the volume, E_max, and the energy change over the window tau by
D = E_max (|v| tau + a1 E_max tau^2 / 2) (the field does work -q E.v, and
|v| grows at most by a1 E_max per unit time; a magnetic field does no work).
Null-collision thinning is exact only while the majorant covers the true
rate along the whole flight (Skullerud's technique, Sec. 1), so these tests
check, independently of the oracle's running sums:

- E_max itself against a brute-force maximum of |E| for each field kind
  (coax: the closed form at the wire surface; grid and mesh: every node and
  random interior points, since an interpolated field is a convex
  combination of node values);
- the rate along sub-stepped flights in coax (with and without B), grid and
  mesh fields: each sub-step moves exactly in the field at its start, and at
  fine points along it the total rate interpolated from the per-level input
  table (np.interp of the summed levels) never exceeds the majorant;
- that the walk has the power to see a wrong bound: with E_max halved, some
  flights reach a rate above the majorant.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import workloads as W

from tests import physics as P

GAS = W.argon_like_gas()
NODES = np.arange(GAS.n_nodes) * GAS.d_eps
TOTAL = GAS.rate.sum(axis=1)        # the input table's levels summed, not the oracle's sums


def _field(kind):
    if kind == "coax":
        return W.Field(W.COAX, wire_r=25e-4, tube_r=0.5, voltage=1500.0)
    if kind == "coax_b":
        return W.Field(W.COAX, wire_r=25e-4, tube_r=0.5, voltage=1500.0, b=(0.0, 0.0, 1.0))
    if kind == "grid":
        return W.coax_grid_map(n=48, half_width=0.02, length=0.05, voltage=1500.0)
    if kind == "mesh":
        return W.coax_mesh_map(cells=6, half_width=0.02, length=0.05, voltage=1500.0, seed=5,
                               grading=1.5)
    raise ValueError(kind)


def _node_emax(field):
    if field.kind == W.GRID:
        v = field.grid.reshape(-1, 4).astype(np.float64)
    else:
        v = field.mesh_values.astype(np.float64)
    return float(np.sqrt((v[:, :3] ** 2).sum(axis=1)).max())


def _random_inside(field, rng, n):
    """Random points strictly inside the volume (status 0)."""
    pts = []
    while len(pts) < n:
        if field.kind == W.COAX:
            r = rng.uniform(field.wire_r, 0.2)
            phi = rng.uniform(0.0, 2.0 * math.pi)
            p = np.array([r * math.cos(phi), r * math.sin(phi), rng.uniform(-1.0, 1.0)])
        elif field.kind == W.GRID:
            n_xyz = np.array(field.grid.shape[2::-1]) - 1
            hi = np.array(field.origin) + np.array(field.spacing) * n_xyz
            p = rng.uniform(np.array(field.origin), hi)
        else:
            lo, hi = field.mesh_nodes.min(axis=0), field.mesh_nodes.max(axis=0)
            p = rng.uniform(lo, hi)
        if oracle.boundary(field, p) == 0:
            pts.append(p)
    return pts


@pytest.mark.parametrize("kind", ["coax", "grid", "mesh"])
def test_field_emax_is_the_largest_field_magnitude(kind):
    field = _field(kind)
    emax = oracle.field_emax(field)
    if kind == "coax":
        closed = field.voltage / (field.wire_r * math.log(field.tube_r / field.wire_r))
        assert emax == pytest.approx(closed, rel=1e-12)
        rs = field.wire_r * np.exp(np.linspace(0.0, math.log(field.tube_r / field.wire_r), 2000))
        mags = [np.linalg.norm(oracle.field_eval(field, [r, 0.0, 0.0])) for r in rs]
        assert max(mags) == pytest.approx(emax, rel=1e-12)
    else:
        assert emax == pytest.approx(_node_emax(field), rel=1e-12)
    rng = np.random.default_rng(17)
    worst = max(np.linalg.norm(oracle.field_eval(field, p)) for p in _random_inside(field, rng, 3000))
    assert worst <= emax * (1.0 + 1e-12)


def _starts(field, rng, n):
    """Flight starts where the field is close to its largest magnitude (near
    the wire, or near the node of the largest field), half of them moving
    along the electron's acceleration, mixed with random starts."""
    if field.kind == W.COAX:
        anchor = None
    else:
        vals = field.grid.reshape(-1, 4) if field.kind == W.GRID else field.mesh_values
        i = int(np.argmax((vals[:, :3].astype(np.float64) ** 2).sum(axis=1)))
        if field.kind == W.GRID:
            nz, ny, nx = field.grid.shape[:3]
            k, rem = divmod(i, ny * nx)
            j, ii = divmod(rem, nx)
            anchor = np.array(field.origin) + np.array(field.spacing) * np.array([ii, j, k])
        else:
            anchor = field.mesh_nodes[i].copy()
    out = []
    while len(out) < n:
        if rng.uniform() < 0.75:
            if anchor is None:
                r = field.wire_r * rng.uniform(1.0, 1.6)
                phi = rng.uniform(0.0, 2.0 * math.pi)
                p = np.array([r * math.cos(phi), r * math.sin(phi), 0.0])
            else:
                p = anchor + rng.normal(scale=3e-4, size=3)
            if oracle.boundary(field, p) != 0:
                continue
        else:
            p = _random_inside(field, rng, 1)[0]
        e = oracle.field_eval(field, p)
        eps0 = rng.choice([0.0, rng.uniform(0.0, 5.0), rng.uniform(0.0, 30.0)])
        if rng.uniform() < 0.5 and np.linalg.norm(e) > 0.0:
            d = -e / np.linalg.norm(e)          # along the electron's acceleration
        else:
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
        out.append((p, math.sqrt(P.speed_sq(eps0)) * d))
    return out


def _walk(field, r, v, dt, n_sub, n_fine):
    """Energies (eV) at fine points of a flight of length dt in n_sub equal
    sub-steps, each in the field at its own start (the sub-step reading),
    up to the end of the first sub-step that ends outside the volume."""
    w = -P.OMEGA_PER_T * np.asarray(field.b, np.float64)
    has_b = bool(np.any(w != 0.0))
    h = dt / n_sub
    eps = [float(v @ v) / (2.0 * P.ACCEL_PER_VCM)]
    for _ in range(n_sub):
        acc = -P.ACCEL_PER_VCM * oracle.field_eval(field, r)
        for m in range(1, n_fine + 1):
            t = h * m / n_fine
            if has_b:
                _, u = oracle.flight(r, v, acc, w, t)   # exact Lorentz motion (pinned against RK4)
            else:
                u = v + acc * t
            eps.append(float(u @ u) / (2.0 * P.ACCEL_PER_VCM))
        if has_b:
            r, v = oracle.flight(r, v, acc, w, h)
        else:
            r, v = r + v * h + 0.5 * acc * h * h, v + acc * h
        if oracle.boundary(field, r) != 0:
            break
    return np.array(eps)


def _excess(kind, emax_scale, n_flights, seed):
    """Largest ratio of the true rate along a flight to its majorant, over
    random sub-stepped flights, with the oracle's majorant computed from
    emax_scale x E_max."""
    field = _field(kind)
    emax = oracle.field_emax(field) * emax_scale
    rng = np.random.default_rng(seed)
    ratios = []
    for r0, v0 in _starts(field, rng, n_flights):
        bw = float(rng.choice([0.25, 1.0]))
        window = float(rng.choice([0.002, 0.01, 0.05, 2.0]))
        nu_w, tau = oracle.majorant_reach(GAS, bw, v0, emax, window)
        dt = tau if rng.uniform() < 0.5 else rng.uniform(0.0, tau)
        n_sub = int(rng.choice([2, 8, 32]))
        eps = _walk(field, r0, v0, dt, n_sub, 6)
        ratios.append(float(np.interp(eps, NODES, TOTAL).max()) / nu_w)
    return np.array(ratios)


@pytest.mark.parametrize("kind", ["coax", "coax_b", "grid", "mesh"])
def test_reach_majorant_bounds_the_rate_along_substepped_flights(kind):
    ratios = _excess(kind, 1.0, 160, seed=23)
    assert ratios.max() <= 1.0 + 1e-12, ratios.max()
    assert ratios.max() > 0.9  # the bound comes close somewhere (not vacuous)


@pytest.mark.parametrize("kind", ["coax", "coax_b", "grid", "mesh"])
def test_halved_field_bound_is_caught(kind):
    """Planted mistake: the oracle's majorant built from E_max / 2 lets some
    flights reach a rate above it."""
    ratios = _excess(kind, 0.5, 160, seed=23)
    assert ratios.max() > 1.0 + 1e-9, ratios.max()
