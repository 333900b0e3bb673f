"""The seeded synthetic inputs follow their stated recipes (CPU): the
per-avalanche fields and primary counts of the 4096-avalanche plate
workload, the gas half-space of plate primaries, the radii of the tube's
primaries, the start of the grid-map primaries, and reproducibility by
seed."""
import math

import numpy as np
from scipy import stats

from paper_2509_15377_gb300 import workloads as W


def test_plate_batched_recipe():
    w = W.plate_batched(n_avalanches=4096, seed=0)
    p = w.primaries
    assert p.n_avalanches == 4096
    # per-avalanche field ~ U(30, 50) kV/cm
    f = p.aval_field
    assert f.shape == (4096,) and f.min() >= 30_000.0 and f.max() <= 50_000.0
    assert stats.kstest((f - 30_000.0) / 20_000.0, "uniform").pvalue > 0.001
    # Poisson(3) primaries per avalanche, empty avalanches kept
    counts = np.bincount(p.aval, minlength=4096)
    assert abs(counts.mean() - 3.0) < 3 * math.sqrt(3.0 / 4096)
    assert abs(counts.var() / counts.mean() - 1.0) < 0.1
    assert (counts == 0).sum() > 0
    # on the cathode, 0.1 eV, at t = 0, ids = input indices
    assert np.all(p.x == 0) and np.all(p.y == 0) and np.all(p.z == 0) and np.all(p.t == 0)
    assert np.all(p.e == 0.1)
    assert np.array_equal(p.uid, np.arange(p.n, dtype=np.uint64))
    # unit directions, isotropic in the gas half-space: cos(theta) ~ U(0, 1)
    assert np.allclose(p.dx ** 2 + p.dy ** 2 + p.dz ** 2, 1.0, atol=1e-12)
    assert p.dz.min() >= 0.0
    assert stats.kstest(p.dz, "uniform").pvalue > 0.001
    phi = np.arctan2(p.dy, p.dx)
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 0.001
    # gap, field kind, time limit
    assert w.field.kind == W.PLATE and w.field.gap == 0.0128 and w.t_max == 100.0


def test_plate_recipe():
    w = W.plate(n_avalanches=1000, e_field=40_000.0, seed=0)
    p = w.primaries
    assert p.n == 1000 and np.array_equal(p.aval, np.arange(1000))
    assert w.field.e0 == 40_000.0 and p.dz.min() >= 0.0


def test_coax_recipe():
    w = W.coax(n_avalanches=2048, seed=0)
    p = w.primaries
    r = np.hypot(p.x, p.y)
    assert p.n == 2048 and r.min() >= 0.1 and r.max() <= 0.45
    assert stats.kstest((r - 0.1) / 0.35, "uniform").pvalue > 0.001
    phi = np.arctan2(p.y, p.x)
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 0.001
    assert np.all(p.z == 0.0) and w.t_max == 10_000.0
    assert w.field.kind == W.COAX and tuple(w.field.b) == (0.0, 0.0, 1.0)
    # isotropic in full: cos(theta) ~ U(-1, 1)
    assert stats.kstest((p.dz + 1.0) / 2.0, "uniform").pvalue > 0.001


def test_grid_stress_recipe():
    w = W.grid_stress(n_avalanches=64, n=16, seed=0)
    p = w.primaries
    f = w.field
    assert f.kind == W.GRID and f.grid.shape == (16, 16, 16, 4)
    assert np.allclose(np.hypot(p.x, p.y), 0.1, rtol=1e-12)
    zc = f.origin[2] + 0.5 * f.spacing[2] * 15
    assert np.allclose(p.z, zc, rtol=1e-12)


def test_inputs_are_reproducible_by_seed():
    a = W.plate_batched(n_avalanches=256, seed=3).primaries
    b = W.plate_batched(n_avalanches=256, seed=3).primaries
    c = W.plate_batched(n_avalanches=256, seed=4).primaries
    for k in ("dx", "dy", "dz", "aval", "aval_field"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    assert not np.array_equal(a.aval_field, c.aval_field)


def test_subset_keeps_avalanche_numbers_and_ids():
    p = W.plate_batched(n_avalanches=64, seed=1).primaries
    s = p.subset([3, 10, 11])
    assert set(np.unique(s.aval).tolist()) <= {3, 10, 11}
    keep = np.isin(p.aval, [3, 10, 11])
    assert np.array_equal(s.uid, p.uid[keep]) and np.array_equal(s.dz, p.dz[keep])
    assert s.n_avalanches == 64 and np.array_equal(s.aval_field, p.aval_field)
