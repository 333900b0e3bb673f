"""GPU parity for fields on tetrahedral meshes: FP64 per electron against the
oracle (held field, sub-steps with crossings, induced signals, a mesh with a
hole), mixed precision against the oracle's distributions, and a mesh that
carries a constant field against the uniform field kind."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import (assert_same_electrons, by_uid, paired_avalanche_ks, ratio_se,
                               run_gpu, two_sample_ks)

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


def _near_wire(n, seed, cells=6, hole=False):
    """Coax field on a jittered mesh of a 400 um box around the wire; the
    primaries start at r = 80 um, mid-length.  `hole` drops the elements of
    one quadrant whose centre is within 75 um of the axis, on the way of the
    electrons drifting in from that quadrant (points there are in no element)."""
    f = W.coax_mesh_map(cells=cells, half_width=0.02, length=0.05, voltage=1500.0, seed=seed)
    if hole:
        c = f.mesh_nodes[f.mesh_tets].mean(axis=1)
        keep = ~((c[:, 0] > 0.0) & (c[:, 1] > 0.0) & (np.hypot(c[:, 0], c[:, 1]) < 0.0075))
        f.mesh_tets = np.ascontiguousarray(f.mesh_tets[keep])
    w = W.mesh_coax(n_avalanches=n, cells=2, seed=seed)
    w.field = f
    ph = np.random.default_rng(seed).uniform(0, 2 * math.pi, n)
    w.primaries.x[:] = 0.008 * np.cos(ph)
    w.primaries.y[:] = 0.008 * np.sin(ph)
    w.primaries.z[:] = 0.025
    return w


def _setup(av, w):
    av.set_gas(w.gas)
    av.set_field(w.field)


@pytest.mark.parametrize("mode", [A.GT_BATCHED, A.GT_PLAIN])
@pytest.mark.parametrize("majorant", [0, 1])
def test_fp64_mesh_per_collision(av, mode, majorant):
    w = _near_wire(20, seed=21)
    _setup(av, w)
    t_max = 0.3
    ref = oracle.run(w.gas, w.field, w.primaries, seed=21, t_max=t_max, majorant=majorant,
                     window=2.0)
    st, out = run_gpu(av, w, seed=21, t_max=t_max, mode=mode, majorant=majorant,
                      majorant_window=2.0, capacity=4 * len(ref["uid"]) + 64)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=t_max)
    assert np.array_equal(out["tallies"], ref["tallies"])


def test_fp64_mesh_with_a_hole(av):
    """Electrons that enter the missing quadrant end there, out of the map."""
    w = _near_wire(24, seed=23, hole=True)
    _setup(av, w)
    t_max = 1.0
    ref = oracle.run(w.gas, w.field, w.primaries, seed=23, t_max=t_max)
    assert (ref["status"] == W.OUT_OF_MAP).sum() > 0
    st, out = run_gpu(av, w, seed=23, t_max=t_max, capacity=4 * len(ref["uid"]) + 64)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=t_max)


def test_fp64_mesh_substeps_and_crossing(av):
    w = _near_wire(16, seed=25)
    _setup(av, w)
    t_max = 0.2
    ref = oracle.run(w.gas, w.field, w.primaries, seed=25, t_max=t_max, substeps=3, crossing=True,
                     majorant=1, window=2.0)
    _, out = run_gpu(av, w, seed=25, t_max=t_max, substeps=3, crossing=1, majorant=1,
                     majorant_window=2.0, capacity=4 * len(ref["uid"]) + 64)
    assert_same_electrons(out, ref, scale_pos=0.01, scale_t=t_max)


def test_fp64_mesh_signal_per_bin(av):
    w = _near_wire(16, seed=27)
    _setup(av, w)
    sig = (W.W_MAP, 100, 0.0, 0.003)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=27, t_max=0.3, signal=sig)
    _, out = run_gpu(av, w, seed=27, t_max=0.3, capacity=4 * len(ref["uid"]) + 64,
                     signal_kind=sig[0], signal_bins=sig[1], signal_t0=sig[2], signal_dt=sig[3])
    scale = np.abs(ref["signal"]).max()
    assert scale > 0.0
    assert np.allclose(out["signal"], ref["signal"], rtol=1e-9, atol=1e-9 * scale)


@pytest.mark.parametrize("precision", [A.GT_FP64, A.GT_MIXED])
def test_constant_field_mesh_equals_uniform_kind(av, precision):
    """On the GPU, a mesh carrying E = (0, 0, -E0) at every node transports
    exactly as the uniform field (its gradients are zero, so the field is
    the same number, and every electron stays inside)."""
    w = W.drift_model(n_electrons=256, n_coll=3000, e_field=2000.0, seed=29)
    _setup(av, w)
    _, a = run_gpu(av, w, seed=29, precision=precision, majorant=1, majorant_window=2.0)
    av.set_field(W.uniform_mesh_map(2000.0, half_width=0.5, cells=5, seed=4))
    _, b = run_gpu(av, w, seed=29, precision=precision, majorant=1, majorant_window=2.0)
    ga, gb = by_uid(a), by_uid(b)
    assert np.array_equal(ga["uid"], gb["uid"])
    assert np.array_equal(ga["status"], gb["status"])
    for k in ("x1", "y1", "z1", "t1", "e1"):
        assert np.array_equal(ga[k], gb[k]), k


def test_mixed_mesh_distributions(av):
    """Mixed precision against the FP64 oracle on the same mesh: electrons
    per avalanche, end radius and end energy after a fixed time."""
    n = 96
    w = _near_wire(n, seed=31)
    _setup(av, w)
    t_max = 0.3
    ref = oracle.run(w.gas, w.field, w.primaries, seed=31, t_max=t_max)
    _, out = run_gpu(av, w, seed=32, t_max=t_max, precision=A.GT_MIXED,
                     capacity=8 * len(ref["uid"]) + 64)
    c_ref = np.bincount(ref["aval"], minlength=n).astype(float)
    c_gpu = np.bincount(out["aval"], minlength=n).astype(float)
    se = math.sqrt(c_ref.var() / n + c_gpu.var() / n)
    assert abs(c_ref.mean() - c_gpu.mean()) < 3 * se + 1e-12, (c_ref.mean(), c_gpu.mean(), se)
    assert two_sample_ks(np.log1p(c_ref), np.log1p(c_gpu)).pvalue > 0.01
    # end radius and energy: KS over the electrons, with the p-value from
    # swapping whole avalanches between the runs (electrons of an avalanche
    # are correlated)
    for key in ("r", "e1"):
        va = ref[key] if key != "r" else np.hypot(ref["x1"], ref["y1"])
        vb = out[key] if key != "r" else np.hypot(out["x1"], out["y1"])
        p = paired_avalanche_ks(va, ref["aval"], vb, out["aval"], n)
        assert p > 0.001, (key, p)
    # fractions of the electrons by status, within 3 sigma of bootstrap
    # errors over avalanches (from one seed to the next the oracle's own
    # fraction on the wire ranges over 0.23-0.37 here)
    for s in (W.WIRE, W.TIME, W.OUT_OF_MAP):
        fr, fg = (ref["status"] == s).mean(), (out["status"] == s).mean()
        se = math.hypot(
            ratio_se(np.bincount(ref["aval"][ref["status"] == s], minlength=n), c_ref),
            ratio_se(np.bincount(out["aval"][out["status"] == s], minlength=n), c_gpu))
        assert abs(fr - fg) < 3 * se + 1e-12, (s, fr, fg, se)


@pytest.mark.parametrize("geo", [{}, {"substeps": 2, "crossing": True}, {"hole": True}])
def test_mixed_mesh_follows_fp64_over_a_few_flights(av, geo):
    """Over a few flights the mixed step stays on the FP64 trajectories, on a
    mesh graded towards the wire where electrons cross elements often: a
    wrong element (a search or walk slip) would show as a field error.  Also
    with sub-steps and exact crossings (the FP32 bisection on the mesh), and
    with a hole on the electrons' way (the decision that a point is in no
    element, taken in FP64 near the hole's faces)."""
    n = 200
    geo = dict(geo)
    hole = geo.pop("hole", False)
    w = _near_wire(n, seed=33)
    w.field = W.coax_mesh_map(cells=12, half_width=0.02, length=0.05, voltage=1500.0, seed=33,
                              grading=3.0)
    if hole:  # the elements of one quadrant between 40 and 55 um from the axis
        c = w.field.mesh_nodes[w.field.mesh_tets].mean(axis=1)
        rc = np.hypot(c[:, 0], c[:, 1])
        keep = ~((c[:, 0] > 0.0) & (c[:, 1] > 0.0) & (rc > 0.004) & (rc < 0.0055))
        w.field.mesh_tets = np.ascontiguousarray(w.field.mesh_tets[keep])
    r = np.random.default_rng(34).uniform(0.003, 0.008, n)
    ph = np.random.default_rng(35).uniform(0, 2 * math.pi, n)
    w.primaries.x[:] = r * np.cos(ph)
    w.primaries.y[:] = r * np.sin(ph)
    _setup(av, w)
    t_max = 0.01
    ref = oracle.run(w.gas, w.field, w.primaries, seed=33, t_max=t_max, **geo)
    _, out = run_gpu(av, w, seed=33, t_max=t_max, precision=A.GT_MIXED,
                     capacity=4 * len(ref["uid"]) + 64, substeps=geo.get("substeps", 0),
                     crossing=int(geo.get("crossing", False)))
    g, o = by_uid(out), by_uid(ref)
    prim = (g["uid"] < n) & np.isin(g["uid"], o["uid"])
    gi = np.nonzero(prim)[0]
    oi = np.searchsorted(o["uid"], g["uid"][gi])
    d = np.max(np.abs(np.stack([g[k][gi] - o[k][oi] for k in ("x1", "y1", "z1")])), axis=0)
    same = (d < 1e-6) & (g["status"][gi] == o["status"][oi]) & (g["n_flight"][gi] == o["n_flight"][oi])
    assert np.mean(o["n_flight"][oi]) > 3
    assert same.mean() > 0.9, (same.mean(), np.sort(d)[-10:])
    if hole:
        assert (o["status"] == W.OUT_OF_MAP).sum() > 0
        assert abs((g["status"] == W.OUT_OF_MAP).mean() - (o["status"] == W.OUT_OF_MAP).mean()) < 0.05


def test_mesh_setup_rejects_bad_meshes(av):
    f = W.coax_mesh_map(cells=2, half_width=0.02, length=0.05, seed=1)
    bad = W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets.copy(),
                  mesh_values=f.mesh_values)
    bad.mesh_tets[3, 1] = f.mesh_nodes.shape[0]          # node index out of range
    with pytest.raises(Exception):
        av.set_field(bad)
    flat = W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets.copy(),
                   mesh_values=f.mesh_values)
    flat.mesh_tets[0, 3] = flat.mesh_tets[0, 2]          # a zero-volume element
    with pytest.raises(Exception):
        av.set_field(flat)
    nan = W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets,
                  mesh_values=f.mesh_values.copy())
    nan.mesh_values[5, 0] = np.nan
    with pytest.raises(Exception):
        av.set_field(nan)
    av.set_field(f)                                       # a good mesh still sets up
