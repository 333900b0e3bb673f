"""Pins of the oracle's tetrahedral-mesh field (Sec. 3.1: field maps are
finite-element solutions on tetrahedral meshes; a point's element is searched
and the element's nodal values interpolated) against facts that do not come
from the oracle: the mesh tiles its box, linear interpolation reproduces an
affine field, a value next to a node is the node's value, and a mesh that
carries a constant field transports exactly like the uniform field.

A slip in the oracle's element search or interpolation (a node order, a sign
of a barycentric coordinate, a transposed edge vector, a wrong value column)
fails one of these.
"""
import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import workloads as W


@pytest.fixture(scope="module")
def coax_mesh():
    return W.coax_mesh_map(cells=6, seed=3)


def _tet_volumes(f):
    v = f.mesh_nodes[f.mesh_tets]
    return np.einsum("ij,ij->i", v[:, 1] - v[:, 0],
                     np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0])) / 6.0


@pytest.mark.parametrize("grading", [0.0, 3.0])
def test_mesh_tiles_its_box(coax_mesh, grading):
    """Positive volumes summing to the box; every interior point lies in
    exactly one element (counted with a separate linear solve per element);
    also for a mesh graded towards the axis."""
    f = coax_mesh if grading == 0.0 else W.coax_mesh_map(cells=6, seed=3, grading=grading)
    vol = _tet_volumes(f)
    assert vol.min() > 0.0
    assert vol.sum() == pytest.approx(0.3 * 0.3 * 1.0, rel=1e-12)
    rng = np.random.default_rng(5)
    pts = rng.uniform([-0.15, -0.15, 0.0], [0.15, 0.15, 1.0], (40, 3))
    v = f.mesh_nodes[f.mesh_tets]
    edges = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)  # [m, 3, 3]
    for p in pts:
        lam = np.linalg.solve(edges, (p - v[:, 0])[:, :, None])[:, :, 0]
        full = np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)
        holders = np.nonzero(full.min(axis=1) > 1e-9)[0]
        assert len(holders) == 1
        t, bary = oracle.mesh_locate(f, p)
        assert t == holders[0]
        np.testing.assert_allclose(bary, full[t], atol=1e-12)
        np.testing.assert_allclose(bary @ v[t], p, atol=1e-14)


def test_mesh_interpolation_exact_on_affine_values():
    """Nodal values of an affine field are reproduced everywhere inside (to
    the float32 rounding of the stored nodal values)."""
    f = W.coax_mesh_map(cells=5, seed=7)
    A = np.array([[120.0, -35.0, 8.0], [22.0, 61.0, -14.0], [-9.0, 17.0, 250.0]])
    c = np.array([300.0, -150.0, 75.0])
    vals = np.zeros((f.mesh_nodes.shape[0], 4), np.float32)
    vals[:, :3] = f.mesh_nodes @ A.T + c
    vals[:, 3] = f.mesh_nodes @ np.array([0.5, -2.0, 1.25]) + 0.3
    g = W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets, mesh_values=vals)
    rng = np.random.default_rng(11)
    for p in rng.uniform([-0.15, -0.15, 0.0], [0.15, 0.15, 1.0], (30, 3)):
        e = oracle.field_eval(g, p)
        np.testing.assert_allclose(e, A @ p + c, rtol=2e-6, atol=2e-4)
        phi = oracle.weighting_potential(g, W.W_MAP, p)
        assert phi == pytest.approx(0.5 * p[0] - 2.0 * p[1] + 1.25 * p[2] + 0.3, abs=1e-6)


def test_mesh_value_next_to_a_node(coax_mesh):
    """Just inside an element, next to one of its nodes, the field is that
    node's stored value."""
    f = coax_mesh
    rng = np.random.default_rng(2)
    for t in rng.choice(f.mesh_tets.shape[0], 20, replace=False):
        q = f.mesh_tets[t]
        v = f.mesh_nodes[q]
        k = int(rng.integers(4))
        p = v[k] + 1e-9 * (v.mean(axis=0) - v[k])
        e = oracle.field_eval(f, p)
        np.testing.assert_allclose(e, f.mesh_values[q[k], :3].astype(np.float64), rtol=1e-6,
                                   atol=1e-3)


def test_mesh_boundary_status(coax_mesh):
    f = coax_mesh
    assert oracle.boundary(f, np.array([0.05, 0.02, 0.5])) == 0
    assert oracle.boundary(f, np.array([0.0, 0.001, 0.5])) == W.WIRE
    assert oracle.boundary(f, np.array([0.2, 0.0, 0.5])) == W.OUT_OF_MAP
    assert oracle.boundary(f, np.array([0.05, 0.0, -1e-6])) == W.OUT_OF_MAP
    assert oracle.mesh_locate(f, np.array([0.05, 0.0, 1.0 + 1e-9]))[0] == -1


def test_mesh_coax_field_approaches_the_closed_form(coax_mesh):
    """Far from the wire the mesh's linear interpolation of the coax field
    is close to the closed form (refining the mesh brings it closer)."""
    errs = []
    rng = np.random.default_rng(4)
    pts = []
    while len(pts) < 12:
        p = rng.uniform([-0.14, -0.14, 0.1], [0.14, 0.14, 0.9])
        if np.hypot(p[0], p[1]) > 0.09:
            pts.append(p)
    for cells in (4, 12):
        f = W.coax_mesh_map(cells=cells, seed=1)
        err = 0.0
        for p in pts:
            r2 = p[0] ** 2 + p[1] ** 2
            s = f.voltage / (np.log(f.tube_r / f.wire_r) * r2)
            exact = np.array([s * p[0], s * p[1], 0.0])
            err = max(err, np.linalg.norm(oracle.field_eval(f, p) - exact) / np.linalg.norm(exact))
        errs.append(err)
    assert errs[1] < 0.5 * errs[0]
    assert errs[1] < 0.05


def test_constant_field_mesh_transports_like_uniform():
    """A mesh that carries E = (0, 0, -E0) at every node is, inside, the
    uniform field: same electrons, same endpoints (held field per flight)."""
    w = W.drift_model(n_electrons=40, n_coll=2000, e_field=2000.0, seed=6)
    mesh = W.uniform_mesh_map(2000.0, half_width=0.5, cells=4, seed=2)
    a = oracle.run(w.gas, w.field, w.primaries, seed=9, coll_limit=w.coll_limit, majorant=1)
    b = oracle.run(w.gas, mesh, w.primaries, seed=9, coll_limit=w.coll_limit, majorant=1)
    ia, ib = np.argsort(a["uid"]), np.argsort(b["uid"])
    assert np.array_equal(a["uid"][ia], b["uid"][ib])
    assert np.array_equal(a["status"][ia], b["status"][ib])
    for k in ("x1", "y1", "z1", "t1", "e1"):
        np.testing.assert_allclose(b[k][ib], a[k][ia], rtol=1e-9, atol=1e-12)
    assert np.abs(np.stack([b["x1"], b["y1"], b["z1"]])).max() < 0.5


def test_mesh_arrays_of_the_wrong_shape_are_refused():
    """The binding and the oracle wrapper refuse mesh arrays whose shapes
    the C code would read past."""
    from paper_2509_15377_gb300 import avalanche as A
    f = W.coax_mesh_map(cells=2, seed=1)
    bad = [W.Field(W.MESH, mesh_nodes=f.mesh_nodes[:, :2], mesh_tets=f.mesh_tets,
                   mesh_values=f.mesh_values),
           W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets[:, :3],
                   mesh_values=f.mesh_values),
           W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets,
                   mesh_values=f.mesh_values[:-1]),
           W.Field(W.MESH, mesh_nodes=f.mesh_nodes, mesh_tets=f.mesh_tets,
                   mesh_values=f.mesh_values[:, :3])]
    for g in bad:
        with pytest.raises(ValueError):
            A.mesh_arrays(g)
        with pytest.raises(ValueError):
            oracle.field_eval(g, np.zeros(3))
    nodes, tets, vals = A.mesh_arrays(f)
    assert nodes.shape[1] == 3 and tets.shape[1] == 4 and vals.shape == (nodes.shape[0], 4)



def test_mesh_signal_telescopes():
    """Shockley-Ramo on a mesh: an avalanche's signal summed over its bins is
    the sum over its electrons of the weighting potential at the end minus
    at the start (every electron's life inside the binned window)."""
    f = W.coax_mesh_map(cells=6, half_width=0.02, length=0.05, voltage=1500.0, seed=9)
    w = W.mesh_coax(n_avalanches=12, cells=2, seed=9)
    w.field = f
    ph = np.random.default_rng(9).uniform(0, 2 * np.pi, 12)
    w.primaries.x[:] = 0.008 * np.cos(ph)
    w.primaries.y[:] = 0.008 * np.sin(ph)
    w.primaries.z[:] = 0.025
    t_max = 0.3
    out = oracle.run(w.gas, f, w.primaries, seed=9, t_max=t_max, signal=(W.W_MAP, 100, 0.0, 0.003))
    phi = lambda x, y, z: np.array([oracle.weighting_potential(f, W.W_MAP, np.array(p))
                                    for p in zip(x, y, z)])
    d = phi(out["x1"], out["y1"], out["z1"]) - phi(out["x0"], out["y0"], out["z0"])
    expect = np.bincount(out["aval"], weights=d, minlength=12)
    assert np.abs(expect).max() > 0.0
    np.testing.assert_allclose(out["signal"].sum(axis=1), expect, rtol=1e-9,
                               atol=1e-12 * np.abs(expect).max())


def test_crossing_out_of_a_mesh_closed_form():
    """Collisionless electrons pushed out of the top face of a constant-field
    mesh: with exact crossings each ends on that face, at the closed-form
    time of uniform acceleration t* = (sqrt(vz^2 + 2 a h) - vz) / a, h the
    distance to the face; without them, far beyond it."""
    from tests import physics as P
    w = W.plate(n_avalanches=40, e_field=30_000.0, seed=71)
    w.gas = W.model_gas(1e-9)
    half = 0.02
    mesh = W.uniform_mesh_map(30_000.0, half_width=half, cells=4, seed=5)
    w.primaries.z[:] = 0.0  # the centre of the cube; the field pushes them to +z
    a = P.ACCEL_PER_VCM * 30_000.0
    vz = w.primaries.dz * np.sqrt(P.speed_sq(w.primaries.e))
    ts = (np.sqrt(vz * vz + 2 * a * half) - vz) / a
    o = oracle.run(w.gas, mesh, w.primaries, seed=71, t_max=100.0, crossing=True)
    idx = np.argsort(o["uid"])
    assert np.all(o["status"] == W.OUT_OF_MAP)
    np.testing.assert_allclose((o["t1"] - o["t0"])[idx], ts, rtol=1e-9)
    assert np.all(np.abs(o["z1"] - half) < 1e-12)
    p = oracle.run(w.gas, mesh, w.primaries, seed=71, t_max=100.0)
    assert np.all(p["z1"] > 1.0)
