"""Mixed precision against the FP64 oracle on the transport observables.

The GPU's mixed-precision path (FP32 kinematics, table and scattering; FP64
position, time and decisions) runs with another seed than the FP64 oracle,
so the two are independent samples of the same process.  For each
configuration every observable must agree within 3 sigma, sigma from a
bootstrap over avalanches on each side (the electrons of one avalanche are
correlated, so avalanches are the independent units), and the per-avalanche
values must pass a two-sample KS test at p > 0.01:

- gain G (electrons collected per primary, Sec. 2) and the Townsend
  coefficient alpha = ln<G> / gap;
- drift velocity v_d = sum dz / sum dt of the collected electrons;
- transverse diffusion D_T = <dx^2 + dy^2> / (4 <dt>) and longitudinal
  D_L = var(dz) / (2 <dt>) of the collected electrons.

Configurations: the argon-like plate at 40 kV/cm (1 primary per avalanche,
400 avalanches), the batched plate workload (per-avalanche field in 30-50
kV/cm, Poisson(3) primaries, avalanches 0..511) and the coaxial tube with a
1 T axial field (256 avalanches from r in 1-4.5 mm); in the tube the drift
quantities are radial (v_r = sum (r0 - r1) / sum dt), azimuthal (the mean
turn of the collected electrons about the wire, from the Lorentz force) and
along the wire (var(dz) / (2 <dt>)); the same quantities on the 256^3
grid-map configuration (48 avalanches at gain ~1e5).

The measured differences are printed (pytest -s) for the error table.
"""
import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import observables as O
from paper_2509_15377_gb300 import workloads as W
from tests.gpu_helpers import run_gpu, two_sample_ks

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


def _compare(name, sums_ref, sums_gpu, gap, geometry):
    rows = O.compare(O.with_errors(sums_ref, gap, geometry, seed=1),
                     O.with_errors(sums_gpu, gap, geometry, seed=2))
    for k, r in rows.items():
        print(f"OBS {name} {k}: oracle {r['a']:.6g} +- {r['se_a']:.3g}, mixed {r['b']:.6g} +- "
              f"{r['se_b']:.3g}, rel diff {r['rel_diff']:+.4f}, {r['sigma']:+.2f} sigma")
    for k, r in rows.items():
        assert r["within_3sigma"], (name, k, r)
    # one value per avalanche: KS on the distributions of the collected
    # electrons per avalanche and of their mean drift time
    for key in ("n", "dt"):
        va, vb = sums_ref[key][sums_ref["n"] > 0], sums_gpu[key][sums_gpu["n"] > 0]
        if key != "n":
            va, vb = va / sums_ref["n"][sums_ref["n"] > 0], vb / sums_gpu["n"][sums_gpu["n"] > 0]
        p = two_sample_ks(va, vb).pvalue
        print(f"OBS {name} KS per-avalanche {key}: p = {p:.3f}")
        assert p > 0.01, (name, key, p)


def _n_prim(prim):
    return np.bincount(prim.aval, minlength=prim.n_avalanches)


def test_mixed_plate_observables_vs_oracle(av):
    n = 400
    w = W.plate(n_avalanches=n, e_field=40_000.0, seed=0)
    av.set_gas(w.gas)
    av.set_field(w.field)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, t_max=w.t_max, majorant=1)
    st, out = run_gpu(av, w, seed=101, precision=A.GT_MIXED, capacity=4_000_000,
                      majorant=A.GT_MAJORANT_BANDED)
    np_ = _n_prim(w.primaries)
    _compare("plate_40kV", O.per_avalanche(ref, n, W.ANODE, np_),
             O.per_avalanche(out, n, W.ANODE, np_), w.field.gap, "plate")
    # the library's own observables kernel gives the same numbers
    obs = av.observables(st["n_endpoints"], w.primaries, collect_status=W.ANODE,
                         drift_status=W.ANODE, gap=w.field.gap)
    g = O.estimates(O.per_avalanche(out, n, W.ANODE, np_), w.field.gap)
    assert obs[0] == pytest.approx(g["gain"], rel=1e-12)
    assert obs[3] == pytest.approx(g["vd"], rel=1e-9)
    assert obs[4] == pytest.approx(g["DT"], rel=1e-9)
    assert obs[5] == pytest.approx(g["DL"], rel=1e-6)
    assert obs[7] == pytest.approx(g["alpha"], rel=1e-12)


def test_mixed_batched_observables_vs_oracle(av):
    n = 512
    w = W.plate_batched(n_avalanches=4096, seed=0)
    sub = w.primaries.subset(list(range(n)))
    av.set_gas(w.gas)
    av.set_field(w.field)
    ref = oracle.run(w.gas, w.field, sub, seed=0, t_max=w.t_max, majorant=1)
    # the GPU runs the same avalanches (ids 0..511) with another seed
    st, out = run_gpu(av, w, seed=202, precision=A.GT_MIXED, capacity=20_000_000, prim=sub,
                      majorant=A.GT_MAJORANT_BANDED)
    np_ = _n_prim(sub)
    _compare("plate_batched_0..511", O.per_avalanche(ref, n, W.ANODE, np_),
             O.per_avalanche(out, n, W.ANODE, np_), w.field.gap, "plate")


def test_mixed_coax_b_observables_vs_oracle(av):
    """The tube's gain is heavy-tailed (a primary from 1-4.5 mm multiplies
    near the wire), so the oracle takes 256 avalanches and the GPU runs the
    same avalanches with 8 seeds, each (avalanche, seed) pair a unit."""
    n = 256
    w = W.coax(n_avalanches=n, seed=0)
    av.set_gas(w.gas)
    av.set_field(w.field)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, t_max=w.t_max, majorant=1)
    np_ = _n_prim(w.primaries)
    parts = []
    for sd in range(303, 311):
        _, out = run_gpu(av, w, seed=sd, precision=A.GT_MIXED, capacity=20_000_000,
                         majorant=A.GT_MAJORANT_BANDED)
        parts.append(O.per_avalanche(out, n, W.WIRE, np_, "coax"))
    gpu = {k: np.concatenate([q[k] for q in parts]) for k in parts[0]}
    _compare("coax_1T", O.per_avalanche(ref, n, W.WIRE, np_, "coax"), gpu, 0.0, "coax")


def test_mixed_grid_map_observables_vs_oracle(av):
    """The 256^3 coax-sampled grid map at gain ~1e5 (the high-gain stress
    configuration): the oracle transports 48 avalanches through the same
    map, the GPU the same avalanches with 8 seeds; gain, radial drift
    velocity, turn about the wire (no B: zero within errors) and D_L along
    the wire, as for the tube."""
    n = 48
    w = W.grid_stress(n_avalanches=n, n=256, seed=0)
    av.set_gas(w.gas)
    av.set_field(w.field)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, t_max=w.t_max, majorant=1)
    np_ = _n_prim(w.primaries)
    parts = []
    for sd in range(404, 412):
        _, out = run_gpu(av, w, seed=sd, precision=A.GT_MIXED, capacity=12_000_000,
                         majorant=A.GT_MAJORANT_BANDED)
        parts.append(O.per_avalanche(out, n, W.WIRE, np_, "coax"))
    gpu = {k: np.concatenate([q[k] for q in parts]) for k in parts[0]}
    _compare("grid_256^3", O.per_avalanche(ref, n, W.WIRE, np_, "coax"), gpu, 0.0, "coax")
