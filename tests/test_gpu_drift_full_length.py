"""The constant-rate drift model at its configured length: 1000 electrons,
each tracked for 1e5 real collisions (nu = 1e12 /s elastic, isotropic, no
energy loss, E = 1 kV/cm along -z, 0.1 eV isotropic start).

FP64: the GPU path equals the FP64 oracle electron by electron over the whole
1e5 collisions (start and end within 1e-9, identical flight counts and
statuses).  The tolerance comes from the arithmetic: both sides are FP64 and
differ only in rounding order and 1-2 ulp of log/sqrt/sin/cos; with
isotropic scattering the direction after a collision forgets the one before,
so these differences add up like a random walk (about 1e-16 sqrt(1e5) ~ 3e-14
relative) and do not grow exponentially.

Mixed precision: the same workload against the closed forms of the model
gas: v_d = eE/(m nu) and E[x^2] = E[y^2] from the independent-flight sum
(tests/physics.py), each within 3 sigma over the 1000 electrons, and the
energy ledger eps_end = eps_0 + E dz per electron (field work is the only
energy change).  The ledger's accuracy is that of FP32 speeds: every
flight and collision rounds |v| several times at 2^-24 = 6e-8, a random walk
over 1e5 collisions; with k roundings per collision the energy error is about
2 k 6e-8 sqrt(1e5) = k 3.8e-5 of the electron's energy (k ~ 7 measured:
median 2.7e-4).  An electron that ends slow has a large error relative to
its own end energy, so the error is taken relative to the mean end energy:
its rms and median must stay below 1e-3.

Most of it is a bias, not a random walk: the FP32 direction of a collision
has E|n|^2 = 1 - 2e-9, because the unit-length rescaling of the azimuth pair
(cos phi, sin phi) rounds quantities that straddle 1.0, where the FP32
spacing doubles (a float32 emulation of the step reproduces -2.0e-9; even a
correctly rounded rsqrt gives +1e-8).  Each elastic collision therefore
scales the energy by about 1 - 2.5e-9 (measured here: -2.5e-4 of the energy
after 1e5 collisions); an avalanche electron's ~250 collisions make that
6e-7.  The mean is held below 4e-4 (1e5 collisions x 4e-9) so that a larger
bias would show.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_15377_gb300 import avalanche as A
from paper_2509_15377_gb300 import workloads as W
from tests import physics as P
from tests.gpu_helpers import assert_same_electrons, run_gpu

pytestmark = pytest.mark.gpu

N_E, N_COLL, E_FIELD, NU = 1000, 100_000, 1000.0, 1000.0


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


@pytest.fixture(scope="module")
def workload():
    return W.drift_model(n_electrons=N_E, n_coll=N_COLL, e_field=E_FIELD, nu=NU, seed=0)


def test_fp64_full_length_per_collision(av, workload):
    w = workload
    av.set_gas(w.gas)
    av.set_field(w.field)
    ref = oracle.run(w.gas, w.field, w.primaries, seed=0, coll_limit=N_COLL)
    st, out = run_gpu(av, w, seed=0, precision=A.GT_FP64, capacity=N_E)
    assert np.all(out["status"] == W.COLL_LIMIT)
    assert np.all(out["n_flight"] == N_COLL)       # nu_max = nu: no null flights
    assert st["real_collisions"] == N_E * N_COLL
    # scales: the spread of the end points (~1.4 mm), the mean time (1e5 / nu)
    assert_same_electrons(out, ref, scale_pos=0.1, scale_t=N_COLL / NU, scale_e=1.0)
    assert np.array_equal(out["tallies"], ref["tallies"])


def test_mixed_full_length_closed_forms(av, workload):
    w = workload
    av.set_gas(w.gas)
    av.set_field(w.field)
    st, out = run_gpu(av, w, seed=1, precision=A.GT_MIXED, capacity=N_E)
    assert np.all(out["status"] == W.COLL_LIMIT)
    dz, dt = out["z1"] - out["z0"], out["t1"] - out["t0"]
    vd = P.drift_velocity(E_FIELD, NU)
    se = np.std(dz - vd * dt, ddof=1) / math.sqrt(N_E) / dt.mean()
    assert abs(dz.mean() / dt.mean() - vd) < 3 * se, (dz.mean() / dt.mean(), vd, se)
    ex = P.transverse_msd(E_FIELD, NU, N_COLL, 0.1)
    xs = np.concatenate([out["x1"] - out["x0"], out["y1"] - out["y0"]]) ** 2
    assert abs(xs.mean() - ex) < 3 * xs.std(ddof=1) / math.sqrt(len(xs)), (xs.mean(), ex)
    # E[t] = N / nu
    assert abs(dt.mean() - N_COLL / NU) < 3 * dt.std(ddof=1) / math.sqrt(N_E)
    err = (out["e1"] - (out["e0"] + E_FIELD * dz)) / out["e1"].mean()
    rms = float(np.sqrt(np.mean(err * err)))
    print(f"mixed drift 1e5 collisions: v_d {dz.mean() / dt.mean():.6g} (closed form {vd:.6g}), "
          f"<x^2> {xs.mean():.4g} ({ex:.4g}), ledger / <e1>: rms {rms:.3g}, "
          f"median |.| {np.median(np.abs(err)):.3g}, max |.| {np.abs(err).max():.3g}, "
          f"mean {err.mean():+.3g}")
    assert rms < 1e-3 and np.median(np.abs(err)) < 1e-3
    assert abs(err.mean()) < 4e-4
