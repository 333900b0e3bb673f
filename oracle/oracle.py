"""ctypes wrapper around the plain-C FP64 oracle (avalanche_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by bench.py's CPU-baseline leg; never by the product path.

`build()` compiles the oracle with gcc (-O2, no floating-point contraction);
`run()` transports a workload and returns numpy arrays of endpoints, the
electron count of every avalanche and its collision tallies.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "avalanche_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = ["build", "philox4x32_10", "splitmix64_mix", "child_uid", "flight", "elastic", "field_eval",
           "boundary", "mesh_locate", "select", "majorant", "field_emax", "majorant_reach", "scatter",
           "ionisation_share", "weighting_potential", "run", "default_threads"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, a second or two)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Gas(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_nodes", C.c_int32), ("d_eps", C.c_double),
                ("level_type", C.c_void_p), ("threshold", C.c_void_p), ("rate", C.c_void_p),
                ("recoil", C.c_double), ("nu_max", C.c_double), ("xi0", C.c_void_p),
                ("screen", C.c_void_p), ("split_w", C.c_double)]


class _Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("e0", C.c_double), ("gap", C.c_double),
                ("wire_r", C.c_double), ("tube_r", C.c_double), ("voltage", C.c_double),
                ("b", C.c_double * 3), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("origin", C.c_double * 3), ("spacing", C.c_double * 3), ("grid", C.c_void_p),
                ("n_mesh_nodes", C.c_int64), ("n_tets", C.c_int64), ("mesh_nodes", C.c_void_p),
                ("mesh_tets", C.c_void_p), ("mesh_values", C.c_void_p)]


class _Run(C.Structure):
    _fields_ = [("n_primaries", C.c_int64), ("n_avalanches", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("t", C.c_void_p),
                ("e", C.c_void_p), ("dx", C.c_void_p), ("dy", C.c_void_p), ("dz", C.c_void_p),
                ("aval", C.c_void_p), ("uid", C.c_void_p), ("aval_field", C.c_void_p),
                ("seed", C.c_uint64), ("t_max", C.c_double), ("coll_limit", C.c_uint32),
                ("n_threads", C.c_int32), ("majorant", C.c_int32), ("window", C.c_double),
                ("band_width", C.c_double), ("substeps", C.c_int32), ("crossing", C.c_int32),
                ("signal_kind", C.c_int32), ("signal_bins", C.c_int32),
                ("signal_t0", C.c_double), ("signal_dt", C.c_double), ("aval_base", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.or_philox4x32_10.restype = None
            lib.or_splitmix64_mix.argtypes = [C.c_uint64]
            lib.or_splitmix64_mix.restype = C.c_uint64
            lib.or_child_uid.argtypes = [C.c_uint64, C.c_uint32]
            lib.or_child_uid.restype = C.c_uint64
            lib.or_flight.argtypes = [C.c_void_p] * 4 + [C.c_double]
            lib.or_flight.restype = None
            lib.or_elastic.argtypes = [C.c_double, C.c_double, C.c_void_p, C.c_double,
                                       C.c_double, C.c_void_p]
            lib.or_elastic.restype = None
            lib.or_scatter.argtypes = [C.c_double, C.c_void_p, C.c_double, C.c_double,
                                       C.c_void_p]
            lib.or_scatter.restype = C.c_double
            lib.or_ionisation_share.argtypes = [C.c_double, C.c_double, C.c_double]
            lib.or_ionisation_share.restype = C.c_double
            lib.or_field_eval.argtypes = [C.POINTER(_Field), C.c_double, C.c_void_p, C.c_void_p]
            lib.or_field_eval.restype = None
            lib.or_boundary.argtypes = [C.POINTER(_Field), C.c_void_p]
            lib.or_boundary.restype = C.c_int
            lib.or_mesh_locate.argtypes = [C.POINTER(_Field), C.c_void_p, C.c_void_p]
            lib.or_mesh_locate.restype = C.c_int64
            lib.or_select.argtypes = [C.POINTER(_Gas), C.c_double, C.c_double,
                                      C.POINTER(C.c_double)]
            lib.or_select.restype = C.c_int
            lib.or_majorant.argtypes = [C.POINTER(_Gas), C.c_double, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.c_int, C.c_double,
                                        C.POINTER(C.c_double)]
            lib.or_majorant.restype = C.c_double
            lib.or_field_emax.argtypes = [C.POINTER(_Field)]
            lib.or_field_emax.restype = C.c_double
            lib.or_majorant_reach.argtypes = [C.POINTER(_Gas), C.c_double, C.POINTER(C.c_double),
                                              C.c_double, C.c_double, C.POINTER(C.c_double)]
            lib.or_majorant_reach.restype = C.c_double
            lib.or_run.argtypes = [C.POINTER(_Gas), C.POINTER(_Field), C.POINTER(_Run),
                                   C.POINTER(C.c_void_p)]
            lib.or_run.restype = C.c_int
            lib.or_result_count.argtypes = [C.c_void_p]
            lib.or_result_count.restype = C.c_int64
            lib.or_result_fetch.argtypes = [C.c_void_p] + [C.c_void_p] * 17
            lib.or_result_fetch.restype = C.c_int
            lib.or_result_signal.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
            lib.or_result_signal.restype = C.c_int
            lib.or_weighting_potential.argtypes = [C.POINTER(_Field), C.c_int, C.c_void_p]
            lib.or_weighting_potential.restype = C.c_double
            lib.or_result_free.argtypes = [C.c_void_p]
            lib.or_result_free.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _gas_struct(gas, keep):
    lt = np.ascontiguousarray(gas.level_type, np.int32)
    th = np.ascontiguousarray(gas.threshold, np.float64)
    rt = np.ascontiguousarray(gas.rate, np.float64)
    keep += [lt, th, rt]
    xi = sc = None
    if getattr(gas, "xi0", None) is not None:
        xi = np.ascontiguousarray(gas.xi0, np.float64)
        keep.append(xi)
    if getattr(gas, "screen", None) is not None:
        sc = np.ascontiguousarray(gas.screen, np.float64)
        keep.append(sc)
    return _Gas(rt.shape[1], rt.shape[0], gas.d_eps, _ptr(lt).value, _ptr(th).value,
                _ptr(rt).value, gas.recoil, gas.nu_max, _ptr(xi).value if xi is not None else None,
                _ptr(sc).value if sc is not None else None, float(getattr(gas, "split_w", 0.0)))


def _field_struct(field, keep):
    f = _Field()
    f.kind = field.kind
    f.e0, f.gap = field.e0, field.gap
    f.wire_r, f.tube_r, f.voltage = field.wire_r, field.tube_r, field.voltage
    f.b = (C.c_double * 3)(*field.b)
    f.origin = (C.c_double * 3)(*field.origin)
    f.spacing = (C.c_double * 3)(*field.spacing)
    if field.grid is not None:
        g = np.ascontiguousarray(field.grid, np.float32)
        keep.append(g)
        f.nz, f.ny, f.nx = g.shape[0], g.shape[1], g.shape[2]
        f.grid = _ptr(g).value
    if getattr(field, "mesh_tets", None) is not None:
        nodes = np.ascontiguousarray(field.mesh_nodes, np.float64)
        tets = np.ascontiguousarray(field.mesh_tets, np.int32)
        vals = np.ascontiguousarray(field.mesh_values, np.float32)
        if (nodes.ndim != 2 or nodes.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4 or
                vals.shape != (nodes.shape[0], 4)):
            raise ValueError("mesh arrays must be nodes [n, 3], tets [m, 4], values [n, 4]")
        keep.extend([nodes, tets, vals])
        f.n_mesh_nodes, f.n_tets = nodes.shape[0], tets.shape[0]
        f.mesh_nodes, f.mesh_tets, f.mesh_values = _ptr(nodes).value, _ptr(tets).value, _ptr(vals).value
    return f


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


# ------------------------------------------------------------------ hooks
def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def splitmix64_mix(z: int) -> int:
    return int(_load().or_splitmix64_mix(C.c_uint64(z & (2**64 - 1))))


def child_uid(parent: int, flight: int) -> int:
    return int(_load().or_child_uid(C.c_uint64(parent & (2**64 - 1)), C.c_uint32(flight)))


def flight(r, v, a, w, dt):
    """One exact flight under constant acceleration a (cm/ns^2) and magnetic
    rotation vector w (rad/ns); returns the new (r, v)."""
    lib = _load()
    r = np.array(r, np.float64)
    v = np.array(v, np.float64)
    a = np.ascontiguousarray(a, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    lib.or_flight(_ptr(r), _ptr(v), _ptr(a), _ptr(w), float(dt))
    return r, v


def elastic(recoil: float, v, u_cos: float, u_phi: float, xi: float = 0.0):
    """Velocity after an elastic collision (direction from the two uniforms,
    isotropic for xi = 0 else screened-Coulomb about v; recoil loss with
    recoil = 2m/M)."""
    v = np.ascontiguousarray(v, np.float64)
    out = np.zeros(3)
    _load().or_elastic(float(recoil), float(xi), _ptr(v), float(u_cos), float(u_phi), _ptr(out))
    return out


def scatter(xi: float, v, u_cos: float, u_phi: float):
    """(new unit direction, cos chi) after a collision with anisotropy xi."""
    v = np.ascontiguousarray(v, np.float64)
    out = np.zeros(3)
    mu = _load().or_scatter(float(xi), _ptr(v), float(u_cos), float(u_phi), _ptr(out))
    return out, mu


def ionisation_share(w: float, rest: float, u: float) -> float:
    """Energy of the new electron of an ionisation from the remainder `rest`."""
    return float(_load().or_ionisation_share(float(w), float(rest), float(u)))


def field_eval(field, r, plate_e=0.0):
    keep = []
    f = _field_struct(field, keep)
    r = np.ascontiguousarray(r, np.float64)
    e = np.zeros(3)
    _load().or_field_eval(C.byref(f), float(plate_e), _ptr(r), _ptr(e))
    return e


def boundary(field, r) -> int:
    keep = []
    f = _field_struct(field, keep)
    r = np.ascontiguousarray(r, np.float64)
    return int(_load().or_boundary(C.byref(f), _ptr(r)))


def select(gas, eps: float, u1: float):
    """Level chosen at energy eps for the uniform u1 (-1 = null) and nu_max."""
    keep = []
    g = _gas_struct(gas, keep)
    nm = C.c_double(0.0)
    j = _load().or_select(C.byref(g), float(eps), float(u1), C.byref(nm))
    if j == -2:
        raise ValueError("bad gas table")
    return j, nm.value


def mesh_locate(field, r):
    """Element of a tetrahedral-mesh field that holds r (the lowest index,
    -1 for none) and r's barycentric coordinates in it."""
    keep = []
    f = _field_struct(field, keep)
    r = np.ascontiguousarray(r, np.float64)
    lam = np.zeros(4, np.float64)
    t = _load().or_mesh_locate(C.byref(f), _ptr(r), _ptr(lam))
    return int(t), lam


def weighting_potential(field, kind: int, r) -> float:
    """Weighting potential of the readout electrode (kind 1 plate anode,
    2 coax wire, 3 the grid map's 4th component) at r."""
    keep = []
    f = _field_struct(field, keep)
    r = np.ascontiguousarray(r, np.float64)
    return float(_load().or_weighting_potential(C.byref(f), int(kind), _ptr(r)))


def majorant(gas, band_width: float, v, e_field, has_b: bool, window: float):
    """Banded majorant (1/ns) and window tau (ns) of a flight with velocity
    v (cm/ns) in the held field e_field (V/cm); has_b selects the bound for
    a flight that also turns in a magnetic field."""
    keep = []
    g = _gas_struct(gas, keep)
    vv = (C.c_double * 3)(*[float(x) for x in v])
    ee = (C.c_double * 3)(*[float(x) for x in e_field])
    tau = C.c_double(0.0)
    nu = _load().or_majorant(C.byref(g), float(band_width), vv, ee, int(bool(has_b)),
                             float(window), C.byref(tau))
    if nu < 0.0:
        raise ValueError("bad gas table")
    return nu, tau.value


def field_emax(field) -> float:
    """Largest field magnitude (V/cm) the oracle assumes for `field` when the
    field is re-evaluated along a flight (sub-steps); 0 for uniform fields."""
    keep = []
    f = _field_struct(field, keep)
    return float(_load().or_field_emax(C.byref(f)))


def majorant_reach(gas, band_width: float, v, emax: float, window: float):
    """Banded majorant (1/ns) and window tau (ns) of a flight with velocity v
    (cm/ns) along which the field may change, its magnitude bounded by emax
    (V/cm): the bound runs with sub-steps use."""
    keep = []
    g = _gas_struct(gas, keep)
    vv = (C.c_double * 3)(*[float(x) for x in v])
    tau = C.c_double(0.0)
    nu = _load().or_majorant_reach(C.byref(g), float(band_width), vv, float(emax), float(window),
                                   C.byref(tau))
    if nu < 0.0:
        raise ValueError("bad gas table or emax")
    return nu, tau.value


# -------------------------------------------------------------------- run
def run(gas, field, prim, seed: int = 0, t_max: float = 0.0, coll_limit: int = 0,
        n_threads: int | None = None, majorant: int = 0, window: float = 2.0,
        band_width: float = 1.0, substeps: int = 1, crossing: bool = False,
        signal: tuple | None = None, aval_base: int = 0) -> dict:
    """Transport every avalanche of `prim` and return a dict of arrays
    (majorant 0: one global nu_max; 1: the banded majorant with flight
    window `window` / band rate and bands of `band_width` eV; `substeps`
    field evaluations per flight; `crossing`: an electron that leaves ends
    at its first boundary crossing; `signal` = (electrode kind, bins, t0, dt)
    for the induced signal per avalanche, out["signal"] [n_avalanches, bins]
    in units of e; `aval_base`: the workload number of avalanche 0, which keys
    the random streams, for a part of a larger workload):
    x0..e0 (start), x1..e1 (end), status, aval, uid, n_flight, ledger [n, 4]
    (field work, inelastic loss, recoil loss, secondary share; eV),
    electrons [n_avalanches], tallies [n_avalanches, L+1] (real collisions
    per level, then null flights)."""
    lib = _load()
    keep = []
    g = _gas_struct(gas, keep)
    f = _field_struct(field, keep)
    cols = {}
    for k in ("x", "y", "z", "t", "e", "dx", "dy", "dz"):
        cols[k] = np.ascontiguousarray(getattr(prim, k), np.float64)
    av = np.ascontiguousarray(prim.aval, np.int32)
    ud = np.ascontiguousarray(prim.uid, np.uint64)
    keep += list(cols.values()) + [av, ud]
    af = None
    if prim.aval_field is not None:
        af = np.ascontiguousarray(prim.aval_field, np.float64)
        keep.append(af)
    ra = _Run()
    ra.n_primaries = prim.n
    ra.n_avalanches = prim.n_avalanches
    for k, a in cols.items():
        setattr(ra, k, _ptr(a).value)
    ra.aval, ra.uid = _ptr(av).value, _ptr(ud).value
    ra.aval_field = _ptr(af).value if af is not None else None
    ra.seed = seed & (2**64 - 1)
    ra.t_max = t_max
    ra.coll_limit = coll_limit
    ra.n_threads = n_threads or default_threads()
    ra.majorant = majorant
    ra.window = window
    ra.band_width = band_width
    ra.substeps = int(substeps)
    ra.crossing = int(bool(crossing))
    ra.aval_base = int(aval_base)
    if signal is not None:
        ra.signal_kind, ra.signal_bins = int(signal[0]), int(signal[1])
        ra.signal_t0, ra.signal_dt = float(signal[2]), float(signal[3])
    handle = C.c_void_p()
    rc = lib.or_run(C.byref(g), C.byref(f), C.byref(ra), C.byref(handle))
    if rc != 0:
        raise RuntimeError(f"oracle run failed ({rc})")
    try:
        n = int(lib.or_result_count(handle))
        out = {k: np.zeros(n, np.float64) for k in
               ("x0", "y0", "z0", "t0", "e0", "x1", "y1", "z1", "t1", "e1")}
        out["status"] = np.zeros(n, np.int32)
        out["aval"] = np.zeros(n, np.int32)
        out["uid"] = np.zeros(n, np.uint64)
        out["n_flight"] = np.zeros(n, np.uint32)
        out["ledger"] = np.zeros((n, 4), np.float64)
        A, L = prim.n_avalanches, gas.n_levels
        out["electrons"] = np.zeros(A, np.uint64)
        out["tallies"] = np.zeros((A, L + 1), np.uint64)
        order = ("x0", "y0", "z0", "t0", "e0", "x1", "y1", "z1", "t1", "e1", "status", "aval",
                 "uid", "n_flight", "ledger", "electrons", "tallies")
        lib.or_result_fetch(handle, *[_ptr(out[k]) for k in order])
        if signal is not None:
            out["signal"] = np.zeros((A, int(signal[1])), np.float64)
            lib.or_result_signal(handle, int(signal[1]), _ptr(out["signal"]))
    finally:
        lib.or_result_free(handle)
    return out
