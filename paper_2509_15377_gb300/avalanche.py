"""ctypes binding of the C ABI in include/gt_avalanche.h.

Argument marshalling only: every step of the transport runs in the CUDA
library.  The functions keep the ABI's names (gas_table_upload, field_setup,
avalanche_run, avalanche_observables); `Avalanche` bundles a context with
torch-allocated device buffers (PyTorch supplies device memory and streams).

Importing this module never falls back to anything: if the library cannot be
loaded, `load()` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import workloads as W

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgt_avalanche.so")

GT_OK, GT_ERR_ARG, GT_ERR_STATE, GT_ERR_WORKSPACE = 0, -1, -2, -3
GT_ERR_QUEUE_OVERFLOW, GT_ERR_TIMEOUT, GT_ERR_CUDA, GT_ERR_NO_DEVICE = -4, -5, -6, -7
GT_ERR_UNSUPPORTED = -8
GT_ERR_HOST_MEMORY = -9
GT_FP64, GT_MIXED = 0, 1
GT_BATCHED, GT_PLAIN = 0, 1
GT_DEBUG_UNFILLED_SLOT = 1
GT_MAJORANT_GLOBAL, GT_MAJORANT_BANDED = 0, 1
GT_OBS_COUNT = 8
GT_ABI_VERSION = 4
PARTIAL_OK = (GT_OK, GT_ERR_QUEUE_OVERFLOW, GT_ERR_TIMEOUT)


class GtError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code}){' - ' + detail if detail else ''}")


# ------------------------------------------------------------- structs
class gt_gas(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_nodes", C.c_int32), ("d_eps", C.c_double),
                ("level_type", C.c_void_p), ("threshold", C.c_void_p), ("rate", C.c_void_p),
                ("recoil", C.c_double), ("nu_max", C.c_double), ("band_width", C.c_double),
                ("xi0", C.c_void_p), ("screen", C.c_void_p), ("split_w", C.c_double)]


class gt_field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("e0", C.c_double), ("gap", C.c_double),
                ("wire_r", C.c_double), ("tube_r", C.c_double), ("voltage", C.c_double),
                ("b", C.c_double * 3), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("origin", C.c_double * 3), ("spacing", C.c_double * 3), ("grid", C.c_void_p),
                ("n_mesh_nodes", C.c_int64), ("n_tets", C.c_int64), ("mesh_nodes", C.c_void_p),
                ("mesh_tets", C.c_void_p), ("mesh_values", C.c_void_p)]


class gt_run(C.Structure):
    _fields_ = [("n_primaries", C.c_int64), ("n_avalanches", C.c_int32),
                ("primaries_on_device", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("t", C.c_void_p),
                ("e", C.c_void_p), ("dx", C.c_void_p), ("dy", C.c_void_p), ("dz", C.c_void_p),
                ("aval", C.c_void_p), ("uid", C.c_void_p), ("aval_field", C.c_void_p),
                ("seed", C.c_uint64), ("t_max", C.c_double), ("coll_limit", C.c_uint32),
                ("precision", C.c_int32), ("mode", C.c_int32), ("block", C.c_int32),
                ("refill_period", C.c_int32), ("grid", C.c_int32),
                ("size_limit", C.c_uint64), ("spin_limit_ms", C.c_double),
                ("time_limit_ms", C.c_double), ("debug_flags", C.c_int32),
                ("flights_per_phase", C.c_int32), ("majorant", C.c_int32), ("aval_base", C.c_int32),
                ("majorant_window", C.c_double), ("substeps", C.c_int32),
                ("crossing", C.c_int32), ("signal_kind", C.c_int32), ("signal_bins", C.c_int32),
                ("signal_t0", C.c_double), ("signal_dt", C.c_double)]


_EP_ARRAYS = ("x0", "y0", "z0", "t0", "e0", "x1", "y1", "z1", "t1", "e1", "status", "aval",
              "uid", "n_flight")


class gt_endpoints(C.Structure):
    _fields_ = [("capacity", C.c_int64)] + [(k, C.c_void_p) for k in _EP_ARRAYS] + \
               [("electrons", C.c_void_p), ("tallies", C.c_void_p), ("signal", C.c_void_p)]


class gt_stats(C.Structure):
    _fields_ = [("n_endpoints", C.c_int64), ("n_dropped", C.c_int64),
                ("real_collisions", C.c_uint64), ("null_collisions", C.c_uint64),
                ("flights", C.c_uint64), ("transport_ms", C.c_double),
                ("launches", C.c_int32), ("iterations", C.c_int32), ("status", C.c_int32),
                ("block", C.c_int32), ("refill_period", C.c_int32), ("grid", C.c_int32),
                ("flights_per_phase", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class gt_tune_point(C.Structure):
    _fields_ = [("block", C.c_int32), ("refill_period", C.c_int32),
                ("flights_per_phase", C.c_int32), ("pad", C.c_int32),
                ("real_per_ms", C.c_double), ("transport_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ("gt_abi_version", "gt_strerror", "gt_abi_sizes", "gt_last_cuda_error", "gt_create",
           "gt_destroy", "gas_table_upload", "gt_gas_nu_max", "field_setup",
           "gt_workspace_bytes", "avalanche_run", "avalanche_run_static", "gt_autotune",
           "avalanche_observables", "gt_graph_create", "gt_graph_launch", "gt_graph_stats",
           "gt_graph_destroy")

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (build it first with paper_2509_15377_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    sig = {
        "gt_abi_version": ([], C.c_int),
        "gt_strerror": ([C.c_int], C.c_char_p),
        "gt_abi_sizes": ([C.POINTER(sz), C.c_int], C.c_int),
        "gt_last_cuda_error": ([vp], C.c_char_p),
        "gt_create": ([C.POINTER(vp), C.c_int], C.c_int),
        "gt_destroy": ([vp], C.c_int),
        "gas_table_upload": ([vp, C.POINTER(gt_gas)], C.c_int),
        "gt_gas_nu_max": ([vp, C.POINTER(C.c_double)], C.c_int),
        "field_setup": ([vp, C.POINTER(gt_field)], C.c_int),
        "gt_workspace_bytes": ([vp, C.POINTER(gt_run), i64, C.POINTER(sz)], C.c_int),
        "avalanche_run": ([vp, C.POINTER(gt_run), C.POINTER(gt_endpoints), vp, sz, vp,
                           C.POINTER(gt_stats)], C.c_int),
        "avalanche_observables": ([vp, C.POINTER(gt_endpoints), i64, i32, vp, i32, i32,
                                   C.c_double, vp, vp], C.c_int),
        "avalanche_run_static": ([vp, C.POINTER(gt_run), C.POINTER(gt_endpoints), vp,
                                  C.POINTER(gt_stats)], C.c_int),
        "gt_autotune": ([vp, C.POINTER(gt_run), C.POINTER(gt_endpoints), vp, sz, vp,
                         C.POINTER(gt_tune_point), i32, C.POINTER(i32),
                         C.POINTER(gt_tune_point)], C.c_int),
        "gt_graph_create": ([vp, C.POINTER(gt_run), C.POINTER(gt_endpoints), vp, sz,
                             C.POINTER(vp)], C.c_int),
        "gt_graph_launch": ([vp, C.c_uint64, vp], C.c_int),
        "gt_graph_stats": ([vp, C.POINTER(gt_stats)], C.c_int),
        "gt_graph_destroy": ([vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if lib.gt_abi_version() != GT_ABI_VERSION:
        raise RuntimeError(f"library ABI {lib.gt_abi_version()}, binding {GT_ABI_VERSION}")
    sizes = (sz * 5)()
    if lib.gt_abi_sizes(sizes, 5) != GT_OK:
        raise RuntimeError("gt_abi_sizes failed")
    mine = [C.sizeof(s) for s in (gt_gas, gt_field, gt_run, gt_endpoints, gt_stats)]
    if list(sizes) != mine:
        raise RuntimeError(f"struct layout mismatch with the library: {list(sizes)} vs {mine}")
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().gt_strerror(code).decode()


def _check(rc: int, what: str, ctx=None, allow=(GT_OK,)):
    if rc not in allow:
        detail = load().gt_last_cuda_error(ctx).decode() if (ctx and rc == GT_ERR_CUDA) else ""
        raise GtError(rc, what, detail)
    return rc


# --------------------------------------------------- ABI-named wrappers
def gt_create(device: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().gt_create(C.byref(h), device), "gt_create")
    return h


def gt_destroy(ctx) -> None:
    load().gt_destroy(ctx)


def gas_table_upload(ctx, gas: W.Gas) -> None:
    lt = np.ascontiguousarray(gas.level_type, np.int32)
    th = np.ascontiguousarray(gas.threshold, np.float64)
    rt = np.ascontiguousarray(gas.rate, np.float64)
    xi = None if gas.xi0 is None else np.ascontiguousarray(gas.xi0, np.float64)
    sc = None if gas.screen is None else np.ascontiguousarray(gas.screen, np.float64)
    if rt.ndim != 2:
        raise ValueError(f"rate must be [n_nodes, n_levels], got {rt.shape}")
    for name, a in (("level_type", lt), ("threshold", th), ("xi0", xi), ("screen", sc)):
        # the library reads one value per level from each
        if a is not None and a.shape != (rt.shape[1],):
            raise ValueError(f"{name} needs one value per level ({rt.shape[1]}), got {a.shape}")
    g = gt_gas(rt.shape[1], rt.shape[0], gas.d_eps, lt.ctypes.data, th.ctypes.data,
               rt.ctypes.data, gas.recoil, gas.nu_max, gas.band_width,
               xi.ctypes.data if xi is not None else None,
               sc.ctypes.data if sc is not None else None, gas.split_w)
    _check(load().gas_table_upload(ctx, C.byref(g)), "gas_table_upload", ctx)


def gas_nu_max(ctx) -> float:
    v = C.c_double()
    _check(load().gt_gas_nu_max(ctx, C.byref(v)), "gt_gas_nu_max", ctx)
    return v.value


def mesh_arrays(field: W.Field):
    """The mesh's node, element and value arrays as the C ABI reads them
    (float64 [n, 3], int32 [m, 4], float32 [n, 4], contiguous); ValueError for
    other shapes, which the library would read past."""
    if field.mesh_nodes is None or field.mesh_tets is None or field.mesh_values is None:
        raise ValueError("a MESH field needs mesh_nodes, mesh_tets and mesh_values")
    nodes = np.ascontiguousarray(field.mesh_nodes, np.float64)
    tets = np.ascontiguousarray(field.mesh_tets, np.int32)
    vals = np.ascontiguousarray(field.mesh_values, np.float32)
    if nodes.ndim != 2 or nodes.shape[1] != 3:
        raise ValueError(f"mesh_nodes must be [n, 3], got {nodes.shape}")
    if tets.ndim != 2 or tets.shape[1] != 4:
        raise ValueError(f"mesh_tets must be [m, 4], got {tets.shape}")
    if vals.shape != (nodes.shape[0], 4):
        raise ValueError(f"mesh_values must be [{nodes.shape[0]}, 4], got {vals.shape}")
    return nodes, tets, vals


def field_setup(ctx, field: W.Field, grid_ptr: int = 0) -> None:
    f = gt_field()
    f.kind = field.kind
    f.e0, f.gap = field.e0, field.gap
    f.wire_r, f.tube_r, f.voltage = field.wire_r, field.tube_r, field.voltage
    f.b = (C.c_double * 3)(*field.b)
    f.origin = (C.c_double * 3)(*field.origin)
    f.spacing = (C.c_double * 3)(*field.spacing)
    if field.kind == W.GRID:
        f.nz, f.ny, f.nx = field.grid.shape[:3]
        f.grid = grid_ptr
    keep = []
    if field.kind == W.MESH:
        nodes, tets, vals = mesh_arrays(field)
        keep.extend([nodes, tets, vals])  # host arrays, copied by field_setup
        f.n_mesh_nodes, f.n_tets = nodes.shape[0], tets.shape[0]
        f.mesh_nodes, f.mesh_tets, f.mesh_values = (nodes.ctypes.data, tets.ctypes.data,
                                                    vals.ctypes.data)
    _check(load().field_setup(ctx, C.byref(f)), "field_setup", ctx)


def workspace_bytes(ctx, run: gt_run, capacity: int) -> int:
    n = C.c_size_t()
    _check(load().gt_workspace_bytes(ctx, C.byref(run), capacity, C.byref(n)),
           "gt_workspace_bytes", ctx)
    return n.value


def avalanche_run(ctx, run: gt_run, out: gt_endpoints, workspace_ptr: int, workspace_nbytes: int,
                  stream_ptr: int, allow=PARTIAL_OK) -> gt_stats:
    st = gt_stats()
    rc = load().avalanche_run(ctx, C.byref(run), C.byref(out), workspace_ptr, workspace_nbytes,
                              stream_ptr, C.byref(st))
    _check(rc, "avalanche_run", ctx, allow)
    st.status = rc
    return st


GT_STATIC_MAX_ELECTRONS = 1 << 18
GT_STATIC_MAX_AVALANCHES = 16384


def avalanche_run_static(ctx, run: gt_run, out: gt_endpoints, stream_ptr: int,
                         allow=PARTIAL_OK) -> gt_stats:
    """The batched run with the library's fixed internal scratch: allocates
    nothing (for callers that cannot allocate device memory at this point);
    limits GT_STATIC_MAX_ELECTRONS slots and GT_STATIC_MAX_AVALANCHES."""
    st = gt_stats()
    rc = load().avalanche_run_static(ctx, C.byref(run), C.byref(out), stream_ptr, C.byref(st))
    _check(rc, "avalanche_run_static", ctx, allow)
    st.status = rc
    return st


def gt_autotune(ctx, run: gt_run, out: gt_endpoints, workspace_ptr: int, workspace_nbytes: int,
                stream_ptr: int):
    """Coordinate-descent search over launch shapes; returns (best, [points])."""
    pts = (gt_tune_point * 128)()
    n = C.c_int32()
    best = gt_tune_point()
    _check(load().gt_autotune(ctx, C.byref(run), C.byref(out), workspace_ptr, workspace_nbytes,
                              stream_ptr, pts, 128, C.byref(n), C.byref(best)), "gt_autotune", ctx)
    return best.as_dict(), [pts[i].as_dict() for i in range(min(n.value, 128))]


def avalanche_observables(ctx, out: gt_endpoints, n_endpoints: int, n_avalanches: int,
                          n_prim_ptr: int, collect_status: int, drift_status: int, gap: float,
                          obs_ptr: int, stream_ptr: int) -> None:
    _check(load().avalanche_observables(ctx, C.byref(out), n_endpoints, n_avalanches, n_prim_ptr,
                                        collect_status, drift_status, gap, obs_ptr, stream_ptr),
           "avalanche_observables", ctx)


# --------------------------------------------------- torch convenience
@dataclass
class RunOptions:
    seed: int = 0
    t_max: float = 0.0
    coll_limit: int = 0
    precision: int = GT_MIXED
    mode: int = GT_BATCHED
    block: int = 0
    refill_period: int = 0
    flights_per_phase: int = 0
    grid: int = 0
    majorant: int = 0          # GT_MAJORANT_GLOBAL / GT_MAJORANT_BANDED
    majorant_window: float = 0.0
    aval_base: int = 0         # workload number of avalanche 0 (a part of a larger workload)
    size_limit: int = 0
    spin_limit_ms: float = 0.0
    time_limit_ms: float = 0.0
    debug_flags: int = 0
    substeps: int = 0          # field evaluations per flight (<= 1: held field)
    crossing: int = 0          # 1: leaving electrons end at the first crossing
    signal_kind: int = 0       # readout electrode for induced signals (workloads.W_*)
    signal_bins: int = 0
    signal_t0: float = 0.0
    signal_dt: float = 0.0


class Avalanche:
    """One context on one GPU with torch-owned device buffers.

    gas, field, primaries come from `workloads`; outputs are torch CUDA
    tensors that stay on the device (`endpoints`), the run summary comes
    back as a dict."""

    PRIM_KEYS = ("x", "y", "z", "t", "e", "dx", "dy", "dz")

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = gt_create(device)
        self._grid = None
        self.gas = None
        self.field = None
        self.ep = None
        self.ws = None

    def close(self):
        if self.ctx is not None:
            gt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup (outside the timed region, as field maps in the paper)
    def set_gas(self, gas: W.Gas):
        gas_table_upload(self.ctx, gas)
        self.gas = gas

    def set_field(self, field: W.Field):
        ptr = 0
        if field.kind == W.GRID:
            g = np.ascontiguousarray(field.grid, np.float32)
            if g.ndim != 4 or g.shape[3] != 4 or min(g.shape[:3]) < 2:
                # the kernels read one float4 per node of an [nz, ny, nx] map
                raise ValueError(f"grid must be [nz, ny, nx, 4] with every n >= 2, got {g.shape}")
            t = self.torch.from_numpy(g)
            self._grid = t.to(f"cuda:{self.device}")
            ptr = self._grid.data_ptr()
        field_setup(self.ctx, field, ptr)
        self.field = field

    def nu_max(self) -> float:
        return gas_nu_max(self.ctx)

    # ---- buffers
    def alloc(self, capacity: int, n_avalanches: int, run: gt_run):
        torch = self.torch
        dev = f"cuda:{self.device}"
        L = self.gas.n_levels
        f64, i32 = torch.float64, torch.int32
        bins = run.signal_bins if run.signal_kind else 0
        need = dict(capacity=capacity, n_avalanches=n_avalanches, L=L, bins=bins)
        if self.ep is None or self.ep["_need"] != need:
            ep = {k: torch.empty(capacity, dtype=f64, device=dev)
                  for k in ("x0", "y0", "z0", "t0", "e0", "x1", "y1", "z1", "t1", "e1")}
            ep["status"] = torch.empty(capacity, dtype=i32, device=dev)
            ep["aval"] = torch.empty(capacity, dtype=i32, device=dev)
            ep["uid"] = torch.empty(capacity, dtype=torch.int64, device=dev)
            ep["n_flight"] = torch.empty(capacity, dtype=i32, device=dev)
            ep["electrons"] = torch.empty(max(n_avalanches, 1), dtype=torch.int64, device=dev)
            ep["tallies"] = torch.empty((max(n_avalanches, 1), L + 1), dtype=torch.int64, device=dev)
            ep["signal"] = (torch.empty((max(n_avalanches, 1), bins), dtype=f64, device=dev)
                            if bins else None)
            ep["_need"] = need
            self.ep = ep
        nbytes = workspace_bytes(self.ctx, run, capacity)
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        return self.ep

    def endpoints_struct(self, capacity: int) -> gt_endpoints:
        o = gt_endpoints()
        o.capacity = capacity
        for k in _EP_ARRAYS:
            setattr(o, k, self.ep[k].data_ptr())
        o.electrons = self.ep["electrons"].data_ptr()
        o.tallies = self.ep["tallies"].data_ptr()
        o.signal = self.ep["signal"].data_ptr() if self.ep.get("signal") is not None else None
        return o

    def check_primaries(self, prim: W.Primaries) -> None:
        """Every per-primary array one-dimensional and of the same length, and
        the per-avalanche fields (if any) one per avalanche: the seed kernel
        reads them all by primary (or avalanche) index."""
        n = prim.n
        for k in self.PRIM_KEYS + ("aval", "uid"):
            a = np.asarray(getattr(prim, k))
            if a.ndim != 1 or a.shape[0] != n:
                raise ValueError(f"primaries.{k} must have shape ({n},), got {a.shape}")
        if prim.aval_field is not None:
            a = np.asarray(prim.aval_field)
            if a.ndim != 1 or a.shape[0] != prim.n_avalanches:
                raise ValueError(f"primaries.aval_field must have shape ({prim.n_avalanches},), "
                                 f"got {a.shape}")

    def primaries_device(self, prim: W.Primaries) -> dict:
        """Primaries as device tensors (resident in HBM)."""
        self.check_primaries(prim)
        torch = self.torch
        dev = f"cuda:{self.device}"
        d = {k: torch.from_numpy(np.ascontiguousarray(getattr(prim, k), np.float64)).to(dev)
             for k in self.PRIM_KEYS}
        d["aval"] = torch.from_numpy(np.ascontiguousarray(prim.aval, np.int32)).to(dev)
        d["uid"] = torch.from_numpy(np.ascontiguousarray(prim.uid).view(np.int64)).to(dev)
        if prim.aval_field is not None:
            d["aval_field"] = torch.from_numpy(np.ascontiguousarray(prim.aval_field, np.float64)).to(dev)
        d["_n"] = prim.n
        d["_n_avalanches"] = prim.n_avalanches
        d["_on_device"] = 1
        return d

    def primaries_pinned(self, prim: W.Primaries) -> dict:
        """Primaries in pinned host memory (copied inside each run)."""
        self.check_primaries(prim)
        torch = self.torch
        d = {k: torch.from_numpy(np.ascontiguousarray(getattr(prim, k), np.float64)).pin_memory()
             for k in self.PRIM_KEYS}
        d["aval"] = torch.from_numpy(np.ascontiguousarray(prim.aval, np.int32)).pin_memory()
        d["uid"] = torch.from_numpy(np.ascontiguousarray(prim.uid).view(np.int64)).pin_memory()
        if prim.aval_field is not None:
            d["aval_field"] = torch.from_numpy(np.ascontiguousarray(prim.aval_field, np.float64)).pin_memory()
        d["_n"] = prim.n
        d["_n_avalanches"] = prim.n_avalanches
        d["_on_device"] = 0
        return d

    def make_run(self, prim: dict, opt: RunOptions) -> gt_run:
        r = gt_run()
        r.n_primaries = prim["_n"]
        r.n_avalanches = prim["_n_avalanches"]
        r.primaries_on_device = prim["_on_device"]
        for k in self.PRIM_KEYS + ("aval", "uid"):
            setattr(r, k, prim[k].data_ptr())
        r.aval_field = prim["aval_field"].data_ptr() if "aval_field" in prim else None
        r.seed = opt.seed & (2**64 - 1)
        r.t_max = opt.t_max
        r.coll_limit = opt.coll_limit
        r.precision = opt.precision
        r.mode = opt.mode
        r.block = opt.block
        r.refill_period = opt.refill_period
        r.flights_per_phase = opt.flights_per_phase
        r.majorant = opt.majorant
        r.majorant_window = opt.majorant_window
        r.aval_base = opt.aval_base
        r.grid = opt.grid
        r.size_limit = opt.size_limit
        r.spin_limit_ms = opt.spin_limit_ms
        r.time_limit_ms = opt.time_limit_ms
        r.debug_flags = opt.debug_flags
        r.substeps = opt.substeps
        r.crossing = opt.crossing
        r.signal_kind = opt.signal_kind
        r.signal_bins = opt.signal_bins
        r.signal_t0 = opt.signal_t0
        r.signal_dt = opt.signal_dt
        return r

    def run(self, prim: dict, opt: RunOptions, capacity: int, stream=None,
            allow=PARTIAL_OK) -> dict:
        torch = self.torch
        r = self.make_run(prim, opt)
        self.alloc(capacity, r.n_avalanches, r)
        o = self.endpoints_struct(capacity)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        st = avalanche_run(self.ctx, r, o, self.ws.data_ptr(), self.ws.numel(), s.cuda_stream,
                           allow)
        return st.as_dict()

    def graph(self, prim: dict, opt: RunOptions, capacity: int) -> "Graph":
        """Record a batched run with device primaries as a CUDA graph
        (gt_graph_create); replay it with Graph.launch(seed)."""
        r = self.make_run(prim, opt)
        self.alloc(capacity, r.n_avalanches, r)
        o = self.endpoints_struct(capacity)
        h = C.c_void_p()
        _check(load().gt_graph_create(self.ctx, C.byref(r), C.byref(o), self.ws.data_ptr(),
                                      self.ws.numel(), C.byref(h)), "gt_graph_create", self.ctx)
        return Graph(self, h)

    def autotune(self, prim: dict, opt: RunOptions, capacity: int, stream=None):
        """Pick the batched launch shape for this precision and field kind
        (remembered by the context for runs that leave it at 0)."""
        torch = self.torch
        r = self.make_run(prim, opt)
        self.alloc(capacity, r.n_avalanches, r)
        o = self.endpoints_struct(capacity)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return gt_autotune(self.ctx, r, o, self.ws.data_ptr(), self.ws.numel(), s.cuda_stream)

    def fetch(self, n: int) -> dict:
        """Copy the first n endpoints and the per-avalanche arrays to numpy."""
        out = {}
        for k in _EP_ARRAYS:
            a = self.ep[k][:n].cpu().numpy()
            if k == "uid":
                a = a.view(np.uint64)
            if k == "n_flight":
                a = a.view(np.uint32)
            out[k] = a
        out["electrons"] = self.ep["electrons"].cpu().numpy().view(np.uint64)
        out["tallies"] = self.ep["tallies"].cpu().numpy().view(np.uint64)
        if self.ep.get("signal") is not None:
            out["signal"] = self.ep["signal"].cpu().numpy()
        return out

    def observables(self, n_endpoints: int, prim: W.Primaries, collect_status: int,
                    drift_status: int = -1, gap: float = 0.0, stream=None) -> np.ndarray:
        torch = self.torch
        dev = f"cuda:{self.device}"
        n_prim = np.bincount(prim.aval, minlength=prim.n_avalanches).astype(np.int32)
        n_prim_t = torch.from_numpy(n_prim).to(dev)
        obs = torch.zeros(GT_OBS_COUNT, dtype=torch.float64, device=dev)
        cap = self.ep["x0"].numel()
        o = self.endpoints_struct(cap)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        avalanche_observables(self.ctx, o, n_endpoints, prim.n_avalanches, n_prim_t.data_ptr(),
                              collect_status, drift_status, gap, obs.data_ptr(), s.cuda_stream)
        return obs.cpu().numpy()


class Graph:
    """A batched run recorded as a CUDA graph (gt_graph_* in the C ABI)."""

    def __init__(self, owner: "Avalanche", handle: C.c_void_p):
        self.owner = owner
        self.h = handle

    def launch(self, seed: int, stream=None) -> None:
        torch = self.owner.torch
        s = stream if stream is not None else torch.cuda.current_stream(self.owner.device)
        _check(load().gt_graph_launch(self.h, seed & (2**64 - 1), s.cuda_stream),
               "gt_graph_launch", self.owner.ctx)

    def stats(self, allow=PARTIAL_OK) -> dict:
        st = gt_stats()
        rc = load().gt_graph_stats(self.h, C.byref(st))
        _check(rc, "gt_graph_stats", self.owner.ctx, allow)
        return st.as_dict()

    def close(self) -> None:
        if self.h:
            load().gt_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
