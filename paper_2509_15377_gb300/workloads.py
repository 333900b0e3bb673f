"""Seeded synthetic inputs for microscopic avalanche transport.

This module only *describes* workloads: gas rate tables, field geometries and
primary electrons, drawn from fixed seeds with numpy.  It holds none of the
transport arithmetic; both the CUDA library and the CPU oracle take its
arrays as inputs.

The paper's own workloads (single and triple GEM with ANSYS field maps and
Magboltz gas files, Sec. 4) are not available, so synthetic stand-ins are
used: a constant-rate model gas (drift closed forms), an argon-like
12-level gas, parallel-plate, coaxial (optionally with axial B) and a
regular-grid field map sampled from the coaxial field.

Units: cm, ns, eV, V/cm, T; collision rates in 1/ns (1e12/s = 1000/ns).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Level kinds of a gas table (interface values of the C ABI).
ELASTIC, EXCITATION, IONISATION, ATTACHMENT = 0, 1, 2, 3
# Field kinds (interface values of the C ABI).
UNIFORM, PLATE, COAX, GRID, MESH = 0, 1, 2, 3, 4
# Electron status codes written to the endpoints (non-zero = finished).
STATUS_NAMES = {
    0: "active", 1: "anode", 2: "cathode", 3: "wire", 4: "tube",
    5: "out_of_map", 6: "time", 7: "coll_limit", 8: "flight_limit",
}
ANODE, CATHODE, WIRE, TUBE, OUT_OF_MAP, TIME, COLL_LIMIT = 1, 2, 3, 4, 5, 6, 7
W_NONE, W_PLATE, W_COAX, W_MAP = 0, 1, 2, 3   # readout electrode of induced signals
FLIGHT_LIMIT, ATTACHED = 8, 9

# Electron mass in unified atomic mass units (CODATA 2018).
ELECTRON_MASS_U = 5.48579909065e-4
ARGON_MASS_U = 39.948

# Excitation slope of the argon-like gas (1/ns per eV above threshold),
# chosen once with the oracle so that the mean gain at 40 kV/cm over a
# 128 um gap is about 1e3.
ARGON_LIKE_K_EXC = 7.25


@dataclasses.dataclass
class Gas:
    """Tabulated per-level collision rates on a uniform energy grid."""
    level_type: np.ndarray   # int32 [L]
    threshold: np.ndarray    # float64 [L] eV lost by the level
    rate: np.ndarray         # float64 [N, L] 1/ns at node energies k * d_eps
    d_eps: float             # eV
    recoil: float = 0.0      # 2m/M (elastic recoil loss), 0 = no loss
    nu_max: float = 0.0      # 1/ns, 0 = derived by the consumer
    band_width: float = 1.0  # eV per energy band of the banded majorant
    # angular model per level: anisotropy xi0 (constant) where screen == 0,
    # else xi = eps / (eps + screen); None = all isotropic
    xi0: Optional[np.ndarray] = None      # float64 [L] in (-1, 1)
    screen: Optional[np.ndarray] = None   # float64 [L] eV, >= 0
    split_w: float = 0.0     # ionisation sharing width (eV); 0 = uniform split

    @property
    def n_levels(self) -> int:
        return int(self.rate.shape[1])

    @property
    def n_nodes(self) -> int:
        return int(self.rate.shape[0])


@dataclasses.dataclass
class Field:
    kind: int
    e0: float = 0.0                 # UNIFORM / PLATE |E| (V/cm), E = (0,0,-e0)
    gap: float = 0.0                # PLATE gap (cm)
    wire_r: float = 0.0             # COAX / GRID wire radius (cm)
    tube_r: float = 0.0             # COAX tube radius (cm)
    voltage: float = 0.0            # COAX wire voltage (V)
    b: tuple = (0.0, 0.0, 0.0)      # uniform B (T)
    grid: Optional[np.ndarray] = None   # GRID float32 [nz, ny, nx, 4]
    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1.0, 1.0, 1.0)
    mesh_nodes: Optional[np.ndarray] = None   # MESH float64 [n, 3] node positions (cm)
    mesh_tets: Optional[np.ndarray] = None    # MESH int32 [m, 4] node indices
    mesh_values: Optional[np.ndarray] = None  # MESH float32 [n, 4] (Ex, Ey, Ez, weighting potential)


@dataclasses.dataclass
class Primaries:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    t: np.ndarray
    e: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    aval: np.ndarray          # int32
    uid: np.ndarray           # uint64
    n_avalanches: int
    aval_field: Optional[np.ndarray] = None   # PLATE per-avalanche |E| (V/cm)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, avalanches) -> "Primaries":
        """Only the primaries of the listed avalanches.

        Avalanche numbers, electron ids and the per-avalanche fields are
        kept unchanged (the other avalanches are simply empty), so a run
        keyed by (seed, avalanche, electron id) reproduces exactly the same
        avalanches as the full workload."""
        sel = np.zeros(self.n_avalanches, dtype=bool)
        sel[np.asarray(avalanches, dtype=np.int64)] = True
        keep = sel[self.aval]
        af = None if self.aval_field is None else self.aval_field.copy()
        return Primaries(
            *(getattr(self, k)[keep].copy() for k in ("x", "y", "z", "t", "e", "dx", "dy", "dz")),
            aval=self.aval[keep].copy(), uid=self.uid[keep].copy(),
            n_avalanches=self.n_avalanches, aval_field=af)


@dataclasses.dataclass
class Workload:
    name: str
    gas: Gas
    field: Field
    primaries: Primaries
    t_max: float = 0.0          # ns, 0 = none
    coll_limit: int = 0         # real collisions per electron, 0 = none
    seed: int = 0


# ------------------------------------------------------------------ gases
def model_gas(nu_elastic: float = 1000.0, nu_ion: float = 0.0, ion_threshold: float = 0.0,
              recoil: float = 0.0, n_nodes: int = 2, d_eps: float = 1000.0,
              exact_nu_max: bool = True, nu_att: float = 0.0, xi_elastic: float = 0.0) -> Gas:
    """Energy-independent rates: elastic (isotropic, or with the constant
    anisotropy xi_elastic) and optionally an ionisation level and an
    attachment level (threshold 0) with fixed rates."""
    types = [ELASTIC]
    thr = [0.0]
    cols = [np.full(n_nodes, nu_elastic)]
    if nu_ion > 0.0:
        types.append(IONISATION)
        thr.append(ion_threshold)
        cols.append(np.full(n_nodes, nu_ion))
    if nu_att > 0.0:
        types.append(ATTACHMENT)
        thr.append(0.0)
        cols.append(np.full(n_nodes, nu_att))
    rate = np.stack(cols, axis=1).astype(np.float64)
    xi0 = None
    if xi_elastic != 0.0:
        xi0 = np.zeros(len(types))
        xi0[0] = xi_elastic
    return Gas(np.array(types, np.int32), np.array(thr, np.float64), rate, float(d_eps),
               float(recoil), float(rate[0].sum()) if exact_nu_max else 0.0, xi0=xi0)


def argon_like_gas(k_exc: float = ARGON_LIKE_K_EXC) -> Gas:
    """Argon-like synthetic gas: 0-100 eV in 2000 bins (2001 nodes), elastic
    1e12*sqrt(eps/eV)/s, ten excitation levels with thresholds spread evenly
    over 11.5-15 eV and rates k_exc*(eps - E_j), one ionisation level at
    15.7 eV with rate 5e10*(eps - 15.7)/s; elastic recoil on M = 39.948 u."""
    n_nodes, d_eps = 2001, 0.05
    eps = np.arange(n_nodes, dtype=np.float64) * d_eps
    thr_exc = 11.5 + np.arange(10) * (3.5 / 9.0)
    rates = [1000.0 * np.sqrt(eps)]
    for ej in thr_exc:
        rates.append(np.where(eps >= ej, k_exc * (eps - ej), 0.0))
    rates.append(np.where(eps >= 15.7, 50.0 * (eps - 15.7), 0.0))
    rate = np.stack(rates, axis=1)
    types = np.array([ELASTIC] + [EXCITATION] * 10 + [IONISATION], np.int32)
    thr = np.concatenate([[0.0], thr_exc, [15.7]]).astype(np.float64)
    recoil = 2.0 * ELECTRON_MASS_U / ARGON_MASS_U
    return Gas(types, thr, rate, d_eps, recoil, 0.0)


def argon_like_physical_gas(k_exc: float = ARGON_LIKE_K_EXC, screen: float = 6.8,
                            split_w: float = 10.0, nu_att: float = 2.0) -> Gas:
    """The argon-like gas with the physics of the next level of detail:
    every level scatters with the screened-Coulomb anisotropy
    xi = eps / (eps + screen); the ionisation remainder is shared with the
    Opal-Peterson-Beaty form of width split_w; and an attachment level with
    the constant rate nu_att (1/ns, threshold 0) stands in for an
    electronegative admixture.  All three are synthetic choices."""
    g = argon_like_gas(k_exc)
    rate = np.concatenate([g.rate, np.full((g.n_nodes, 1), nu_att)], axis=1)
    types = np.concatenate([g.level_type, [ATTACHMENT]]).astype(np.int32)
    thr = np.concatenate([g.threshold, [0.0]])
    return Gas(types, thr, rate, g.d_eps, g.recoil, 0.0,
               screen=np.full(len(types), float(screen)), split_w=float(split_w))


# -------------------------------------------------------------- primaries
def _isotropic(rng: np.random.Generator, n: int, forward_z: bool = False):
    c = rng.uniform(-1.0, 1.0, n)
    if forward_z:
        c = np.abs(c)
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    return s * np.cos(phi), s * np.sin(phi), c


def _primaries(rng, x, y, z, aval, n_aval, e0=0.1, forward_z=False, aval_field=None):
    n = len(x)
    dx, dy, dz = _isotropic(rng, n, forward_z)
    return Primaries(np.asarray(x, np.float64), np.asarray(y, np.float64),
                     np.asarray(z, np.float64), np.zeros(n), np.full(n, e0),
                     dx, dy, dz, np.asarray(aval, np.int32),
                     np.arange(n, dtype=np.uint64), int(n_aval), aval_field)


# -------------------------------------------------------------- workloads
def drift_model(n_electrons: int = 1000, n_coll: int = 100_000, e_field: float = 1000.0,
                nu: float = 1000.0, b=(0.0, 0.0, 0.0), seed: int = 0) -> Workload:
    """Constant-rate elastic model gas, uniform E = (0,0,-E0); every electron
    is its own avalanche and stops after `n_coll` real collisions."""
    rng = np.random.default_rng(seed)
    z = np.zeros(n_electrons)
    prim = _primaries(rng, z, z, z, np.arange(n_electrons), n_electrons)
    return Workload("drift_model", model_gas(nu), Field(UNIFORM, e0=e_field, b=tuple(b)),
                    prim, 0.0, n_coll, seed)


def plate(n_avalanches: int = 1000, e_field: float = 40_000.0, gap: float = 0.0128,
          k_exc: float = ARGON_LIKE_K_EXC, t_max: float = 100.0, seed: int = 0) -> Workload:
    """Argon-like gas, parallel-plate gap, one primary per avalanche released
    from the cathode (x = y = z = 0) with 0.1 eV into the gas half-space."""
    rng = np.random.default_rng(seed)
    z = np.zeros(n_avalanches)
    prim = _primaries(rng, z, z, z, np.arange(n_avalanches), n_avalanches, forward_z=True)
    return Workload("plate", argon_like_gas(k_exc), Field(PLATE, e0=e_field, gap=gap),
                    prim, t_max, 0, seed)


def plate_batched(n_avalanches: int = 4096, e_lo: float = 30_000.0, e_hi: float = 50_000.0,
                  mean_primaries: float = 3.0, gap: float = 0.0128,
                  k_exc: float = ARGON_LIKE_K_EXC, t_max: float = 100.0,
                  seed: int = 0) -> Workload:
    """Many parallel-plate avalanches with per-avalanche field ~ U(e_lo, e_hi)
    and Poisson(mean) primaries (empty avalanches kept)."""
    rng = np.random.default_rng(seed)
    fields = rng.uniform(e_lo, e_hi, n_avalanches)
    counts = rng.poisson(mean_primaries, n_avalanches)
    aval = np.repeat(np.arange(n_avalanches), counts)
    z = np.zeros(len(aval))
    prim = _primaries(rng, z, z, z, aval, n_avalanches, forward_z=True, aval_field=fields)
    return Workload("plate_batched", argon_like_gas(k_exc), Field(PLATE, e0=40_000.0, gap=gap),
                    prim, t_max, 0, seed)


def coax(n_avalanches: int = 2048, wire_r: float = 25e-4, tube_r: float = 0.5,
         voltage: float = 1500.0, b_axial: float = 1.0, r_lo: float = 0.1, r_hi: float = 0.45,
         k_exc: float = ARGON_LIKE_K_EXC, t_max: float = 10_000.0, seed: int = 0) -> Workload:
    """Coaxial tube with axial B; one primary per avalanche at r ~ U(r_lo, r_hi),
    phi ~ U(0, 2 pi), z = 0 (the tube is infinite in z)."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_lo, r_hi, n_avalanches)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_avalanches)
    prim = _primaries(rng, r * np.cos(phi), r * np.sin(phi), np.zeros(n_avalanches),
                      np.arange(n_avalanches), n_avalanches)
    f = Field(COAX, wire_r=wire_r, tube_r=tube_r, voltage=voltage, b=(0.0, 0.0, b_axial))
    return Workload("coax", argon_like_gas(k_exc), f, prim, t_max, 0, seed)


def coax_grid_map(n: int = 256, half_width: float = 0.15, length: float = 1.0,
                  wire_r: float = 25e-4, tube_r: float = 0.5, voltage: float = 1500.0) -> Field:
    """A regular n^3 float32 map of the coaxial field on
    [-w, w]^2 x [0, length]; nodes inside the wire take the field at r = a.
    The 4th component holds the wire's weighting potential
    ln(r/b) / ln(a/b) (1 on the wire, 0 on the tube) for induced signals."""
    xs = np.linspace(-half_width, half_width, n)
    zs = np.linspace(0.0, length, n)
    X, Y = np.meshgrid(xs, xs, indexing="xy")          # [ny, nx]
    r2 = np.maximum(X * X + Y * Y, wire_r * wire_r)
    s = voltage / (math.log(tube_r / wire_r) * r2)
    plane = np.zeros((n, n, 4), np.float32)
    plane[..., 0] = s * X
    plane[..., 1] = s * Y
    plane[..., 3] = np.log(np.sqrt(r2) / tube_r) / math.log(wire_r / tube_r)
    grid = np.broadcast_to(plane, (len(zs), n, n, 4)).astype(np.float32)
    sp = 2.0 * half_width / (n - 1)
    return Field(GRID, wire_r=wire_r, tube_r=tube_r, voltage=voltage, grid=np.ascontiguousarray(grid),
                 origin=(-half_width, -half_width, 0.0), spacing=(sp, sp, length / (n - 1)))


# The six tetrahedra of a cube that share its main diagonal, corner c = the
# bits (x, y, z): one per order in which the three axes are stepped from
# corner 0 to corner 7.  Every cube cut the same way gives a conforming mesh.
_CUBE_TETS = ((0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7))


def box_mesh(cells, lo, hi, jitter: float = 0.15, seed: int = 0):
    """A synthetic FEM-like tetrahedral mesh of the box [lo, hi]: a lattice of
    cells[0] x cells[1] x cells[2] cubes, each cut into six tetrahedra, with
    every node moved by up to `jitter` lattice spacings along each axis in
    which it is not on the box's surface (the box faces stay planar).
    Returns (nodes float64 [n, 3], tets int32 [m, 4]), every tetrahedron
    positively oriented."""
    cells = tuple(int(c) for c in cells)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    rng = np.random.default_rng(seed)
    axes = [np.linspace(lo[d], hi[d], cells[d] + 1) for d in range(3)]
    I, J, K = np.meshgrid(np.arange(cells[0] + 1), np.arange(cells[1] + 1), np.arange(cells[2] + 1),
                          indexing="ij")
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    nodes = np.stack([axes[d][idx[:, d]] for d in range(3)], axis=1)
    h = (hi - lo) / np.asarray(cells, np.float64)
    for d in range(3):
        inner = (idx[:, d] > 0) & (idx[:, d] < cells[d])
        nodes[inner, d] += rng.uniform(-jitter, jitter, int(inner.sum())) * h[d]

    def node(i, j, k):
        return (i * (cells[1] + 1) + j) * (cells[2] + 1) + k

    ci, cj, ck = np.meshgrid(np.arange(cells[0]), np.arange(cells[1]), np.arange(cells[2]),
                             indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    corner = np.stack([node(ci + (c & 1), cj + ((c >> 1) & 1), ck + ((c >> 2) & 1))
                       for c in range(8)], axis=1)
    tets = np.concatenate([corner[:, list(t)] for t in _CUBE_TETS], axis=0).astype(np.int32)
    v = nodes[tets]
    det = np.einsum("ij,ij->i", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))
    flip = det < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    if np.min(np.abs(det)) <= 0.05 * float(np.prod(h)):
        raise ValueError("jitter too large: a tetrahedron is nearly flat")
    return nodes, tets


def coax_mesh_map(cells: int = 8, half_width: float = 0.15, length: float = 1.0,
                  jitter: float = 0.15, wire_r: float = 25e-4, tube_r: float = 0.5,
                  voltage: float = 1500.0, seed: int = 0, grading: float = 0.0) -> Field:
    """The coaxial field on a jittered tetrahedral mesh of [-w, w]^2 x
    [0, length] (cells^3 cubes, six tetrahedra each), sampled at the nodes
    as coax_grid_map samples its grid (r clamped at the wire radius); the
    4th nodal value is the wire's weighting potential.  grading = a > 0
    refines the mesh towards the wire: x and y become w sinh(a x/w)/sinh(a)
    (cells about cosh(a) times finer on the axis than at the box's side)."""
    nodes, tets = box_mesh((cells, cells, cells), (-half_width, -half_width, 0.0),
                           (half_width, half_width, length), jitter, seed)
    if grading > 0.0:
        nodes[:, :2] = half_width * np.sinh(grading * nodes[:, :2] / half_width) / math.sinh(grading)
        v = nodes[tets]
        det = np.einsum("ij,ij->i", v[:, 1] - v[:, 0],
                        np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))
        if not np.all(det > 0.0):
            raise ValueError("grading turned an element over")
    x, y = nodes[:, 0], nodes[:, 1]
    r2 = np.maximum(x * x + y * y, wire_r * wire_r)
    s = voltage / (math.log(tube_r / wire_r) * r2)
    vals = np.zeros((nodes.shape[0], 4), np.float32)
    vals[:, 0] = s * x
    vals[:, 1] = s * y
    vals[:, 3] = np.log(np.sqrt(r2) / tube_r) / math.log(wire_r / tube_r)
    return Field(MESH, wire_r=wire_r, tube_r=tube_r, voltage=voltage, mesh_nodes=nodes,
                 mesh_tets=tets, mesh_values=vals)


def uniform_mesh_map(e0: float, half_width: float, cells: int = 6, jitter: float = 0.15,
                     seed: int = 0) -> Field:
    """E = (0, 0, -e0) given at the nodes of a jittered tetrahedral mesh of
    the cube [-w, w]^3: inside it the same field as Field(UNIFORM, e0)."""
    nodes, tets = box_mesh((cells, cells, cells), (-half_width,) * 3, (half_width,) * 3, jitter, seed)
    vals = np.zeros((nodes.shape[0], 4), np.float32)
    vals[:, 2] = -e0
    return Field(MESH, mesh_nodes=nodes, mesh_tets=tets, mesh_values=vals)


def mesh_coax(n_avalanches: int = 64, cells: int = 8, voltage: float = 1810.0,
              r_start: float = 0.1, k_exc: float = ARGON_LIKE_K_EXC, t_max: float = 1000.0,
              seed: int = 0, grading: float = 0.0) -> Workload:
    """The grid workload's geometry on a tetrahedral mesh: coax field sampled
    at the nodes of a jittered (optionally graded) mesh of the map box; one
    primary per avalanche at r = r_start, random phi, mid-length."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_avalanches)
    f = coax_mesh_map(cells=cells, voltage=voltage, seed=seed, grading=grading)
    prim = _primaries(rng, r_start * np.cos(phi), r_start * np.sin(phi),
                      np.full(n_avalanches, 0.5), np.arange(n_avalanches), n_avalanches)
    return Workload("mesh_coax", argon_like_gas(k_exc), f, prim, t_max, 0, seed)


def grid_stress(n_avalanches: int = 256, n: int = 256, voltage: float = 1810.0,
                r_start: float = 0.1, k_exc: float = ARGON_LIKE_K_EXC, t_max: float = 1000.0,
                seed: int = 0) -> Workload:
    """Coax-sampled regular-grid map; one primary per avalanche at
    r = r_start, random phi, mid-length.  The default voltage gives a mean
    gain near 1e5 with the argon-like gas (oracle: 1.14e5 +- 0.12e5 at
    1820 V over 64 avalanches, 6.9e4 +- 1.1e4 at 1775 V over 16)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_avalanches)
    f = coax_grid_map(n=n, voltage=voltage)
    zc = 0.5 * (f.origin[2] + f.spacing[2] * (n - 1))
    prim = _primaries(rng, r_start * np.cos(phi), r_start * np.sin(phi),
                      np.full(n_avalanches, zc), np.arange(n_avalanches), n_avalanches)
    return Workload("grid_stress", argon_like_gas(k_exc), f, prim, t_max, 0, seed)
