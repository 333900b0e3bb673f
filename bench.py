"""Benchmark: real electron-collisions per second of the batched mixed-precision
avalanche transport on one GB300 (configuration: 4096 parallel-plate
avalanches in the argon-like gas, per-avalanche field U(30, 50) kV/cm,
Poisson(3) primaries, one persistent launch per step), with the plain
one-avalanche-at-a-time FP64 GPU path and the FP64 CPU oracle as
comparators.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line on rank 0.  Under torchrun with N ranks the workload
is one batched workload of N x 4096 avalanches (one seed); rank r transports
the contiguous avalanche range r x 4096 .. (r+1) x 4096 - 1 with its random
streams keyed by the workload's avalanche numbers, and rank 0 gathers the
per-avalanche electron counts and collision tallies over the host at the
end: weak scaling, no collective during the runs.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "electron-collisions/sec on 1 GB300 (batched mixed vs plain FP64) at matched gain/v_d"
UNIT = "electron-collisions/s"
WORKLOAD = "plate_batched_4096"

# Roofline of the batched transport kernel (bound: instruction issue of the
# SM's ALU/FMA pipes).  Work per flight, two ways:
# - calibrated: lane instructions of the kernel's own straight-line step,
#   ncu smsp__thread_inst_executed.sum / flights on `bench.py --calibrate
#   --steps 1 --block B --refill-period 32 --flights-per-phase 1` with the
#   banded majorant (the step's build for one flight per round, band bounds
#   rising with energy and no magnetic field), per launch bound B (the
#   register allocation differs).  Lanes
#   switched off by divergence are not counted, so divergence, stalls and
#   queue work all show as lost efficiency;
# - algorithmic: the operations the method needs per flight of the mixed
#   step on this workload (Philox-10 block, majorant window and reach, log,
#   exact flight, energy, table interpolation, and per real collision the
#   level choice, tally, isotropic direction and speed), counted from its
#   arithmetic, one lane instruction per operation; what the kernel issues
#   beyond it (spill code, addressing, control, FP64 folds) is overhead.
LANE_INST_PER_FLIGHT_BY_BLOCK = {768: 321.2, 896: 323.2, 1024: 313.5}
ALGORITHMIC_LANE_INST_PER_FLIGHT = 190.0
# The same calibration for the field-map line on the 256^3 grid (`bench.py
# --calibrate --calibrate-field grid --block B --refill-period 16
# --flights-per-phase 1`: straight-line flights at r = 1 mm in the map, the
# step plus eight float4 gathers and the trilinear interpolation per flight).
GRID_LANE_INST_PER_FLIGHT_BY_BLOCK = {512: 419.7, 768: 442.3, 1024: 414.1}


def lane_inst_per_flight(block: int, table=None) -> float:
    """The calibration of the launch bound a block size runs under (None
    when the table has none)."""
    table = LANE_INST_PER_FLIGHT_BY_BLOCK if table is None else table
    if not table:
        return None
    for bound in sorted(table):
        if block <= bound:
            return table[bound]
    return table[max(table)]


def issue_peak(sm_max_mhz) -> float:
    """Lane instructions per second of the whole GPU, in G: 152 SMs x 4
    schedulers x 32 lanes x the SM clock."""
    return SM_COUNT * ISSUE_PER_SM_PER_CLK * LANES_PER_WARP * (sm_max_mhz or 2070.0) * 1e6 / 1e9


SM_COUNT = 152
ISSUE_PER_SM_PER_CLK = 4       # warp schedulers per SM, one instruction each per clock
LANES_PER_WARP = 32
# DRAM bytes per electron of the batched kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum on the 256-avalanche case at 1024 threads: 139.5 MB +
# 321.1 MB for 2,005,010 electrons; traffic grows with electrons, so it is
# scaled to a launch by the electrons the launch stores).  Set back to None
# when the kernel changes, until the next capture.
DRAM_BYTES_PER_ELECTRON = 229.7
# Bytes per electron that the batched transport kernel must move by its
# data layout: at birth the start record (x0 y0 z0 t0 e0, 40 B), id (8),
# avalanche (4), birth velocity (24), birth element (4) and ready flag (4)
# are written (84 B); the lane that takes the electron reads them back
# without e0 (76 B); at the end x1 y1 z1 t1 e1 (40), status (4) and flight
# count (4) are written (48 B).
ALGORITHMIC_BYTES_PER_ELECTRON = 84 + 76 + 48


# ---------------------------------------------------------------- sharding
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, backend_device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, backend_device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU baseline
def oracle_baseline(w, seed: int, n_aval: int, args, keep: bool = False) -> dict:
    """The FP64 oracle as it stands on the host cores, on the first n_aval
    avalanches of the workload (a bounded sample), with the same majorant
    as the GPU run.  keep: also return the oracle's endpoints ("_out")."""
    import oracle
    sub = w.primaries.subset(list(range(n_aval)))
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    o = oracle.run(w.gas, w.field, sub, seed=seed, t_max=w.t_max, n_threads=threads,
                   majorant=int(args.majorant == "banded"), window=args.window,
                   band_width=w.gas.band_width)
    dt = time.perf_counter() - t0
    L = w.gas.n_levels
    real = int(o["tallies"][:, :L].sum())
    res = {"value": real / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"avalanches 0..{n_aval - 1} of {w.primaries.n_avalanches} "
                     f"({real:.3g} real collisions in {dt:.1f} s, {args.majorant} majorant)",
           "seconds": dt, "real_collisions": real}
    if keep:
        res["_out"] = o
        res["_prim"] = sub
    return res


# ---------------------------------------------------- matched observables
def matched_check(av, w, ref_out, ref_prim, n_aval: int, opt, seeds, cap, stream, collect,
                  geometry: str = "plate") -> dict:
    """The batched mixed-precision GPU path against the FP64 oracle on the
    same avalanche numbers 0..n_aval-1 with independent seeds (the oracle
    run `ref_out` with its seed; the GPU once per seed in `seeds`): gain,
    Townsend coefficient, drift velocity and diffusion, each with its
    bootstrap standard error over avalanches, the difference in units of
    the combined error and a pass at 3 sigma."""
    from paper_2509_15377_gb300 import avalanche as A
    from paper_2509_15377_gb300 import observables as O
    gap = w.field.gap
    n_prim = np.bincount(ref_prim.aval, minlength=ref_prim.n_avalanches)[:n_aval]
    ref = O.with_errors(O.per_avalanche(ref_out, n_aval, collect, n_prim, geometry), gap,
                        geometry, seed=1)
    dev_prim = av.primaries_device(ref_prim)
    parts = []
    for sd in seeds:
        st = av.run(dev_prim, dataclasses.replace(opt, seed=sd), cap, stream=stream,
                    allow=(A.GT_OK,))
        out = av.fetch(st["n_endpoints"])
        parts.append(O.per_avalanche(out, n_aval, collect, n_prim, geometry))
    # (avalanche, seed) pairs are the independent units of the GPU sample
    gpu = O.with_errors({k: np.concatenate([p_[k] for p_ in parts]) for k in parts[0]}, gap,
                        geometry, seed=2)
    rows = O.compare(ref, gpu)
    return {"avalanches": n_aval, "oracle_runs": 1, "gpu_seeds": len(seeds),
            "observables": {k: {"oracle": r["a"], "oracle_se": r["se_a"], "mixed": r["b"],
                                "mixed_se": r["se_b"], "rel_diff": r["rel_diff"],
                                "sigma": r["sigma"], "pass_3sigma": r["within_3sigma"]}
                            for k, r in rows.items()},
            "gain_window_3sigma_rel": 3.0 * math.hypot(rows["gain"]["se_a"], rows["gain"]["se_b"])
            / rows["gain"]["a"],
            "matched": all(r["within_3sigma"] for r in rows.values())}


# ---------------------------------------------------------------- our arm
def field_map_lines(av, args, seed: int, cap: int, stream, flush, majorant) -> dict:
    """Field maps of the coax geometry (the grid workload's box, 1810 V, one
    primary at r = 1 mm per avalanche): the regular 256^3 grid and a
    tetrahedral mesh of the same box (48^3 jittered cubes graded towards the
    wire, six elements each), batched mixed.  Each map's launch shape comes
    from the autotuner on its first --map-tune-avalanches avalanches (about
    1e5 electrons each: enough to keep every SM busy for most of a run),
    unless given on the command line."""
    from paper_2509_15377_gb300 import avalanche as A
    from paper_2509_15377_gb300 import workloads as W
    maps = {}
    n_map = args.map_avalanches
    chosen = [m for m in args.maps.split(",") if m]
    for name in chosen:
        if name == "grid":
            wl = W.grid_stress(n_avalanches=n_map, n=256, seed=seed)
        else:
            wl = W.mesh_coax(n_avalanches=n_map, cells=48, seed=seed, grading=4.0)
        av.set_gas(wl.gas)
        av.set_field(wl.field)
        m_opt = A.RunOptions(seed=seed, t_max=wl.t_max, precision=A.GT_MIXED, mode=A.GT_BATCHED,
                             block=args.block, refill_period=args.refill_period,
                             flights_per_phase=args.flights_per_phase,
                             majorant=majorant, majorant_window=args.window)
        tuned = None
        if not args.no_autotune:
            tsub = wl.primaries.subset(list(range(min(args.map_tune_avalanches, n_map))))
            tb, tp = av.autotune(av.primaries_device(tsub), m_opt, cap, stream=stream)
            tuned = {"best": [tb["block"], tb["refill_period"], tb["flights_per_phase"]],
                     "runs": len(tp), "sample_avalanches": len(set(tsub.aval.tolist()))}
        m_dev = av.primaries_device(wl.primaries)
        m_real, m_ms, m_fl = 0, 0.0, 0
        for _ in range(2):
            flush.fill_(1)
            m_st = av.run(m_dev, m_opt, cap, stream=stream, allow=(A.GT_OK,))
            m_real += m_st["real_collisions"]
            m_ms += m_st["transport_ms"]
            m_fl += m_st["flights"]
        maps[name] = {"value_kernel_time": m_real / (m_ms / 1e3), "unit": UNIT,
                      "flights_per_real": m_fl / max(m_real, 1), "avalanches": n_map,
                      "electrons_per_avalanche": m_st["n_endpoints"] / n_map,
                      "shape": [m_st["block"], m_st["refill_period"], m_st["flights_per_phase"]],
                      "autotune": tuned}
        if name == "grid":
            maps[name]["map"] = "256^3 float4 nodes, trilinear"
            lipf = lane_inst_per_flight(m_st["block"], GRID_LANE_INST_PER_FLIGHT_BY_BLOCK)
            if lipf:
                # issue roofline of the line: the calibrated work per flight
                # times the line's flights per second of transport time; the
                # line's first ~15 ns run only its 256 primaries (latency)
                ach = lipf * m_fl / (m_ms / 1e3) / 1e9
                peak = issue_peak(None)
                maps[name]["roofline"] = {
                    "bound": "alu", "achieved": ach, "peak": peak, "unit": "Glane-inst/s",
                    "frac": ach / peak, "lane_inst_per_flight": lipf,
                    "flights_per_s": m_fl / (m_ms / 1e3),
                    "kernel": "k_batched<MixedElectron, GRID, smem table>",
                    "peak_note": "152 SMs x 4 schedulers x 32 lanes x 2070 MHz"}
        else:
            maps[name]["map"] = (f"{wl.field.mesh_tets.shape[0]} tetrahedra, "
                                 f"{wl.field.mesh_nodes.shape[0]} nodes, linear, "
                                 "graded towards the wire (sinh, a = 4)")
    return maps


def run_maps_only(args) -> None:
    """Only the field-map lines (a profiling aid): prints their JSON."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_15377_gb300 import avalanche as A
    torch.cuda.set_device(0)
    av = A.Avalanche(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda:0")
    majorant = A.GT_MAJORANT_BANDED if args.majorant == "banded" else A.GT_MAJORANT_GLOBAL
    maps = field_map_lines(av, args, 0, args.capacity, stream, flush, majorant)
    print(json.dumps({"field_maps": maps}))
    av.close()


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    # the gather at the end goes over the host (gloo), not the GPUs
    host_group = dist.new_group(backend="gloo") if ws > 1 else None

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier()
    from paper_2509_15377_gb300 import avalanche as A
    from paper_2509_15377_gb300 import shard
    from paper_2509_15377_gb300 import workloads as W

    # one workload of ws x 4096 avalanches, one seed; this rank's contiguous
    # range of avalanche numbers (rank 0's part of the 1-GPU run is the
    # whole 4096-avalanche workload)
    seed = 0
    n_total = args.avalanches * ws
    whole = W.plate_batched(n_avalanches=n_total, seed=seed)
    a0, a1 = shard.partition(n_total, ws, rank)
    w = dataclasses.replace(whole, primaries=shard.part_primaries(whole.primaries, a0, a1))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w, seed, args.cpu_avalanches, args, keep=True)

    av = A.Avalanche(local)
    av.set_gas(w.gas)
    av.set_field(w.field)
    prim_dev = av.primaries_device(w.primaries)
    majorant = A.GT_MAJORANT_BANDED if args.majorant == "banded" else A.GT_MAJORANT_GLOBAL
    opt = A.RunOptions(seed=seed, t_max=w.t_max, precision=A.GT_MIXED, mode=A.GT_BATCHED,
                       block=args.block, refill_period=args.refill_period,
                       flights_per_phase=args.flights_per_phase, majorant=majorant,
                       majorant_window=args.window, aval_base=a0)
    cap = args.capacity
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    tune = None
    if not args.no_autotune and not (args.block or args.refill_period or args.flights_per_phase):
        # launch shape chosen by the library's autotuner on a sample of the
        # workload (outside the timed region); later runs use it
        sample = w.primaries.subset(list(range(min(args.tune_avalanches, args.avalanches))))
        best, pts = av.autotune(av.primaries_device(sample), opt, cap, stream=stream)
        tune = {"best": best, "sample_avalanches": args.tune_avalanches,
                "points": [[q["block"], q["refill_period"], q["flights_per_phase"],
                            round(q["real_per_ms"] / 1e6, 4)] for q in pts],
                "points_unit": "[block, refill_period, flights_per_phase, 1e9 real collisions/s]"}

    # the timed steps replay the batched run as a captured CUDA graph (a new
    # seed per step: different avalanches, same work); --no-graph calls
    # avalanche_run instead
    graph = None if args.no_graph else av.graph(prim_dev, opt, cap)
    step_no = [0]

    def step(prim):
        flush.fill_(1)
        step_no[0] += 1
        if graph is None:
            return av.run(prim, dataclasses.replace(opt, seed=seed + 7919 * step_no[0]), cap,
                          stream=stream, allow=(A.GT_OK,))
        graph.launch(seed + 7919 * step_no[0], stream=stream)
        return graph.stats(allow=(A.GT_OK,))

    for _ in range(args.warmup):
        step(prim_dev)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    real = flights = 0
    kernel_ms = []
    stats = []
    for _ in range(args.steps):
        st = step(prim_dev)
        real += st["real_collisions"]
        flights += st["flights"]
        kernel_ms.append(st["transport_ms"])
        stats.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    t_max_rank = max_over_ranks(elapsed, dev)
    total_real = sum_over_ranks(float(real), dev)
    value = total_real / t_max_rank

    # the gather: every rank's per-avalanche electron counts and tallies of
    # the last step, placed at its avalanche range on rank 0 (over the host)
    last = stats[-1]
    part = {"electrons": av.ep["electrons"][:a1 - a0].cpu().numpy().view(np.uint64),
            "tallies": av.ep["tallies"][:a1 - a0].cpu().numpy().view(np.uint64)}
    merged = shard.gather(part, a0, n_total, group=host_group) if ws > 1 else part
    gathered = None
    if rank == 0:
        L = w.gas.n_levels
        gathered = {"avalanches": int(merged["electrons"].shape[0]),
                    "electrons": int(merged["electrons"].sum()),
                    "real_collisions_last_step": int(merged["tallies"][:, :L].sum()),
                    "ranges": [list(shard.partition(n_total, ws, r)) for r in range(ws)]}

    # observables of the last step (gain, drift velocity)
    obs = av.observables(last["n_endpoints"], w.primaries, collect_status=W.ANODE,
                         drift_status=W.ANODE, gap=w.field.gap)

    # end to end through the public API: pinned host inputs copied inside
    # every step, the per-avalanche results read back (the endpoints stay on
    # the device, as the C ABI's output arrays are the caller's)
    prim_host = av.primaries_pinned(w.primaries)
    h_elec = torch.empty(w.primaries.n_avalanches, dtype=torch.int64).pin_memory()
    h_tal = torch.empty((w.primaries.n_avalanches, w.gas.n_levels + 1), dtype=torch.int64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_real = 0
    for _ in range(e2e_steps):
        flush.fill_(1)
        st = av.run(prim_host, opt, cap, stream=stream, allow=(A.GT_OK,))
        h_elec.copy_(av.ep["electrons"], non_blocking=True)
        h_tal.copy_(av.ep["tallies"], non_blocking=True)
        torch.cuda.synchronize()
        e2e_real += st["real_collisions"]
    e2e_t = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = sum_over_ranks(float(e2e_real), dev) / e2e_t
    h2d = sum(prim_host[k].numel() * prim_host[k].element_size()
              for k in list(A.Avalanche.PRIM_KEYS) + ["aval", "uid", "aval_field"])
    d2h = h_elec.numel() * 8 + h_tal.numel() * 8 + 256

    if rank != 0:
        av.close()
        return
    extra = not args.no_plain

    def timed_runs(o, prim, n=2):
        """Real collisions per second of transport-kernel time over n runs."""
        r_, ms_, fl_ = 0, 0.0, 0
        for _ in range(n):
            flush.fill_(1)
            s_ = av.run(prim, o, cap, stream=stream, allow=(A.GT_OK,))
            r_ += s_["real_collisions"]
            ms_ += s_["transport_ms"]
            fl_ += s_["flights"]
        return {"value_kernel_time": r_ / (ms_ / 1e3), "unit": UNIT,
                "flights_per_real": fl_ / max(r_, 1),
                "shape": [s_["block"], s_["refill_period"], s_["flights_per_phase"]]}, s_

    # the same batched mixed run with the other majorant (one global nu_max):
    # what the banded majorant alone buys
    other = None
    if extra:
        o_opt = dataclasses.replace(
            opt, majorant=A.GT_MAJORANT_GLOBAL if majorant == A.GT_MAJORANT_BANDED
            else A.GT_MAJORANT_BANDED)
        other, _ = timed_runs(o_opt, prim_dev)
        other["majorant"] = "global" if o_opt.majorant == A.GT_MAJORANT_GLOBAL else "banded"

    # the same batched run in FP64 (the FP64 kernel, autotuned): what mixed
    # precision alone buys, at the same batching
    fp64_batched = None
    tune_sample = av.primaries_device(
        w.primaries.subset(list(range(min(args.tune_avalanches, args.avalanches)))))
    if extra:
        f_opt = dataclasses.replace(opt, precision=A.GT_FP64, block=0, refill_period=0,
                                    flights_per_phase=0)
        if not args.no_autotune:
            av.autotune(tune_sample, f_opt, cap, stream=stream)
        fp64_batched, _ = timed_runs(f_opt, prim_dev, n=1)
        fp64_batched["note"] = "same 4096-avalanche workload, FP64 batched kernel"

    # the same batched mixed step with the physical gas (screened-Coulomb
    # anisotropy, Opal-Peterson-Beaty sharing, attachment)
    physical = None
    if extra:
        av.set_gas(W.argon_like_physical_gas())
        if not args.no_autotune:  # each kernel build has its own best shape
            av.autotune(tune_sample, opt, cap, stream=stream)
        physical, p_st = timed_runs(opt, prim_dev)
        p_obs = av.observables(p_st["n_endpoints"], w.primaries, collect_status=W.ANODE,
                               drift_status=W.ANODE, gap=w.field.gap)
        physical.update(gas="argon-like + screened-Coulomb anisotropy, OPB sharing, attachment",
                        gain=p_obs[0])
        av.set_gas(w.gas)
        # the basic gas with exact boundary crossings (the general kernel)
        c_opt = dataclasses.replace(opt, crossing=1)
        if not args.no_autotune:
            av.autotune(tune_sample, c_opt, cap, stream=stream)
        physical["crossing"], _ = timed_runs(c_opt, prim_dev)
        physical["crossing"]["note"] = "basic gas, endpoints at the first boundary crossing"
        # the basic gas with the anode's induced signal, 2000 bins of 50 ps
        s_opt = dataclasses.replace(opt, signal_kind=W.W_PLATE, signal_bins=2000,
                                    signal_t0=0.0, signal_dt=0.05)
        if not args.no_autotune:  # a kernel build of its own (crossings alone have another)
            av.autotune(tune_sample, s_opt, cap, stream=stream)
        physical["signal"], _ = timed_runs(s_opt, prim_dev)
        physical["signal"]["note"] = ("basic gas, Shockley-Ramo anode signal per avalanche, "
                                      "2000 bins x 0.05 ns")

    # the coaxial tube with a 1 T axial field: 2048 avalanches, one primary
    # each at r in 1-4.5 mm, batched mixed (E x B flights)
    coax = None
    if extra:
        cw = W.coax(n_avalanches=2048, seed=seed)
        av.set_gas(cw.gas)
        av.set_field(cw.field)
        c_prim = av.primaries_device(cw.primaries)
        c_opt = dataclasses.replace(opt, t_max=cw.t_max, block=0, refill_period=0,
                                    flights_per_phase=0, aval_base=0)
        if not args.no_autotune:
            av.autotune(av.primaries_device(cw.primaries.subset(list(range(512)))), c_opt, cap,
                        stream=stream)
        coax, c_st = timed_runs(c_opt, c_prim)
        c_obs = av.observables(c_st["n_endpoints"], cw.primaries, collect_status=W.WIRE)
        coax.update(avalanches=2048, gain=c_obs[0], gain_se=c_obs[1],
                    electrons_per_avalanche=c_st["n_endpoints"] / 2048,
                    field="coax a = 25 um, b = 5 mm, 1500 V, B = 1 T axial")

    maps = None
    if extra:
        maps = field_map_lines(av, args, seed, cap, stream, flush, majorant)
    av.set_gas(w.gas)
    av.set_field(w.field)

    # plain FP64 GPU path (the paper's structure: one avalanche at a time, one
    # launch per generation) on a sample, with both majorants
    plain = None
    if extra:
        sub = w.primaries.subset(list(range(args.plain_avalanches)))
        psub = av.primaries_device(sub)
        plain = {"sample": f"avalanches 0..{args.plain_avalanches - 1}", "unit": UNIT}
        for name, mj in (("global", A.GT_MAJORANT_GLOBAL), ("banded", A.GT_MAJORANT_BANDED)):
            popt = A.RunOptions(seed=seed, t_max=w.t_max, precision=A.GT_FP64, mode=A.GT_PLAIN,
                                majorant=mj, majorant_window=args.window)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pst = av.run(psub, popt, cap, stream=stream, allow=(A.GT_OK,))
            torch.cuda.synchronize()
            pdt = time.perf_counter() - t0
            plain["value_" + name] = pst["real_collisions"] / pdt
            if mj == majorant:
                # like for like: the speedup compares runs with the same majorant
                plain.update(value=plain["value_" + name], majorant=name,
                             launches=pst["launches"], generations=pst["iterations"])

    # matched observables: the batched mixed path against the FP64 oracle on
    # the same avalanche numbers with independent seeds
    matched = None
    if extra and cpu is not None:
        matched = {"plate_batched_sample": matched_check(
            av, w, cpu.pop("_out"), cpu.pop("_prim"), args.cpu_avalanches, opt,
            [seed + 1001, seed + 1002], cap, stream, W.ANODE)}
        import oracle
        pw = W.plate(n_avalanches=1000, e_field=40_000.0, seed=seed)
        t0 = time.perf_counter()
        p_ref = oracle.run(pw.gas, pw.field, pw.primaries, seed=seed, t_max=pw.t_max,
                           majorant=int(majorant == A.GT_MAJORANT_BANDED), window=args.window,
                           band_width=pw.gas.band_width)
        p_secs = time.perf_counter() - t0
        av.set_field(pw.field)
        matched["plate_40kV_1000"] = matched_check(
            av, pw, p_ref, pw.primaries, 1000, dataclasses.replace(opt, t_max=pw.t_max,
                                                                  aval_base=0),
            [seed + 2001, seed + 2002, seed + 2003, seed + 2004], cap, stream, W.ANODE)
        matched["plate_40kV_1000"]["oracle_seconds"] = p_secs
        matched["matched"] = all(v["matched"] for v in matched.values() if isinstance(v, dict))
        av.set_field(w.field)
    elif cpu is not None:
        cpu.pop("_out")
        cpu.pop("_prim")

    kms = statistics.mean(kernel_ms)
    fl_per_launch = flights / len(kernel_ms)
    peak_clk = clk.get("sm_max_mhz") or 2070.0
    peak = issue_peak(peak_clk)
    lipf = lane_inst_per_flight(stats[-1]["block"])
    achieved = lipf * fl_per_launch / (kms / 1e3) / 1e9
    achieved_alg = ALGORITHMIC_LANE_INST_PER_FLIGHT * fl_per_launch / (kms / 1e3) / 1e9
    electrons_per_launch = statistics.mean(s["n_endpoints"] for s in stats)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Glane-inst/s",
            "frac": achieved / peak,
            "traffic": (DRAM_BYTES_PER_ELECTRON * electrons_per_launch
                        if DRAM_BYTES_PER_ELECTRON else None),
            "traffic_unit": "bytes per launch (ncu DRAM bytes per electron x electrons)",
            "algorithmic_bytes": ALGORITHMIC_BYTES_PER_ELECTRON * electrons_per_launch,
            "kernel": "k_batched<MixedElectron, PLATE, smem table>", "kernel_ms": kms,
            "flights_per_launch": fl_per_launch,
            "lane_inst_per_flight": lipf,
            "algorithmic": {"lane_inst_per_flight": ALGORITHMIC_LANE_INST_PER_FLIGHT,
                            "achieved": achieved_alg, "frac": achieved_alg / peak},
            "peak_note": "152 SMs x 4 schedulers x 32 lanes x max SM clock (measured max)",
            "clock_frac": (clk.get("sm_mhz") or peak_clk) / peak_clk}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max_rank * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "avalanches_per_gpu": args.avalanches,
                   "avalanches_total": n_total,
                   "field_kv_cm": [30, 50], "primaries_mean": 3, "gap_um": 128,
                   "gas": "argon-like 12-level", "precision": "mixed", "mode": "batched",
                   "block": stats[-1]["block"], "grid": stats[-1]["grid"],
                   "refill_period": stats[-1]["refill_period"],
                   "flights_per_phase": stats[-1]["flights_per_phase"],
                   "autotune": tune,
                   "launch": "avalanche_run per step" if args.no_graph else
                             "captured CUDA graph replay per step (new seed each)",
                   "l2": "flushed (256 MB write) before every step",
                   "parallelism": f"{ws} GPU(s), contiguous avalanche ranges, host gather"},
        "flights_per_s": sum_over_ranks(float(flights), dev) / t_max_rank,
        "null_fraction": 1.0 - real / max(flights, 1),
        "electrons_per_step": stats[-1]["n_endpoints"],
        "gathered": gathered,
        "observables": {"gain": obs[0], "gain_se": obs[1], "vd_cm_per_ns": obs[3],
                        "dt_cm2_per_ns": obs[4], "dl_cm2_per_ns": obs[5], "alpha_per_cm": obs[7]},
        "matched": matched,
        "majorant": args.majorant,
        "flights_per_real": flights / max(real, 1),
        "other_majorant": other,
        "fp64_batched": fp64_batched,
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (value / plain["value"]) if plain else None,
        "speedup_vs_fp64_batched": (value / fp64_batched["value_kernel_time"])
        if fp64_batched else None,
        "physical_gas": physical,
        "coax_b": coax,
        "field_maps": maps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "readback": "per-avalanche electron counts and tallies; endpoints stay on the device"},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    av.close()


# ------------------------------------------------------------- calibration
def calibration_workload(n_electrons: int, coll_limit: int = 1000, field: str = "plate"):
    """Straight-line flights for the instruction count per flight, run by the
    same kernel instantiation as the benchmark line: the argon-like table
    with its ionisation rate set to zero (same 12-level selection, no
    secondaries), one electron per thread, each stopped after `coll_limit`
    real collisions.  plate: 40 kV/cm, an anode too far away to reach, from
    mid-gap; grid: the field-map line's 256^3 coax map (1810 V), from
    r = 1 mm at mid-length (1000 collisions move an electron a few um)."""
    from paper_2509_15377_gb300 import workloads as W
    g = W.argon_like_gas()
    g.rate = g.rate.copy()
    g.rate[:, -1] = 0.0
    w = W.drift_model(n_electrons=n_electrons, n_coll=coll_limit, e_field=40_000.0, seed=0)
    w.gas = g
    if field == "grid":
        gs = W.grid_stress(n_avalanches=n_electrons, n=256, seed=0)
        w.field = gs.field
        w.primaries = gs.primaries
        return w
    w.field = W.Field(W.PLATE, e0=40_000.0, gap=1.0e3)
    w.primaries.z[:] = 500.0
    return w


def run_calibration(args) -> None:
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_15377_gb300 import avalanche as A
    av = A.Avalanche(0)
    threads = SM_COUNT * (args.block or 1024)
    w = calibration_workload(threads, field=args.calibrate_field)
    av.set_gas(w.gas)
    av.set_field(w.field)
    prim = av.primaries_device(w.primaries)
    opt = A.RunOptions(seed=0, coll_limit=w.coll_limit, precision=A.GT_MIXED, mode=A.GT_BATCHED,
                       block=args.block, refill_period=args.refill_period,
                       flights_per_phase=args.flights_per_phase,
                       majorant=(A.GT_MAJORANT_BANDED if args.majorant == "banded"
                                 else A.GT_MAJORANT_GLOBAL),
                       majorant_window=args.window)
    for _ in range(max(1, args.steps)):
        st = av.run(prim, opt, threads, allow=(A.GT_OK,))
    torch.cuda.synchronize()
    print(json.dumps({"calibration": args.calibrate_field, "electrons": threads,
                      "flights": st["flights"],
                      "warp_flights": st["flights"] / 32.0, "real": st["real_collisions"],
                      "transport_ms": st["transport_ms"], "block": st["block"],
                      "grid": st["grid"]}), flush=True)
    av.close()


# ----------------------------------------------------------- reference arm
def run_reference(args) -> None:
    """The reference arm is the FP64 CPU oracle on the host cores, on a
    bounded sample of this workload per step (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2509_15377_gb300 import workloads as W
    import oracle
    oracle.build()
    w = W.plate_batched(n_avalanches=args.avalanches, seed=0)
    per_step = max(1, args.ref_avalanches)
    for _ in range(args.warmup):
        oracle_baseline(w, 0, max(1, per_step // 8), args)
    real = 0
    secs = 0.0
    res = None
    for _ in range(args.steps):
        res = oracle_baseline(w, 0, per_step, args)
        real += res["real_collisions"]
        secs += res["seconds"]
    value = real / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "avalanches_per_gpu": args.avalanches},
            "cpu_baseline": {"kind": "oracle", "cores": res["cores"], "sample": res["sample"],
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def parse(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--avalanches", type=int, default=4096)
    ap.add_argument("--capacity", type=int, default=100_000_000)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--refill-period", type=int, default=0)
    ap.add_argument("--flights-per-phase", type=int, default=0)
    # the oracle's sample: ~17 s of CPU work on 16 Arm cores (banded majorant),
    # also the oracle side of the matched check; the reference arm takes
    # --ref-avalanches per step
    ap.add_argument("--cpu-avalanches", type=int, default=1024)
    ap.add_argument("--ref-avalanches", type=int, default=256,
                    help="oracle avalanches per step of the reference arm")
    ap.add_argument("--plain-avalanches", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="time avalanche_run calls instead of captured graph replays")
    ap.add_argument("--majorant", default="banded", choices=["banded", "global"])
    ap.add_argument("--window", type=float, default=2.0)
    ap.add_argument("--tune-avalanches", type=int, default=1024)
    ap.add_argument("--maps-only", action="store_true",
                    help="only the grid / mesh field-map lines (profiling aid)")
    ap.add_argument("--maps", default="grid,mesh")
    ap.add_argument("--map-avalanches", type=int, default=256)
    ap.add_argument("--map-tune-avalanches", type=int, default=96)
    ap.add_argument("--calibrate", action="store_true",
                    help="run the straight-line calibration workload (for ncu)")
    ap.add_argument("--calibrate-field", default="plate", choices=["plate", "grid"])
    return ap.parse_args(argv)


def main(argv=None):
    args = parse(argv)
    if args.maps_only:
        run_maps_only(args)
    elif args.calibrate:
        run_calibration(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
