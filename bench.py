"""Benchmark: real electron-collisions per second of the batched mixed-precision
avalanche transport on one GB300 (configuration: 4096 parallel-plate
avalanches in the argon-like gas, per-avalanche field U(30, 50) kV/cm,
Poisson(3) primaries, one persistent launch per step), with the plain
one-avalanche-at-a-time FP64 GPU path and the FP64 CPU oracle as
comparators.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line on rank 0.  Under torchrun every rank runs its own
4096 avalanches (seed = rank): weak scaling, no collective on the data path.
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
# SM's ALU/FMA pipes).  Algorithmic work per flight = lane instructions of
# the straight-line step: ncu smsp__thread_inst_executed.sum / flights on
# `bench.py --calibrate --steps 1 --block B --refill-period 32
# --flights-per-phase 1` with the default banded majorant, per launch bound
# B (the spill code differs; profiles/k_batched_mixed_plate_batched_4096.md).
# Lanes switched off by divergence are not counted, so divergence, stalls
# and queue work all show as lost efficiency.
LANE_INST_PER_FLIGHT_BY_BLOCK = {768: 413.3, 896: 402.1, 1024: 423.8}


def lane_inst_per_flight(block: int) -> float:
    """The calibration of the launch bound a block size runs under."""
    for bound in sorted(LANE_INST_PER_FLIGHT_BY_BLOCK):
        if block <= bound:
            return LANE_INST_PER_FLIGHT_BY_BLOCK[bound]
    return LANE_INST_PER_FLIGHT_BY_BLOCK[max(LANE_INST_PER_FLIGHT_BY_BLOCK)]


SM_COUNT = 152
ISSUE_PER_SM_PER_CLK = 4       # warp schedulers per SM, one instruction each per clock
LANES_PER_WARP = 32
# DRAM bytes per electron of the batched kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum on the 256-avalanche case, divided by its
# electrons; traffic grows with electrons, so it is scaled to a launch by
# the electrons the launch stores).  None once the kernel has changed: the
# last capture (199.8 B per electron) predates the 4-byte birth-element
# field that every new electron now stores.
DRAM_BYTES_PER_ELECTRON = None


# ---------------------------------------------------------------- sharding
def shard_seed(rank: int) -> int:
    """Each rank transports its own statistically identical workload."""
    return rank


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
def oracle_baseline(w, seed: int, n_aval: int, args) -> dict:
    """The FP64 oracle as it stands on the host cores, on the first n_aval
    avalanches of the workload (a bounded sample), with the same majorant
    as the GPU run."""
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
    return {"value": real / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"avalanches 0..{n_aval - 1} of {w.primaries.n_avalanches} "
                      f"({real:.3g} real collisions in {dt:.1f} s, {args.majorant} majorant)",
            "seconds": dt, "real_collisions": real}


# ---------------------------------------------------------------- our arm
def field_map_lines(av, args, seed: int, cap: int, stream, flush, majorant) -> dict:
    """Field maps of the coax geometry (the grid workload's box, 1810 V, one
    primary at r = 1 mm per avalanche): the regular 256^3 grid and a
    tetrahedral mesh of the same box (48^3 jittered cubes graded towards the
    wire, six elements each), batched mixed.  Launch shapes are fixed per map
    (the best of fixed-shape runs of the full workload; the autotuner's small
    samples, a few avalanches growing from one electron each, are starved of
    parallelism and pick poorly) unless given on the command line."""
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
        given = args.block or args.refill_period or args.flights_per_phase
        shape = ((args.block, args.refill_period, args.flights_per_phase) if given
                 else (512, 4, 1) if name == "grid" else (512, 32, 1))
        m_opt = A.RunOptions(seed=seed, t_max=wl.t_max, precision=A.GT_MIXED, mode=A.GT_BATCHED,
                             block=shape[0], refill_period=shape[1], flights_per_phase=shape[2],
                             majorant=majorant, majorant_window=args.window)
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
                      "shape": [m_st["block"], m_st["refill_period"], m_st["flights_per_phase"]]}
        if name == "grid":
            maps[name]["map"] = "256^3 float4 nodes, trilinear"
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

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier()
    from paper_2509_15377_gb300 import avalanche as A
    from paper_2509_15377_gb300 import workloads as W

    seed = shard_seed(rank)
    w = W.plate_batched(n_avalanches=args.avalanches, seed=seed)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w, seed, args.cpu_avalanches, args)

    av = A.Avalanche(local)
    av.set_gas(w.gas)
    av.set_field(w.field)
    prim_dev = av.primaries_device(w.primaries)
    majorant = A.GT_MAJORANT_BANDED if args.majorant == "banded" else A.GT_MAJORANT_GLOBAL
    opt = A.RunOptions(seed=seed, t_max=w.t_max, precision=A.GT_MIXED, mode=A.GT_BATCHED,
                       block=args.block, refill_period=args.refill_period,
                       flights_per_phase=args.flights_per_phase, majorant=majorant,
                       majorant_window=args.window)
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
            return av.run(prim, opt, cap, stream=stream, allow=(A.GT_OK,))
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

    # observables of the last step (gain, drift velocity) for the matched check
    last = stats[-1]
    obs = av.observables(last["n_endpoints"], w.primaries, collect_status=W.ANODE,
                         drift_status=W.ANODE, gap=w.field.gap)

    # end to end through the public API: pinned host inputs copied inside
    # every step, the per-avalanche results read back
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

    # plain FP64 GPU path (one avalanche per launch sequence) on a sample
    # the same batched mixed run with the global majorant (one nu_max), for
    # the gain of the banded majorant alone
    other = None
    if rank == 0 and not args.no_plain:
        o_opt = dataclasses.replace(
            opt, majorant=A.GT_MAJORANT_GLOBAL if majorant == A.GT_MAJORANT_BANDED
            else A.GT_MAJORANT_BANDED)
        o_real, o_ms = 0, 0.0
        for _ in range(2):
            flush.fill_(1)
            o_st = av.run(prim_dev, o_opt, cap, stream=stream, allow=(A.GT_OK,))
            o_real += o_st["real_collisions"]
            o_ms += o_st["transport_ms"]
        other = {"majorant": "global" if o_opt.majorant == A.GT_MAJORANT_GLOBAL else "banded",
                 "value_kernel_time": o_real / (o_ms / 1e3), "unit": UNIT,
                 "flights_per_real": o_st["flights"] / max(o_st["real_collisions"], 1)}

    # the same batched mixed step with the physical gas (screened-Coulomb
    # anisotropy, Opal-Peterson-Beaty sharing, attachment)
    physical = None
    if rank == 0 and not args.no_plain:
        av.set_gas(W.argon_like_physical_gas())
        tune_sample = av.primaries_device(w.primaries.subset(list(range(args.tune_avalanches))))
        if not args.no_autotune:  # each kernel build has its own best shape
            av.autotune(tune_sample, opt, cap, stream=stream)
        p_real, p_ms, p_fl = 0, 0.0, 0
        for _ in range(2):
            flush.fill_(1)
            p_st = av.run(prim_dev, opt, cap, stream=stream, allow=(A.GT_OK,))
            p_real += p_st["real_collisions"]
            p_ms += p_st["transport_ms"]
            p_fl += p_st["flights"]
        p_obs = av.observables(p_st["n_endpoints"], w.primaries, collect_status=W.ANODE,
                               drift_status=W.ANODE, gap=w.field.gap)
        physical = {"gas": "argon-like + screened-Coulomb anisotropy, OPB sharing, attachment",
                    "value_kernel_time": p_real / (p_ms / 1e3), "unit": UNIT,
                    "flights_per_real": p_fl / max(p_real, 1), "gain": p_obs[0],
                    "shape": [p_st["block"], p_st["refill_period"], p_st["flights_per_phase"]]}
        av.set_gas(w.gas)
        # the basic gas with exact boundary crossings (the general kernel)
        c_opt = dataclasses.replace(opt, crossing=1)
        if not args.no_autotune:
            av.autotune(tune_sample, c_opt, cap, stream=stream)
        c_real, c_ms = 0, 0.0
        for _ in range(2):
            flush.fill_(1)
            c_st = av.run(prim_dev, c_opt, cap, stream=stream, allow=(A.GT_OK,))
            c_real += c_st["real_collisions"]
            c_ms += c_st["transport_ms"]
        physical["crossing"] = {"value_kernel_time": c_real / (c_ms / 1e3), "unit": UNIT,
                                "note": "basic gas, endpoints at the first boundary crossing",
                                "shape": [c_st["block"], c_st["refill_period"],
                                          c_st["flights_per_phase"]]}
        # the basic gas with the anode's induced signal, 2000 bins of 50 ps
        s_opt = dataclasses.replace(opt, signal_kind=W.W_PLATE, signal_bins=2000,
                                    signal_t0=0.0, signal_dt=0.05)
        s_real, s_ms = 0, 0.0
        for _ in range(2):
            flush.fill_(1)
            s_st = av.run(prim_dev, s_opt, cap, stream=stream, allow=(A.GT_OK,))
            s_real += s_st["real_collisions"]
            s_ms += s_st["transport_ms"]
        physical["signal"] = {"value_kernel_time": s_real / (s_ms / 1e3), "unit": UNIT,
                              "note": "basic gas, Shockley-Ramo anode signal per avalanche, "
                                      "2000 bins x 0.05 ns"}

    maps = None
    if rank == 0 and not args.no_plain:
        maps = field_map_lines(av, args, seed, cap, stream, flush, majorant)
        av.set_gas(w.gas)
        av.set_field(w.field)

    # plain FP64 GPU path (the paper's structure: one avalanche at a time, one
    # launch per generation) on a sample, with both majorants
    plain = None
    if rank == 0 and not args.no_plain:
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
                pobs = av.observables(pst["n_endpoints"], sub, collect_status=W.ANODE,
                                      drift_status=W.ANODE, gap=w.field.gap)
                plain.update(value=plain["value_" + name], majorant=name,
                             launches=pst["launches"], generations=pst["iterations"])
        # the mixed batched run restricted to the same avalanches, for the gain match
        st_m = av.run(psub, opt, cap, stream=stream, allow=(A.GT_OK,))
        mobs = av.observables(st_m["n_endpoints"], sub, collect_status=W.ANODE,
                              drift_status=W.ANODE, gap=w.field.gap)
        se = math.hypot(pobs[1], mobs[1])
        plain.update(gain_fp64_plain=pobs[0], gain_mixed_batched=mobs[0], gain_sigma=se,
                     matched_gain_3sigma=bool(abs(pobs[0] - mobs[0]) <= 3 * se),
                     vd_fp64_plain=pobs[3], vd_mixed_batched=mobs[3])

    if rank != 0:
        av.close()
        return
    kms = statistics.mean(kernel_ms)
    fl_per_launch = flights / len(kernel_ms)
    peak_clk = clk.get("sm_max_mhz") or 2070.0
    # G lane-instructions/s: SMs x schedulers x lanes x max SM clock
    peak = SM_COUNT * ISSUE_PER_SM_PER_CLK * LANES_PER_WARP * peak_clk * 1e6 / 1e9
    lipf = lane_inst_per_flight(stats[-1]["block"])
    achieved = lipf * fl_per_launch / (kms / 1e3) / 1e9
    electrons_per_launch = statistics.mean(s["n_endpoints"] for s in stats)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Glane-inst/s",
            "frac": achieved / peak,
            "traffic": (DRAM_BYTES_PER_ELECTRON * electrons_per_launch
                        if DRAM_BYTES_PER_ELECTRON else None),
            "traffic_unit": "bytes per launch (ncu, scaled from the 256-avalanche capture)",
            "kernel": "k_batched<MixedElectron, PLATE, smem table>", "kernel_ms": kms,
            "flights_per_launch": fl_per_launch,
            "lane_inst_per_flight": lipf,
            "peak_note": "152 SMs x 4 schedulers x 32 lanes x max SM clock (measured max)",
            "clock_frac": (clk.get("sm_mhz") or peak_clk) / peak_clk}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max_rank * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "avalanches_per_gpu": args.avalanches,
                   "field_kv_cm": [30, 50], "primaries_mean": 3, "gap_um": 128,
                   "gas": "argon-like 12-level", "precision": "mixed", "mode": "batched",
                   "block": stats[-1]["block"], "grid": stats[-1]["grid"],
                   "refill_period": stats[-1]["refill_period"],
                   "flights_per_phase": stats[-1]["flights_per_phase"],
                   "autotune": tune,
                   "launch": "avalanche_run per step" if args.no_graph else
                             "captured CUDA graph replay per step (new seed each)",
                   "l2": "flushed (256 MB write) before every step"},
        "flights_per_s": sum_over_ranks(float(flights), dev) / t_max_rank,
        "null_fraction": 1.0 - real / max(flights, 1),
        "electrons_per_step": stats[-1]["n_endpoints"],
        "observables": {"gain": obs[0], "gain_se": obs[1], "vd_cm_per_ns": obs[3],
                        "dt_cm2_per_ns": obs[4], "dl_cm2_per_ns": obs[5]},
        "majorant": args.majorant,
        "flights_per_real": flights / max(real, 1),
        "other_majorant": other,
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (value / plain["value"]) if plain else None,
        "physical_gas": physical,
        "field_maps": maps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    av.close()


# ------------------------------------------------------------- calibration
def calibration_workload(n_electrons: int, coll_limit: int = 1000):
    """Straight-line flights for the instruction count per flight, run by the
    same kernel instantiation as the benchmark (plate field): the argon-like
    table with its ionisation rate set to zero (same 12-level selection, no
    secondaries), 40 kV/cm, an anode too far away to reach, one electron per
    thread from mid-gap, each stopped after `coll_limit` real collisions."""
    from paper_2509_15377_gb300 import workloads as W
    g = W.argon_like_gas()
    g.rate = g.rate.copy()
    g.rate[:, -1] = 0.0
    w = W.drift_model(n_electrons=n_electrons, n_coll=coll_limit, e_field=40_000.0, seed=0)
    w.gas = g
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
    w = calibration_workload(threads)
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
    print(json.dumps({"calibration": True, "electrons": threads, "flights": st["flights"],
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
    per_step = max(1, args.cpu_avalanches // 2)
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
    # the oracle's sample: ~10-15 s of CPU work on 16 Arm cores (banded majorant);
    # the reference arm takes half of it per step
    ap.add_argument("--cpu-avalanches", type=int, default=512)
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
    ap.add_argument("--calibrate", action="store_true",
                    help="run the straight-line calibration workload (for ncu)")
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
