"""A workload's avalanches split over GPUs, and the parts gathered.

Avalanches do not interact (Sec. 2: the work is embarrassingly parallel):
each is a pure function of the seed, its avalanche number and its
primaries, because the random streams are keyed by (seed, avalanche number,
electron id, flight).  A workload of A avalanches therefore splits into
contiguous ranges of avalanche numbers, one per process and GPU.  Each part
runs alone with `aval_base` = the first avalanche of its range (the number
that keys its random streams), its avalanches renumbered from 0 for its own
per-avalanche arrays, and the workload's electron ids.  The only exchange is
the gather at the end: rank 0 concatenates the endpoint records and places
each part's per-avalanche arrays at its range.  The union is the result of
one run of the whole workload, electron for electron.

Host logic only (numpy and torch.distributed); the transport runs in the
CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

# per-avalanche arrays of a result dict (the rest are per-electron arrays)
PER_AVALANCHE = ("electrons", "tallies", "signal")


def partition(n_avalanches: int, world_size: int, rank: int) -> tuple[int, int]:
    """Contiguous range [a0, a1) of avalanche numbers for `rank`: sizes differ
    by at most one, lower ranks take the larger parts."""
    if world_size < 1 or not 0 <= rank < world_size or n_avalanches < 0:
        raise ValueError("bad partition arguments")
    q, r = divmod(n_avalanches, world_size)
    a0 = rank * q + min(rank, r)
    return a0, a0 + q + (1 if rank < r else 0)


def part_primaries(prim: W.Primaries, a0: int, a1: int) -> W.Primaries:
    """The primaries of avalanches [a0, a1), renumbered from 0; electron ids
    and per-avalanche fields are those of the workload.  Run it with
    aval_base = a0."""
    if not 0 <= a0 <= a1 <= prim.n_avalanches:
        raise ValueError(f"range [{a0}, {a1}) outside 0..{prim.n_avalanches}")
    keep = (prim.aval >= a0) & (prim.aval < a1)
    af = None if prim.aval_field is None else prim.aval_field[a0:a1].copy()
    return W.Primaries(
        *(getattr(prim, k)[keep].copy() for k in ("x", "y", "z", "t", "e", "dx", "dy", "dz")),
        aval=(prim.aval[keep] - a0).astype(np.int32), uid=prim.uid[keep].copy(),
        n_avalanches=a1 - a0, aval_field=af)


def merge(parts, n_avalanches: int) -> dict:
    """One result from the parts' results, given as (a0, result) pairs whose
    ranges tile [0, n_avalanches): per-electron arrays concatenated in part
    order (the endpoint's avalanche number shifted by a0), per-avalanche
    arrays placed at their ranges."""
    parts = sorted(parts, key=lambda p: p[0])
    out: dict = {}
    covered = 0
    for a0, res in parts:
        n_av = int(np.asarray(res["electrons"]).shape[0])
        if a0 != covered:
            raise ValueError(f"parts do not tile the avalanches: gap or overlap at {covered}")
        covered = a0 + n_av
        for k, v in res.items():
            v = np.asarray(v)
            if k in PER_AVALANCHE:
                if k not in out:
                    out[k] = np.zeros((n_avalanches,) + v.shape[1:], v.dtype)
                out[k][a0:a0 + n_av] = v
            else:
                if k == "aval":
                    v = v.astype(np.int64) + a0
                out.setdefault(k, []).append(v)
    if covered != n_avalanches:
        raise ValueError(f"parts cover {covered} of {n_avalanches} avalanches")
    for k, v in list(out.items()):
        if isinstance(v, list):
            out[k] = np.concatenate(v)
            if k == "aval":
                out[k] = out[k].astype(np.int32)
    return out


def gather(result: dict, a0: int, n_avalanches: int, group=None, dst: int = 0):
    """Collective over the ranks of `group` (torch.distributed): every rank
    passes its part's result (numpy arrays); rank `dst` returns the merged
    result of the whole workload, the others None."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    payload = (int(a0), {k: np.asarray(v) for k, v in result.items()})
    got = [None] * world if rank == dst else None
    dist.gather_object(payload, got, dst=dist.get_global_rank(group, dst) if group else dst,
                       group=group)
    if rank != dst:
        return None
    return merge(got, n_avalanches)
