"""Autotuner of the packet-pool launch: for a grid (or a batch of grids), time the
transport of a package prefix under each candidate (resident blocks per SM, threads
per block, interaction batch, refill period, and for a single grid the walk) with CUDA
events and keep the fastest.
Results are cached in a JSON file keyed by the workload class (cells to the nearest
power of two, species, levels, bins, optical-depth decade; for a batch, its models'
classes)."""
from __future__ import annotations

import itertools
import json
import math
import os
from typing import Dict, Optional

from . import rt

# the batched launch runs the linked walk; a single grid also tries the path walk
BATCH_CANDIDATES = dict(blocks_per_sm=(0, 5), threads=(128, 256), interaction_batch=(4, 8, 12),
                        refill_period=(16, 32))
CANDIDATES = dict(BATCH_CANDIDATES, walk=(rt.WALK_LINKED, rt.WALK_PATH))


def single_grid_candidates():
    """The launch options tried for one grid. Five resident blocks of 256 threads
    select the linked walk's variant compiled for that occupancy; the path walk is
    compiled for four such blocks only, so there a cap of five is the occupancy itself
    and that launch is tried (and reported) once, as blocks_per_sm = 0."""
    for values in itertools.product(*CANDIDATES.values()):
        opts = dict(zip(CANDIDATES, values))
        if (opts["walk"] == rt.WALK_PATH and opts["blocks_per_sm"] == 5 and
                opts["threads"] == 256):
            continue
        yield opts
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1201_3588_gb300",
                             "autotune.json")


def workload_key(grid: "rt.Grid", tau_v: float) -> str:
    return (f"cells2^{int(round(math.log2(max(grid.N, 1))))}-S{grid.S}-"
            f"L{grid.model.tree.max_level}-bins{grid.B}-"
            f"tau1e{int(math.floor(math.log10(max(tau_v, 1e-30))))}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(grid: "rt.Grid", tau_v: float, n_probe: int = 2_000_000, cache: Optional[str] = None,
         force: bool = False) -> Dict[str, int]:
    """Best launch options for this grid's class (the grid must have a source with at
    least n_probe planned packages; its tallies are reset afterwards)."""
    import torch
    path = cache or DEFAULT_CACHE
    db = _load(path)
    key = workload_key(grid, tau_v)
    if key in db and not force:
        return db[key]["opts"]
    s = torch.cuda.current_stream()
    n_probe = min(n_probe, getattr(grid, "n_total", n_probe))
    grid.transport(min(n_probe, 100_000), seed=1)      # warm
    best = None
    for opts in single_grid_candidates():
        grid.reset(s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        grid.transport(n_probe, seed=7, stream=s, **opts)
        b.record(s)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        if best is None or ms < best[0]:
            best = (ms, opts)
    grid.reset(s)
    torch.cuda.synchronize()
    db[key] = {"opts": best[1], "ms_per_probe": best[0], "n_probe": n_probe}
    _store(path, db)
    return best[1]


def _store(path, db):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def batch_key(grids, tau_vs, n_packages) -> str:
    classes = sorted(workload_key(g, t) for g, t in zip(grids, tau_vs))
    h = 0
    for c in classes:
        for ch in c.encode():
            h = (h * 131 + ch) % (1 << 61)
    pk = int(round(math.log2(max(sum(n_packages), 1))))
    return f"batch{len(grids)}-pk2^{pk}-{h:016x}"


def tune_batch(grids, tau_vs, n_packages, fraction: float = 0.05, seed: int = 0,
               cache: Optional[str] = None, force: bool = False) -> Dict[str, int]:
    """Best launch options for one batched launch of these grids: every candidate
    runs the whole batch on `fraction` of each model's packages (at least one each),
    so the choice weighs every model class by the work it brings."""
    import torch
    path = cache or DEFAULT_CACHE
    db = _load(path)
    key = batch_key(grids, tau_vs, n_packages)
    if key in db and not force:
        return db[key]["opts"]
    probe = [max(1, int(n * fraction)) for n in n_packages]
    s = torch.cuda.current_stream()
    best = None
    for values in itertools.product(*BATCH_CANDIDATES.values()):
        opts = dict(zip(BATCH_CANDIDATES, values))
        b = rt.Batch(grids, probe, seed=seed, **opts)
        b.run(reset=True, temperatures=False, stream=s)       # warm
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        b.run(reset=True, temperatures=False, stream=s)
        e.record(s)
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        b.close()
        if best is None or ms < best[0]:
            best = (ms, opts)
    for g in grids:
        g.reset(s)
    torch.cuda.synchronize()
    db[key] = {"opts": best[1], "ms_per_probe": best[0], "probe_packages": sum(probe)}
    _store(path, db)
    return best[1]

