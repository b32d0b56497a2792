#!/usr/bin/env python
"""Throughput of the photon-package transport on GB300: packages/s.

A step is one pass of the whole path over one batch of packages: zero the tallies,
transport the batch (Bjorkman-Wood re-emission, persistent packet-pool kernel,
FP32), invert the counts into per-cell temperatures (FP64), gather the escaped
spectrum and, where the model holds PAHs, compute the emission of every PAH-active
cell with the BF16 tensor-core surrogate and the exact transient-heating solution
as its fallback. The default workload is the large disk: gap and spiral, 256^3
base cubes with three levels of 2x2x2 refinement (1.73e8 cells), 400 frequency
bins, silicate, carbon and PAHs of 30 and 200 C atoms, 2.5e8 packages per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large_disk|disk|disk_pah|disk_images|sphere|batch]

Prints one JSON line. With several ranks (torchrun) every rank follows its own
package-id range (weak scaling), the integer counts are summed over ranks, and the
step time is the maximum over ranks. ``--impl reference`` times the CPU oracle
on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "photon packages/sec on 1 GB300 (chosen form vs plain) at stated T/count tolerance"
UNIT = "packages/s"
L2_BYTES = 129 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--packages", type=float, default=None,
                   help="packages per GPU per step (default: 2.5e8 for the large disk, "
                        "1e8 otherwise)")
    p.add_argument("--workload", choices=["disk", "sphere", "batch", "disk_pah", "disk_images",
                                          "large_disk", "disk4", "disk_pah_small", "surrogate"],
                   default="large_disk")
    p.add_argument("--rows", type=float, default=5e5,
                   help="surrogate workload: feature rows per forward pass")
    p.add_argument("--full-run", action="store_true",
                   help="after the timed steps, one untimed-by-the-line run of the "
                        "workload's full package count (1e10 for the large disk), reported "
                        "in the line's 'full_run'")
    p.add_argument("--batch-models", type=int, default=256)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--plain-packages", type=float, default=1e7)
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--walk", choices=["auto", "linked", "path"], default="auto",
                   help="the pool kernel's walk (auto: the path walk when the face-link "
                        "records exceed 4 GB)")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the autotuning of the pool launch before the timed steps")
    p.add_argument("--no-pah", action="store_true",
                   help="leave the PAH emission out of the step (the transport still "
                        "tallies PAH absorptions); for profiling the transport alone")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--cpu-one-thread", action="store_true",
                   help="time the oracle on one host thread instead of one process per core")
    a = p.parse_args()
    if a.packages is None:
        a.packages = DEFAULT_PACKAGES.get(a.workload, 1e8)
    return a


# packages per step: config 5 is timed on a prefix of its 1e10 packages, sized so
# that 20 timed steps take under a minute
DEFAULT_PACKAGES = {"large_disk": 2.5e8}
WALKS = {"auto": 0, "linked": 1, "path": 2}
FULL_PACKAGES = {"large_disk": 1e10, "disk": 1e8, "disk_pah": 1e8, "disk_images": 1e8,
                 "sphere": 1e5}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def build_model(name):
    from paper_1201_3588_gb300 import workloads as w
    if name == "sphere":
        return w.sphere_model(), "dust sphere 16^3, 64 bins, 2 species, tau_V=1"
    if name == "disk_images":
        return (w.disk_model(),
                "flared disk 128^3 base + 2 levels of 2x2x2 refinement, 200 bins, 2 species, "
                "midplane tau_V=1e3, r 0.1-100 AU; peel-off images at the 10 and 11.3 micron "
                "bins, 256x256 pixels over +-100 AU, inclination 60 deg, and their dual-band "
                "major-axis profile")
    if name == "large_disk":
        return (w.large_disk_model(),
                "large disk with gap and spiral, 256^3 base + 3 levels (1.73e8 cells), 400 bins, "
                "silicate, carbon, PAH 30 C and 200 C; PAH emission by the BF16 surrogate with "
                "exact fallback (tol 0.05)")
    if name == "disk4":
        return (w.disk4_model(),
                "flared disk with gap and spiral, 128^3 base + 2 levels, 400 bins, four dust "
                "species with the PAH disk's opacities and no PAH tallies (transport profiling)")
    if name == "disk_pah_small":
        return (w.disk_pah_model(n_base=64, max_level=1),
                "flared disk with gap and spiral, 64^3 base + 1 level, 200 bins, silicate, "
                "carbon, PAH 30 C and 200 C (PAH-kernel profiling)")
    if name == "disk_pah":
        return (w.disk_pah_model(),
                "flared disk with gap and spiral, 128^3 base + 2 levels, 200 bins, silicate, "
                "carbon, PAH 30 C and 200 C; PAH emission by the BF16 surrogate with exact "
                "fallback (tol 0.05)")
    return (w.disk_model(),
            "flared disk 128^3 base + 2 levels of 2x2x2 refinement, 200 bins, 2 species, "
            "midplane tau_V=1e3, r 0.1-100 AU")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_prefix(model, first, n_total, seconds, mode=0):
    """The oracle on one host thread: packages first, first + 1, ... of the workload,
    in chunks, until `seconds` have passed. Returns (packages, seconds)."""
    import oracle
    om = oracle.OracleModel(model)
    tally = oracle.new_tally(om)
    done, chunk = 0, 4
    t0 = time.perf_counter()
    while True:
        oracle.transport(om, chunk, seed=1000, first_id=first + done, n_total=n_total,
                         mode=mode, tally=tally)
        done += chunk
        el = time.perf_counter() - t0
        if el >= seconds:
            break
        chunk = max(1, min(chunk * 2, int(done / el * (seconds - el)) + 1))
    return done, el


_POOL_MODEL = None


def _oracle_worker(job):
    first, n_total, seconds, mode = job
    return _oracle_prefix(_POOL_MODEL, first, n_total, seconds, mode)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(model):
    """One oracle process per host core, forked while the process has not touched
    CUDA (they share the model's pages; none of them uses the GPU)."""
    global _POOL_MODEL
    _POOL_MODEL = model
    import multiprocessing as mp
    n = host_cores()
    pool = mp.get_context("fork").Pool(n)
    pool.n_workers = n
    return pool


def cpu_oracle_rate(model, n_total, seconds, mode=0, pool=None):
    """Oracle packages/s on the host cores: with a pool, every process follows its
    own range of package ids (disjoint, spread over the workload) for `seconds`;
    packages of all processes / the longest wall time. Returns (rate, packages,
    seconds, processes)."""
    if pool is None:
        done, el = _oracle_prefix(model, 0, n_total, seconds, mode)
        return done / el, done, el, 1
    w = pool.n_workers
    stride = max(1, n_total // w)
    res = pool.map(_oracle_worker, [(i * stride, n_total, seconds, mode) for i in range(w)])
    done = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return done / el, done, el, w


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    model, desc = build_model(args.workload)
    pool = oracle_pool(model) if not args.cpu_one_thread else None
    n_total = int(args.packages)
    per_step = max(1.0, args.cpu_seconds / 3.0)
    times, counts = [], []
    for i in range(args.warmup + args.steps):
        rate, n, el, cores = cpu_oracle_rate(model, n_total, per_step, pool=pool)
        if i >= args.warmup:
            times.append(el)
            counts.append(n)
    if pool is not None:
        pool.close()
        pool.join()
    value = sum(counts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "packages_per_step": sum(counts) // len(counts),
                       "sample": "oracle prefix of the same workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sum(counts)} packages over {args.steps} steps, "
                                       f"{cores} processes on disjoint package ranges"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Figures of the pool kernel from ncu captures, per workload, valid only for the
# kernel source they were measured on (the hash covers the code of the sources with
# comments and blank lines removed): DRAM traffic (dram__bytes_read.sum +
# dram__bytes_write.sum) per package of a prefix launch, and the mean active lanes
# per executed warp instruction (warp execution efficiency x 32).
PROFILE_SOURCES = ("paper_1201_3588_gb300/csrc/rt_transport.cu",
                   "paper_1201_3588_gb300/csrc/rt_internal.h")
PROFILE = {
    # 1-pass counters of one 2e7-package launch on the full large disk (path walk):
    # dram 174.27 GB read + 0.11 GB written; 6.759e10 warp and 1.053e12 thread
    # instructions over 5.24e9 crossings
    "large_disk": {"sha256": "37df585bc0db86db4b62d16c47608a40489a74d084f398b36c592e962be6373b",
                   "dram_bytes_per_package": 8718.9, "warp_lanes_active": 15.58,
                   "warp_instr_per_crossing": 12.89,
                   "file": "profiles/k_transport_pool_large_disk.md"},
    # the same counters of one 1e8-package launch on the flared disk (linked walk):
    # dram 103.92 GB read + 0.24 GB written; 1.496e11 warp and 2.543e12 thread
    # instructions over 1.41e10 crossings
    "disk": {"sha256": "37df585bc0db86db4b62d16c47608a40489a74d084f398b36c592e962be6373b",
             "dram_bytes_per_package": 1041.6, "warp_lanes_active": 17.0,
             "warp_instr_per_crossing": 10.62, "file": "profiles/k_transport_pool_disk.md"},
}


def source_code_hash(paths):
    """SHA-256 of C/C++ sources with comments, trailing blanks and empty lines
    removed, so that an edit of a comment does not void a capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in paths:
        with open(os.path.join(ROOT, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()


def profile_figures(workload):
    """The ncu figures of this workload when they belong to the current source."""
    p = PROFILE.get(workload)
    if not p or source_code_hash(PROFILE_SOURCES) != p["sha256"]:
        return None
    return p


def crossing_bytes(c, S, L):
    """Algorithmic bytes of one transport launch by the per-unit count of the
    method's data: every cell crossing reads the base-cube id (4 B), the child ids
    of the L refinement levels (4 B each) and the S densities (4 B each); every
    absorption is one 8-byte read-modify-write of a count (16 B)."""
    return c["crossings"] * (4 + 4 * L + 4 * S) + 16 * c["absorptions"]


def walk_bytes(c, S, path=False):
    """Bytes the walk that ran reads per launch. Linked walk: every cell entered reads
    its face link (4 B) and S densities (4 B each), every descent into a finer
    neighbour one child id (4 B). Path walk: every crossing reads one slot row (S
    densities or a block code, 4 B each), every level descended one more row (the
    `levels` counter), every interaction the leaf id (4 B) and its densities. Both:
    every absorption is one 8-byte read-modify-write of a count (16 B). Peel-off:
    every cell a sight line crosses reads a link and densities, every peeled event
    adds into an FP64 pixel (16 B)."""
    events = c["absorptions"] + c["scatters"] + c["capped"]
    if path:
        walk = 4 * S * (c["crossings"] + c["levels"]) + (4 + 4 * S) * events
    else:
        walk = (c["crossings"] + events) * (4 + 4 * S) + 4 * c["levels"]
    return (walk + 16 * c["absorptions"]
            + c.get("peel_crossings", 0) * (4 + 4 * S) + 16 * c.get("peel_events", 0))


def grid_bytes(model, path):
    """Device bytes of the grid arrays the transport reads and of the counts:
    densities, levels, the walk's own array (slot rows for the path walk, face-link
    records for the linked walk), tree, counts."""
    t = model.tree
    N, S = t.n_leaves, model.n_species
    slots = t.n_base ** 3 + 8 * t.n_blocks
    walk = 4 * S * slots if path else 32 * N
    return 4 * N * S + N + walk + 4 * slots + 8 * N * S


def path_walk_runs(walk, N, S, L, n_slots, images=False):
    """Whether the pool kernel runs the path walk (the same rule as rt_transport):
    walk is rt.WALK_* (0 automatic), n_slots the tree's base cells plus 8 per block."""
    fits = L <= 4 and n_slots < 2 ** 31 - 1
    if images or not fits:
        return False
    if walk == 0:
        return S == 4 or 32 * N > 4e9
    return walk == 2


def walk_label(choice, N, S, L):
    """The pool walk the library runs for this grid (the same rule as rt_transport)."""
    if choice == "auto":
        choice = "path" if L <= 4 and (S == 4 or 32 * N > 4e9) else "linked"
        return f"{choice} (automatic)"
    return choice


def has_pah(model):
    return any(sp.is_pah for sp in model.species)


def train_surrogate(g, n, first, stream, dev):
    """The PAH surrogate trained on the exact solutions of one untimed transport
    pass of the same model (at most 1e6 (cell, PAH) pairs, 8 epochs)."""
    import torch
    from paper_1201_3588_gb300 import rt, surrogate
    g.transport(n, seed=999, first_id=first, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, Y = surrogate.training_pairs(g)
    keep = torch.randperm(X.shape[0], device=dev)[:1_000_000]
    X, Y = X[keep].contiguous(), Y[keep].contiguous()
    net = rt.MLP(X.shape[1], surrogate.N_HIDDEN, surrogate.N_LAYERS, g.B, seed=0)
    hist = surrogate.train(net, X, Y, epochs=8)
    xp = X[:, -2]
    net.set_range(float(xp.min()) - 0.25, float(xp.max()) + 0.25)
    torch.cuda.synchronize()
    info = {"training_pairs": int(X.shape[0]), "train_s": time.perf_counter() - t0,
            "train_loss_first_last": [hist[0], hist[-1]]}
    del X, Y
    g.reset(stream)
    return net, info


def pah_step_launches(n_active, n_fallback, n_pah):
    """Kernels of one active-cell PAH emission pass: the compaction of PAH-active
    cells; per batch of at most 2^20 of them and per PAH the features, the fused
    network and the check, per PAH the add, and the compaction of failed cells;
    then one exact launch for those."""
    if n_active == 0:
        return 1
    batches = (n_active + (1 << 20) - 1) >> 20
    return 1 + batches * (4 * n_pah + 1) + (1 if n_fallback else 0)


def surrogate_error(g, net, cells_dev, j_dev, tol, stream):
    """Surrogate-with-fallback emission against the exact emission of the same cells
    (both from the library): energy-weighted L1 error, its median and 90th
    percentile over cells, and the time of each."""
    import torch
    from paper_1201_3588_gb300 import rt
    dev = j_dev.device
    cells_ex = torch.empty_like(cells_dev)
    j_ex = torch.empty_like(j_dev)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("pah_exact_all")  # lets a profiler select this pass
    a.record(stream)
    c_ex, r_ex, _ = g.pah_emission_active(mode=rt.PAH_EXACT, cells=cells_ex, out=j_ex,
                                          stream=stream)
    e.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t_exact = a.elapsed_time(e)
    a.record(stream)
    c_au, r_au, nf = g.pah_emission_active(mode=rt.PAH_AUTO, surrogate=net, tol=tol,
                                           cells=cells_dev, out=j_dev, stream=stream)
    e.record(stream)
    torch.cuda.synchronize()
    t_auto = a.elapsed_time(e)
    o_ex = torch.argsort(c_ex.long())
    o_au = torch.argsort(c_au.long())
    same_cells = bool(torch.equal(c_ex.long()[o_ex], c_au.long()[o_au]))
    rx = r_ex[o_ex].double()
    ra = r_au[o_au].double()
    tot = rx.sum(dim=1).clamp_min(1e-300)
    err = (ra - rx).abs().sum(dim=1) / tot
    return {"active_cells": int(c_ex.shape[0]), "fallback_cells": int(nf),
            "exact_ms": t_exact, "surrogate_auto_ms": t_auto,
            "exact_over_auto": t_exact / max(t_auto, 1e-9),
            "l1_vs_exact_energy_weighted": float((err * tot).sum() / tot.sum()),
            "l1_vs_exact_median": float(err.median()),
            "l1_vs_exact_p90": float(torch.quantile(err.float(), 0.9)),
            "same_cells": same_cells}, r_au.shape[0]


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1201_3588_gb300 import rt, shard

    rank, world, local = dist_env()
    model, desc = build_model(args.workload)
    # the host-core oracle processes are forked before this process touches CUDA
    pool = oracle_pool(model) if rank == 0 and args.cpu_seconds > 0 \
        and not args.cpu_one_thread else None
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n = int(args.packages)
    S, N, B = model.n_species, model.tree.n_leaves, model.n_bins
    L = model.tree.max_level
    stream = torch.cuda.Stream(device=dev)
    g = rt.Grid(model)
    g.emit_star(n * world)
    T_dev = torch.empty((S, N), dtype=torch.float32, device=dev)
    sed_dev = torch.empty((2, model.n_sed_dirs, B), dtype=torch.int64, device=dev)
    cnt_dev = torch.empty((S, N), dtype=torch.int64, device=dev) if world > 1 else None
    first = rank * n
    pah = has_pah(model) and not args.no_pah
    images = args.workload == "disk_images"
    img_dev = prof_dev = None
    if images:
        import numpy as np
        from paper_1201_3588_gb300 import workloads as w
        lam = w.bin_centre_wavelength(model.nu_edges) / w.MICRON
        pob = np.full(B, -1, np.int32)
        pob[int(np.argmin(np.abs(lam - 11.3)))] = 0       # the band
        pob[int(np.argmin(np.abs(lam - 10.0)))] = 1       # the continuum beside it
        inc = math.radians(60.0)
        g.set_images((0.0, math.sin(inc), math.cos(inc)), pob, 256, 256, model.half_size)
        img_dev = torch.empty((2, 256, 256), dtype=torch.float64, device=dev)
        prof_dev = torch.empty(256, dtype=torch.float64, device=dev)
    # the pool launch (blocks per SM, threads, interaction batch, refill period, walk)
    # tuned on prefixes of this grid, before anything is timed
    opts = {}
    if not args.no_tune and not images:
        from paper_1201_3588_gb300 import autotune
        tau = model.recipe.get("tau_v_mid", model.recipe.get("tau_v", 1.0))
        opts = autotune.tune(g, tau, n_probe=min(n, 20_000_000))
    if args.walk != "auto":
        opts["walk"] = WALKS[args.walk]
    net, pah_info = None, {}
    tol = 0.05
    cells_dev = j_dev = None
    pah_state = {"active": 0, "fallback": 0}
    if pah:
        net, pah_info = train_surrogate(g, n, first, stream, dev)
        # rows for the PAH-active cells, at most 8 GiB of them
        max_cells = max(1, min(N, (8 << 30) // (4 * B)))
        cells_dev = torch.empty(max_cells, dtype=torch.int32, device=dev)
        j_dev = torch.empty((max_cells, B), dtype=torch.float32, device=dev)

    def step(k, ev=None):
        g.reset(stream)
        if ev:
            ev[0].record(stream)
        g.transport(n, seed=1000 + k, first_id=first, stream=stream,
                    count_scale=shard.count_scale(world), **opts)
        if ev:
            ev[1].record(stream)
        if world > 1:  # sum the integer counts over ranks (package ranges are disjoint)
            shard.reduce_counts(g, cnt_dev, stream=stream)
        g.temperatures(out=T_dev, stream=stream)
        g.sed(out=sed_dev, stream=stream)
        if pah:
            c, _, nf = g.pah_emission_active(mode=rt.PAH_AUTO, surrogate=net, tol=tol,
                                             cells=cells_dev, out=j_dev, stream=stream)
            pah_state["active"], pah_state["fallback"] = int(c.shape[0]), nf
        if images:
            g.images(out=img_dev, stream=stream)
            g.image_profile(0, 1, 2, out=prof_dev, stream=stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    counters_warm = g.counters()

    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    launches = 0
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select these launches
        t_start.record(stream)
        for k in range(args.steps):
            step(args.warmup + k, kev[k])
            # transport, temperatures, the reset's clearing of PAH rows; the PAH pass
            # (counted from its own sizes)
            launches += 2 + (1 if g.n_pah else 0) + (
                pah_step_launches(pah_state["active"], pah_state["fallback"], g.n_pah)
                if pah else 0) + (4 if images else 0)
        t_end.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.summary()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    kern_s = [a.elapsed_time(b) / 1e3 for a, b in kev]
    c = g.counters()  # last step's counters (each step starts from zero)
    if world > 1:
        t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    value = n * world * args.steps / elapsed

    # roofline of the dominant kernel (the transport launch), per unit of the method's
    # data: crossings x (base id + L child ids + S densities) + absorptions x 16 B
    hbm, src = peaks()
    kmean = sum(kern_s) / len(kern_s)
    bytes_launch = crossing_bytes(c, S, L)
    achieved = bytes_launch / kmean / 1e9
    path = path_walk_runs(opts.get("walk", WALKS[args.walk]), N, S, L,
                          model.tree.n_base ** 3 + 8 * model.tree.n_blocks, images)
    prof = profile_figures(args.workload)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm,
            "traffic": prof["dram_bytes_per_package"] * n if prof else None,
            "peak_source": src,
            "kernel": "k_transport_pool" + (" (peel-off variant)" if images else ""),
            "kernel_ms": 1e3 * kmean,
            "bytes_per_crossing": 4 + 4 * L + 4 * S,
            "algorithmic_bytes_per_launch": bytes_launch,
            "walk": "path" if path else "linked",
            "walk_bytes_per_launch": walk_bytes(c, S, path),
            "walk_frac": walk_bytes(c, S, path) / kmean / 1e9 / hbm}
    if prof:
        roof["warp_lanes_active_per_instruction"] = prof["warp_lanes_active"]
        roof["warp_execution_efficiency"] = prof["warp_lanes_active"] / 32.0
        roof["warp_instructions_per_crossing"] = prof.get("warp_instr_per_crossing")
        roof["profile"] = prof["file"]

    extra = {}
    if pah:
        err, n_rows = surrogate_error(g, net, cells_dev, j_dev, tol, stream)
        pah_info.update(err)
        pah_info["tol"] = tol
        extra["pah"] = pah_info
    if images:
        extra["images"] = {"peel_events": c["peel_events"],
                           "peel_crossings": c["peel_crossings"],
                           "band_minus_continuum_total": float((img_dev[0] - img_dev[1]).sum()),
                           "profile_peak": float(prof_dev.max())}
    if rank == 0 and not args.no_plain and not images:
        extra["plain"] = plain_rates(g, model, int(args.plain_packages), stream,
                                     net if pah else None, cells_dev, j_dev, tol, opts)
    if args.full_run and rank == 0:
        extra["full_run"] = full_run(g, args.workload, stream, net, cells_dev, j_dev, tol, opts)
    params = net.get_params() if pah else None
    n_active = pah_state["active"]
    del T_dev, cells_dev, j_dev
    g.close()
    torch.cuda.empty_cache()
    e2e = e2e_rate(model, n, world, first, args.e2e_steps, net, params, tol,
                   max(1, 2 * n_active), opts) if args.e2e_steps > 0 and not images else None
    if rank == 0:
        cpu_rate, cpu_n, cpu_s, cpu_cores = cpu_oracle_rate(model, n * world, args.cpu_seconds,
                                                            pool=pool)
        if pool is not None:
            pool.close()
            pool.join()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "packages_per_gpu_per_step": n,
                       "packages_full_workload": FULL_PACKAGES.get(args.workload),
                       "leaves": N, "bins": B, "species": S, "levels": L,
                       "reemission": "bjorkman-wood",
                       "walk": walk_label(args.walk, N, S, L) if "walk" not in opts else
                       {1: "linked", 2: "path"}[opts["walk"]] + " (autotuned)",
                       "launch": opts or "defaults",
                       "form": "FP32 packet-pool transport" +
                               (" + BF16 tcgen05 PAH surrogate with exact fallback"
                                if pah else ""),
                       "l2": f"inputs larger than L2: grid + counts "
                             f"{grid_bytes(model, path) / 2**20:.0f} MiB > 129 MiB"},
            "roofline": roof,
            "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cpu_cores,
                             "kind": "oracle",
                             "sample": f"{cpu_n} packages of the same workload (BW mode, "
                                       f"{cpu_cores} processes on disjoint package ranges, "
                                       f"{cpu_s:.1f} s)"},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "per_step": {"crossings": c["crossings"], "absorptions": c["absorptions"],
                         "scatters": c["scatters"], "capped": c["capped"],
                         "errors": c["errors"], "crossings_per_s": c["crossings"] / kmean,
                         "interactions_per_s": (c["absorptions"] + c["scatters"]) / kmean,
                         "warmup_crossings": counters_warm["crossings"],
                         "pah_active_cells": pah_state["active"] if pah else None,
                         "pah_fallback_cells": pah_state["fallback"] if pah else None},
            "oracle_error": ORACLE_ERROR,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Agreement of each result with the FP64 oracle, as the GPU tests establish it
# (tests/test_gpu_*.py; the bound each test asserts).
ORACLE_ERROR = {
    "temperatures": "the same counts inverted by both: max relative difference <= 2e-4 "
                    "(sphere, disk, large disk: 2e-5 measured); replay on a refined box: "
                    "cells with >= 1e4 counts within 0.5 %",
    "absorption_counts": "BW mode, per cell: means of 16 oracle and 64 GPU runs within 4 "
                         "sigma (no more cells beyond than chance allows; refined disk, "
                         "refined box, 4 batch models, 4 rank-scaled shards)",
    "histories": "frozen-mode replay of 300 sampled packages: 0.94 (disk) and 0.91 (large "
                 "disk) identical event by event; every first divergence explained (a "
                 "re-emission table interval, an FP32 face decision, a rounding tie, an "
                 "edge crossing)",
    "pah_exact_emission": "sampled cells vs the oracle's level solution: 2e-3 on bins "
                          "above 1e-6 of the peak; emitted = absorbed to 2e-4",
    "surrogate": "forward vs the oracle's FP64 network: BF16 error (1e-2 per output); "
                 "gradients: cosine > 0.999; accuracy vs exact: the line's pah block",
}


def plain_rates(g, model, n_prefix, stream, net=None, cells_dev=None, j_dev=None, tol=0.05,
                opts=None):
    """The plain form (one thread per package, global tables, per-lane atomics; FP64
    and FP32) against the pool on a package prefix of the same workload; with PAHs,
    also the plain form's exact PAH emission of every active cell against the
    surrogate with fallback, on the pool prefix's tallies."""
    import torch
    from paper_1201_3588_gb300 import rt
    out = {"packages": n_prefix}
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for name, kern in (("pool_f32", rt.KERNEL_POOL), ("plain_f32", rt.KERNEL_PLAIN_F32),
                       ("plain_f64", rt.KERNEL_PLAIN_F64)):
        a, b = ev()
        g.reset(stream)
        a.record(stream)
        g.transport(n_prefix, seed=77, kernel=kern, stream=stream,
                    **(opts if kern == rt.KERNEL_POOL and opts else {}))
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = n_prefix / (a.elapsed_time(b) / 1e3)
    out["pool_over_plain_f32"] = out["pool_f32"] / out["plain_f32"]
    out["pool_over_plain_f64"] = out["pool_f32"] / out["plain_f64"]
    if net is not None:
        g.reset(stream)
        g.transport(n_prefix, seed=77, stream=stream, **(opts or {}))
        times = {}
        for name, mode in (("exact", rt.PAH_EXACT), ("auto", rt.PAH_AUTO)):
            a, b = ev()
            a.record(stream)
            g.pah_emission_active(mode=mode, surrogate=net, tol=tol, cells=cells_dev,
                                  out=j_dev, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            times[name] = a.elapsed_time(b) / 1e3
        # per package of the prefix: plain = plain FP64 transport + exact PAH,
        # chosen = pool FP32 transport + surrogate with fallback
        t_plain = n_prefix / out["plain_f64"] + times["exact"]
        t_chosen = n_prefix / out["pool_f32"] + times["auto"]
        out["pah_exact_s"], out["pah_auto_s"] = times["exact"], times["auto"]
        out["plain_form"] = n_prefix / t_plain
        out["chosen_form"] = n_prefix / t_chosen
        out["chosen_over_plain"] = t_plain / t_chosen
    g.reset(stream)
    torch.cuda.synchronize()
    return out


def full_run(g, workload, stream, net, cells_dev, j_dev, tol, opts=None):
    """One pass of the workload's full package count in launches of 1e9 packages
    (consecutive id ranges), then temperatures, spectrum and PAH emission."""
    import torch
    from paper_1201_3588_gb300 import rt
    n_full = int(FULL_PACKAGES.get(workload, 1e8))
    T = torch.empty((g.S, g.N), dtype=torch.float32, device=j_dev.device if j_dev is not None
                    else torch.device("cuda"))
    torch.cuda.synchronize()
    g.emit_star(n_full)  # the source's package energy for the full count
    g.reset(stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    chunk = 10 ** 9
    torch.cuda.synchronize()
    a.record(stream)
    for f0 in range(0, n_full, chunk):
        g.transport(min(chunk, n_full - f0), seed=4242, first_id=f0, stream=stream,
                    **(opts or {}))
    g.temperatures(out=T, stream=stream)
    g.sed(stream=stream)
    nf = na = 0
    if net is not None:
        c, _, nf = g.pah_emission_active(mode=rt.PAH_AUTO, surrogate=net, tol=tol,
                                         cells=cells_dev, out=j_dev, stream=stream)
        na = int(c.shape[0])
    b.record(stream)
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1e3
    c = g.counters()
    return {"packages": n_full, "seconds": s, "packages_per_s": n_full / s,
            "emitted": c["emitted"], "escaped": c["escaped"], "capped": c["capped"],
            "errors": c["errors"], "crossings": c["crossings"],
            "absorptions": c["absorptions"], "clamped": c["clamped"],
            "pah_active_cells": na, "pah_fallback_cells": nf}


def pinned_model(model):
    """A shallow copy of the model whose large input arrays live in pinned host
    memory (page-locked, so that the library's copies to the device run at full
    speed)."""
    import copy
    import numpy as np
    import torch

    def pin(a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        t = torch.empty(a.shape, dtype=getattr(torch, np.dtype(dtype).name), pin_memory=True)
        v = t.numpy()
        v[...] = a
        return v, t

    m = copy.copy(model)
    m.tree = copy.copy(model.tree)
    keep = []
    m.tree.base, k1 = pin(model.tree.base, np.int32)
    m.tree.child, k2 = pin(model.tree.child, np.int32)
    m.rho, k3 = pin(model.rho, np.float64)
    keep += [k1, k2, k3]
    return m, keep


def e2e_rate(model, n, world, first, steps, net=None, params=None, tol=0.05, max_cells=1,
             opts=None):
    """Same metric through the public API with host buffers: every step creates the
    grid from pinned host arrays (tree, densities, opacities, PAH data), loads the
    surrogate's weights from the host, transports, and reads the temperatures, the
    escaped spectrum and the PAH emission of the active cells back into pinned host
    buffers, then destroys the grid -- all inside the timed region."""
    import numpy as np
    import torch
    from paper_1201_3588_gb300 import rt
    S, N, B = model.n_species, model.tree.n_leaves, model.n_bins
    pm, keep = pinned_model(model)
    T_t = torch.empty((S, N), dtype=torch.float32, pin_memory=True)
    T_host = T_t.numpy()
    sed_host = np.zeros((2, model.n_sed_dirs, B), dtype=np.uint64)
    pah = net is not None
    if pah:
        cells_t = torch.empty(max_cells, dtype=torch.int32, pin_memory=True)
        rows_t = torch.empty((max_cells, B), dtype=torch.float32, pin_memory=True)
        cells_host, rows_host = cells_t.numpy(), rows_t.numpy()
    times, parts, na = [], [], 0
    for k in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = rt.Grid(pm)
        try:
            if pah:
                net.set_params(params)
            g.emit_star(n * world)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g.transport(n, seed=5000 + k, first_id=first, **(opts or {}))
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            g.temperatures(out=T_host)
            g.sed(out=sed_host)
            if pah:
                c, _, _ = g.pah_emission_active(mode=rt.PAH_AUTO, surrogate=net, tol=tol,
                                                cells=cells_host, out=rows_host)
                na = int(c.shape[0])
            torch.cuda.synchronize()
            t3 = time.perf_counter()
        finally:
            g.close()
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        if k > 0:  # the first pass warms the process
            times.append(t4 - t0)
            parts.append((t1 - t0, t2 - t1, t3 - t2, t4 - t3))
    t = model.tree
    h2d = (4 * t.n_base ** 3 + 32 * t.n_blocks + 8 * S * N + 8 * (B + 1) + 24 * S * B
           + (4 * params.size if pah else 0))
    d2h = 4 * S * N + 16 * model.n_sed_dirs * B + 8 + (4 * na * (B + 1) if pah else 0)
    del keep
    return {"value": n * world / (sum(times) / len(times)), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1e3 * sum(times) / len(times),
            "ms_by_part": {name: 1e3 * sum(p[i] for p in parts) / len(parts) for i, name in
                           enumerate(("create_and_load", "transport", "outputs", "destroy"))},
            "host_buffers": "pinned"}


def _oracle_batch_worker(job):
    i, seconds = job
    m, n = _POOL_MODEL[i % len(_POOL_MODEL)]
    return _oracle_prefix(m, 0, n, seconds)


def run_batch(args):
    """Config of many uneven models in one graph-captured persistent launch: a step is
    one replay of (reset, batched transport, every model's temperatures)."""
    global _POOL_MODEL
    from paper_1201_3588_gb300 import workloads as w
    rank, world, local = dist_env()
    models = w.batch_models(n_models=args.batch_models, seed=0, n_bins=100)
    pool = None
    if args.cpu_seconds > 0:  # forked before CUDA; each process follows one model
        import multiprocessing as mp
        _POOL_MODEL = models
        pool = mp.get_context("fork").Pool(host_cores())
    import torch
    from paper_1201_3588_gb300 import autotune, rt
    torch.cuda.set_device(local)
    grids = []
    for m, n in models:
        g = rt.Grid(m)
        g.emit_star(n)
        grids.append(g)
    npk = [n for _, n in models]
    total = sum(npk)
    # one launch configuration for the whole batch, tuned on whole-batch probes
    opts = autotune.tune_batch(grids, [m.recipe["tau_v"] for m, _ in models], npk,
                               fraction=0.02)
    b = rt.Batch(grids, npk, seed=0, **opts)
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        b.run_graph(stream)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        a.record(stream)
        for _ in range(args.steps):
            b.run_graph(stream)
        e.record(stream)
        torch.cuda.synchronize()
    el = a.elapsed_time(e) / 1e3
    c = [g.counters() for g in grids]
    # the batched transport launch alone, for the roofline
    kt = []
    for _ in range(3):
        for g in grids:
            g.reset(stream)
        a.record(stream)
        b.run(reset=False, temperatures=False, stream=stream)
        e.record(stream)
        torch.cuda.synchronize()
        kt.append(a.elapsed_time(e) / 1e3)
    kmean = sum(kt) / len(kt)
    c2 = [g.counters() for g in grids]
    bytes_launch = sum(crossing_bytes(x, m.n_species, m.tree.max_level)
                       for x, (m, _) in zip(c2, models))
    hbm, src = peaks()
    achieved = bytes_launch / kmean / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "peak_source": src,
            "kernel": "k_transport_batch", "kernel_ms": 1e3 * kmean,
            "algorithmic_bytes_per_launch": bytes_launch}
    b.close()
    for g in grids:
        g.close()
    torch.cuda.empty_cache()
    e2e = batch_e2e(models, opts, args.e2e_steps) if args.e2e_steps > 0 else None
    cpu = None
    if pool is not None:
        res = pool.map(_oracle_batch_worker,
                       [(i, args.cpu_seconds) for i in range(host_cores())])
        pool.close()
        pool.join()
        done = sum(r[0] for r in res)
        secs = max(r[1] for r in res)
        cpu = {"value": done / secs, "unit": UNIT, "cores": len(res), "kind": "oracle",
               "sample": f"{done} packages of the batch's first {min(len(res), len(models))} "
                         f"models (one process each, BW mode, {secs:.1f} s)"}
    emitted = sum(x["emitted"] for x in c)
    line = {"metric": METRIC, "value": total * args.steps / el, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batch of {len(models)} uneven sphere/disk models, 100 bins, "
                                   "one graph-captured persistent launch",
                       "packages_per_step": total, "leaves_total": sum(m.tree.n_leaves
                                                                       for m, _ in models),
                       "autotuned": opts},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": (1 + len(models)) * args.steps, "clocks": clk.summary(),
            "per_step": {"crossings": sum(x["crossings"] for x in c),
                         "absorptions": sum(x["absorptions"] for x in c),
                         "emitted": emitted, "errors": sum(x["errors"] for x in c)}}
    print(json.dumps(line), flush=True)


def batch_e2e(models, opts, steps):
    """The batch through the public API from host arrays: every step creates all the
    grids, plans and runs the batched launch, reads every model's temperatures and
    escaped spectrum back to host memory and destroys everything."""
    import numpy as np
    import torch
    from paper_1201_3588_gb300 import rt
    T_host = [np.zeros((m.n_species, m.tree.n_leaves), dtype=np.float32) for m, _ in models]
    npk = [n for _, n in models]
    times = []
    for k in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grids = []
        for m, n in models:
            g = rt.Grid(m)
            g.emit_star(n)
            grids.append(g)
        b = rt.Batch(grids, npk, seed=100 + k, **opts)
        b.run(reset=True, temperatures=True)
        for i, g in enumerate(grids):
            b.temperatures(i, out=T_host[i])
            g.sed()
        b.close()
        for g in grids:
            g.close()
        torch.cuda.synchronize()
        if k > 0:
            times.append(time.perf_counter() - t0)
    h2d = sum(4 * m.tree.n_base ** 3 + 32 * m.tree.n_blocks + 8 * m.n_species * m.tree.n_leaves
              + 8 * (m.n_bins + 1) + 24 * m.n_species * m.n_bins for m, _ in models)
    d2h = sum(4 * m.n_species * m.tree.n_leaves + 16 * m.n_sed_dirs * m.n_bins + 8
              for m, _ in models)
    return {"value": sum(npk) / (sum(times) / len(times)), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1e3 * sum(times) / len(times), "host_buffers": "pageable"}


def peaks_tensor():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (burst)"
    except Exception:
        return 1900.0, "fallback"


def run_surrogate(args):
    """The PAH emission network alone (the large disk's shape: 64 coarse bins + 2
    features -> 3 x 256 SiLU -> 400 bins): a step is one fused tensor-core forward
    pass over `--rows` synthetic feature rows; the line reports its tensor roofline
    (2 sum(in x out) FLOP per row against the bf16 peak) and the time of one training
    step (loss, gradients and Adam on 1024 rows, layer-by-layer tcgen05 GEMMs)."""
    import torch
    from paper_1201_3588_gb300 import rt
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_in, n_h, n_l, n_out = 66, 256, 3, 400
    M = int(args.rows)
    net = rt.MLP(n_in, n_h, n_l, n_out, seed=0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    x = torch.rand((M, n_in), device=dev, generator=gen) * 2.0 - 1.0
    y = torch.empty((M, n_out), device=dev)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        net.forward(x, y, stream=stream)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        a.record(stream)
        for _ in range(args.steps):
            net.forward(x, y, stream=stream)
        e.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    el = a.elapsed_time(e) / 1e3 / args.steps
    flops = 2.0 * (n_in * n_h + (n_l - 1) * n_h * n_h + n_h * n_out) * M
    peak, src = peaks_tensor()
    achieved = flops / el / 1e12
    xb = x[:1024].contiguous()
    tb = torch.rand((1024, n_out), device=dev, generator=gen)
    for _ in range(3):
        net.loss_grad(xb, tb, want_loss=False, stream=stream)
        net.adam_step(1e-4, stream=stream)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(50):
        net.loss_grad(xb, tb, want_loss=False, stream=stream)
        net.adam_step(1e-4, stream=stream)
    e.record(stream)
    torch.cuda.synchronize()
    train_ms = a.elapsed_time(e) / 50
    line = {"metric": "surrogate forward rows/s (PAH emission network, fused tcgen05)",
            "value": M / el, "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"{M} feature rows, network {n_in} -> {n_l} x {n_h} SiLU "
                                   f"-> {n_out}", "rows": M},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": src, "kernel": "k_mlp_forward_tc",
                         "flop_per_row": flops / M},
            "training_step_ms_1024_rows": train_ms,
            "gpu_launches": args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "surrogate":
        run_surrogate(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
