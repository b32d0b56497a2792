#!/usr/bin/env python
"""Throughput of the photon-package transport on GB300: packages/s.

A step is one pass of the whole path over one batch: zero the counts, transport
the batch of packages (Bjorkman-Wood re-emission, persistent packet-pool kernel,
FP32), invert the counts into per-cell temperatures (FP64) and gather the escaped
spectrum. The workload is the flared proto-planetary disk (128^3 base cubes, two
levels of 2x2x2 refinement at the inner rim and midplane, 200 frequency bins,
midplane V-band optical depth 1e3, 1e8 packages per GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
    p.add_argument("--packages", type=float, default=1e8, help="packages per GPU per step")
    p.add_argument("--workload", choices=["disk", "sphere", "batch", "disk_pah", "disk_images",
                                          "large_disk"],
                   default="disk")
    p.add_argument("--batch-models", type=int, default=256)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--plain-packages", type=float, default=1e7)
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--cpu-one-thread", action="store_true",
                   help="time the oracle on one host thread instead of one process per core")
    return p.parse_args()


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


# DRAM traffic of the pool kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum over a 2e6-package launch on the disk, scaled per package),
# valid only for that workload and the kernel source it was measured on (the hash
# covers the code of the sources with comments and blank lines removed).
TRAFFIC = {"sources": ("paper_1201_3588_gb300/csrc/rt_transport.cu",
                       "paper_1201_3588_gb300/csrc/rt_internal.h"),
           "sha256": "d50f24fa339fca45dfc7626db83c4a47413a6771b8e1acd8f0d2cc88bb82dfe8",
           "dram_bytes_per_package": 1035.3}


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


def traffic_per_launch(n_packages):
    if not TRAFFIC["sha256"] or not TRAFFIC["dram_bytes_per_package"]:
        return None
    if source_code_hash(TRAFFIC["sources"]) != TRAFFIC["sha256"]:
        return None
    return TRAFFIC["dram_bytes_per_package"] * n_packages


def walk_bytes(c, S):
    """Algorithmic bytes of one transport launch (per unit of work):
    every cell entered reads its face link (4 B) and S densities (4 B each), every
    descent into a finer neighbour one child id (4 B); every absorption is one 8-byte
    read-modify-write of a count (16 B). Peel-off: every cell a sight line crosses
    reads the same link and densities, every peeled event adds into an FP64 pixel
    (16 B)."""
    entered = c["crossings"] + c["absorptions"] + c["scatters"] + c["capped"]
    return (entered * (4 + 4 * S) + 4 * c["levels"] + 16 * c["absorptions"]
            + c.get("peel_crossings", 0) * (4 + 4 * S) + 16 * c.get("peel_events", 0))


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1201_3588_gb300 import rt

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
    stream = torch.cuda.Stream(device=dev)
    g = rt.Grid(model)
    g.emit_star(n * world)
    T_dev = torch.empty((S, N), dtype=torch.float32, device=dev)
    sed_dev = torch.empty((2, model.n_sed_dirs, B), dtype=torch.int64, device=dev)
    cnt_dev = torch.empty((S, N), dtype=torch.int64, device=dev) if world > 1 else None
    first = rank * n
    pah = args.workload in ("disk_pah", "large_disk")
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
    net, pah_info = None, {}
    # cells per PAH-emission call: the output buffer held at <= 16 GiB
    pah_chunk = max(1, min(N, (16 << 30) // (4 * B)))
    j_dev = torch.empty((min(pah_chunk, N), B), dtype=torch.float32, device=dev) if pah else None

    def pah_emission(mode=rt.PAH_AUTO, count=False):
        nf = 0
        for c0 in range(0, N, pah_chunk):
            nc = min(pah_chunk, N - c0)
            _, f = g.pah_emission(first=c0, n=nc, mode=mode, surrogate=net, tol=0.05,
                                  out=j_dev[:nc], stream=stream, count_fallback=count)
            nf += f
        return nf

    if pah:  # train the surrogate on the exact solutions of a first (untimed) pass
        from paper_1201_3588_gb300 import surrogate
        g.transport(n, seed=999, first_id=first, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, Y = surrogate.training_pairs(g)
        keep = torch.randperm(X.shape[0], device=dev)[:1_000_000]
        X, Y = X[keep].contiguous(), Y[keep].contiguous()
        net = rt.MLP(X.shape[1], surrogate.N_HIDDEN, surrogate.N_LAYERS, B, seed=0)
        hist = surrogate.train(net, X, Y, epochs=8)
        xp = X[:, -2]
        net.set_range(float(xp.min()) - 0.25, float(xp.max()) + 0.25)
        torch.cuda.synchronize()
        pah_info = {"training_pairs": int(X.shape[0]), "train_s": time.perf_counter() - t0,
                    "train_loss_first_last": [hist[0], hist[-1]]}
        del X, Y
        g.reset(stream)

    def step(k, ev=None):
        g.reset(stream)
        if ev:
            ev[0].record(stream)
        g.transport(n, seed=1000 + k, first_id=first, stream=stream)
        if ev:
            ev[1].record(stream)
        if world > 1:  # sum the integer counts over ranks (package ranges are disjoint)
            g.counts(out=cnt_dev, stream=stream)
            with torch.cuda.stream(stream):
                dist.all_reduce(cnt_dev)
            g.set_counts(cnt_dev, stream=stream)
        g.temperatures(out=T_dev, stream=stream)
        g.sed(out=sed_dev, stream=stream)
        if pah:
            pah_emission()
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
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for k in range(args.steps):
            step(args.warmup + k, kev[k])
        t_end.record(stream)
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

    # roofline of the dominant kernel (the transport launch)
    hbm, src = peaks()
    kmean = sum(kern_s) / len(kern_s)
    bytes_launch = walk_bytes(c, S)
    achieved = bytes_launch / kmean / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm,
            "traffic": traffic_per_launch(n) if args.workload == "disk" else None,
            "peak_source": src,
            "kernel": "k_transport_pool" + (" (peel-off variant)" if images else ""),
            "kernel_ms": 1e3 * kmean,
            "algorithmic_bytes_per_launch": bytes_launch}

    extra = {}
    if pah:
        torch.cuda.synchronize()
        pah_info["fallback_cells_last_step"] = pah_emission(count=True)
        pah_info["pah_cells"] = int((torch.from_numpy(g.pah_absorbed().sum(axis=(0, 2)).astype("int64")) > 0).sum())
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pah_emission(mode=rt.PAH_EXACT)
        e.record(stream)
        torch.cuda.synchronize()
        pah_info["exact_pah_ms"] = a.elapsed_time(e)
        a.record(stream)
        pah_emission()
        e.record(stream)
        torch.cuda.synchronize()
        pah_info["surrogate_auto_pah_ms"] = a.elapsed_time(e)
        extra["pah"] = pah_info
    if images:
        extra["images"] = {"peel_events": c["peel_events"],
                           "peel_crossings": c["peel_crossings"],
                           "band_minus_continuum_total": float((img_dev[0] - img_dev[1]).sum()),
                           "profile_peak": float(prof_dev.max())}
    if rank == 0 and not args.no_plain and not images:
        extra["plain"] = plain_rates(g, model, int(args.plain_packages), stream, c, n)
    e2e = e2e_rate(model, n, world, first, args.e2e_steps) \
        if args.e2e_steps > 0 and not pah and not images else None
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
            "config": {"workload": desc, "packages_per_gpu_per_step": n, "leaves": N,
                       "bins": B, "species": S, "reemission": "bjorkman-wood",
                       "kernel": "persistent packet pool",
                       "l2": f"inputs larger than L2: grid + counts "
                             f"{(4 * N * S + N + 8 * N * S) / 2**20:.0f} MiB > 129 MiB"},
            "roofline": roof,
            "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cpu_cores,
                             "kind": "oracle",
                             "sample": f"{cpu_n} packages of the same workload (BW mode, "
                                       f"{cpu_cores} processes on disjoint package ranges, "
                                       f"{cpu_s:.1f} s)"},
            "e2e": e2e,
            "gpu_launches": (2 + (pah_launches(N, pah_chunk) if pah else 0)
                             + (4 if images else 0)) * args.steps,
            "clocks": clocks,
            "per_step": {"crossings": c["crossings"], "absorptions": c["absorptions"],
                         "scatters": c["scatters"], "capped": c["capped"],
                         "errors": c["errors"], "crossings_per_s": c["crossings"] / kmean,
                         "warmup_crossings": counters_warm["crossings"]},
            **extra,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


def pah_launches(N, chunk, n_pah=2):
    """Kernels of one surrogate pass over N cells, per call (chunk of cells): the
    compaction of PAH-active cells; per batch of at most 2^20 of them (one batch on
    these disks) and per PAH the features, the fused network and the check, per PAH
    the add, and the compaction of failed cells; then their exact solution."""
    chunks = (N + chunk - 1) // chunk
    return chunks * (1 + (3 * n_pah + n_pah + 1) + 1)


def plain_rates(g, model, n_prefix, stream, c_pool, n_full):
    """The plain forms (one thread per package, global tables, per-lane atomics) on a
    package prefix of the same workload, FP32 and FP64, against the pool on the same
    prefix."""
    import torch
    from paper_1201_3588_gb300 import rt
    out = {"packages": n_prefix}
    for name, kern in (("pool_f32", rt.KERNEL_POOL), ("plain_f32", rt.KERNEL_PLAIN_F32),
                       ("plain_f64", rt.KERNEL_PLAIN_F64)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        g.reset(stream)
        a.record(stream)
        g.transport(n_prefix, seed=77, kernel=kern, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        s = a.elapsed_time(b) / 1e3
        out[name] = n_prefix / s
    out["pool_over_plain_f32"] = out["pool_f32"] / out["plain_f32"]
    out["pool_over_plain_f64"] = out["pool_f32"] / out["plain_f64"]
    return out


def e2e_rate(model, n, world, first, steps):
    """Same metric through the public API with host buffers: create the grid from
    host arrays, set dust and source, transport, temperatures and spectrum back to
    host, destroy -- all inside the timed region."""
    import numpy as np
    import torch
    from paper_1201_3588_gb300 import rt
    S, N, B = model.n_species, model.tree.n_leaves, model.n_bins
    T_host = np.zeros((S, N), dtype=np.float32)
    times = []
    for k in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with rt.Grid(model) as g:
            g.emit_star(n * world)
            g.transport(n, seed=5000 + k, first_id=first)
            g.temperatures(out=T_host)
            sed, eps = g.sed()
        torch.cuda.synchronize()
        if k > 0:  # the first pass warms the process
            times.append(time.perf_counter() - t0)
    t = model.tree
    h2d = 4 * t.n_base ** 3 + 32 * t.n_blocks + 4 * S * N + N + 8 * (B + 1) + 24 * S * B
    d2h = 4 * S * N + 16 * model.n_sed_dirs * B + 8 * S * 1024 + 8
    return {"value": n * world / (sum(times) / len(times)), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1e3 * sum(times) / len(times)}


def run_batch(args):
    """Config of many uneven models in one graph-captured persistent launch: a step is
    one replay of (reset, batched transport, every model's temperatures)."""
    import torch
    from paper_1201_3588_gb300 import autotune, rt, workloads as w
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    models = w.batch_models(n_models=args.batch_models, seed=0, n_bins=100)
    grids = []
    for m, n in models:
        g = rt.Grid(m)
        g.emit_star(n)
        grids.append(g)
    npk = [n for _, n in models]
    total = sum(npk)
    # tune on the largest model's class
    big = max(range(len(models)), key=lambda i: grids[i].N)
    opts = autotune.tune(grids[big], models[big][0].recipe["tau_v"], n_probe=1_000_000)
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
    emitted = sum(x["emitted"] for x in c)
    line = {"metric": METRIC, "value": total * args.steps / el, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batch of {len(models)} uneven sphere/disk models, 100 bins, "
                                   "one graph-captured persistent launch",
                       "packages_per_step": total, "leaves_total": sum(g.N for g in grids),
                       "autotuned": opts},
            "gpu_launches": (1 + len(grids)) * args.steps, "clocks": clk.summary(),
            "check": {"emitted_last_step": emitted,
                      "errors": sum(x["errors"] for x in c)}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
