"""The multi-rank path through the library.

* Two ranks (processes with a gloo process group, both on cuda:0, their kernels
  independent) each transport their own package range; the library's counts go
  through shard.reduce_counts (rt_counts, all_reduce, rt_set_counts) and the
  spectra through shard.reduce_spectrum. In the frozen mode the summed counts, the
  spectrum and the temperatures from the summed counts equal one process following
  all packages, bit for bit.
* Bjorkman-Wood with rank-local counts: W shards, each from zeroed counts, summed.
  Without a scale every shard re-emits as if its cells held a W-th of their energy:
  the escaped spectrum is far from the oracle's unsharded BW runs. With the
  temperature index scaled by W (count_scale) the per-cell counts agree within 4
  sigma and the spectrum's deviation falls to a small fraction; what remains comes
  from the spread of a cell's counts over the shards (T(n) is not linear in n) and
  shrinks as the counts per cell and shard grow."""
import multiprocessing
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import rt, shard, workloads as w
from _helpers import assert_runs_agree, frozen_field, runs_z

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, n_per, out_dir):
    import torch.distributed as dist
    here = os.path.dirname(os.path.abspath(__file__))
    for p in (os.path.dirname(here), here):
        if p not in sys.path:
            sys.path.insert(0, p)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    m = w.sphere_model()
    Tf = frozen_field(m)
    first, n = shard.package_range(rank, world, n_per)
    with rt.Grid(m) as g:
        g.emit_star(shard.total_packages(world, n_per))
        g.set_frozen_temperatures(Tf)
        g.transport(n, seed=9, first_id=first, mode=rt.REEMIT_FROZEN)
        cnt = torch.zeros((m.n_species, m.tree.n_leaves), dtype=torch.int64)
        sed = torch.zeros((2, m.n_sed_dirs, m.n_bins), dtype=torch.int64)
        shard.reduce_counts(g, cnt)
        shard.reduce_spectrum(g, sed)
        T = g.temperatures()
        if rank == 0:
            np.savez(os.path.join(out_dir, "ranks.npz"), cnt=cnt.numpy(), sed=sed.numpy(), T=T)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_through_the_library_equal_one_process(tmp_path):
    import torch.multiprocessing as tmp
    world, n_per = 2, 200_000
    tmp.start_processes(_rank, args=(world, _free_port(), n_per, str(tmp_path)), nprocs=world,
                        start_method="spawn", join=True)
    got = np.load(tmp_path / "ranks.npz")
    m = w.sphere_model()
    with rt.Grid(m) as g:
        g.emit_star(world * n_per)
        g.set_frozen_temperatures(frozen_field(m))
        g.transport(world * n_per, seed=9, mode=rt.REEMIT_FROZEN)
        ref_cnt, (ref_sed, _), ref_T = g.counts(), g.sed(), g.temperatures()
    assert np.array_equal(got["cnt"], ref_cnt.astype(np.int64))
    assert np.array_equal(got["sed"], ref_sed.astype(np.int64))
    assert np.array_equal(got["T"], ref_T)


N_BW = 400_000


def _sphere():
    return w.sphere_model(n_base=8, n_bins=64)


def _oracle_bw(seed):
    t = oracle.transport(_sphere(), N_BW, seed=seed, n_total=N_BW, mode=oracle.MODE_BW)
    return t.count.astype(np.float64), t.sed[0, 0].astype(np.float64)


def test_rank_scaled_bw_index_matches_the_unsharded_oracle():
    world, reps = 4, 32
    n = N_BW // world
    ctx = multiprocessing.get_context("spawn")
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    with ctx.Pool(max(1, min(16, cores))) as pool:
        res = pool.map(_oracle_bw, [9000 + k for k in range(16)])
    o_cnt = np.array([r[0] for r in res])
    o_sed = np.array([r[1] for r in res])
    runs = {1: ([], []), world: ([], [])}
    with rt.Grid(_sphere()) as g:
        g.emit_star(N_BW)
        for rep in range(reps):
            for scale in runs:
                cnt, sed = 0.0, 0.0
                for r in range(world):
                    g.reset()
                    first, _ = shard.package_range(r, world, n)
                    g.transport(n, seed=500 + rep, first_id=first, mode=rt.REEMIT_BW,
                                count_scale=scale)
                    cnt = cnt + g.counts().astype(np.float64)
                    sed = sed + g.sed()[0][0, 0].astype(np.float64)
                runs[scale][0].append(cnt)
                runs[scale][1].append(sed)
    print("absorptions per (cell, species) and run:", float(o_cnt.mean(axis=0).mean()))
    assert_runs_agree(o_cnt, np.array(runs[world][0]), "scaled shards, counts")
    dev = {}
    for scale in runs:
        g_sed = np.array(runs[scale][1])
        z, ok = runs_z(o_sed, g_sed)
        dev[scale] = float(np.abs(g_sed.mean(axis=0) - o_sed.mean(axis=0)).sum()
                           / o_sed.mean(axis=0).sum())
        print(f"count_scale {scale}: escaped spectrum mean z^2 {float((z[ok] ** 2).mean()):.2f}, "
              f"relative L1 deviation {dev[scale]:.4f}")
        if scale == 1:
            assert float((z[ok] ** 2).mean()) > 4.0
    assert dev[world] < 0.25 * dev[1], dev
