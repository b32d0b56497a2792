"""Bjorkman-Wood transport on refined grids, GPU against the FP64 oracle.

* Per-cell absorption counts of the BW mode on two refined grids: a disk (32^3 base
  cubes, two levels of subcubes near the rim and midplane, 100 bins) and a dusty box
  (16^3 base cubes refined twice around the star, so that cells of all three levels
  absorb). Both exercise the walk the benchmark times: face links, descents into
  finer neighbours, eps/V per level. The oracle makes 16 independent BW runs (one
  host process each), the GPU 64, all of 1e5 packages. Each cell's mean count must
  lie within 4 sigma of the GPU's, sigma from the spread of the runs. With up to
  ~10^4 cells compared a few may lie beyond 4 sigma by chance: the test bounds their
  number by the chance rate, and bounds the mean square z of well-measured cells (a
  small bias common to many cells raises it).
* Temperatures under replay: the frozen mode on a small refined box, GPU and oracle
  following the same packages; cells with >= 1e4 absorptions agree within 0.5 %.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import rt, workloads as w
from _helpers import assert_runs_agree, frozen_field

pytestmark = pytest.mark.gpu

N_RUN = 100_000          # packages per run (eps = L / N_RUN in every run)
ORACLE_RUNS = 16
GPU_RUNS = 64


def _disk():
    return w.disk_model(n_base=32, max_level=2, n_bins=100, tau_v_mid=30.0)


def _dusty_box():
    nu = w.frequency_edges(100)
    return w.uniform_box_model(16, 100, 5.0, w.two_species(nu), max_level=2,
                               refine=w.sphere_refine_fn(16, 0.3))


MODELS = {"disk": _disk, "box": _dusty_box}


def _oracle_bw_run(job):
    name, seed = job
    m = MODELS[name]()
    t = oracle.transport(m, N_RUN, seed=seed, n_total=N_RUN, mode=oracle.MODE_BW)
    return t.count.astype(np.float64), t.sed[0, 0].astype(np.float64), t.emitted, t.escaped


def _pool(n):
    # spawned processes: this process may already hold a CUDA context
    return mp.get_context("spawn").Pool(n)


def _procs():
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return max(1, min(ORACLE_RUNS, cores))


@pytest.mark.parametrize("name", ["disk", "box"])
def test_bw_counts_on_refined_grids_match_oracle(name):
    model = MODELS[name]()
    assert model.tree.max_level == 2 and (model.tree.leaf_level == 1).any()
    with _pool(_procs()) as pool:
        res = pool.map(_oracle_bw_run, [(name, 7000 + k) for k in range(ORACLE_RUNS)])
    o_cnt = np.array([r[0] for r in res])
    o_sed = np.array([r[1] for r in res])
    assert all(r[2] == N_RUN == r[3] for r in res)
    g_cnt, g_sed = [], []
    with rt.Grid(model) as g:
        g.emit_star(N_RUN)
        for k in range(GPU_RUNS):
            g.reset()
            g.transport(N_RUN, seed=100 + k, mode=rt.REEMIT_BW)
            c = g.counters()
            assert c["emitted"] == N_RUN == c["escaped"] and c["errors"] == 0
            g_cnt.append(g.counts().astype(np.float64))
            g_sed.append(g.sed()[0][0, 0].astype(np.float64))
    g_cnt, g_sed = np.array(g_cnt), np.array(g_sed)
    assert_runs_agree(o_cnt, g_cnt, f"{name} counts")
    assert_runs_agree(o_sed, g_sed, f"{name} escaped spectrum")
    if name == "box":  # cells of every refinement level absorbed and were compared
        lev = model.tree.leaf_level
        mean = g_cnt.mean(axis=0)
        for L in range(3):
            assert (mean[:, lev == L] > 5).sum() >= 10, L


def _box():
    # 2^3 base cubes, all split, the eight around the star split again: 120 cells of
    # levels 1 and 2; a grey absorber-scatterer (albedo 0.3, g 0.5) thick enough that
    # packages are absorbed ~9 times each
    sp = [w.grey_species(64, 0.7, 0.3, 0.5)]
    return w.uniform_box_model(2, 64, 4.0, sp, max_level=2, refine=w.sphere_refine_fn(2, 0.45))


def _oracle_frozen_shard(job):
    first, n, n_total, seed = job
    m = _box()
    Tf = frozen_field(m, T0=60.0, r0_frac=0.2).astype(np.float64)
    t = oracle.transport(m, n, seed=seed, first_id=first, n_total=n_total,
                         mode=oracle.MODE_FROZEN, T_frozen=Tf)
    return t.count.astype(np.int64)


def test_temperatures_under_replay_on_refined_box():
    model = _box()
    assert model.tree.max_level == 2
    N = 300_000
    seed = 31
    Tf = frozen_field(model, T0=60.0, r0_frac=0.2)
    with rt.Grid(model) as g:
        g.emit_star(N)
        g.set_frozen_temperatures(Tf)
        g.transport(N, seed=seed, mode=rt.REEMIT_FROZEN)
        c = g.counters()
        cnt_g = g.counts().astype(np.int64)
        T_g = g.temperatures().astype(np.float64)
        _, eps = g.sed()
    assert c["emitted"] == N == c["escaped"] and c["errors"] == 0
    # the oracle follows the same packages in disjoint id ranges (the frozen mode
    # shards exactly), then inverts its own counts
    k = _procs()
    step = (N + k - 1) // k
    jobs = [(f, min(step, N - f), N, seed) for f in range(0, N, step)]
    with _pool(k) as pool:
        cnt_o = sum(pool.map(_oracle_frozen_shard, jobs))
    T_o = oracle.temperatures(model, cnt_o.astype(np.uint64), eps)
    big = (cnt_g >= 10_000) & (cnt_o >= 10_000)
    print("cells with >= 1e4 counts:", int(big.sum()), "of", cnt_g.size,
          "max |T_gpu/T_oracle - 1|:", float(np.abs(T_g[big] / T_o[big] - 1).max()),
          "max count difference:", float(np.abs(cnt_g[big] / cnt_o[big] - 1).max()))
    assert big.sum() >= 0.5 * cnt_g.size
    np.testing.assert_allclose(T_g[big], T_o[big], rtol=5e-3)
