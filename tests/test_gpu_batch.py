"""Batched persistent launch of uneven models: in the frozen-temperature mode every
package's history is a pure function of (seed, id), so the batch must reproduce the
per-model launches and the oracle's counts of the same packages; in the BW mode its
per-cell counts agree with independent oracle runs in distribution; graph replays
must reproduce the direct run; the autotuner returns a valid configuration and
caches it."""
import json

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import autotune, rt, workloads as w
from _helpers import assert_runs_agree, frozen_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def models():
    return w.batch_models(n_models=8, seed=3, n_bins=40, sizes=(16, 24, 32))


def _grids(models, frozen=True):
    grids = []
    for m, n in models:
        g = rt.Grid(m)
        g.emit_star(n)
        if frozen:
            g.set_frozen_temperatures(frozen_field(m))
        grids.append(g)
    return grids


def test_batch_equals_per_model_launches(models):
    npk = [min(n, 300_000) for _, n in models]
    grids = _grids(models)
    b = rt.Batch(grids, npk, seed=11, mode=rt.REEMIT_FROZEN)
    b.run(reset=True, temperatures=False)
    got = [(g.counts().astype(np.int64), g.sed()[0].astype(np.int64), g.counters())
           for g in grids]
    for m, g in enumerate(grids):
        g.reset()
        g.transport(npk[m], seed=11 + m, mode=rt.REEMIT_FROZEN)
        cnt, sed, c = g.counts().astype(np.int64), g.sed()[0].astype(np.int64), g.counters()
        gc, gs, gcn = got[m]
        assert gcn["emitted"] == c["emitted"] == npk[m]
        assert gcn["escaped"] + gcn["capped"] == npk[m] and gcn["errors"] == 0
        assert np.abs(gc - cnt).sum() <= 1e-3 * cnt.sum() + 2
        assert np.abs(gs - sed).sum() <= 1e-3 * npk[m] + 2
    b.close()
    for g in grids:
        g.close()


def test_graph_replay_matches_direct_run(models):
    npk = [min(n, 200_000) for _, n in models]
    grids = _grids(models)
    b = rt.Batch(grids, npk, seed=5, mode=rt.REEMIT_FROZEN)
    b.run(reset=True, temperatures=True)
    ref = [(g.counts().copy(), b.temperatures(i)) for i, g in enumerate(grids)]
    for _ in range(2):
        b.run_graph()
        for i, g in enumerate(grids):
            cnt = g.counts()
            T = b.temperatures(i)
            assert np.abs(cnt.astype(np.int64) - ref[i][0].astype(np.int64)).sum() <= \
                1e-3 * ref[i][0].sum() + 2
            np.testing.assert_allclose(T, g.temperatures(), rtol=1e-6)
    b.close()
    for g in grids:
        g.close()


def test_autotuner_picks_and_caches(tmp_path, models):
    m, n = models[0]
    with rt.Grid(m) as g:
        g.emit_star(10 ** 6)
        path = str(tmp_path / "tune.json")
        opts = autotune.tune(g, m.recipe["tau_v"], n_probe=200_000, cache=path)
        assert set(opts) == {"blocks_per_sm", "threads", "interaction_batch", "refill_period",
                             "walk"}
        db = json.load(open(path))
        assert len(db) == 1 and list(db.values())[0]["opts"] == opts
        assert autotune.tune(g, m.recipe["tau_v"], cache=path) == opts
        g.transport(10 ** 6, **opts)
        assert g.counters()["emitted"] == 10 ** 6


def _oracle_models():
    """Four uneven models sharing 40 bins and two species: spheres and disks of
    different grids, refinement and optical depth."""
    nu = w.frequency_edges(40)
    sp = w.two_species(nu)
    return [w.sphere_model(n_base=8, n_bins=40, tau_v=1.0, species=sp),
            w.disk_model(n_base=16, max_level=1, n_bins=40, tau_v_mid=10.0, species=sp),
            w.uniform_box_model(8, 40, 2.0, sp, max_level=2, refine=w.sphere_refine_fn(8, 0.3)),
            w.disk_model(n_base=16, max_level=2, n_bins=40, tau_v_mid=3.0, species=sp,
                         perturbed=True)]


ORACLE_NPK = [20_000, 30_000, 10_000, 25_000]


def _oracle_job(job):
    m_idx, seed, mode, frozen = job
    m = _oracle_models()[m_idx]
    kw = {}
    if frozen:
        kw["T_frozen"] = frozen_field(m).astype(np.float64)
    t = oracle.transport(m, ORACLE_NPK[m_idx], seed=seed, n_total=ORACLE_NPK[m_idx], mode=mode,
                         **kw)
    return t.count.astype(np.float64), t.sed[0, 0].astype(np.float64)


def _spawn_pool(n):
    import multiprocessing as mp
    import os
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(max(1, min(n, cores)))


def test_batch_frozen_replay_matches_oracle():
    """Frozen mode: each model's packages, followed in the one batched launch, give the
    oracle's per-cell counts and spectrum of the same packages."""
    models = _oracle_models()
    grids = []
    for m, n in zip(models, ORACLE_NPK):
        g = rt.Grid(m)
        g.emit_star(n)
        g.set_frozen_temperatures(frozen_field(m))
        grids.append(g)
    seed = 21
    b = rt.Batch(grids, ORACLE_NPK, seed=seed, mode=rt.REEMIT_FROZEN)
    b.run(reset=True, temperatures=False)
    with _spawn_pool(len(models)) as pool:
        res = pool.map(_oracle_job, [(i, seed + i, oracle.MODE_FROZEN, True)
                                     for i in range(len(models))])
    for i, g in enumerate(grids):
        c = g.counters()
        assert c["emitted"] == ORACLE_NPK[i] == c["escaped"] and c["errors"] == 0
        cnt = g.counts().astype(np.int64)
        sed = g.sed()[0][0, 0].astype(np.int64)
        ocnt, osed = res[i][0].astype(np.int64), res[i][1].astype(np.int64)
        diff = np.abs(cnt - ocnt)
        print(f"model {i}: counts {ocnt.sum()}, differing {diff.sum()}")
        assert diff.sum() <= 0.03 * ocnt.sum() + 5
        assert (diff <= 4 * np.sqrt(cnt + ocnt) + 1).all()
        assert np.abs(sed - osed).sum() <= 0.03 * ORACLE_NPK[i] + 5
    b.close()
    for g in grids:
        g.close()


def test_batch_bw_statistics_match_oracle():
    """BW mode: per-cell counts and escaped spectra of every model over 48 batched
    launches agree with 12 independent oracle runs within 4 sigma."""
    models = _oracle_models()
    grids = []
    for m, n in zip(models, ORACLE_NPK):
        g = rt.Grid(m)
        g.emit_star(n)
        grids.append(g)
    runs = [[] for _ in models]
    for k in range(48):
        b = rt.Batch(grids, ORACLE_NPK, seed=1000 + 10 * k, mode=rt.REEMIT_BW)
        b.run(reset=True, temperatures=False)
        for i, g in enumerate(grids):
            c = g.counters()
            assert c["emitted"] == ORACLE_NPK[i] == c["escaped"] and c["errors"] == 0
            runs[i].append((g.counts().astype(np.float64), g.sed()[0][0, 0].astype(np.float64)))
        b.close()
    jobs = [(i, 50_000 + 100 * k + i, oracle.MODE_BW, False)
            for k in range(12) for i in range(len(models))]
    with _spawn_pool(16) as pool:
        res = pool.map(_oracle_job, jobs)
    for i in range(len(models)):
        o = [r for (j, r) in zip(jobs, res) if j[0] == i]
        o_cnt = np.array([r[0] for r in o])
        o_sed = np.array([r[1] for r in o])
        g_cnt = np.array([r[0] for r in runs[i]])
        g_sed = np.array([r[1] for r in runs[i]])
        assert_runs_agree(o_cnt, g_cnt, f"model {i} counts")
        assert_runs_agree(o_sed, g_sed, f"model {i} escaped spectrum")
    for g in grids:
        g.close()


def test_batch_autotuner_covers_the_batch(tmp_path, models):
    """The batch tuner times whole-batch probes over the block shapes too, caches its
    choice per batch class, and the choice runs the batch."""
    grids = _grids(models, frozen=False)
    npk = [min(n, 400_000) for _, n in models]
    path = str(tmp_path / "tune.json")
    taus = [m.recipe["tau_v"] for m, _ in models]
    opts = autotune.tune_batch(grids, taus, npk, fraction=0.05, cache=path)
    assert set(opts) == set(autotune.BATCH_CANDIDATES) and opts["threads"] in (128, 256)
    assert autotune.tune_batch(grids, taus, npk, cache=path) == opts
    b = rt.Batch(grids, npk, seed=1, **opts)
    b.run(reset=True, temperatures=False)
    for g, n in zip(grids, npk):
        c = g.counters()
        assert c["emitted"] == n == c["escaped"] + c["capped"] and c["errors"] == 0
    b.close()
    for g in grids:
        g.close()

