"""Batched persistent launch of uneven models: in the frozen-temperature mode every
package's history is a pure function of (seed, id), so the batch must reproduce the
per-model launches; graph replays must reproduce the direct run; the autotuner
returns a valid configuration and caches it."""
import json

import numpy as np
import pytest

from paper_1201_3588_gb300 import autotune, rt, workloads as w
from _helpers import frozen_field

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
        assert set(opts) == {"blocks_per_sm", "interaction_batch", "refill_period"}
        db = json.load(open(path))
        assert len(db) == 1 and list(db.values())[0]["opts"] == opts
        assert autotune.tune(g, m.recipe["tau_v"], cache=path) == opts
        g.transport(10 ** 6, **opts)
        assert g.counters()["emitted"] == 10 ** 6
