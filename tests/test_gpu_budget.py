"""The transport's time budget: every warp of the persistent pool compares the device
clock with the launch's budget between steps and returns once it is spent, setting
the status word. The next synchronising call reports RT_ERR_TIMEOUT (partial
results), and the handle and the CUDA context stay usable: after a reset the same
grid transports again to the full count. The kernel ends by itself; nothing hangs
or faults."""
import pytest

from paper_1201_3588_gb300 import rt, workloads as w

pytestmark = pytest.mark.gpu


def test_transport_stops_at_its_budget_and_the_grid_recovers():
    m = w.disk_model(n_base=64, max_level=1, n_bins=100)
    N = 5 * 10 ** 7                          # far more than 2 ms of work
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.transport(N, seed=1, budget_s=0.002)
        with pytest.raises(rt.RTError) as err:
            g.counters()
        assert err.value.code == 4           # RT_ERR_TIMEOUT
        g.reset()
        g.transport(100_000, seed=2)
        c = g.counters()
        assert c["emitted"] == 100_000 == c["escaped"]
        assert c["errors"] == 0 and c["capped"] == 0


def test_batch_stops_at_its_budget():
    models = w.batch_models(n_models=4, seed=0, n_bins=50)
    grids = [rt.Grid(m) for m, _ in models]
    try:
        for (m, n), g in zip(models, grids):
            g.emit_star(10 ** 7)
        b = rt.Batch(grids, [10 ** 7] * len(grids), seed=0, budget_s=0.001)
        b.run()
        timed_out = 0
        for g in grids:
            try:
                g.counters()
            except rt.RTError as e:
                assert e.code == 4
                timed_out += 1
        assert timed_out >= 1
        b.close()
    finally:
        for g in grids:
            g.close()
