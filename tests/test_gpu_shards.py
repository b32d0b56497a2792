"""Sharding by package range on one GPU: K sequential shards (each its own
first_id range, its own grid) whose integer counts and spectra are summed on the
host equal the unsharded run bit for bit in the frozen mode, where histories do not
depend on arrival order. The same sum through rt_set_counts reproduces the
temperatures of the unsharded run."""
import numpy as np
import pytest

from paper_1201_3588_gb300 import rt, shard, workloads as w
from _helpers import frozen_field

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 4])
def test_shards_sum_to_the_single_run(world):
    m = w.sphere_model()
    Tf = frozen_field(m)
    n_per = 250_000
    N = shard.total_packages(world, n_per)
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.set_frozen_temperatures(Tf)
        g.transport(N, seed=9, mode=rt.REEMIT_FROZEN)
        ref_cnt, (ref_sed, eps) = g.counts(), g.sed()
        ref_T = g.temperatures()
    cnt = np.zeros_like(ref_cnt)
    sed = np.zeros_like(ref_sed)
    for r in range(world):
        first, n = shard.package_range(r, world, n_per)
        with rt.Grid(m) as g:
            g.emit_star(N)
            g.set_frozen_temperatures(Tf)
            g.transport(n, seed=9, first_id=first, mode=rt.REEMIT_FROZEN)
            cnt += g.counts()
            sed += g.sed()[0]
            assert g.counters()["emitted"] == n
    assert np.array_equal(cnt, ref_cnt)
    assert np.array_equal(sed, ref_sed)
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.set_counts(cnt)
        assert np.array_equal(g.temperatures(), ref_T)
