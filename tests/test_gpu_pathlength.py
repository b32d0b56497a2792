"""Lucy path-length estimator on the GPU: tallies equal the oracle's under frozen-mode
replay, temperatures from them invert like the oracle's, and the Lucy iteration
settles to the Bjorkman-Wood temperatures in well-sampled cells."""
import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import lucy, rt, workloads as w
from _helpers import frozen_field

pytestmark = pytest.mark.gpu


def test_pathlength_tallies_match_oracle():
    m = w.sphere_model()
    Tf = frozen_field(m)
    N = 20000
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.set_frozen_temperatures(Tf)
        g.transport(N, seed=3, mode=rt.REEMIT_FROZEN, estimators=rt.EST_PATHLENGTH)
        P = g.pathlength().astype(np.float64)
        Tp = g.temperatures_pathlength()
        _, eps = g.sed()
    o = oracle.transport(m, N, seed=3, mode=oracle.MODE_FROZEN, T_frozen=Tf.astype(np.float64),
                         n_total=N)
    assert abs(P.sum() / o.pathabs.sum() - 1) < 0.01
    big = o.pathabs > 0.05 * o.pathabs.max()
    assert np.abs(P[big] / o.pathabs[big] - 1).max() < 0.05
    # temperatures from the tallies: the oracle's inversion of the same sums
    d0 = 2 * m.half_size / m.tree.n_base
    kabs, _, _ = m.opacity_arrays()
    rng = np.random.default_rng(0)
    for s in range(m.n_species):
        for c in rng.choice(np.nonzero(P[s] > 0)[0], 40, replace=False):
            u = P[s, c] * eps / (m.rho[s, c] * d0 ** 3)
            assert Tp[s, c] == pytest.approx(oracle.temperature(kabs[s], m.nu_edges, u), rel=2e-4)


def test_lucy_iteration_settles_to_bw_temperatures():
    m = w.sphere_model(tau_v=1.0)
    N = 200_000_000
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.transport(N, seed=1)
        T_bw = g.temperatures()
        cnt = g.counts()
        T_lucy, changes = lucy.iterate(g, N, iterations=3, seed=10)
    print("Lucy iteration max relative change per iteration", changes)
    assert changes[-1] < 0.05
    well = cnt > 1e4
    assert well.sum() > 200, well.sum()
    assert np.median(np.abs(T_lucy[well] / T_bw[well] - 1)) < 0.005
