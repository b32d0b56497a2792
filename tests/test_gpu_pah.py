"""PAH path on the GPU against the oracle: transport with PAH species (absorbed-
spectrum tallies, template re-emission) under frozen-mode replay, and the exact
transient-heating emission of sampled cells (thermal-discrete steady state)."""
import numpy as np
import pytest

import oracle
from oracle import pah
from paper_1201_3588_gb300 import rt, workloads as w
from _helpers import frozen_field, trace_agreement

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pah_model():
    B = 64
    nu = w.frequency_edges(B)
    sp = w.two_species(nu) + [w.pah_species(nu, 30), w.pah_species(nu, 200)]
    return w.sphere_model(n_base=8, n_bins=B, tau_v=3.0, species=sp,
                          fractions=[0.70, 0.25, 0.03, 0.02])


@pytest.fixture(scope="module")
def pah_oracle(pah_model):
    return oracle.OracleModel(pah_model)


def test_pah_replay_and_tallies_match_oracle(pah_model, pah_oracle):
    N = 20000
    Tf = frozen_field(pah_model)
    with rt.Grid(pah_model) as g:
        g.emit_star(N)
        g.set_frozen_temperatures(Tf)
        g.transport(N, seed=4, mode=rt.REEMIT_FROZEN)
        cnt = g.counts().astype(np.int64)
        tal = g.pah_absorbed().astype(np.int64)
        c = g.counters()
        ids = np.arange(2000, dtype=np.uint64) * 7
        rec = g.trace(ids, seed=4)
    o = oracle.transport(pah_oracle, N, seed=4, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf.astype(np.float64), n_total=N)
    assert c["emitted"] == N == c["escaped"] and c["errors"] == 0
    # every PAH absorption is tallied once
    assert tal.sum(axis=(1, 2)).tolist() == cnt[2:].sum(axis=1).tolist()
    otal = o.pahabs.astype(np.int64)
    assert np.abs(tal - otal).sum() <= 0.03 * otal.sum() + 3
    assert np.abs(cnt - o.count.astype(np.int64)).sum() <= 0.03 * o.count.sum() + 5
    orc = oracle.trace(pah_oracle, ids, Tf.astype(np.float64), seed=4, n_total=N)
    frac, _ = trace_agreement(rec, orc)
    print("PAH replay agreement", frac)
    assert frac >= 0.97


def test_exact_pah_emission_matches_oracle(pah_model, pah_oracle):
    N = 2 * 10 ** 6
    with rt.Grid(pah_model) as g:
        g.emit_star(N)
        g.transport(N, seed=9)
        tal = g.pah_absorbed().astype(np.float64)
        _, eps = g.sed()
        J, nf = g.pah_emission()
    m = pah_model
    assert nf == 0 and J.shape == (m.tree.n_leaves, m.n_bins)
    d0 = 2 * m.half_size / m.tree.n_base
    V = d0 ** 3
    e = pah.coarse_photon_energy(m.nu_edges)
    absorbed = (tal * eps).sum(axis=(0, 2))
    has = absorbed > 0
    assert (J[~has] == 0).all()
    # emitted = absorbed, cell by cell (FP32 tables)
    np.testing.assert_allclose(J[has].sum(axis=1), absorbed[has], rtol=2e-4)
    # sampled cells against the oracle's level solution
    rng = np.random.default_rng(0)
    cells = rng.choice(np.nonzero(has)[0], 12, replace=False)
    tabs = {}
    for p, si in enumerate(pah_oracle.pah_species):
        sp = m.species[si]
        tabs[p] = (sp, pah.level_tables(sp.kabs * sp.mol_mass, sp.modes, m.nu_edges,
                                        n_levels=400, t_top=2500.0))
    for c in cells:
        ref = np.zeros(m.n_bins)
        for p, (sp, tab) in tabs.items():
            si = pah_oracle.pah_species[p]
            n_mol = m.rho[si, c] * V / sp.mol_mass
            if tal[p, c].sum() == 0:
                continue
            R = pah.cell_rates(tal[p, c], eps, n_mol, e)
            P, _ = pah.populations(R, e, tab)
            ref += n_mol * pah.emission(P, tab)
        big = ref > 1e-6 * ref.max()
        np.testing.assert_allclose(J[c][big], ref[big], rtol=2e-3)
