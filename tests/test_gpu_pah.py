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


def test_active_cell_emission_equals_range_form(pah_model):
    """rt_pah_emission_active returns, for every PAH-active cell and no other, the
    row rt_pah_emission writes for it -- exact, surrogate and auto (with fallback)
    modes, device and host outputs, all PAHs and one PAH -- and refuses a buffer
    smaller than the number of active cells."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    N = 10 ** 6
    net = rt.MLP(64 + 2, 64, 2, pah_model.n_bins, seed=3)  # untrained: many fallbacks
    with rt.Grid(pah_model) as g:
        g.emit_star(N)
        g.transport(N, seed=5)
        tal = g.pah_absorbed()
        for mode, pah_sel in ((rt.PAH_EXACT, -1), (rt.PAH_SURROGATE, -1), (rt.PAH_AUTO, -1),
                              (rt.PAH_AUTO, 1)):
            sur = None if mode == rt.PAH_EXACT else net
            tol = 0.05 if mode == rt.PAH_AUTO else 0.0
            J, nf_range = g.pah_emission(mode=mode, surrogate=sur, tol=tol, pah=pah_sel)
            sel = tal if pah_sel < 0 else tal[pah_sel:pah_sel + 1]
            active = np.nonzero(sel.sum(axis=(0, 2)) > 0)[0]
            assert len(active) > 50
            # device output
            cells_d = torch.full((g.N,), -1, dtype=torch.int32, device=dev)
            rows_d = torch.zeros((g.N, g.B), dtype=torch.float32, device=dev)
            c_d, r_d, nf_d = g.pah_emission_active(mode=mode, surrogate=sur, tol=tol,
                                                   cells=cells_d, out=rows_d, pah=pah_sel)
            c_d, r_d = c_d.cpu().numpy(), r_d.cpu().numpy()
            # host output
            c_h, r_h, nf_h = g.pah_emission_active(mode=mode, surrogate=sur, tol=tol,
                                                   pah=pah_sel)
            for cells, rows, nf in ((c_d, r_d, nf_d), (c_h, r_h, nf_h)):
                assert sorted(cells.tolist()) == active.tolist()
                assert nf == nf_range
                np.testing.assert_allclose(rows, J[cells], rtol=1e-6, atol=0)
            if mode == rt.PAH_AUTO:
                assert 0 < nf_range <= len(active)
        small_c = np.zeros(10, dtype=np.int32)
        small_r = np.zeros((10, g.B), dtype=np.float32)
        with pytest.raises(rt.RTError) as e:
            g.pah_emission_active(cells=small_c, out=small_r)
        assert e.value.code == 6


def test_reset_clears_pah_tallies(pah_model):
    """rt_reset clears the absorbed spectra of exactly the cells that hold counts:
    after a first run and a reset, a second run's tallies and active cells equal
    those of the same run on a fresh grid (frozen mode: package histories are pure
    functions of the seed, so the sums are identical)."""
    N = 200_000
    Tf = frozen_field(pah_model)
    out = []
    for first_seed in (1, None):
        with rt.Grid(pah_model) as g:
            g.emit_star(N)
            g.set_frozen_temperatures(Tf)
            if first_seed is not None:
                g.transport(N, seed=first_seed, mode=rt.REEMIT_FROZEN)
                assert g.pah_absorbed().sum() > 0
                g.reset()
                assert g.pah_absorbed().sum() == 0
            g.transport(N, seed=2, mode=rt.REEMIT_FROZEN)
            cells, _, _ = g.pah_emission_active()
            out.append((g.pah_absorbed(), np.sort(cells)))
    (a1, c1), (a2, c2) = out
    assert np.array_equal(a1, a2)
    assert np.array_equal(c1, c2)
    assert np.array_equal(c2, np.nonzero(a2.sum(axis=(0, 2)) > 0)[0])
