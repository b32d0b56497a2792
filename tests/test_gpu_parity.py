"""GPU parity of the CUDA transport (through the C ABI) against the FP64 oracle.

* Philox blocks: bit-exact.
* Frozen-temperature mode: package histories are pure functions of (seed, id), so
  GPU and oracle replay the same packages; FP32 rounding (and the tabulated
  re-emission spectra) lets a small fraction diverge.
* BW mode: counts depend on the arrival order, so GPU and oracle agree in
  distribution: per-cell counts within 4 sigma (sigma from GPU batch means,
  floored at Poisson; no more cells beyond than chance allows).
* Temperatures: the GPU kernel and the oracle invert the same counts.
* Closed forms on the GPU at large N: Beer-Lambert slab, 2x2x2 first interactions,
  the optically thin r^-1/2 law (0.5% where counts > 1e4).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import rt, workloads as w
from _helpers import (assert_runs_agree, binom_ok, escape_fraction_cube, frozen_field,
                      grey_box, trace_agreement)

pytestmark = pytest.mark.gpu
SIGMA = 5.670374419e-5


@pytest.fixture(scope="module")
def sphere():
    return w.sphere_model()          # 16^3, 64 bins, 2 species, tau_V = 1


def test_philox_bit_exact():
    ids = np.concatenate([np.arange(500, dtype=np.uint64),
                          np.array([2 ** 32 - 1, 2 ** 32, 2 ** 63 + 12345], dtype=np.uint64)])
    for seed, ev, blk in [(0, 0, 0), (1234567890123, 7, 1), (2 ** 64 - 1, 2 ** 31, 0)]:
        got = rt.philox(ids, ev, blk, seed)
        for i in range(0, len(ids), 37):
            idv = int(ids[i])
            exp = oracle.philox([idv & 0xFFFFFFFF, idv >> 32, ev, blk],
                                [seed & 0xFFFFFFFF, seed >> 32])
            assert got[i].tolist() == exp


def test_frozen_replay_matches_oracle(sphere):
    Tf = frozen_field(sphere)
    n_total = 10 ** 6
    with rt.Grid(sphere) as g:
        g.emit_star(n_total)
        g.set_frozen_temperatures(Tf)
        ids = np.arange(3000, dtype=np.uint64) * 331 + 17
        gr = g.trace(ids, seed=5)
    orc = oracle.trace(sphere, ids, Tf.astype(np.float64), seed=5, n_total=n_total)
    frac, same = trace_agreement(gr, orc)
    print("replay agreement (sphere)", frac)
    assert frac >= 0.98, frac
    # every history accounted: escaped (no cap at the default limit)
    assert (gr[:, 4] == 1).all() and (orc["escaped"] == 1).all()


@pytest.mark.parametrize("kernel", [rt.KERNEL_POOL, rt.KERNEL_PLAIN_F32, rt.KERNEL_PLAIN_F64])
def test_frozen_counts_match_oracle(sphere, kernel):
    Tf = frozen_field(sphere)
    N = 20000
    with rt.Grid(sphere) as g:
        g.emit_star(N)
        g.set_frozen_temperatures(Tf)
        g.transport(N, seed=3, mode=rt.REEMIT_FROZEN, kernel=kernel)
        c = g.counters()
        cnt = g.counts().astype(np.int64)
        sed, eps = g.sed()
    o = oracle.transport(sphere, N, seed=3, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf.astype(np.float64), n_total=N)
    ocnt = o.count.astype(np.int64)
    assert c["emitted"] == N == c["escaped"] + c["capped"]
    assert c["errors"] == 0 and c["capped"] == 0
    assert int(cnt.sum()) == c["absorptions"]
    diff = np.abs(cnt - ocnt)
    assert diff.sum() <= 0.03 * ocnt.sum() + 5, (diff.sum(), ocnt.sum())
    assert (diff <= 4 * np.sqrt(cnt + ocnt) + 1).all()
    assert np.abs(sed.astype(np.int64) - o.sed.astype(np.int64)).sum() <= 0.03 * N
    assert eps == pytest.approx(oracle.package_energy(sphere, N), rel=1e-12)


def test_frozen_pool_and_plain_agree(sphere):
    """Same per-package FP32 code under two schedulers: the pool must neither lose nor
    repeat packages."""
    Tf = frozen_field(sphere)
    N = 200000
    out = []
    for kernel in (rt.KERNEL_POOL, rt.KERNEL_PLAIN_F32):
        with rt.Grid(sphere) as g:
            g.emit_star(N)
            g.set_frozen_temperatures(Tf)
            g.transport(N, seed=11, mode=rt.REEMIT_FROZEN, kernel=kernel)
            out.append((g.counts().astype(np.int64), g.sed()[0].astype(np.int64),
                        g.counters()))
    (a, sa, ca), (b, sb, cb) = out
    assert ca["emitted"] == cb["emitted"] == N
    assert np.abs(a - b).sum() <= 1e-3 * a.sum() + 2
    assert np.abs(sa - sb).sum() <= 1e-3 * N + 2


def _gpu_batches(model, N, n_batches, mode, kernel=rt.KERNEL_POOL):
    runs, seds = [], []
    with rt.Grid(model) as g:
        g.emit_star(N)
        for k in range(n_batches):
            g.reset()
            g.transport(N, seed=1000 + k, mode=mode, kernel=kernel)
            c = g.counters()
            assert c["emitted"] == N == c["escaped"] + c["capped"] and c["errors"] == 0
            runs.append(g.counts().astype(np.float64))
            seds.append(g.sed()[0][0].astype(np.float64))
    return np.array(runs), np.array(seds)


@pytest.mark.parametrize("mode", [rt.REEMIT_BW, rt.REEMIT_NOCORR])
def test_counts_statistics_match_oracle(sphere, mode):
    N = 20000
    runs, seds = _gpu_batches(sphere, N, 32, mode)
    o = oracle.transport(sphere, N, seed=77, mode=mode, n_total=N)
    # one oracle run against 32 GPU runs, per cell within 4 sigma (the variance from
    # the GPU runs, floored at Poisson and at one count; beyond 4 sigma no more cells
    # than chance allows over the 8192 compared)
    assert_runs_agree(o.count.astype(np.float64)[None], runs, f"mode {mode} counts")
    assert_runs_agree(o.sed[0, 0].astype(np.float64)[None], seds, f"mode {mode} spectrum")


def test_temperature_kernel_inverts_like_oracle(sphere):
    N = 10 ** 6
    with rt.Grid(sphere) as g:
        g.emit_star(N)
        g.transport(N, seed=2)
        cnt = g.counts()
        T = g.temperatures()
        _, eps = g.sed()
    To = oracle.temperatures(sphere, cnt, eps)
    pos = cnt > 0
    assert (T[~pos] == 0).all()
    rel = np.abs(T[pos] / To[pos] - 1)
    assert rel.max() < 2e-4, rel.max()


@pytest.mark.parametrize("kernel", [rt.KERNEL_POOL, rt.KERNEL_PLAIN_F32, rt.KERNEL_PLAIN_F64])
@pytest.mark.parametrize("tau,oblique", [(0.1, False), (1.0, False), (3.0, True)])
def test_slab_beer_lambert(kernel, tau, oblique):
    H = w.AU
    ang = math.radians(20.0) if oblique else 0.0
    d = (math.sin(ang), 0.0, math.cos(ang))
    star = w.Star(pos_cm=(-0.5 * H if oblique else 0.13 * H, 0.21 * H, -H),
                  kind=w.SOURCE_BEAM, beam_dir=d)
    m = grey_box(4, tau / 2.0, star=star)
    N = 10 ** 6
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.transport(N, seed=7, kernel=kernel, max_events=1)
        sed, _ = g.sed()
    assert binom_ok(int(sed[1].sum()), N, math.exp(-tau / math.cos(ang)))


def test_first_interactions_2x2x2():
    tree = w.build_tree(2, 0)
    albedo, B = 0.4, 4
    sp = [w.grey_species(B, 1.0 - albedo, albedo, 0.0)]
    taus = np.array([0.05, 0.2, 0.5, 1.0, 1.5, 2.5, 0.0, 3.5])
    H = w.AU
    m = w.explicit_model(tree, taus / H, B, sp, half_size_cm=H)
    N = 2 * 10 ** 6
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.transport(N, seed=3, max_events=1)
        cnt = g.counts()[0]
        c = g.counters()
    tot = 0.0
    for leaf in range(8):
        pc = (1.0 - escape_fraction_cube(taus[leaf])) / 8.0
        tot += pc
        assert binom_ok(int(cnt[leaf]), N, (1 - albedo) * pc), leaf
    assert binom_ok(c["scatters"], N, albedo * tot)


def test_optically_thin_temperature_law():
    """Grey absorber, first absorptions: T matches T*(R*/2r)^(1/2) (with attenuation,
    cell-averaged) within max(0.5%, 4 sigma) where counts exceed 1e4."""
    from test_oracle_transport import _cell_integral, _corner_cell_integral
    H = w.AU
    n_base, B = 6, 8
    sp = [w.grey_species(B, 1.0)]
    m = w.uniform_box_model(n_base, B, 0.08, sp, half_size_cm=H)
    m = dataclasses.replace(m, nu_edges=w.frequency_edges(B, 0.01, 1.0e5))
    N = 3 * 10 ** 8
    with rt.Grid(m) as g:
        g.emit_star(N)
        g.transport(N, seed=21, max_events=1)
        T = g.temperatures()[0]
        cnt = g.counts()[0]
        _, eps = g.sed()
    d0 = 2 * H / n_base
    rho = m.rho[0, 0]
    lo, hi = w.leaf_bounds_cm(m.tree, H)
    checked = 0
    for c in range(m.tree.n_leaves):
        corner = np.all(np.isclose(np.minimum(np.abs(lo[c]), np.abs(hi[c])), 0.0))
        I = _corner_cell_integral(rho, d0) if corner else _cell_integral(rho, lo[c], hi[c])
        En = N * rho * I
        Texp = (En * (m.star.L / N) / (rho * d0 ** 3) / (4 * SIGMA)) ** 0.25
        tol = max(0.005, 4 / (4 * math.sqrt(En)))
        if cnt[c] > 1e4:
            checked += 1
            assert abs(T[c] / Texp - 1) < tol, (c, T[c], Texp)
    assert checked > 150, checked


def test_edge_cases_and_errors(sphere):
    with rt.Grid(sphere) as g:
        with pytest.raises(rt.RTError) as e:
            g.transport(10)                       # no source yet
        assert e.value.code == 5
        g.emit_star(1000)
        g.transport(0)                            # empty launch is a no-op
        assert g.counters()["emitted"] == 0
        with pytest.raises(rt.RTError) as e:
            g.transport(10, first_id=995)         # beyond the planned total
        assert e.value.code == 6
        with pytest.raises(rt.RTError) as e:
            g.transport(10, mode=rt.REEMIT_FROZEN)  # no frozen field
        assert e.value.code == 5
        with pytest.raises(rt.RTError):
            g.transport(10, threads=48)
        g.transport(1000, seed=1)
        assert g.counters()["emitted"] == 1000


def test_empty_and_single_cell_grids():
    # no dust anywhere: every package escapes uncollided, at its stellar bin
    m = grey_box(4, 1.0)
    m = dataclasses.replace(m, rho=np.zeros_like(m.rho))
    with rt.Grid(m) as g:
        g.emit_star(5000)
        g.transport(5000)
        sed, _ = g.sed()
        c = g.counters()
    assert c["escaped"] == 5000 and int(sed[1].sum()) == 5000 and c["absorptions"] == 0
    # one base cube, star on its lower corner (the domain's centre is a corner only
    # for even n, so place the source explicitly)
    t = w.build_tree(1, 0)
    sp = [w.grey_species(4, 1.0)]
    m1 = w.explicit_model(t, np.full(1, 1.0 / w.AU), 4, sp, half_size_cm=w.AU)
    with rt.Grid(m1) as g:
        g.emit_star(20000)
        g.transport(20000, max_events=1)
        sed, _ = g.sed()
    assert int(sed[1].sum()) > 0 and g is not None


def test_max_bins_and_many_directions():
    """1024 bins with 64 direction bins: the escaped histogram no longer fits in
    shared memory and goes to global memory; results stay consistent."""
    B = 1024
    sp = [w.grey_species(B, 1.0, 0.5, 0.3)]
    m = w.uniform_box_model(4, B, 0.5, sp, half_size_cm=w.AU, n_sed_dirs=64)
    with rt.Grid(m) as g:
        g.emit_star(50000)
        g.transport(50000, seed=4)
        sed, _ = g.sed()
        c = g.counters()
    assert c["escaped"] == 50000 and int(sed[0].sum()) == 50000
    assert sed.shape == (2, 64, B)


def test_bw_and_no_correction_agree_where_counts_are_large(sphere):
    """Sec. 2: the vectorised code re-emits without the Bjorkman-Wood correction, and
    the two agree when a cell's counts are not small. Cells with more than 1e4
    absorptions: the mean temperatures of 6 runs per mode agree within 0.5 %, or
    within 4 standard errors of the difference where the runs scatter more."""
    N, runs = 40_000_000, 6
    res = {}
    for mode in (rt.REEMIT_BW, rt.REEMIT_NOCORR):
        Ts, Cs = [], []
        with rt.Grid(sphere) as g:
            g.emit_star(N)
            for k in range(runs):
                g.reset()
                g.transport(N, seed=300 + k, mode=mode)
                Ts.append(g.temperatures().astype(np.float64))
                Cs.append(g.counts().astype(np.float64))
        res[mode] = (np.array(Ts), np.array(Cs))
    (Tb, Cb), (Tn, Cn) = res[rt.REEMIT_BW], res[rt.REEMIT_NOCORR]
    mb, mn = Tb.mean(axis=0), Tn.mean(axis=0)
    se = np.sqrt(Tb.var(axis=0, ddof=1) / runs + Tn.var(axis=0, ddof=1) / runs)
    big = (Cb.mean(axis=0) > 1e4) & (Cn.mean(axis=0) > 1e4)
    d = np.abs(mb - mn)[big]
    rel = d / mb[big]
    print(f"{int(big.sum())} cells above 1e4 counts: max relative difference {rel.max():.4f}, "
          f"max |d|/se {float((d / se[big]).max()):.2f}")
    assert big.sum() > 50
    assert np.all((rel <= 5e-3) | (d <= 4 * se[big]))
