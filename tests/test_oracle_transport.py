"""Pins of the oracle's transport against closed forms and brute force:
Beer-Lambert transmission of a pure absorber (slab, normal and oblique), uncollided
escape from a uniform cube (angular quadrature), first-interaction counts on a 2x2x2
grid, exact photon accounting, the optically thin T ~ r^-1/2 law, and the three
re-emission rules against their defining spectra."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1201_3588_gb300 import workloads as w

SIGMA = 5.670374419e-5


def _binom_ok(k, n, p, z=4.0):
    return abs(k - n * p) <= z * math.sqrt(max(n * p * (1 - p), 1e-300)) + 1e-9


def _grey_box(n_base, tau_half, albedo=0.0, B=4, star=None, g=0.0):
    sp = [w.grey_species(B, 1.0 - albedo, albedo, g)]
    return w.uniform_box_model(n_base, B, tau_half, sp, half_size_cm=w.AU, star=star)


def _escape_fraction_cube(tau_face):
    """Fraction of isotropic packages from the centre of a uniform cube that leave it
    without interacting: 6/(4 pi) * integral over the +z face of
    exp(-tau sqrt(1+x^2+y^2)) / (1+x^2+y^2)^(3/2) dx dy, tau the centre-to-face depth."""
    x, wt = np.polynomial.legendre.leggauss(200)
    X, Y = np.meshgrid(x, x)
    W = np.outer(wt, wt)
    r2 = 1 + X ** 2 + Y ** 2
    return 6 / (4 * math.pi) * float((W * np.exp(-tau_face * np.sqrt(r2)) / r2 ** 1.5).sum())


@pytest.mark.parametrize("tau", [0.1, 1.0, 3.0])
@pytest.mark.parametrize("oblique", [False, True])
def test_slab_transmission_is_beer_lambert(tau, oblique):
    H = w.AU
    ang = math.radians(20.0) if oblique else 0.0
    d = (math.sin(ang), 0.0, math.cos(ang))
    star = w.Star(pos_cm=(-0.5 * H if oblique else 0.13 * H, 0.21 * H, -H),
                  kind=w.SOURCE_BEAM, beam_dir=d)
    m = _grey_box(4, tau / 2.0, star=star)          # bottom-to-top depth tau
    N = 20000
    # max_events=0 stops each package at its first interaction: only the uncollided
    # escape matters here
    t = oracle.transport(m, N, seed=7, max_events=0)
    assert t.errors == 0
    k = int(t.sed[1].sum())                          # escaped without interacting
    p = math.exp(-tau / math.cos(ang))
    assert _binom_ok(k, N, p), (k, N * p)


@pytest.mark.parametrize("tau_face", [0.3, 2.0])
def test_uncollided_escape_from_uniform_cube(tau_face):
    m = _grey_box(4, tau_face)
    N = 40000
    t = oracle.transport(m, N, seed=11, max_events=0)
    p = _escape_fraction_cube(tau_face)
    assert _binom_ok(int(t.sed[1].sum()), N, p), (int(t.sed[1].sum()), N * p)


def test_first_interactions_on_2x2x2_grid():
    """Point source on the corner shared by all 8 cubes: every ray stays in one octant
    and crosses its cube from the corner to the far faces, so the first-interaction
    probability of cube c is (1/8) [1 - F(tau_c)], F the uncollided fraction of a
    uniform cube with centre-to-face depth tau_c; absorption takes (1 - albedo)."""
    tree = w.build_tree(2, 0)
    albedo = 0.4
    B = 4
    sp = [w.grey_species(B, 1.0 - albedo, albedo, 0.0)]
    taus = np.array([0.05, 0.2, 0.5, 1.0, 1.5, 2.5, 0.0, 3.5])   # per cube, corner to face
    H = w.AU
    d0 = H                                                      # cube edge (n = 2)
    rho = taus / (1.0 * d0)                                     # kappa_ext = 1 cm^2/g
    m = w.explicit_model(tree, rho, B, sp, half_size_cm=H)
    N = 60000
    t = oracle.transport(m, N, seed=3, max_events=1)
    assert t.errors == 0 and t.emitted == N
    ext_total = 0.0
    for leaf in range(8):
        pc = (1.0 - _escape_fraction_cube(taus[leaf])) / 8.0
        ext_total += pc
        assert _binom_ok(int(t.count[0, leaf]), N, (1 - albedo) * pc), leaf
    # capped packages are those whose second interaction was cut; first scatters:
    assert _binom_ok(t.scatters, N, albedo * ext_total)


def test_photon_accounting_identities():
    m = w.sphere_model(n_base=8, n_bins=16, tau_v=3.0)
    t = oracle.transport(m, 3000, seed=5)
    assert t.errors == 0 and t.capped == 0
    assert t.emitted == 3000 == t.escaped + t.capped
    assert int(t.count.sum()) == t.absorptions
    assert int(t.sed[0].sum()) == t.escaped
    assert int(t.sed[1].sum()) <= t.escaped
    # resuming from a package id continues the same streams: two halves == whole (in
    # the frozen mode, where trajectories do not depend on the counts)
    Tf = np.full((m.n_species, m.tree.n_leaves), 30.0)
    a = oracle.transport(m, 2000, seed=9, mode=oracle.MODE_FROZEN, T_frozen=Tf, n_total=2000)
    b = oracle.transport(m, 1200, seed=9, mode=oracle.MODE_FROZEN, T_frozen=Tf, n_total=2000)
    b = oracle.transport(m, 800, seed=9, first_id=1200, mode=oracle.MODE_FROZEN,
                         T_frozen=Tf, n_total=2000, tally=b)
    assert (a.count == b.count).all() and (a.sed == b.sed).all()
    assert a.crossings == b.crossings


def test_event_cap_accounting():
    m = _grey_box(4, 6.0, albedo=0.9)
    t = oracle.transport(m, 500, seed=2, max_events=3)
    assert t.capped > 0
    assert t.emitted == t.escaped + t.capped


def _corner_cell_integral(k, L):
    """(1/4 pi) * integral over the octant of (1 - exp(-k L(d)))/k dOmega, L(d) the
    distance from the corner to the cube's far faces (edge L)."""
    x, wt = np.polynomial.legendre.leggauss(120)
    X, Y = np.meshgrid((x + 1) / 2, (x + 1) / 2)          # the +z face of the octant cube
    W = np.outer(wt, wt) / 4
    r2 = 1 + X ** 2 + Y ** 2
    path = L * np.sqrt(r2)
    f = (1 - np.exp(-k * path)) / k if k > 0 else path
    return 3 * float((W * f / r2 ** 1.5).sum()) / (4 * math.pi)


def _cell_integral(k, lo, hi):
    """(1/4 pi) * integral over the box of exp(-k r)/r^2 dV (box away from the origin)."""
    x, wt = np.polynomial.legendre.leggauss(10)
    pts = [(lo[a] + hi[a]) / 2 + (hi[a] - lo[a]) / 2 * x for a in range(3)]
    ws = [(hi[a] - lo[a]) / 2 * wt for a in range(3)]
    X, Y, Z = np.meshgrid(*pts, indexing="ij")
    W = ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    return float((W * np.exp(-k * r) / r ** 2).sum()) / (4 * math.pi)


def test_optically_thin_temperature_follows_r_to_minus_half():
    """Grey absorber, first absorptions only: n_c = N int_c rho kappa e^{-rho kappa r}
    /(4 pi r^2) dV in expectation, and 4 kappa sigma T^4 = n eps / M gives
    T = T* (R*/2r)^(1/2) (times the attenuation) -- the r^-1/2 law."""
    H = w.AU
    n_base, B = 6, 8
    sp = [w.grey_species(B, 1.0)]
    m = w.uniform_box_model(n_base, B, 0.08, sp, half_size_cm=H)
    m = dataclasses.replace(m, nu_edges=w.frequency_edges(B, 0.01, 1.0e5))
    N = 300000
    t = oracle.transport(m, N, seed=21, max_events=1)
    eps = m.star.L / N
    T = oracle.temperatures(m, t.count, eps)[0]
    d0 = 2 * H / n_base
    rho = m.rho[0, 0]
    k = rho * 1.0                                     # kappa_ext = kappa_abs = 1
    lo, hi = w.leaf_bounds_cm(m.tree, H)
    V = d0 ** 3
    zs, rs, Ts = [], [], []
    for c in range(m.tree.n_leaves):
        corner = np.all(np.isclose(np.minimum(np.abs(lo[c]), np.abs(hi[c])), 0.0))
        I = _corner_cell_integral(k, d0) if corner else _cell_integral(k, lo[c], hi[c])
        En = N * rho * 1.0 * I
        Texp = (En * eps / (rho * V) / (4 * 1.0 * SIGMA)) ** 0.25
        sig = Texp / (4 * math.sqrt(En))
        zs.append((T[c] - Texp) / sig)
        rs.append(np.linalg.norm((lo[c] + hi[c]) / 2))
        Ts.append(Texp)
    zs = np.array(zs)
    assert np.abs(zs).max() < 4.5, np.abs(zs).max()
    assert abs(zs.mean()) < 4.0 / math.sqrt(len(zs))
    # the closed-form field itself falls close to r^-1/2 (attenuation adds a little)
    slope = np.polyfit(np.log(rs), np.log(Ts), 1)[0]
    assert -0.56 < slope < -0.44


def _pmf_of_sampler(m, mode, n, e, uf, tmin, K=24, M=400):
    cnt = np.zeros(m.B)
    for a in (np.arange(K) + 0.5) / K:
        for b in (np.arange(M) + 0.5) / M:
            cnt[oracle.reemit_bin(m, 0, mode, n, e, uf, tmin, a, b)] += 1
    return cnt / cnt.sum()


def _exact_spectrum(m, Ta, Tb):
    ka = m.species[0].kabs
    nu = m.nu_edges
    Pa = np.array([oracle.planck_bin(nu[i], nu[i + 1], Ta) for i in range(m.n_bins)])
    Pb = np.array([oracle.planck_bin(nu[i], nu[i + 1], Tb) for i in range(m.n_bins)])
    d = ka * (Pb - Pa)
    return d / d.sum()


@pytest.mark.parametrize("n", [0, 3, 40])
def test_bw_reemission_is_the_difference_spectrum(n):
    B = 12
    nu = w.frequency_edges(B)
    sp = [w.powerlaw_species("sil", nu, 1e4, 0.5, 1.5)]
    m = w.explicit_model(w.build_tree(2, 0), np.ones((1, 8)), B, sp)
    ka = sp[0].kabs
    e = oracle.emission_per_mass(ka, nu, 20.0) * 0.3         # big steps in T
    Ta = oracle.temperature(ka, nu, n * e)
    Tb = oracle.temperature(ka, nu, (n + 1) * e)
    pmf = _pmf_of_sampler(oracle.as_oracle(m), oracle.MODE_BW, n, e, 0.0, 1.0)
    assert np.abs(pmf - _exact_spectrum(m, Ta, Tb)).max() < 6e-3


@pytest.mark.parametrize("mode", ["nocorr", "frozen"])
def test_nocorr_and_frozen_reemission_follow_kappa_B(mode):
    B = 12
    nu = w.frequency_edges(B)
    sp = [w.powerlaw_species("carb", nu, 2e4, 0.3, 1.0)]
    m = w.explicit_model(w.build_tree(2, 0), np.ones((1, 8)), B, sp)
    ka = sp[0].kabs
    if mode == "nocorr":
        e = oracle.emission_per_mass(ka, nu, 35.0) / 5
        T = oracle.temperature(ka, nu, 5 * e)                  # T(n) before absorbing
        pmf = _pmf_of_sampler(oracle.as_oracle(m), oracle.MODE_NOCORR, 5, e, 0.0, 1.0)
    else:
        T = 80.0
        uf = oracle.emission_per_mass(ka, nu, T)
        pmf = _pmf_of_sampler(oracle.as_oracle(m), oracle.MODE_FROZEN, 0, 1.0, uf, 1.0)
    assert np.abs(pmf - _exact_spectrum(m, 0.0, T)).max() < 6e-3


def test_bw_difference_spectra_telescope():
    """Summed over n = 0..N-1 the BW spectra equal kappa B(T(N)) (Bjorkman & Wood's
    property), so the whole cell re-emits at its final temperature."""
    B = 10
    nu = w.frequency_edges(B)
    sp = [w.powerlaw_species("sil", nu, 1e4, 0.5, 1.5)]
    m = oracle.as_oracle(w.explicit_model(w.build_tree(2, 0), np.ones((1, 8)), B, sp))
    ka = sp[0].kabs
    Nn = 6
    e = oracle.emission_per_mass(ka, nu, 50.0) / Nn
    tot = np.zeros(B)
    for n in range(Nn):
        tot += _pmf_of_sampler(m, oracle.MODE_BW, n, e, 0.0, 1.0, K=16, M=300)
    TN = oracle.temperature(ka, nu, Nn * e)
    assert np.abs(tot / Nn - _exact_spectrum(m.model, 0.0, TN)).max() < 6e-3
