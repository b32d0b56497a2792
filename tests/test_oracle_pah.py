"""Pins of the oracle's PAH transient-heating solution (thermal-discrete steady
state): normalisation, exact energy balance, agreement with a dense solve of the
full master equation, the flux written as a convolution with the cumulative upward
rates (the form the GPU solves), the equilibrium limit of a large molecule in a strong field,
the single-photon ceiling of a weak monochromatic field, and the classical limit of
the heat content."""
import math

import numpy as np
import pytest

import oracle
from oracle import pah
from paper_1201_3588_gb300 import workloads as w

NU = w.frequency_edges(200)


def _species(nc):
    sp = w.pah_species(NU, nc)
    return sp, sp.kabs * sp.mol_mass


def _stellar_rates(sigma_mol, flux, T_star=5800.0):
    """Absorption rates per molecule in the 64 coarse bins for a diluted blackbody
    of bolometric flux `flux` (erg s^-1 cm^-2)."""
    e = pah.coarse_photon_energy(NU)
    Pst = np.array([oracle.planck_bin(NU[b], NU[b + 1], T_star) for b in range(200)])
    fb = flux * Pst / Pst.sum()
    cm = pah.coarse_map(200)
    R = np.zeros(64)
    for b in range(200):
        R[cm[b]] += fb[b] * sigma_mol[b] / e[cm[b]]
    return R, e


@pytest.mark.parametrize("flux", [1e4, 1e7])
def test_normalised_and_energy_conserving(flux):
    sp, sig = _species(30)
    tab = pah.level_tables(sig, sp.modes, NU, n_levels=300)
    R, e = _stellar_rates(sig, flux)
    P, _ = pah.populations(R, e, tab)
    assert P.sum() == pytest.approx(1.0, abs=1e-12) and (P >= 0).all()
    assert pah.emission(P, tab).sum() == pytest.approx((R * e).sum(), rel=1e-9)


def test_level_recursion_equals_dense_master_equation():
    sp, sig = _species(30)
    tab = pah.level_tables(sig, sp.modes, NU, n_levels=50)
    for scale in (1.0, 1e3, 1e6):
        R, e = _stellar_rates(sig, 1e4 * scale)
        P1, _ = pah.populations(R, e, tab)
        P2 = pah.dense_populations(R, e, tab)
        assert np.abs(P1 - P2).max() < 1e-10


def _convolution_populations(R, e, tab):
    """The same steady state written as the GPU solves it: with uniform levels the
    rate from level i to the levels at or above f depends on f - i alone, G(d), so
    the upward flux across the boundary below f is sum_{d>=1} G(d) P_{f-d} (FP64
    here; independent of the oracle's scatter of arrivals)."""
    dE, L = tab["dE"], tab["L"]
    M = len(L)
    H = np.zeros(M + 1)
    for k in range(len(R)):
        if R[k] <= 0.0:
            continue
        x = e[k] / dE
        q = int(math.floor(x))
        w_k = x - q
        H[min(q, M - 1)] += R[k] * (1.0 - w_k) if q >= 1 else 0.0
        H[min(q + 1, M - 1)] += R[k] * w_k
    G = np.cumsum(H[::-1])[::-1]             # G[d] = sum_{q >= d} H[q]
    P = np.zeros(M)
    P[0] = 1.0
    for f in range(1, M):
        d = np.arange(1, f + 1)
        C = L[f] / dE
        P[f] = (G[d] * P[f - d]).sum() / C if C > 0 else 0.0
    return P / P.sum()


@pytest.mark.parametrize("nc,flux", [(30, 1e2), (30, 1e6), (200, 1e4), (200, 1e9)])
def test_flux_as_convolution_equals_level_recursion(nc, flux):
    # the form of the GPU's FP32 solution against the oracle's carried recursion
    sp, sig = _species(nc)
    tab = pah.level_tables(sig, sp.modes, NU, n_levels=200)
    R, e = _stellar_rates(sig, flux)
    P1, _ = pah.populations(R, e, tab)
    P2 = _convolution_populations(R, e, tab)
    # deep in the tail the carried difference of the oracle loses digits even in
    # FP64 (3e-7 at 1e-12 of the peak); every level above 1e-6 of it agrees closely
    big = P1 > 1e-6 * P1.max()
    assert np.abs(P2[big] / P1[big] - 1).max() < 1e-9
    J1, J2 = pah.emission(P1, tab), pah.emission(P2, tab)
    bj = J1 > 1e-6 * J1.max()
    assert np.abs(J2[bj] / J1[bj] - 1).max() < 1e-8


def test_large_molecule_in_strong_field_reaches_equilibrium():
    """Many modes and frequent absorptions: the temperature hardly fluctuates, so the
    mean level temperature tends to the equilibrium T with L(T) = absorbed power."""
    sp, sig = _species(4000)
    R, e = _stellar_rates(sig, 3e8)
    P_abs = (R * e).sum()
    Teq = oracle.temperature(sig, NU, P_abs)            # 4 pi sum sigma_b P_b(T) = P_abs
    tab = pah.level_tables(sig, sp.modes, NU, n_levels=600, t_top=2.0 * Teq)
    P, _ = pah.populations(R, e, tab)
    Tm = float((P * tab["T"]).sum())
    assert Tm == pytest.approx(Teq, rel=0.02)
    assert float(np.sqrt((P * (tab["T"] - Tm) ** 2).sum())) < 0.05 * Teq


def test_weak_monochromatic_field_stays_below_one_photon():
    """Rare absorptions of photons of one energy: the molecule cools fully between
    them, so almost no population lies above one photon's energy."""
    sp, sig = _species(30)
    tab = pah.level_tables(sig, sp.modes, NU, n_levels=400)
    e = pah.coarse_photon_energy(NU)
    k = 60                                             # a UV coarse bin
    R = np.zeros(64)
    R[k] = 1e-6                                        # photons per second
    P, _ = pah.populations(R, e, tab)
    above = tab["E"] > e[k] + 2 * tab["dE"]
    assert P[above].sum() < 1e-5
    # and the emitted power is the absorbed one
    assert pah.emission(P, tab).sum() == pytest.approx(R[k] * e[k], rel=1e-9)


def test_heat_content_limits_and_inverse():
    modes = w.pah_modes(50, w.pah_hydrogens(50))
    n_tot = sum(n for n, _ in modes)
    assert n_tot == 3 * (50 + w.pah_hydrogens(50)) - 6
    T = 1e6                                            # classical: E -> sum n k (T - theta/2)
    cl = sum(n * pah.K_B * (T - th / 2) for n, th in modes)
    assert float(pah.internal_energy(T, modes)) == pytest.approx(cl, rel=1e-8)
    for T in (3.0, 40.0, 700.0, 2500.0):
        E = float(pah.internal_energy(T, modes))
        assert pah.temperature_of_energy(E, modes) == pytest.approx(T, rel=1e-12)
