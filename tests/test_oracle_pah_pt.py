"""Pins of the oracle's P(T) of a PAH in a monochromatic field (Fig. 3 inputs:
100 C atoms, photons of 3.8 eV .. 1 keV at 10^4 erg/s/cm^2): the single-photon
limit in closed form, the energy balance, and the strong-field limit at the
equilibrium temperature."""
import math

import numpy as np
import pytest

import oracle
from oracle import pah
from paper_1201_3588_gb300 import workloads as w

EV = 1.602176634e-12
FIG3_EV = [3.8, 13.6, 50.0, 100.0, 300.0, 1000.0]


def _pah100(B=48):
    nu = w.frequency_edges(B)
    sp = w.pah_species(nu, 100)
    return sp, nu, sp.kabs * sp.mol_mass


def test_single_photon_limit():
    """A rare photon lifts the molecule from the ground level to E = h nu (levels q
    and q + 1 with weights 1 - w, w), then it cools level by level: the time spent
    in level j per absorption is 1/C_j, so P_j = R / C_j for 1 <= j <= q and
    P_{q+1} = w R / C_{q+1}, to first order in R."""
    sp, nu, sig = _pah100()
    h_nu = 13.6 * EV
    r = pah.temperature_distribution(sp.modes, sig, nu, h_nu, flux=1e-8, sigma_line=1e-16,
                                     n_levels=300)
    P, L, dE, R = r["P"], r["L"], r["dE"], r["rate"]
    C = L / dE
    x = h_nu / dE
    q, wq = int(math.floor(x)), x - math.floor(x)
    j = np.arange(1, q + 1)
    np.testing.assert_allclose(P[j] * C[j] / (R * P[0]), 1.0, rtol=1e-5)
    assert P[q + 1] * C[q + 1] / (R * P[0]) == pytest.approx(wq, rel=1e-5, abs=1e-9)
    assert P[q + 2:].sum() < 1e-6 * P[1:q + 2].sum()


@pytest.mark.parametrize("e_ev", FIG3_EV)
def test_energy_balance(e_ev):
    """Emitted power = absorbed power R h nu: the split onto the two levels around
    E_i + h nu keeps the energy and cooling removes L dE/dE per level step (up to
    the energy cut off at the top level, negligible with levels up to 6000 K)."""
    sp, nu, sig = _pah100()
    r = pah.temperature_distribution(sp.modes, sig, nu, e_ev * EV, flux=1e4, sigma_line=2e-16,
                                     n_levels=600, t_top=6000.0)
    assert r["emission"].sum() == pytest.approx(r["rate"] * e_ev * EV, rel=1e-8)
    assert r["P"].sum() == pytest.approx(1.0, abs=1e-12)


def test_strong_field_sits_at_equilibrium():
    """A large molecule with many photons per cooling time: P(T) narrows around the
    temperature at which cooling equals heating, 4 pi sum_b sigma_b P_b(T) = R h nu."""
    nu = w.frequency_edges(48)
    sp = w.pah_species(nu, 4000)
    sig = sp.kabs * sp.mol_mass
    h_nu = 3.8 * EV
    r = pah.temperature_distribution(sp.modes, sig, nu, h_nu, flux=8.86e5, sigma_line=8e-15,
                                     n_levels=1200, t_top=3000.0)
    heat = r["rate"] * h_nu

    def cool(T):
        return 4 * math.pi * sum(sig[b] * oracle.planck_bin(nu[b], nu[b + 1], T)
                                 for b in range(len(nu) - 1))
    lo, hi = 10.0, 3000.0
    for _ in range(100):
        mid = math.sqrt(lo * hi)
        lo, hi = (mid, hi) if cool(mid) < heat else (lo, mid)
    T_eq = math.sqrt(lo * hi)
    mean_T = float((r["P"] * r["T"]).sum())
    width = math.sqrt(float((r["P"] * (r["T"] - mean_T) ** 2).sum()))
    assert 700.0 < T_eq < 900.0
    assert mean_T == pytest.approx(T_eq, rel=0.015)
    assert width < 0.06 * T_eq


def test_harder_photons_reach_higher_temperatures():
    """One absorption from the ground lands on the levels around E = h nu; above
    them the populations fall off sharply (a second photon before cooling is rare
    at 10^4 erg/s/cm^2), so the edge of P(T) sits at T(E = h nu) and rises with h nu."""
    sp, nu, sig = _pah100()
    edge = []
    for e_ev in FIG3_EV:
        r = pah.temperature_distribution(sp.modes, sig, nu, e_ev * EV, flux=1e4,
                                         sigma_line=2e-16, n_levels=600, t_top=6000.0,
                                         t_sub=1000.0)
        P, T, dE = r["P"], r["T"], r["dE"]
        q = int(math.floor(e_ev * EV / dE))
        assert P[q + 2] < 0.5 * P[q], (e_ev, P[q], P[q + 2])
        assert T[q] == pytest.approx(pah.temperature_of_energy(e_ev * EV, sp.modes), rel=0.01)
        assert 0.0 <= r["p_above"] <= 1.0
        edge.append(T[q])
    assert all(b > a for a, b in zip(edge, edge[1:])), edge
