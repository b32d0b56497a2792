"""Transient heating of PAH molecules -- oracle (plain FP64 numpy).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg); the library never
imports it.

The paper (Sec. 1, Sec. 3, Fig. 3) computes the temperature distribution P(T) of
PAHs heated by single photons and their band emission; it gives no equations. This
follows the thermal-discrete steady state of Guhathakurta & Draine (1989) as used
by Draine & Li (2001): internal-energy levels E_f; absorption moves a molecule up
from E_i to E_i + h nu (split between the two levels around it so that the energy
is kept); emission is continuous cooling at the rate L(E) = 4 pi sum_b sigma_b
P_b(T(E)), modelled as a transition to the level below at rate L/dE. With only that
downward step, the probability flux upward across each level boundary must equal
the downward flux C_f P_f, which gives the populations level by level. The
emission of the molecule is sum_f P_f 4 pi sigma_b P_b(T(E_f)) per bin.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

H = 6.62607015e-27
K_B = 1.380649e-16
EV = 1.602176634e-12


def internal_energy(T, modes):
    """E(T) = sum over mode groups of n k theta / (exp(theta/T) - 1) (Einstein modes)."""
    T = np.asarray(T, dtype=np.float64)
    out = np.zeros_like(T)
    pos = T > 0
    with np.errstate(over="ignore"):
        for n, th in modes:
            out[pos] += n * K_B * th / np.expm1(th / T[pos])
    return out


def temperature_of_energy(E, modes):
    """Inverse of internal_energy by bisection in ln T (to 1e-14)."""
    E = float(E)
    if E <= 0.0:
        return 0.0
    lo, hi = 1e-3, 10.0
    while float(internal_energy(hi, modes)) < E:
        hi *= 2.0
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if float(internal_energy(mid, modes)) < E:
            lo = mid
        else:
            hi = mid
        if hi / lo - 1.0 < 1e-14:
            break
    return math.sqrt(lo * hi)


def coarse_map(n_bins: int, n_coarse: int = 64):
    """Coarse absorbed-spectrum bin of every fine frequency bin: floor(b K / B)."""
    return (np.arange(n_bins) * n_coarse) // n_bins


def coarse_photon_energy(nu_edges, n_coarse: int = 64):
    """Photon energy (erg) of each coarse bin: h times the geometric centre of its
    frequency range."""
    B = len(nu_edges) - 1
    cm = coarse_map(B, n_coarse)
    e = np.zeros(n_coarse)
    for k in range(n_coarse):
        idx = np.nonzero(cm == k)[0]
        e[k] = H * math.sqrt(nu_edges[idx[0]] * nu_edges[idx[-1] + 1])
    return e


def level_tables(sigma_mol, modes, nu_edges, n_levels=400, t_top=2500.0, e_photon=None):
    """Energy levels E_f = f dE (dE = E_max/(n_levels-1), E_max = E(t_top) plus the
    largest photon energy: that of the grid, or `e_photon` when given), their
    temperatures, cooling rates L_f and per-bin emission s_fb = 4 pi sigma_b P_b(T_f)
    (erg/s per molecule)."""
    B = len(nu_edges) - 1
    e_top = H * nu_edges[-1] if e_photon is None else float(e_photon)
    e_max = float(internal_energy(t_top, modes)) + e_top
    E = np.linspace(0.0, e_max, n_levels)
    T = np.array([temperature_of_energy(x, modes) for x in E])
    s = np.zeros((n_levels, B))
    for f in range(1, n_levels):
        for b in range(B):
            s[f, b] = 4.0 * math.pi * sigma_mol[b] * oracle.planck_bin(nu_edges[b], nu_edges[b + 1],
                                                                      T[f])
    L = s.sum(axis=1)
    return dict(E=E, T=T, L=L, s=s, dE=E[1] - E[0])


def _targets(E_i, e_k, dE, M):
    """Lower target level and the weight on the level above (energy-keeping split)."""
    x = (E_i + e_k) / dE
    f = int(math.floor(x))
    w = x - f
    if f >= M - 1:
        return M - 1, 0.0, True
    return f, w, False


def populations(R, e, tab):
    """Steady-state level populations for photon absorption rates R_k (per molecule
    per second) at photon energies e_k. Returns (P normalised, truncated) where
    `truncated` flags transitions cut at the top level."""
    E, L, dE = tab["E"], tab["L"], tab["dE"]
    M = len(E)
    C = np.zeros(M)
    C[1:] = L[1:] / dE                       # downward (cooling) rate f -> f-1
    P = np.zeros(M)
    D = np.zeros(M)                          # arrivals into each level from below
    truncated = False
    P[0] = 1.0
    F = 0.0                                  # upward flux across the boundary below f

    def scatter(i):
        nonlocal truncated
        up = 0.0
        for k in range(len(R)):
            if R[k] <= 0.0:
                continue
            f, w, cut = _targets(E[i], e[k], dE, M)
            truncated |= cut
            if f > i:
                D[f] += P[i] * R[k] * (1.0 - w)
                up += R[k] * (1.0 - w)
            if f + 1 > i and f + 1 < M:
                D[f + 1] += P[i] * R[k] * w
                up += R[k] * w
        return up

    U = scatter(0)
    F = P[0] * U
    for f in range(1, M):
        P[f] = F / C[f] if C[f] > 0 else 0.0
        U = scatter(f)
        F = max(F - D[f] + P[f] * U, 0.0)
        if P[f] > 1e250:                     # keep the numbers finite
            P[: f + 1] *= 1e-250
            D *= 1e-250
            F *= 1e-250
    return P / P.sum(), truncated


def emission(P, tab):
    """Emitted power per bin of one molecule (erg/s)."""
    return P @ tab["s"]


def cell_rates(counts_k, eps, n_mol, e):
    """Photon absorption rates per molecule from the coarse absorbed counts."""
    return np.asarray(counts_k, dtype=np.float64) * eps / (e * n_mol)


def dense_populations(R, e, tab):
    """The same steady state from the full rate matrix (numpy least squares), for
    checking the level-by-level solution on small grids."""
    E, L, dE = tab["E"], tab["L"], tab["dE"]
    M = len(E)
    W = np.zeros((M, M))                     # W[j, i]: rate i -> j
    for i in range(M):
        for k in range(len(R)):
            f, w, _ = _targets(E[i], e[k], dE, M)
            if f != i:
                W[f, i] += R[k] * (1.0 - w)
            if f + 1 < M and f + 1 != i:
                W[f + 1, i] += R[k] * w
        if i > 0:
            W[i - 1, i] += L[i] / dE
    A = W - np.diag(W.sum(axis=0))
    A = np.vstack([A, np.ones(M)])
    b = np.zeros(M + 1)
    b[-1] = 1.0
    P, *_ = np.linalg.lstsq(A, b, rcond=None)
    return P


F_REF = 1.0e4   # erg s^-1 cm^-2: the heating bath of the paper's Fig. 3


def stellar_rates(sigma_mol, nu_edges, T_star, flux=F_REF, n_coarse=64):
    """Absorption rates per molecule in the coarse bins for a diluted blackbody of
    temperature T_star and bolometric flux `flux` inside the frequency grid."""
    B = len(nu_edges) - 1
    e = coarse_photon_energy(nu_edges, n_coarse)
    Pst = np.array([oracle.planck_bin(nu_edges[b], nu_edges[b + 1], T_star) for b in range(B)])
    fb = flux * Pst / Pst.sum()
    cm = coarse_map(B, n_coarse)
    R = np.zeros(n_coarse)
    for b in range(B):
        R[cm[b]] += fb[b] * sigma_mol[b] / e[cm[b]]
    return R, e


def template_spectrum(species, nu_edges, T_star, flux=F_REF, n_levels=400, t_top=2500.0):
    """Re-emission spectrum (weights per bin, summing to 1) of a PAH species heated
    by starlight of bolometric flux `flux`: the emission of the steady state."""
    sig = species.kabs * species.mol_mass
    tab = level_tables(sig, species.modes, nu_edges, n_levels=n_levels, t_top=t_top)
    R, e = stellar_rates(sig, nu_edges, T_star, flux, min(64, len(nu_edges) - 1))
    P, _ = populations(R, e, tab)
    J = emission(P, tab)
    return J / J.sum()


def temperature_distribution(modes, sigma_mol, nu_edges, h_nu, flux, sigma_line,
                             n_levels=400, t_top=2500.0, t_sub=2500.0):
    """P(T) of a PAH in a monochromatic field (Fig. 3): photons of energy h_nu (erg)
    at flux `flux` (erg/s/cm^2), absorbed with cross section sigma_line (cm^2) at the
    rate R = sigma_line flux / h_nu; levels span 0 .. E(t_top) + h_nu; cooling by the
    cross sections sigma_mol on the frequency grid. Returns the populations P_f, the
    level temperatures, the time fraction spent above t_sub (the shaded region of
    Fig. 3: hotter than graphite sublimates), the emission per bin and R."""
    tab = level_tables(sigma_mol, modes, nu_edges, n_levels=n_levels, t_top=t_top,
                       e_photon=h_nu)
    R = sigma_line * flux / h_nu
    P, truncated = populations(np.array([R]), np.array([h_nu]), tab)
    return dict(P=P, T=tab["T"], E=tab["E"], L=tab["L"],
                p_above=float(P[tab["T"] > t_sub].sum()), emission=emission(P, tab),
                rate=R, truncated=truncated, dE=tab["dE"])
