"""P(T) of PAHs in monochromatic fields on the GPU (rt_pah_temperature_distribution)
against the FP64 oracle: the Fig. 3 inputs (100 C atoms; 3.8 eV .. 1 keV photons at
10^4 erg/s/cm^2) and a batch over sizes and fluxes, with the time spent above the
sublimation threshold."""
import math
import time

import numpy as np
import pytest

from oracle import pah
from paper_1201_3588_gb300 import rt, workloads as w

pytestmark = pytest.mark.gpu
EV = 1.602176634e-12
FIG3_EV = [3.8, 13.6, 50.0, 100.0, 300.0, 1000.0]


def _cases(sizes, energies, fluxes, nu, sigma_line=2e-18, t_top=4000.0):
    cases, sig, meta = [], [], []
    for nc in sizes:
        sp = w.pah_species(nu, nc)
        for e_ev in energies:
            for F in fluxes:
                s_line = sigma_line * nc
                cases.append(dict(modes=sp.modes, h_nu=e_ev * EV, rate=s_line * F / (e_ev * EV),
                                  t_top=t_top))
                sig.append(sp.kabs * sp.mol_mass)
                meta.append((sp, e_ev, F, s_line))
    return cases, np.array(sig), meta


def _compare(cases, sig, meta, nu, M, t_sub):
    P, T, a, em = rt.pah_temperature_distribution(cases, nu, sig, n_levels=M, t_sub=t_sub)
    for i, (sp, e_ev, F, s_line) in enumerate(meta):
        r = pah.temperature_distribution(sp.modes, sig[i], nu, e_ev * EV, F, s_line,
                                         n_levels=M, t_top=cases[i]["t_top"], t_sub=t_sub)
        np.testing.assert_allclose(T[i], r["T"], rtol=1e-11, atol=0)
        # the level-by-level recursion carries rounding into the far tails
        big = r["P"] > 1e-6 * r["P"].max()
        tail = (r["P"] > 1e-12 * r["P"].max()) & ~big
        np.testing.assert_allclose(P[i][big], r["P"][big], rtol=1e-7)
        np.testing.assert_allclose(P[i][tail], r["P"][tail], rtol=1e-4)
        assert abs(P[i][~(big | tail)]).max(initial=0.0) < 1e-11 * r["P"].max()
        assert a[i] == pytest.approx(r["p_above"], rel=1e-7, abs=1e-15)
        np.testing.assert_allclose(em[i], r["emission"], rtol=1e-7, atol=1e-12 * em[i].max())
        # energy: emitted = absorbed, up to the cut at the top level
        assert em[i].sum() == pytest.approx(cases[i]["rate"] * cases[i]["h_nu"], rel=1e-6)
    return P, T, a, em


def test_fig3_inputs_match_oracle():
    nu = w.frequency_edges(48)
    cases, sig, meta = _cases([100], FIG3_EV, [1e4], nu, t_top=6000.0)
    P, T, a, em = _compare(cases, sig, meta, nu, M=600, t_sub=2500.0)
    print("time above 2500 K per photon energy:",
          {e: float(x) for e, x in zip(FIG3_EV, a)})
    # harder photons reach the sublimation range: no time above 2500 K for 3.8 eV
    assert a[0] < 1e-12 < a[-1]


def test_batch_over_sizes_and_fluxes():
    nu = w.frequency_edges(64)
    cases, sig, meta = _cases([30, 100], [3.8, 13.6, 100.0], [1e2, 1e4, 1e6], nu)
    t0 = time.perf_counter()
    _compare(cases, sig, meta, nu, M=400, t_sub=2000.0)
    print(f"{len(cases)} cases checked in {time.perf_counter() - t0:.1f} s")


def test_arguments():
    nu = w.frequency_edges(8)
    sp = w.pah_species(nu, 50)
    good = dict(modes=sp.modes, h_nu=10 * EV, rate=1.0)
    sig = (sp.kabs * sp.mol_mass)[None]
    for bad_case, kw in [(dict(good, h_nu=0.0), {}), (dict(good, rate=-1.0), {}),
                         (good, dict(n_levels=8)), (good, dict(n_levels=5000)),
                         (dict(good, modes=()), {})]:
        with pytest.raises(rt.RTError) as e:
            rt.pah_temperature_distribution([bad_case], nu, sig, **kw)
        assert e.value.code == 1
    with pytest.raises(rt.RTError):
        rt.pah_temperature_distribution([good], nu, -sig)
