"""Where and why a GPU history and the oracle's history of the same package part.

Under frozen-temperature replay both sides draw the same Philox numbers, so a
package's history on the GPU (FP32 transport, tabulated re-emission spectra) and in
the oracle (FP64, exact re-emission spectra) agree event by event until a decision
falls the other way. The first event whose (kind, cell, bin) differ is the
divergence; it is explained when one of these holds there:

* face: one side's event point lies within an optical depth tau_tol of a face of
  its cell (FP32 accumulates the optical depth and the position as the package
  crosses cells, so the interaction falls just before or just after the face), or
  the two points are
  the same and each lies on the other's cell (a point on a shared face). Two points
  are the same when they lie within POS_TOL, or within an optical depth tau_tol of
  each other (in a thin cell a tiny optical-depth difference moves the point far).
  tau_tol = TAU_TIE + n eps32 (TAU_MAX + kx |p|) bounds the FP32 error linearly over
  the n cells crossed since the previous event (estimated as the distance flown over
  the cell's edge, plus one): per cell one rounding of the remaining optical depth
  (at most TAU_MAX) and of the position (|p| base-cube units, extinction kx per
  unit);
* edge crossing: every event agrees and only the number of cells crossed differs
  (a path through an edge or corner steps one axis at a time on the GPU and crosses
  a cell over zero length; the oracle steps all axes at once);
* decision tie: at the same point and cell, the uniform deviate that decides the
  event (albedo test, species, bin from a discrete spectrum) lies within REL_TIE of
  its threshold recomputed in FP64;
* re-emission table: an absorption at the same point whose new bin differs; the
  GPU samples the temperature-interval mixture of a 1024-row table, the oracle the
  exact spectrum at the energy's temperature T_u. The GPU's bin must lie between
  the bins the exact spectra at the ends of the table intervals around T_u give for
  the same deviate (the mixture over an interval lies between its end spectra,
  which are stochastically ordered in temperature).
"""
import math

import numpy as np

import oracle

TAU_TIE = 1e-4
POS_TOL = 2e-3      # base-cube units
REL_TIE = 1e-5
EPS32 = 2.0 ** -24
TAU_MAX = 16.7      # the largest optical depth a package draws (-ln of the smallest deviate)
KINDS = ("emission", "scatter", "absorption", "escape", "capped")


def first_divergence(ge, oe):
    """Index of the first event whose (kind, cell, bin) differ, None if none does."""
    n = min(len(ge), len(oe))
    for j in range(n):
        if (int(ge["kind"][j]) != int(oe["kind"][j]) or int(ge["leaf"][j]) != int(oe["leaf"][j])
                or int(ge["bin"][j]) != int(oe["bin"][j])):
            return j
    return None if len(ge) == len(oe) else n


def _deviates(seed, pid, event, block):
    w = oracle.philox([pid & 0xFFFFFFFF, pid >> 32, event, block],
                      [seed & 0xFFFFFFFF, seed >> 32])
    return [oracle.uniform(x) for x in w]


def _table_T(n_T, t_min, t_max):
    i = np.arange(n_T, dtype=np.float64)
    T = t_min * (t_max / t_min) ** ((i - 1) / (n_T - 2))
    T[0] = 0.0
    T[-1] = t_max
    return T


def _cum_tie(weights, xi):
    """Is xi (times the total) within REL_TIE of a cumulative boundary?"""
    cum = np.cumsum(weights)
    tot = cum[-1]
    if not tot > 0:
        return False
    return bool(np.min(np.abs(cum[:-1] - xi * tot)) <= REL_TIE * tot) if cum.size > 1 else False


def _bin_at(weights, xi):
    cum = np.cumsum(weights)
    return int(np.searchsorted(cum, xi * cum[-1], side="right"))


class Classifier:
    """Explains the first divergence of GPU and oracle histories of one model under
    frozen temperatures T_frozen [S][N] and Philox key `seed`."""

    def __init__(self, model, T_frozen, seed, om=None, n_temp=1024, t_min=1.0, t_max=3000.0):
        self.m = model
        self.om = om if om is not None else oracle.OracleModel(model)
        self.Tf = np.maximum(np.asarray(T_frozen, dtype=np.float64), t_min)
        self.seed = int(seed)
        self.lo, self.hi = model.tree.leaf_bounds()
        kabs, ksca, _ = model.opacity_arrays()
        self.kabs, self.ksca, self.kext = kabs, ksca, kabs + ksca
        self.d0 = model.cell_size_cm()
        self.nu = model.nu_edges
        self.Tgrid = _table_T(n_temp, t_min, t_max)
        self.pah_of = {s: p for p, s in enumerate(self.om.pah_species)}

    # -- geometry
    def _kx(self, leaf, b):
        return float(self.m.rho[:, leaf] @ self.kext[:, b]) * self.d0

    def _tau_to_face(self, leaf, p, b):
        lo, hi = self.lo[leaf], self.hi[leaf]
        d = max(0.0, float(np.min(np.minimum(p - lo, hi - p))))
        return self._kx(leaf, b) * d

    def _tau_tol(self, leaf, p, p_prev, b):
        n = float(np.linalg.norm(p - p_prev)) / float(self.hi[leaf][0] - self.lo[leaf][0]) + 1.0
        return TAU_TIE + n * EPS32 * (TAU_MAX + self._kx(leaf, b) * float(np.abs(p).max()))

    def _dist_to_box(self, leaf, p):
        q = np.clip(p, self.lo[leaf], self.hi[leaf])
        return float(np.abs(p - q).max())

    # -- spectra
    def _dB(self, s, T):
        return self.kabs[s] * np.array([oracle.dplanck_bin(self.nu[b], self.nu[b + 1], T)
                                        for b in range(self.m.n_bins)])

    def _table_bins(self, s, leaf, xi_u, xi_b):
        """Bin range the table's interval mixtures around the exact T_u allow."""
        uf = oracle.emission_per_mass(self.kabs[s], self.nu, self.Tf[s, leaf])
        Tu = oracle.temperature(self.kabs[s], self.nu, xi_u * uf)
        nT = self.Tgrid.size
        i = int(np.searchsorted(self.Tgrid, Tu, side="right")) - 1
        i0, i1 = max(0, i - 1), min(nT - 2, i + 1)
        T_lo, T_hi = max(self.Tgrid[i0], 1e-3), self.Tgrid[i1 + 1]
        return _bin_at(self._dB(s, T_lo), xi_b), _bin_at(self._dB(s, T_hi), xi_b), Tu

    def classify(self, pid, ge, oe):
        """(category, detail) of package pid's first divergence; 'same' if none."""
        j = first_divergence(ge, oe)
        if j is None:
            return "same", ""
        if j >= min(len(ge), len(oe)):
            return "unexplained", f"event lists of different length agree up to {j}"
        g, o = ge[j], oe[j]
        gp, op = np.asarray(g["pos"], np.float64), np.asarray(o["pos"], np.float64)
        kg, ko = int(g["kind"]), int(o["kind"])
        where = f"event {j}: gpu {KINDS[kg]} cell {int(g['leaf'])} bin {int(g['bin'])}, " \
                f"oracle {KINDS[ko]} cell {int(o['leaf'])} bin {int(o['bin'])}"
        if j == 0:  # the emission bin from the stellar spectrum
            w = np.array([oracle.planck_bin(self.nu[b], self.nu[b + 1], self.m.star.T)
                          for b in range(self.m.n_bins)])
            x = _deviates(self.seed, pid, 0, 0)[0]
            return ("decision tie", where) if _cum_tie(w, x) else ("unexplained", where)
        b_prev = int(oe["bin"][j - 1])
        leaf = int(o["leaf"])
        prev = np.asarray(oe["pos"][j - 1], np.float64)
        tol = self._tau_tol(leaf, op, prev, b_prev)
        dist = float(np.abs(gp - op).max())
        same_point = dist <= POS_TOL or dist * self._kx(leaf, b_prev) <= tol
        if same_point and int(g["leaf"]) == leaf and kg in (1, 2) and ko in (1, 2):
            w0 = _deviates(self.seed, pid, j, 0)
            w1 = _deviates(self.seed, pid, j, 1)
            rho = self.m.rho[:, leaf]
            kext = float(rho @ self.kext[:, b_prev])
            ksca = float(rho @ self.ksca[:, b_prev])
            if kg != ko:  # scatter or absorb
                tie = abs(w0[0] * kext - ksca) <= REL_TIE * kext
                return ("decision tie", where + " (albedo)") if tie else ("unexplained", where)
            s = int(o["species"])
            if kg == 2 and int(g["species"]) != s:
                tie = _cum_tie(rho * self.kabs[:, b_prev], w0[1])
                return ("decision tie", where + " (species)") if tie else ("unexplained", where)
            if kg == 2 and s in self.pah_of:
                w = self.om.pah_template[self.pah_of[s]]
                tie = _cum_tie(w, w1[2])
                return ("decision tie", where + " (PAH bin)") if tie else ("unexplained", where)
            if kg == 2:
                blo, bhi, Tu = self._table_bins(s, leaf, w1[1], w1[2])
                ok = min(blo, bhi) <= int(g["bin"]) <= max(blo, bhi)
                detail = where + f" (T_u {Tu:.2f} K, table bins {blo}..{bhi})"
                return ("re-emission table", detail) if ok else ("unexplained", detail)
        # the walk: an interaction point at a face of its cell, or a point on a shared face
        for k, p, lf in ((kg, gp, int(g["leaf"])), (ko, op, int(o["leaf"]))):
            if k in (1, 2) and self._tau_to_face(lf, p, b_prev) <= \
                    self._tau_tol(lf, p, prev, b_prev):
                return "face", where
        if same_point and self._dist_to_box(leaf, gp) <= POS_TOL and \
                self._dist_to_box(int(g["leaf"]), op) <= POS_TOL:
            return "face", where + " (point on a shared face)"
        return "unexplained", where


def explain(grid, model, ids, T_frozen, seed, n_total, om=None, max_out=1 << 16):
    """Classify the first divergence of every listed package (GPU event replay
    through the library against the oracle's). Returns {category: count} and the
    unexplained cases."""
    cl = Classifier(model, T_frozen, seed, om=om)
    gev, gn = grid.trace_events(ids, seed=seed, max_out=max_out)
    out, bad = {}, []
    for i, pid in enumerate(np.asarray(ids, dtype=np.uint64)):
        oev, on = oracle.trace_events(cl.om, int(pid), cl.Tf, seed=seed, n_total=n_total,
                                      max_out=max_out)
        cat, detail = cl.classify(int(pid), gev[i], oev)
        if cat == "same":
            if gn[i] > max_out or on > max_out:
                cat, detail = "unexplained", f"diverges beyond the first {max_out} events"
            else:  # the summaries differ in the cells crossed only
                cat = "edge crossing"
        out[cat] = out.get(cat, 0) + 1
        if cat == "unexplained":
            bad.append((int(pid), detail))
    return out, bad
