/*
 * rt_oracle.c -- plain FP64 CPU reference of the photon-package Monte Carlo of
 * Siebenmorgen, Heymann & Kruegel, Sec. 2.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library's product path. It shares
 * no code with the CUDA library.
 *
 * One package at a time, in the order Sec. 2 tells it:
 *   1. the star emits a package of constant energy eps at a frequency drawn from
 *      its spectrum;
 *   2. entering a cell, the package may interact there; the interaction
 *      probability follows the extinction optical depth along the path inside
 *      the cell (optical-depth sampling, tau = -ln xi);
 *   3. a scattered package only changes direction, by the phase function
 *      (Henyey-Greenstein);
 *   4. an absorbed package is replaced by one of the same energy, emitted
 *      isotropically from the absorption spot at a new frequency;
 *   5. every absorption raises the cell's energy by eps (an integer count), and
 *      with it the cell's temperature.
 * The new frequency follows one of three rules (Sec. 2 on the correction of
 * Bjorkman & Wood 2001):
 *   BW      difference spectrum kappa_abs * [B(T(n+1)) - B(T(n))], T(n) the
 *           temperature after n absorptions of the cell's species;
 *   NOCORR  kappa_abs * B(T(n)), the temperature before the absorption, with no
 *           correction (T(0) replaced by a floor t_min);
 *   FROZEN  kappa_abs * B(T_frozen), a fixed per-cell temperature.
 * Each spectrum is sampled as an exact mixture: kappa*[B(T_b)-B(T_a)] equals the
 * integral over T in [T_a, T_b] of kappa * dB/dT, so drawing u uniformly in the
 * absorbed-energy interval [S(T_a), S(T_b)], setting T_u = S^-1(u) and drawing the
 * bin from kappa * dP/dT(T_u) reproduces it exactly.
 *
 * Frequencies are discrete bins; P_b(T) is the Planck function integrated over
 * bin b. The random numbers come from Philox4x32-10 (Salmon et al. 2011) with
 * key = seed and counter = (package id lo, hi, event index, block index).
 *
 * Images (Sec. 3, Fig. 2) by peel-off toward an observer at infinity along o: at
 * the emission (point source), at every scattering and at every re-emission the
 * package sends eps * w * exp(-tau) into the pixel its position projects to, with
 * w the probability per steradian of leaving toward o (1/(4 pi) when isotropic, the
 * Henyey-Greenstein phase function at the angle between the incoming direction and
 * o when scattered) and tau the extinction optical depth from the event to the
 * boundary along o at the outgoing frequency. The package's own path is unchanged.
 */
#include "rt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 exact / recommended values, cgs */
#define H_PLANCK 6.62607015e-27
#define K_BOLTZ 1.380649e-16
#define C_LIGHT 2.99792458e10
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------ Philox */
/* Philox4x32 with 10 rounds: each round multiplies counter words 0 and 2 by the
 * published constants, mixes the high halves with words 1, 3 and the round key,
 * and the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 32-bit word -> uniform deviate in the open interval (0,1): the top 23 bits
 * select one of 2^23 equal sub-intervals and the deviate is its midpoint. */
double orc_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

static void draw_block(const uint32_t key[2], uint64_t id, uint32_t event, uint32_t blk,
                       double u[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), event, blk};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = orc_uniform(w[i]);
}

/* ------------------------------------------------------------ Planck integrals */
/* Gauss-Legendre nodes on [-1,1], found by Newton iteration on P_16. */
#define NGL 16
static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;

static void legendre(double x, double *pn, double *dpn)
{
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= NGL; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *dpn = NGL * (x * p1 - p0) / (x * x - 1.0);
}

static void gl_init(void)
{
    if (gl_ready) return;
    for (int i = 0; i < NGL; ++i) {
        double x = cos(PI * (i + 0.75) / (NGL + 0.5)), pn, dpn;
        for (int it = 0; it < 100; ++it) {
            legendre(x, &pn, &dpn);
            double dx = pn / dpn;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        legendre(x, &pn, &dpn);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
    }
    gl_ready = 1;
}

/* B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1), erg s^-1 cm^-2 Hz^-1 sr^-1 */
static double planck_nu(double nu, double T)
{
    if (!(T > 0.0)) return 0.0;
    double x = H_PLANCK * nu / (K_BOLTZ * T);
    double em = exp(-x);
    return 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT) * em / (-expm1(-x));
}

/* dB_nu/dT */
static double dplanck_nu(double nu, double T)
{
    if (!(T > 0.0)) return 0.0;
    double x = H_PLANCK * nu / (K_BOLTZ * T);
    double em = exp(-x);
    double den = -expm1(-x);
    return 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT) * (x / T) * em / (den * den);
}

/* integral of f(nu) over [nu0, nu1] by composite 16-point Gauss-Legendre in ln(nu),
 * panels no wider than 0.25 in ln(nu) */
static double bin_integral(double nu0, double nu1, double T, int deriv)
{
    gl_init();
    double a = log(nu0), b = log(nu1);
    int np = (int)ceil((b - a) / 0.25);
    if (np < 1) np = 1;
    double h = (b - a) / np, s = 0.0;
    for (int p = 0; p < np; ++p) {
        double mid = a + (p + 0.5) * h, half = 0.5 * h;
        for (int i = 0; i < NGL; ++i) {
            double nu = exp(mid + half * gl_x[i]);
            double f = deriv ? dplanck_nu(nu, T) : planck_nu(nu, T);
            s += gl_w[i] * half * f * nu; /* d nu = nu d ln nu */
        }
    }
    return s;
}

/* P_b(T): Planck function integrated over one frequency bin */
double orc_planck_bin(double nu0, double nu1, double T) { return bin_integral(nu0, nu1, T, 0); }

/* dP_b/dT */
double orc_dplanck_bin(double nu0, double nu1, double T) { return bin_integral(nu0, nu1, T, 1); }

/* S(T) = 4 pi sum_b kappa_abs(b) P_b(T): power emitted per gram at temperature T
 * (erg s^-1 g^-1); radiative equilibrium sets it equal to the absorbed power. */
double orc_emission_per_mass(const double *kabs, const double *nu, int nb, double T)
{
    double s = 0.0;
    for (int b = 0; b < nb; ++b)
        if (kabs[b] > 0.0) s += kabs[b] * orc_planck_bin(nu[b], nu[b + 1], T);
    return 4.0 * PI * s;
}

/* S(T) and dS/dT together (one pass over the quadrature nodes) */
static void emission_and_slope(const double *kabs, const double *nu, int nb, double T,
                               double *S, double *dS)
{
    gl_init();
    double s = 0.0, ds = 0.0;
    if (T > 0.0) {
        for (int b = 0; b < nb; ++b) {
            if (!(kabs[b] > 0.0)) continue;
            double a0 = log(nu[b]), a1 = log(nu[b + 1]);
            int np = (int)ceil((a1 - a0) / 0.25);
            if (np < 1) np = 1;
            double h = (a1 - a0) / np, pb = 0.0, dpb = 0.0;
            for (int p = 0; p < np; ++p) {
                double mid = a0 + (p + 0.5) * h, half = 0.5 * h;
                for (int i = 0; i < NGL; ++i) {
                    double f = exp(mid + half * gl_x[i]);
                    double x = H_PLANCK * f / (K_BOLTZ * T);
                    double em = exp(-x), den = -expm1(-x);
                    double bnu = 2.0 * H_PLANCK * f * f * f / (C_LIGHT * C_LIGHT) * em / den;
                    pb += gl_w[i] * half * bnu * f;
                    dpb += gl_w[i] * half * bnu * (x / T) / den * f;
                }
            }
            s += kabs[b] * pb;
            ds += kabs[b] * dpb;
        }
    }
    *S = 4.0 * PI * s;
    *dS = 4.0 * PI * ds;
}

/* T = S^-1(u): Newton on ln S against ln T (S is close to a power of T), kept
 * inside a bracket [lo, hi] that every evaluation tightens; bisection or doubling
 * whenever a Newton step would leave it. Converged to 1e-14 relative. */
double orc_temperature(const double *kabs, const double *nu, int nb, double u)
{
    if (!(u > 0.0)) return 0.0;
    double lo = 0.0, hi = INFINITY, T = 100.0;
    for (int it = 0; it < 500; ++it) {
        double S, dS;
        emission_and_slope(kabs, nu, nb, T, &S, &dS);
        if (S == u) return T;
        if (S > u) hi = T; else lo = T;
        double Tn;
        if (S > 0.0 && dS > 0.0)
            Tn = T * exp(-(log(S) - log(u)) * S / (T * dS));
        else
            Tn = 2.0 * T;
        if (!(Tn > lo && Tn < hi)) Tn = isinf(hi) ? 2.0 * T : 0.5 * (lo + hi);
        if (fabs(Tn - T) <= 1e-14 * T) return Tn;
        T = Tn;
        if (T > 1e9) return T;
    }
    return T;
}

/* ------------------------------------------------------------ scattering */
/* Henyey-Greenstein: invert the cumulative distribution of mu = cos(theta). */
double orc_hg_mu(double g, double xi)
{
    if (fabs(g) < 1e-6) return 2.0 * xi - 1.0;
    double f = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
    double mu = (1.0 + g * g - f * f) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* Turn unit vector d by polar angle acos(mu) and azimuth phi. The azimuth is
 * counted from e1 = (dx dz, dy dz, -(1-dz^2))/sqrt(1-dz^2) towards
 * e2 = (-dy, dx, 0)/sqrt(1-dz^2); near the poles from the x axis towards y. */
void orc_rotate(double d[3], double mu, double phi)
{
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    double cp = cos(phi), sp = sin(phi);
    double ux = d[0], uy = d[1], uz = d[2];
    double nx, ny, nz;
    if (fabs(uz) > 0.99999) {
        nx = s * cp;
        ny = s * sp;
        nz = (uz > 0 ? 1.0 : -1.0) * mu;
    } else {
        double r = sqrt(1.0 - uz * uz);
        nx = mu * ux + s * (ux * uz * cp - uy * sp) / r;
        ny = mu * uy + s * (uy * uz * cp + ux * sp) / r;
        nz = mu * uz - s * r * cp;
    }
    double nrm = sqrt(nx * nx + ny * ny + nz * nz);
    d[0] = nx / nrm; d[1] = ny / nrm; d[2] = nz / nrm;
}

static void isotropic(double xi_mu, double xi_phi, double d[3])
{
    double mu = 2.0 * xi_mu - 1.0;
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    double phi = 2.0 * PI * xi_phi;
    d[0] = s * cos(phi);
    d[1] = s * sin(phi);
    d[2] = mu;
}

/* first index whose running sum exceeds xi * total (inverse cumulative) */
static int sample_discrete(const double *w, int n, double xi)
{
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += w[i];
    if (!(tot > 0.0)) return 0;
    double target = xi * tot, cum = 0.0;
    for (int i = 0; i < n; ++i) {
        cum += w[i];
        if (cum > target) return i;
    }
    for (int i = n - 1; i >= 0; --i)
        if (w[i] > 0.0) return i;
    return 0;
}

/* ------------------------------------------------------------ grid */
/* Index of the cell holding coordinate q when moving with direction component d:
 * on a face (q integral) the cell ahead is taken. */
static int64_t dirfloor(double q, double d)
{
    double f = floor(q);
    if (d < 0.0 && f == q) return (int64_t)f - 1;
    return (int64_t)f;
}

/* Find the leaf holding point p (base-cube units) for a package moving along d:
 * base cube first, then down the 2x2x2 subcubes. out = {leaf, level, i, j, k}
 * with (i, j, k) the leaf's integer corner at its level. Returns 0 inside, 1
 * outside the domain, -1 on a malformed tree. */
int orc_locate(const orc_model *m, const double p[3], const double d[3], int64_t out[5])
{
    int64_t n = m->n_base, I[3];
    for (int a = 0; a < 3; ++a) {
        I[a] = dirfloor(p[a], d[a]);
        if (I[a] < 0 || I[a] >= n) return 1;
    }
    int64_t node = m->base[I[0] + n * (I[1] + n * I[2])];
    int level = 0;
    while (node < 0) {
        int64_t blk = -node - 1;
        if (blk >= m->n_blocks || level >= m->max_level) return -1;
        ++level;
        double sc = ldexp(1.0, level);
        int oct = 0;
        for (int a = 0; a < 3; ++a) {
            int64_t J = dirfloor(p[a] * sc, d[a]);
            int64_t o = J - 2 * I[a];
            if (o < 0 || o > 1) return -1;
            oct |= (int)o << a;
            I[a] = J;
        }
        node = m->child[blk * 8 + oct];
    }
    if (node >= m->n_leaves) return -1;
    out[0] = node; out[1] = level; out[2] = I[0]; out[3] = I[1]; out[4] = I[2];
    return 0;
}

/* Distance (base-cube units) from p along d to the leaf's boundary, and the axis
 * whose face is hit first (lowest axis on ties). */
static double exit_distance(const double p[3], const double d[3], const double lo[3],
                            const double hi[3], int *axis)
{
    double best = INFINITY;
    int ax = 0;
    for (int a = 0; a < 3; ++a) {
        double t;
        if (d[a] > 0.0) t = (hi[a] - p[a]) / d[a];
        else if (d[a] < 0.0) t = (lo[a] - p[a]) / d[a];
        else continue;
        if (t < best) { best = t; ax = a; }
    }
    *axis = ax;
    return best < 0.0 ? 0.0 : best;
}

static void clamp3(double p[3], const double lo[3], const double hi[3])
{
    for (int a = 0; a < 3; ++a) {
        if (p[a] < lo[a]) p[a] = lo[a];
        if (p[a] > hi[a]) p[a] = hi[a];
    }
}

static void leaf_box(const int64_t c[5], double lo[3], double hi[3])
{
    double sz = ldexp(1.0, -(int)c[1]);
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)c[2 + a] * sz;
        hi[a] = lo[a] + sz;
    }
}

/* Free flight without interactions: the leaves a ray crosses and the path length
 * (base-cube units) inside each. Returns the number of leaves, -1 on error. */
int64_t orc_ray_cells(const orc_model *m, const double p0[3], const double d0[3],
                      int64_t max_cells, int64_t *leaves, double *lengths)
{
    double p[3] = {p0[0], p0[1], p0[2]}, d[3] = {d0[0], d0[1], d0[2]};
    int64_t k = 0;
    for (;;) {
        int64_t c[5];
        int rc = orc_locate(m, p, d, c);
        if (rc == 1) return k;
        if (rc < 0 || k >= max_cells) return -1;
        double lo[3], hi[3];
        leaf_box(c, lo, hi);
        int ax;
        double t = exit_distance(p, d, lo, hi, &ax);
        leaves[k] = c[0];
        lengths[k] = t;
        ++k;
        for (int a = 0; a < 3; ++a) p[a] += t * d[a];
        p[ax] = d[ax] > 0.0 ? hi[ax] : lo[ax];
        clamp3(p, lo, hi);
    }
}

/* ------------------------------------------------------------ transport */
typedef struct {
    double d0;            /* base cube edge, cm */
    double eps;           /* package energy (luminosity share), erg/s */
    double *star_w;       /* [B] stellar bin weights P_b(T*) */
    double *kext;         /* [S][B] */
    double src[3];        /* source position, base-cube units */
    double beam[3];
    uint32_t key[2];
} ctx_t;

double orc_package_energy(const orc_model *m, uint64_t n_total)
{
    /* eps = L_in_range / N: the star's luminosity inside the frequency grid,
     * L * pi sum_b P_b(T*) / (sigma T*^4), shared by all packages. sigma is
     * written through its Planck-law expression 2 pi^5 k^4 / (15 c^2 h^3). */
    double sigma = 2.0 * pow(PI, 5) * pow(K_BOLTZ, 4) /
                   (15.0 * C_LIGHT * C_LIGHT * pow(H_PLANCK, 3));
    double s = 0.0;
    for (int b = 0; b < m->n_bins; ++b)
        s += orc_planck_bin(m->nu_edges[b], m->nu_edges[b + 1], m->star_T);
    double frac = PI * s / (sigma * pow(m->star_T, 4));
    return m->star_L * frac / (double)n_total;
}

static int ctx_init(const orc_model *m, const orc_run *r, ctx_t *c)
{
    int S = m->n_species, B = m->n_bins;
    c->d0 = 2.0 * m->half_size / (double)m->n_base;
    c->eps = orc_package_energy(m, r->n_total ? r->n_total : 1);
    c->star_w = (double *)malloc(sizeof(double) * B);
    c->kext = (double *)malloc(sizeof(double) * S * B);
    if (!c->star_w || !c->kext) return -1;
    for (int b = 0; b < B; ++b)
        c->star_w[b] = orc_planck_bin(m->nu_edges[b], m->nu_edges[b + 1], m->star_T);
    for (int i = 0; i < S * B; ++i) c->kext[i] = m->kabs[i] + m->ksca[i];
    for (int a = 0; a < 3; ++a) c->src[a] = (m->star_pos[a] + m->half_size) / c->d0;
    double bn = sqrt(m->beam_dir[0] * m->beam_dir[0] + m->beam_dir[1] * m->beam_dir[1] +
                     m->beam_dir[2] * m->beam_dir[2]);
    for (int a = 0; a < 3; ++a) c->beam[a] = bn > 0 ? m->beam_dir[a] / bn : (a == 2);
    c->key[0] = (uint32_t)r->seed;
    c->key[1] = (uint32_t)(r->seed >> 32);
    return 0;
}

static void ctx_free(ctx_t *c)
{
    free(c->star_w);
    free(c->kext);
}

/* New frequency bin after an absorption by species s (see the file header). */
int orc_reemit_bin(const orc_model *m, int s, int mode, uint64_t n, double e,
                   double u_frozen, double t_min, double xi_u, double xi_bin)
{
    const double *ka = m->kabs + (size_t)s * m->n_bins;
    const double *nu = m->nu_edges;
    int B = m->n_bins;
    double u_lo, u_hi;
    if (mode == ORC_MODE_BW) {
        u_lo = (double)n * e;
        u_hi = (double)(n + 1) * e;
    } else if (mode == ORC_MODE_NOCORR) {
        u_lo = 0.0;
        u_hi = fmax((double)n * e, orc_emission_per_mass(ka, nu, B, t_min));
    } else {
        u_lo = 0.0;
        u_hi = u_frozen;
    }
    double u = u_lo + xi_u * (u_hi - u_lo);
    double Tu = orc_temperature(ka, nu, B, u);
    double *w = (double *)malloc(sizeof(double) * (size_t)B);
    if (!w) return -1;
    for (int b = 0; b < B; ++b)
        w[b] = ka[b] > 0.0 ? ka[b] * orc_dplanck_bin(nu[b], nu[b + 1], Tu) : 0.0;
    int bin = sample_discrete(w, B, xi_bin);
    free(w);
    return bin;
}

static int sed_dir_bin(const double d[3], int ndir)
{
    int k = (int)floor(0.5 * (d[2] + 1.0) * ndir);
    if (k < 0) k = 0;
    if (k >= ndir) k = ndir - 1;
    return k;
}

/* Extinction optical depth from p (base-cube units) along d to the domain boundary
 * at bin `bin`, walking the cells like a package that never interacts. */
static double tau_to_boundary(const orc_model *m, const ctx_t *c, const double p0[3],
                              const double d[3], int bin)
{
    double p[3] = {p0[0], p0[1], p0[2]};
    const int S = m->n_species, B = m->n_bins;
    const int64_t N = m->n_leaves;
    double tau = 0.0;
    for (int guard = 0; guard < 100000000; ++guard) {
        int64_t cell[5];
        int rc = orc_locate(m, p, d, cell);
        if (rc != 0) break;
        double lo[3], hi[3];
        leaf_box(cell, lo, hi);
        int ax;
        double t = exit_distance(p, d, lo, hi, &ax);
        double k = 0.0;
        for (int s = 0; s < S; ++s) k += m->rho[(size_t)s * N + cell[0]] * c->kext[s * B + bin];
        tau += k * c->d0 * t;
        for (int a = 0; a < 3; ++a) p[a] += t * d[a];
        p[ax] = d[ax] > 0.0 ? hi[ax] : lo[ax];
        clamp3(p, lo, hi);
    }
    return tau;
}

double orc_optical_depth(const orc_model *m, const double p_cm[3], const double dir[3], int bin)
{
    orc_run r;
    memset(&r, 0, sizeof(r));
    r.n_total = 1;
    ctx_t c;
    if (ctx_init(m, &r, &c)) { ctx_free(&c); return -1.0; }
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = (p_cm[a] + m->half_size) / c.d0;
    double t = tau_to_boundary(m, &c, p, dir, bin);
    ctx_free(&c);
    return t;
}

/* Peel-off: the share w (per steradian) of the package's energy that leaves the
 * event at p toward the observer, attenuated by the line of sight, into the pixel
 * the position projects to. */
static void peel(const orc_model *m, const orc_run *r, const ctx_t *c, orc_tally *t,
                 const double p[3], int bin, double w)
{
    if (!t || !t->image || r->n_planes <= 0) return;
    int plane = r->plane_of_bin[bin];
    if (plane < 0) return;
    const double *o = r->obs_dir;
    double tau = tau_to_boundary(m, c, p, o, bin);
    /* image axes: e1 = normalise(z x o) (x when o is along z), e2 = o x e1 */
    double e1[3], e2[3];
    if (fabs(o[2]) < 0.999999) {
        double nn = sqrt(o[0] * o[0] + o[1] * o[1]);
        e1[0] = -o[1] / nn; e1[1] = o[0] / nn; e1[2] = 0.0;
    } else {
        e1[0] = 1.0; e1[1] = 0.0; e1[2] = 0.0;
    }
    e2[0] = o[1] * e1[2] - o[2] * e1[1];
    e2[1] = o[2] * e1[0] - o[0] * e1[2];
    e2[2] = o[0] * e1[1] - o[1] * e1[0];
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = p[a] * c->d0 - m->half_size;
    double u = x[0] * e1[0] + x[1] * e1[1] + x[2] * e1[2];
    double v = x[0] * e2[0] + x[1] * e2[1] + x[2] * e2[2];
    int px = (int)floor((u + r->img_half) / (2.0 * r->img_half) * r->nx);
    int py = (int)floor((v + r->img_half) / (2.0 * r->img_half) * r->ny);
    if (px < 0 || px >= r->nx || py < 0 || py >= r->ny) return;
    t->image[((size_t)plane * r->ny + py) * r->nx + px] += c->eps * w * exp(-tau);
}

/* Follow package `id` until it leaves the grid or reaches the event cap.
 * count may be NULL only in the frozen mode (trajectories then do not depend on
 * the counts). */
/* Event log of one package (trace): events beyond cap are counted, not stored. */
typedef struct {
    orc_event *ev;
    int64_t cap, n;
} event_log;

static void log_event(event_log *lg, int kind, int species, int64_t leaf, int bin,
                      const double p[3])
{
    if (!lg) return;
    if (lg->n < lg->cap) {
        orc_event *e = &lg->ev[lg->n];
        e->kind = kind;
        e->species = species;
        e->leaf = leaf;
        e->bin = bin;
        e->pad = 0;
        e->pos[0] = p[0]; e->pos[1] = p[1]; e->pos[2] = p[2];
    }
    lg->n += 1;
}

static int run_package(const orc_model *m, const orc_run *r, const ctx_t *c, uint64_t id,
                       uint64_t *count, orc_tally *t, orc_trace_rec *rec, event_log *lg)
{
    const int S = m->n_species, B = m->n_bins;
    const int64_t N = m->n_leaves;
    double u[4], v[4];
    double p[3], d[3];
    uint64_t n_ev = 0, n_abs = 0, n_sca = 0, n_cross = 0;
    int interacted = 0, escaped = 0, capped = 0, err = 0;
    int64_t last_leaf = -1;

    /* 1. emission: bin from the stellar spectrum, direction, optical depth */
    draw_block(c->key, id, 0, 0, u);
    int bin = sample_discrete(c->star_w, B, u[0]);
    if (m->source_kind == ORC_SOURCE_BEAM) {
        d[0] = c->beam[0]; d[1] = c->beam[1]; d[2] = c->beam[2];
    } else {
        isotropic(u[1], u[2], d);
    }
    double tau = -log(u[3]);
    for (int a = 0; a < 3; ++a) p[a] = c->src[a];
    log_event(lg, 0, -1, -1, bin, p);
    if (m->source_kind != ORC_SOURCE_BEAM) peel(m, r, c, t, p, bin, 1.0 / (4.0 * PI));

    for (;;) {
        int64_t cell[5];
        int rc = orc_locate(m, p, d, cell);
        if (rc == 1) { escaped = 1; break; }
        if (rc < 0) { err = 1; break; }
        int64_t leaf = cell[0];
        last_leaf = leaf;
        double lo[3], hi[3];
        leaf_box(cell, lo, hi);
        int ax;
        double tex = exit_distance(p, d, lo, hi, &ax);
        /* 2. extinction optical depth across the cell (per base-cube unit) */
        double k = 0.0;
        for (int s = 0; s < S; ++s) k += m->rho[(size_t)s * N + leaf] * c->kext[s * B + bin];
        k *= c->d0;
        double dtau = k * tex;
        if (t && t->pathabs) {
            /* Lucy (1999): the absorbed energy of a cell is eps times the sum, over
             * the segments crossing it, of rho kappa_abs times the segment length */
            double seg = (k > 0.0 && dtau > tau) ? tau / k : tex;
            for (int s = 0; s < S; ++s)
                t->pathabs[(size_t)s * N + leaf] +=
                    m->rho[(size_t)s * N + leaf] * m->kabs[s * B + bin] * seg * c->d0;
        }
        if (k > 0.0 && dtau > tau) {
            double sdist = tau / k;
            for (int a = 0; a < 3; ++a) p[a] += sdist * d[a];
            clamp3(p, lo, hi);
            ++n_ev;
            if (n_ev > r->max_events) { capped = 1; log_event(lg, 4, -1, leaf, bin, p); break; }
            interacted = 1;
            draw_block(c->key, id, (uint32_t)n_ev, 0, u);
            draw_block(c->key, id, (uint32_t)n_ev, 1, v);
            double wsca[64], wabs[64];
            double ksca = 0.0, kext = 0.0;
            for (int s = 0; s < S; ++s) {
                double rho = m->rho[(size_t)s * N + leaf];
                wsca[s] = rho * m->ksca[s * B + bin];
                wabs[s] = rho * m->kabs[s * B + bin];
                ksca += wsca[s];
                kext += rho * c->kext[s * B + bin];
            }
            if (u[0] * kext < ksca) {
                /* 3. scattering by the phase function of the scattering species */
                int s = sample_discrete(wsca, S, u[1]);
                if (t && t->image && r->n_planes > 0) {
                    /* Henyey-Greenstein probability per steradian toward the observer */
                    double gg = m->g[s * B + bin];
                    double mo = d[0] * r->obs_dir[0] + d[1] * r->obs_dir[1] + d[2] * r->obs_dir[2];
                    double w = (1.0 - gg * gg) / (4.0 * PI * pow(1.0 + gg * gg - 2.0 * gg * mo, 1.5));
                    peel(m, r, c, t, p, bin, w);
                }
                double mu = orc_hg_mu(m->g[s * B + bin], u[2]);
                orc_rotate(d, mu, 2.0 * PI * u[3]);
                ++n_sca;
                log_event(lg, 1, s, leaf, bin, p);
            } else {
                /* 4.+5. absorption: the cell's energy rises by eps; isotropic
                 * re-emission of the same energy at a new frequency */
                int s = sample_discrete(wabs, S, u[1]);
                size_t ci = (size_t)s * N + leaf;
                uint64_t n = 0;
                if (count) n = count[ci]++;
                int pa = m->pah_index ? m->pah_index[s] : -1;
                if (pa >= 0) {
                    /* PAH: the absorbed photon goes to the cell's coarse absorbed
                     * spectrum; the package leaves at a frequency from the PAH's
                     * emission spectrum in this cell (its template unless a
                     * per-cell spectrum is given) */
                    if (t && t->pahabs) {
                        int kc = (int)(((int64_t)bin * m->n_coarse) / B);
                        t->pahabs[((size_t)pa * N + leaf) * m->n_coarse + kc] += 1;
                    }
                    const double *wrow = m->pah_template + (size_t)pa * B;
                    if (m->pah_cell_w) {
                        /* the cell's own PAH emission spectrum, where one is given */
                        const double *cw = m->pah_cell_w + ((size_t)pa * N + leaf) * B;
                        double tot = 0.0;
                        for (int b = 0; b < B; ++b) tot += cw[b];
                        if (tot > 0.0) wrow = cw;
                    }
                    bin = sample_discrete(wrow, B, v[2]);
                    log_event(lg, 2, s, leaf, bin, p);
                    peel(m, r, c, t, p, bin, 1.0 / (4.0 * PI));
                    isotropic(u[2], u[3], d);
                    ++n_abs;
                    tau = -log(v[0]);
                    continue;
                }
                double mass = m->rho[ci] * pow(c->d0 * ldexp(1.0, -(int)cell[1]), 3);
                double e = c->eps / mass;
                double uf = 0.0;
                if (r->mode == ORC_MODE_FROZEN) {
                    double Tf = fmax(r->T_frozen[ci], r->t_min);
                    uf = orc_emission_per_mass(m->kabs + (size_t)s * B, m->nu_edges, B, Tf);
                }
                bin = orc_reemit_bin(m, s, r->mode, n, e, uf, r->t_min, v[1], v[2]);
                if (bin < 0) { err = 1; break; }
                log_event(lg, 2, s, leaf, bin, p);
                peel(m, r, c, t, p, bin, 1.0 / (4.0 * PI));
                isotropic(u[2], u[3], d);
                ++n_abs;
            }
            tau = -log(v[0]);
        } else {
            tau -= dtau;
            for (int a = 0; a < 3; ++a) p[a] += tex * d[a];
            p[ax] = d[ax] > 0.0 ? hi[ax] : lo[ax];
            clamp3(p, lo, hi);
            ++n_cross;
        }
    }
    if (escaped) log_event(lg, 3, -1, last_leaf, bin, p);
    int db = sed_dir_bin(d, m->n_sed_dirs);
    if (t) {
        t->emitted += 1;
        t->absorptions += n_abs;
        t->scatters += n_sca;
        t->crossings += n_cross;
        if (escaped) {
            t->escaped += 1;
            t->sed[(size_t)db * B + bin] += 1;
            if (!interacted) t->sed[(size_t)(m->n_sed_dirs + db) * B + bin] += 1;
        }
        if (capped) t->capped += 1;
        if (err) t->errors += 1;
    }
    if (rec) {
        rec->id = id;
        rec->events = n_ev;
        rec->absorptions = n_abs;
        rec->scatters = n_sca;
        rec->crossings = n_cross;
        rec->escaped = escaped;
        rec->capped = capped;
        rec->final_bin = bin;
        rec->dir_bin = db;
        rec->last_leaf = last_leaf;
        rec->dir[0] = d[0]; rec->dir[1] = d[1]; rec->dir[2] = d[2];
    }
    return err ? -1 : 0;
}

static int check_model(const orc_model *m)
{
    if (m->n_species < 1 || m->n_species > 64 || m->n_bins < 1 || m->n_base < 1 ||
        m->n_sed_dirs < 1 || m->n_leaves < 1)
        return -1;
    return 0;
}

int orc_transport(const orc_model *m, const orc_run *r, orc_tally *t)
{
    if (check_model(m)) return -1;
    if (r->mode == ORC_MODE_FROZEN && !r->T_frozen) return -1;
    ctx_t c;
    if (ctx_init(m, r, &c)) { ctx_free(&c); return -2; }
    int rc = 0;
    for (uint64_t i = 0; i < r->n_packages; ++i)
        if (run_package(m, r, &c, r->first_id + i, t->count, t, NULL, NULL)) rc = -3;
    ctx_free(&c);
    return rc;
}

int orc_trace(const orc_model *m, const orc_run *r, const uint64_t *ids, int64_t n,
              orc_trace_rec *out)
{
    if (check_model(m)) return -1;
    if (r->mode != ORC_MODE_FROZEN || !r->T_frozen) return -1;
    ctx_t c;
    if (ctx_init(m, r, &c)) { ctx_free(&c); return -2; }
    int rc = 0;
    for (int64_t i = 0; i < n; ++i)
        if (run_package(m, r, &c, ids[i], NULL, NULL, &out[i], NULL)) rc = -3;
    ctx_free(&c);
    return rc;
}

int orc_trace_events(const orc_model *m, const orc_run *r, uint64_t id, int64_t max_out,
                     orc_event *ev, int64_t *n_out)
{
    if (check_model(m)) return -1;
    if (r->mode != ORC_MODE_FROZEN || !r->T_frozen || max_out < 0) return -1;
    ctx_t c;
    if (ctx_init(m, r, &c)) { ctx_free(&c); return -2; }
    event_log lg = {ev, max_out, 0};
    int rc = run_package(m, r, &c, id, NULL, NULL, NULL, &lg) ? -3 : 0;
    *n_out = lg.n;
    ctx_free(&c);
    return rc;
}

/* Cell temperatures from the counts: n eps = M S(T), M = rho V (Sec. 2: each
 * absorption raises the cell's energy by eps, and accordingly its temperature).
 * T = 0 where nothing was absorbed or the species is absent. */
int orc_temperatures(const orc_model *m, const uint64_t *count, double eps, double *T)
{
    if (check_model(m)) return -1;
    const int64_t N = m->n_leaves;
    double d0 = 2.0 * m->half_size / (double)m->n_base;
    /* the leaf level is recovered by descending to each leaf once */
    int32_t *lev = (int32_t *)malloc(sizeof(int32_t) * N);
    if (!lev) return -2;
    for (int64_t i = 0; i < N; ++i) lev[i] = -1;
    int64_t nb = (int64_t)m->n_base * m->n_base * m->n_base;
    /* iterative walk of the tree: (node, level) stack */
    int64_t cap = 64 + 8 * (m->max_level + 1) * 8, top = 0;
    int64_t *stk = (int64_t *)malloc(sizeof(int64_t) * 2 * cap);
    if (!stk) { free(lev); return -2; }
    for (int64_t i = 0; i < nb; ++i) {
        top = 0;
        stk[0] = m->base[i]; stk[1] = 0; top = 1;
        while (top > 0) {
            --top;
            int64_t node = stk[2 * top], l = stk[2 * top + 1];
            if (node >= 0) {
                if (node < N) lev[node] = (int32_t)l;
            } else {
                int64_t blk = -node - 1;
                if (blk >= m->n_blocks) continue;
                for (int o = 0; o < 8; ++o) {
                    if (top >= cap) break;
                    stk[2 * top] = m->child[blk * 8 + o];
                    stk[2 * top + 1] = l + 1;
                    ++top;
                }
            }
        }
    }
    free(stk);
    for (int s = 0; s < m->n_species; ++s) {
        const double *ka = m->kabs + (size_t)s * m->n_bins;
        for (int64_t i = 0; i < N; ++i) {
            size_t ci = (size_t)s * N + i;
            double rho = m->rho[ci];
            if (count[ci] == 0 || !(rho > 0.0) || lev[i] < 0) { T[ci] = 0.0; continue; }
            double V = pow(d0 * ldexp(1.0, -lev[i]), 3);
            T[ci] = orc_temperature(ka, m->nu_edges, m->n_bins,
                                    (double)count[ci] * eps / (rho * V));
        }
    }
    free(lev);
    return 0;
}
