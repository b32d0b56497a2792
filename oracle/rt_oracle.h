/*
 * rt_oracle.h -- plain, slow FP64 CPU reference of Monte Carlo dust radiative
 * transfer with photon packages of constant energy (Siebenmorgen, Heymann &
 * Kruegel, Sec. 2), used to check the CUDA library.
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may call this code; the library's product path never does.
 * It shares no source with the CUDA library: its Philox generator, Planck
 * integrals, cell walk, samplers and temperature inversion are written here
 * independently.
 *
 * Units are cgs. Positions on the grid are measured in base-cube units
 * (0 .. n_base per axis); the domain is [-half_size, half_size]^3 cm.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MODE_BW = 0, ORC_MODE_NOCORR = 1, ORC_MODE_FROZEN = 2 };
enum { ORC_SOURCE_POINT = 0, ORC_SOURCE_BEAM = 1 };

typedef struct {
    double half_size;          /* cm */
    int32_t n_base, max_level;
    const int32_t *base;       /* [n^3], ix + n*(iy + n*iz); >=0 leaf, <0 -(block+1) */
    const int32_t *child;      /* [n_blocks*8], octant = ox | oy<<1 | oz<<2 */
    int64_t n_blocks, n_leaves;
    int32_t n_species, n_bins;
    const double *rho;         /* [S][N] g/cm^3 */
    const double *kabs;        /* [S][B] cm^2/g */
    const double *ksca;        /* [S][B] cm^2/g */
    const double *g;           /* [S][B] Henyey-Greenstein asymmetry */
    const double *nu_edges;    /* [B+1] Hz ascending */
    double star_T, star_L;     /* K, erg/s */
    double star_pos[3];        /* cm */
    int32_t source_kind, n_sed_dirs;
    double beam_dir[3];
    /* PAH species (may be absent): pah_index[s] = PAH number of species s or -1;
     * an absorption by a PAH is tallied in its cell's coarse absorbed spectrum and
     * re-emitted from that PAH's template spectrum (weights per bin) */
    const int32_t *pah_index;  /* [S] or NULL */
    const double *pah_template;/* [n_pah][B] */
    int32_t n_coarse, n_pah;
    /* per-cell PAH re-emission spectra (may be absent): [n_pah][N][B] weights; a
     * cell whose row sums to zero re-emits from the template */
    const double *pah_cell_w;
} orc_model;

typedef struct {
    uint64_t seed;
    uint64_t first_id, n_packages;
    uint64_t n_total;          /* packages sharing the source luminosity */
    int32_t mode, pad;
    uint64_t max_events;       /* interaction cap per package */
    double t_min;              /* temperature floor of the no-correction mode */
    const double *T_frozen;    /* [S][N] for the frozen-temperature mode */
    /* peel-off toward a distant observer (may be absent: n_planes = 0) */
    double obs_dir[3];         /* unit vector from the model to the observer */
    const int32_t *plane_of_bin; /* [B]: image plane of each bin, -1 for none */
    int32_t n_planes, nx, ny, pad2;
    double img_half;           /* half width of the square image, cm */
} orc_run;

typedef struct {
    uint64_t *count;           /* [S][N] absorption counts, accumulated */
    uint64_t *sed;             /* [2][n_dir][B]: all escaped / escaped uncollided */
    uint64_t *pahabs;          /* [n_pah][N][n_coarse] PAH absorptions, or NULL */
    double *pathabs;           /* [S][N] Lucy path-length sums of rho kappa_abs l, or NULL */
    double *image;             /* [n_planes][ny][nx] peel-off images, erg/s/sr, or NULL */
    uint64_t emitted, escaped, capped, absorptions, scatters, crossings, errors;
} orc_tally;

typedef struct {               /* one package's history (frozen mode replay) */
    uint64_t id;
    uint64_t events, absorptions, scatters, crossings;
    int32_t escaped, capped, final_bin, dir_bin;
    int64_t last_leaf;
    double dir[3];
} orc_trace_rec;

typedef struct {               /* one event of a package's history (frozen mode replay) */
    int32_t kind;              /* 0 emission, 1 scattering, 2 absorption, 3 escape,
                                  4 capped */
    int32_t species;           /* interacting species, -1 at the end */
    int64_t leaf;              /* cell of the event (at the end: the last cell) */
    int32_t bin;               /* frequency bin after the event */
    int32_t pad;
    double pos[3];             /* position, base-cube units */
} orc_event;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t x);
double orc_planck_bin(double nu0, double nu1, double T);
double orc_dplanck_bin(double nu0, double nu1, double T);
double orc_emission_per_mass(const double *kabs, const double *nu_edges, int n_bins,
                             double T);
double orc_temperature(const double *kabs, const double *nu_edges, int n_bins, double u);
double orc_hg_mu(double g, double xi);
void orc_rotate(double d[3], double mu, double phi);
int orc_locate(const orc_model *m, const double p[3], const double d[3], int64_t out[5]);
int64_t orc_ray_cells(const orc_model *m, const double p0[3], const double d0[3],
                      int64_t max_cells, int64_t *leaves, double *lengths);
double orc_package_energy(const orc_model *m, uint64_t n_total);
double orc_optical_depth(const orc_model *m, const double p_cm[3], const double dir[3], int bin);
int orc_transport(const orc_model *m, const orc_run *r, orc_tally *t);
int orc_trace(const orc_model *m, const orc_run *r, const uint64_t *ids, int64_t n,
              orc_trace_rec *out);
/* The events of package `id` in the frozen mode: at most max_out are written to
 * ev, *n_out receives the number the history has (it may exceed max_out). */
int orc_trace_events(const orc_model *m, const orc_run *r, uint64_t id, int64_t max_out,
                     orc_event *ev, int64_t *n_out);
int orc_temperatures(const orc_model *m, const uint64_t *count, double eps, double *T_out);
int orc_reemit_bin(const orc_model *m, int species, int mode, uint64_t n, double eps_over_m,
                   double u_frozen, double t_min, double xi_u, double xi_bin);

#ifdef __cplusplus
}
#endif
#endif
