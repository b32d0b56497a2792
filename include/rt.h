/*
 * rt.h -- C ABI of librt_gb300: Monte Carlo dust radiative transfer with photon
 * packages of constant energy through a grid of cubes and subcubes, on one GB300
 * (sm_103a), after Siebenmorgen, Heymann & Kruegel, "PAH in vectorized three
 * dimensional Monte Carlo dust radiative transfer models", Sec. 2.
 *
 * Conventions shared by every entry point:
 *  - Units are cgs (cm, g, s, erg, Hz, K). The domain is the cube
 *    [-half_size_cm, half_size_cm]^3 cut into n_base^3 base cubes.
 *  - Every call returns an rt_status; nothing aborts and no C++ exception crosses
 *    the ABI. rt_status_string() names a status.
 *  - Input arrays are read during the call and copied; the caller keeps
 *    ownership. Output arrays are caller-owned; `mem` says whether a pointer is
 *    host (RT_MEM_HOST) or device (RT_MEM_DEVICE) memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    launch work are asynchronous on that stream, except where a host output is
 *    requested, in which case the call waits for its own copy.
 *  - Device-side faults of the method (a malformed tree reached by a package, a
 *    time budget exceeded) are recorded in a status word on the device; the next
 *    call that synchronises (rt_get_counters, rt_sed, a host-memory output)
 *    returns them as RT_ERR_DEVICE or RT_ERR_TIMEOUT.
 *  - A handle is used by one host thread at a time.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_grid rt_grid;

typedef enum {
    RT_OK = 0,
    RT_ERR_ARG = 1,      /* invalid argument or inconsistent sizes */
    RT_ERR_OOM = 2,      /* device or host allocation failed */
    RT_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    RT_ERR_TIMEOUT = 4,  /* a kernel stopped at its time budget; results partial */
    RT_ERR_STATE = 5,    /* call out of order (e.g. transport before rt_emit_star) */
    RT_ERR_RANGE = 6,    /* package ids beyond the planned total */
    RT_ERR_DEVICE = 7,   /* a package met a malformed tree; results invalid */
    RT_ERR_TOO_LARGE = 8 /* request exceeds a fixed maximum (see the no-alloc entry) */
} rt_status;

/* Re-emission rule after an absorption (Sec. 2, the correction of Bjorkman &
 * Wood 2001 and its omission in the vectorised code). */
enum {
    RT_REEMIT_BW = 0,     /* difference spectrum kappa_abs [B(T(n+1)) - B(T(n))] */
    RT_REEMIT_NOCORR = 1, /* kappa_abs B(T(n)), T(0) floored at t_min */
    RT_REEMIT_FROZEN = 2  /* kappa_abs B(T_frozen), per-cell temperatures given */
};

enum { RT_SOURCE_POINT = 0, RT_SOURCE_BEAM = 1 };

/* Transport kernel forms. POOL is the persistent packet pool (FP32); the PLAIN
 * forms run one thread per package with per-lane global atomics, in FP32 or FP64. */
enum { RT_KERNEL_POOL = 0, RT_KERNEL_PLAIN_F32 = 1, RT_KERNEL_PLAIN_F64 = 2 };

enum { RT_MEM_HOST = 0, RT_MEM_DEVICE = 1 };

/* How rt_pah_emission computes the emission of transiently heated PAHs. */
enum { RT_PAH_EXACT = 0, RT_PAH_SURROGATE = 1, RT_PAH_AUTO = 2 };

/* Grid of cubes and subcubes (Sec. 2: space is cut into cubes, and cubes that
 * need finer resolution are split again into subcubes, the cells).
 * base[ix + n*(iy + n*iz)] and child[8*block + (ox | oy<<1 | oz<<2)] hold a leaf id
 * (>= 0) or -(block+1) for a cube split into 2x2x2 children. Every leaf id in
 * [0, n_leaves) must appear exactly once and no path may exceed max_level. */
typedef struct rt_grid_desc {
    double half_size_cm;
    int32_t n_base;         /* base cubes per axis, 1 .. 2048 */
    int32_t max_level;      /* refinement levels, 0 .. 7 */
    int64_t n_blocks;       /* number of 2x2x2 child blocks */
    int64_t n_leaves;       /* cells (leaves) */
    const int32_t *base;    /* host, [n_base^3] */
    const int32_t *child;   /* host, [n_blocks*8]; may be NULL when n_blocks == 0 */
    int32_t n_species;      /* dust species, 1 .. 8 */
    int32_t n_bins;         /* frequency bins, 1 .. 1024 */
    const double *rho;      /* host, [n_species][n_leaves] density, g cm^-3 */
    const double *nu_edges; /* host, [n_bins+1] bin edges in Hz, ascending */
    int32_t n_sed_dirs;     /* escape direction bins in cos(theta) w.r.t. +z, >= 1 */
    int32_t n_temp;         /* temperature-table rows incl. T = 0; 0 selects 1024 */
    double t_min, t_max;    /* table range in K; 0 selects 1 K and 3000 K */
} rt_grid_desc;

typedef struct rt_run_opts {
    int32_t mode;           /* RT_REEMIT_* */
    int32_t kernel;         /* RT_KERNEL_* */
    uint64_t max_events;    /* interactions per package before it is capped; 0: 1e7 */
    int32_t blocks_per_sm;  /* pool: resident blocks per SM; 0: from occupancy */
    int32_t threads;        /* threads per block, multiple of 32; 0: 256 */
    int32_t refill_period;  /* pool: steps between refills of dead lanes; 0: 32 */
    int32_t interaction_batch; /* pool: lanes of a warp waiting at an interaction
                               point that start an interaction phase, 1..32; 0: 8 */
    double budget_s;        /* device time budget per launch in s; 0: 120 */
    int32_t estimators;     /* RT_EST_* bits: extra tallies kept during the launch */
    int32_t count_scale;    /* BW / no-correction: an absorption that finds n earlier
                               ones in its cell indexes the temperature at
                               count_scale * n (0 or 1: n). When W ranks share the
                               packages and each keeps its own counts, W makes every
                               rank's re-emission spectra telescope to the cell's
                               total in expectation; 1 leaves them at the rank's own
                               share, a W-fold underestimate of the cell's energy. */
    int32_t walk;           /* pool kernel: RT_WALK_* */
    int32_t reserved;
} rt_run_opts;

/* How the pool kernel finds the next cell. LINKED reads the leaf's face-link record
 * (one dependent read per crossing; the record also holds the densities of up to two
 * species); PATH climbs the package's own stack of the blocks on its path to the
 * common ancestor with the neighbour and descends from there, reading one row per
 * slot of the tree (every base cell and block child: a leaf's densities, or the code
 * of the block below it) -- one read per crossing, one more per level descended (no
 * link records; grids of at most 4 levels whose base cells plus 8 x blocks fit an
 * int32). Both give the same histories. AUTO takes the path walk for four species,
 * and for any species count when the link records exceed 4 GB: its randomly read
 * array, (n^3 + 8 n_blocks) x S floats, is smaller, which costs less address
 * translation on large grids. */
enum { RT_WALK_AUTO = 0, RT_WALK_LINKED = 1, RT_WALK_PATH = 2 };

/* Lucy (1999) path-length estimator: every cell segment a package crosses adds
 * rho_s kappa_abs,s(bin) * length (an absorption optical depth) to its cell and
 * species; eps times that sum is the cell's absorbed power, with far less variance
 * than the absorption counts in optically thin cells. */
enum { RT_EST_PATHLENGTH = 1 };

typedef struct rt_counters {
    uint64_t emitted, escaped, capped, absorptions, scatters, crossings, errors;
    uint64_t clamped;       /* absorptions whose energy lay beyond the table's t_max */
    uint64_t levels;        /* tree reads below the base cubes: for the linked and plain
                               walks the sum of the refinement levels of the cells
                               entered; for the path walk the block-slot rows read */
    uint64_t peel_events;   /* scatterings and re-emissions sent toward the observer */
    uint64_t peel_crossings;/* cells crossed by their sight lines (and the source's) */
    uint64_t peel_dropped;  /* events beyond the event buffer's capacity (not imaged) */
} rt_counters;

/* Create a grid handle: copies the tree and densities to the device and walks the
 * tree there, level by level, to find every leaf's level and corner and build its
 * face links (deferred to the first call that reads them -- a linked-walk transport,
 * peel-off images, a replay, a batch -- when the automatic walk is the path walk).
 * The path walk's slot rows are built here when it is the automatic walk, else by
 * the first transport that takes it (which then synchronises). RT_ERR_ARG when a
 * leaf or block is reached twice or never, an id is out of range, a block lies at
 * max_level or deeper, or a density is negative or not finite. Synchronises. */
rt_status rt_grid_create(const rt_grid_desc *d, rt_grid **out);

/* Release every resource of the handle. NULL is accepted. */
rt_status rt_grid_destroy(rt_grid *g);

/* Dust species `species` (0-based): absorption and scattering opacities per bin
 * (cm^2 per gram of that species) and the Henyey-Greenstein asymmetry per bin
 * (Sec. 1-2). is_pah / n_carbon tag PAH species. Host arrays of n_bins. */
rt_status rt_set_dust(rt_grid *g, int species, const double *kabs, const double *ksca,
                      const double *g_hg, int n_bins, int is_pah, int n_carbon);

/* The source (Sec. 2: the star sends out packages that all carry the same energy
 * eps but differ in frequency):
 * a blackbody of temperature T_star (K) and luminosity L_star (erg/s) at pos_cm,
 * emitting isotropically (RT_SOURCE_POINT) or along beam_dir (RT_SOURCE_BEAM).
 * Every package carries eps = L_in / n_packages_total, L_in the part of L_star
 * inside the frequency grid. */
rt_status rt_emit_star(rt_grid *g, double T_star, double L_star, const double pos_cm[3],
                       int source_kind, const double beam_dir[3], uint64_t n_packages_total);

/* Per-cell temperatures [n_species][n_leaves] (K) for RT_REEMIT_FROZEN. */
rt_status rt_set_frozen_temperatures(rt_grid *g, const float *T, int mem, void *stream);

/* Follow packages first_package_id .. first_package_id + n_packages - 1 (Sec. 2:
 * optical-depth sampling cell by cell, Henyey-Greenstein scattering, absorption
 * with isotropic re-emission at nu_new, each absorption adding eps to its cell).
 * Package k draws its random numbers from Philox4x32-10 with key = seed and
 * counter (k, event, block), so ranges may be run in any order or split across
 * calls. Absorption counts and the escaped spectrum accumulate across calls
 * until rt_reset. o may be NULL (defaults). Asynchronous on `stream`. */
rt_status rt_transport(rt_grid *g, uint64_t n_packages, uint64_t seed,
                       uint64_t first_package_id, const rt_run_opts *o, void *stream);

/* Zero the counts, the escaped spectrum and the counters. */
rt_status rt_reset(rt_grid *g, void *stream);

/* Cell temperatures [n_species][n_leaves] (K) from the counts (Sec. 2: every
 * absorption adds eps to the cell's energy, which sets its temperature):
 * n eps = rho V 4 pi sum_b kappa_abs(b) P_b(T), inverted in FP64. Cells without
 * absorptions (or without the species) get 0. */
rt_status rt_cell_temperatures(rt_grid *g, float *T_out, int mem, void *stream);

/* Temperatures [n_species][n_leaves] from the path-length tallies instead of the
 * counts: eps * sum = M S(T) (launches with RT_EST_PATHLENGTH since the last reset). */
rt_status rt_cell_temperatures_pathlength(rt_grid *g, float *T_out, int mem, void *stream);

/* The raw path-length tallies [n_species][n_leaves] (absorption optical depth). */
rt_status rt_pathlength(rt_grid *g, float *out, int mem, void *stream);

/* Escaped packages per direction and frequency bin, [2][n_sed_dirs][n_bins]:
 * index 0 counts all escaped packages, index 1 those that never interacted.
 * eps_out (may be NULL) receives the package energy in erg/s. The spectrum's
 * luminosity per bin is count * eps. */
rt_status rt_sed(rt_grid *g, uint64_t *counts_out, int mem, double *eps_out, void *stream);

/* Raw absorption counts [n_species][n_leaves]. */
rt_status rt_counts(rt_grid *g, uint64_t *out, int mem, void *stream);

/* Replace the absorption counts [n_species][n_leaves] (resuming from a checkpoint,
 * or loading counts summed over several package ranges, e.g. over ranks). */
rt_status rt_set_counts(rt_grid *g, const uint64_t *in, int mem, void *stream);

/* Package totals accumulated since the last reset; synchronises the handle's
 * last stream and reports device-side faults. */
rt_status rt_get_counters(rt_grid *g, rt_counters *out);

/* ---------------------------------------------------------------------------
 * Peel-off images (Sec. 3, Fig. 2: images of the model at chosen wavelengths and
 * flux profiles along the disk's major axis, seen from a distant observer).
 * While images are set, every pool-kernel launch also sends toward the observer,
 * from each point-source emission, scattering and re-emission whose (outgoing) bin
 * has an image plane, the share of the package energy per steradian that leaves
 * in the observer's direction -- 1/(4 pi) for isotropic emission, the
 * Henyey-Greenstein phase function of the scattering species at the scattering
 * angle for a scattering -- attenuated by exp(-tau) along the sight line to the
 * boundary, into the pixel the event's position projects to. The image is the
 * observed intensity integrated over each pixel: erg/s/sr per pixel (divide by the
 * squared distance for the flux). The packages' own paths are unchanged.
 * A launch records its events in a device buffer (20 bytes each) and a second
 * kernel traces their sight lines; events beyond the buffer's capacity are counted
 * as dropped and not imaged.
 * ------------------------------------------------------------------------- */
typedef struct rt_image_desc {
    double obs_dir[3];      /* direction from the model toward the observer (normalised
                               here). Image axes: u along normalise(z x o) (x when o
                               lies along z), v = o x u; pixel (ix, iy) holds
                               u in [-h + ix 2h/nx, ...), v likewise with ny. */
    int32_t nx, ny;         /* pixels (1 .. 16384 each) */
    double half_width_cm;   /* h: the images span [-h, h]^2 around the model centre */
    double tau_max;         /* sight lines deeper than this add nothing (0: 40) */
    uint64_t event_capacity;/* events one transport launch can record (0: 2^24; at
                               most 2^31) */
} rt_image_desc;

/* Set (or, with d == NULL, remove) the images: plane_of_bin (host, [n_bins]) gives
 * each bin's image plane or -1; the planes are 0 .. max(plane_of_bin), all nx by
 * ny. Allocates the images and zeroes them; rt_reset zeroes them too. While set,
 * only the pool kernel may transport (plain kernels: RT_ERR_STATE) and the grid
 * cannot join a batch (RT_ERR_STATE). RT_ERR_TOO_LARGE beyond 2^28 pixels in all. */
rt_status rt_set_images(rt_grid *g, const rt_image_desc *d, const int32_t *plane_of_bin);

/* The images, [n_planes][ny][nx] doubles in erg/s/sr per pixel (scaled by the
 * current package energy eps). mem: where `out` lives; a host copy synchronises and
 * returns RT_ERR_RANGE (after copying) when events were dropped since the last reset
 * (rt_get_counters reports them in either case). */
rt_status rt_images(rt_grid *g, double *out, int mem, void *stream);

/* Profile along the image's u axis (the major axis of a disk in the z = 0 plane
 * seen inclined about the x axis): out[ix] = mean over the rows whose centres lie
 * within half_rows pixels of the centre line of (plane_a - plane_b), plane_b = -1
 * for none (a dual-band difference otherwise). nx doubles, erg/s/sr per pixel. */
rt_status rt_image_profile(rt_grid *g, int plane_a, int plane_b, int half_rows, double *out,
                           int mem, void *stream);

/* ---------------------------------------------------------------------------
 * Batches: many models (grids) of uneven size, optical depth and package count in
 * one persistent launch. Warps take chunks of `chunk` packages (model, index range)
 * from a device queue, interleaved over the models, and run the packet pool on the
 * chunk's model. The plan holds every device array the launch needs, so running it
 * allocates nothing and can be captured in a CUDA graph.
 * ------------------------------------------------------------------------- */
typedef struct rt_batch rt_batch;

/* Plan packages 0 .. n_packages[m]-1 of every grid m (seed + m keys model m's Philox
 * streams; o: as rt_transport, pool kernel only, o->threads the threads per block
 * of the batched launch; chunk 0: 4096). Builds missing
 * tables (synchronising) and allocates the plan's device arrays. The grids must
 * outlive the plan and stay on the current device. */
rt_status rt_batch_create(rt_grid *const *grids, int n, const uint64_t *n_packages,
                          uint64_t seed, const rt_run_opts *o, uint64_t chunk, rt_batch **out);
rt_status rt_batch_destroy(rt_batch *b);

/* One pass: optionally zero every grid's tallies (reset), the batched transport
 * launch, and optionally every grid's temperatures into a buffer of the grid
 * (read with rt_batch_temperatures). Asynchronous on `stream`. */
rt_status rt_batch_run(rt_batch *b, int reset, int temperatures, void *stream);

/* rt_batch_run(b, 1, 1, .) recorded once into a CUDA graph (on a stream of the
 * plan's own), then launched on `stream`; later calls replay the graph. */
rt_status rt_batch_run_graph(rt_batch *b, void *stream);

/* Temperatures [n_species][n_leaves] of model `model` from the last run. */
rt_status rt_batch_temperatures(rt_batch *b, int model, float *T_out, int mem, void *stream);

/* Replay: the histories of the listed packages (host ids) in the frozen mode,
 * one thread per package with the FP32 transport code. Each record holds
 * {events, absorptions, scatters, crossings, escaped, capped, final_bin,
 * dir_bin, last_leaf} as int64; out is host memory [n][9]. */
rt_status rt_trace(rt_grid *g, const uint64_t *ids, int64_t n, uint64_t seed,
                   uint64_t max_events, int64_t *out);

/* One event of a replayed history: kind 0 emission (cell -1), 1 scattering,
 * 2 absorption (species: the absorbing species), 3 escape, 4 capped (species -1
 * except for absorptions); the cell (at an escape: the last cell), the frequency bin
 * after the event and the position in base-cube units (0 .. n_base per axis). */
typedef struct rt_event {
    int32_t kind, species, leaf, bin;
    float pos[3];
    int32_t pad;
} rt_event;

/* Replay at event level: as rt_trace, and the events of package ids[i] in
 * out[i * max_out ...] (host; at most max_out each), n_out[i] (host) the number of
 * events its history has, which may exceed max_out. Diagnostic: compares histories
 * with an independent implementation event by event. */
rt_status rt_trace_events(rt_grid *g, const uint64_t *ids, int64_t n, uint64_t seed,
                          uint64_t max_events, int64_t max_out, rt_event *out,
                          int64_t *n_out);

/* Philox4x32-10 blocks for counters {id_lo, id_hi, event, block} = (ids[i], event,
 * block) under key = seed, written to out[4*i..4*i+3] (host). Diagnostic. */
rt_status rt_philox(const uint64_t *ids, int64_t n, uint32_t event, uint32_t block,
                    uint64_t seed, uint32_t *out);

/* Molecular data of a PAH species (Sec. 1: PAHs of 30 and 200 C atoms; Sec. 3, Fig. 3:
 * their temperature distribution after single-photon heating). `species` must have
 * been declared with is_pah = 1 in rt_set_dust, whose kabs is then the PAH's
 * absorption cross section per gram. modes = {count_0, theta_0, count_1, theta_1, ...}
 * lists n_groups (1..4) groups of vibrational modes with their characteristic
 * temperatures (K): the heat content is sum n k theta / (exp(theta/T) - 1).
 * n_levels internal-energy levels (16..2048; 0: 400) span 0 .. E(t_top) plus the
 * largest photon energy of the grid (t_top 0: 2500 K).
 *
 * In transport, a package absorbed by a PAH is counted in its cell's absorbed
 * spectrum of 64 coarse bins (coarse bin of fine bin b: floor(64 b / n_bins); all
 * bins when n_bins < 64) and leaves at a frequency drawn from the PAH's template
 * spectrum: the exact steady-state emission in a bath of the source's blackbody at
 * a bolometric flux of 1e4 erg s^-1 cm^-2. */
rt_status rt_set_pah(rt_grid *g, int species, int n_carbon, int n_hydrogen, double mol_mass_g,
                     const double *modes, int n_groups, int n_levels, double t_top);

/* PAH absorbed spectra [n_pah][n_leaves][n_coarse] (uint32 counts; PAHs numbered in
 * species order). */
rt_status rt_pah_absorbed(rt_grid *g, uint32_t *out, int mem, void *stream);

/* Emission of the transiently heated PAHs of cells first_cell .. first_cell+n_cells-1
 * into j_out [n_cells][n_bins] (erg/s per bin; all PAH species summed, or only PAH
 * number `pah` when pah >= 0). Exact (RT_PAH_EXACT): for each cell and PAH, the
 * thermal-discrete steady state under the photon absorption rates its absorbed
 * spectrum implies (count * eps / (h nu_k N_molecules)), then N_molecules
 * sum_f P_f 4 pi sigma_b P_b(T_f), a quad of four lanes per cell with FP32
 * populations (the upward flux across each level boundary summed afresh from the
 * arrivals above it, so no cancellation); emitted power equals absorbed power. RT_PAH_SURROGATE: the network `surrogate` (an rt_mlp
 * with n_in = n_coarse + 2, n_out = n_bins, trained on rt_pah_training_pairs)
 * predicts each PAH's emission relative to its absorbed power (decoded as
 * q_b = exp(7 (y_b - 1)) - 1e-6, floored at 0); the prediction is rescaled to
 * conserve energy. RT_PAH_AUTO: as SURROGATE, but a cell goes to the
 * exact solution when for any PAH the prediction's energy residual |sum_b q_b - 1|
 * before rescaling exceeds `tol`, or its absorbed power per molecule lies outside
 * the range set with rt_mlp_set_range. *n_fallback_out (may be NULL) receives the
 * number of such cells. The PAH-active cells of the range are listed first; the
 * surrogate runs over them in batches of up to 2^20 and the cells sent to the exact
 * solution are solved in one launch at the end. Synchronises the stream to size that
 * work (after listing the active cells and after the checks) and for a host output. */
typedef struct rt_mlp rt_mlp;
rt_status rt_pah_emission(rt_grid *g, int64_t first_cell, int64_t n_cells, int pah, int mode,
                          const rt_mlp *surrogate, float tol, float *j_out, int mem,
                          uint64_t *n_fallback_out, void *stream);

/* The same emission for the PAH-active cells only, in compact form (Sec. 2-3: the
 * PAH emission of the cells that absorbed photons). The cells of the whole grid in
 * which a PAH (all PAH species, or only number `pah` when pah >= 0) absorbed
 * anything since the last reset are listed, in no particular order: cells_out[i]
 * (int32 cell id) is the cell of row i of j_out [n_active][n_bins] (erg/s per bin),
 * which holds what rt_pah_emission writes for that cell in the same mode. Cells
 * without PAH absorptions emit nothing and get no row. *n_active_out receives the
 * number of such cells; when it exceeds max_cells the call returns RT_ERR_RANGE and
 * writes no rows. cells_out and j_out both live where `mem` says; a host output
 * synchronises. n_fallback_out, mode, surrogate and tol as for rt_pah_emission.
 * Unlike the range form this writes nothing for inactive cells, so on a grid where
 * few cells hold PAH absorptions the output is small. */
rt_status rt_pah_emission_active(rt_grid *g, int pah, int mode, const rt_mlp *surrogate,
                                 float tol, int64_t max_cells, int32_t *cells_out,
                                 float *j_out, int mem, int64_t *n_active_out,
                                 uint64_t *n_fallback_out, void *stream);

/* Per-cell PAH re-emission spectra, the step that couples the PAH emission back
 * into the transport (Sec. 2: PAH treatment in the Monte Carlo scheme; iterate
 * transport -> rt_pah_emission -> this call -> transport). Rows J [n_cells][n_bins]
 * (erg/s per bin, e.g. rt_pah_emission's output for PAH number `pah`; negative
 * entries count as 0) for cells first_cell .. first_cell+n_cells-1: afterwards a
 * package absorbed by that PAH in such a cell leaves at a bin drawn with
 * probabilities proportional to the cell's row; cells whose row has nothing
 * positive, and cells never set, keep the template spectrum. The spectra stay set
 * until replaced; J == NULL removes them for every PAH. Allocates n_pah x n_leaves x
 * n_bins floats on first use. mem: where J lives; host rows synchronise. */
rt_status rt_set_pah_spectra(rt_grid *g, int pah, int64_t first_cell, int64_t n_cells,
                             const float *J, int mem, void *stream);

/* Temperature distribution P(T) of PAH molecules in a monochromatic radiation field
 * (Sec. 3, Fig. 3: a PAH exposed to photons of 3.8 eV .. 1 keV at a fixed flux), and
 * how long they stay hotter than graphite sublimates (Sec. 4: hard photons destroy
 * PAHs). For every case: internal-energy levels E_f = f dE, f = 0 .. n_levels-1, up
 * to E(t_top) + h_nu (E(T) from Einstein mode groups); absorptions at `rate` move a
 * molecule from E_i to E_i + h_nu (split over the two levels around it so that the
 * energy is kept; cut at the top level); cooling L(E) = 4 pi sum_b sigma_b P_b(T(E))
 * over the frequency grid, a step down at rate L/dE; the steady state follows level
 * by level (the same thermal-discrete solution as rt_pah_emission). Outputs (host):
 * P_out, T_out [n_cases][n_levels] normalised populations and level temperatures;
 * p_above_out [n_cases] the time fraction spent above t_sub; emission_out
 * [n_cases][n_bins] the emitted power per bin, erg/s per molecule (its sum equals
 * rate * h_nu up to the energy cut at the top). Inputs: nu_edges [n_bins+1] (Hz,
 * increasing), sigma [n_cases][n_bins] absorption cross sections per molecule (cm^2),
 * n_levels 16..4096. One GPU block per case; allocates and frees its device arrays;
 * synchronises. */
typedef struct rt_pah_pt_case {
    double modes[4][2];     /* mode groups: (number of modes, Einstein temperature K) */
    int32_t n_groups;       /* 1..4 */
    int32_t reserved;
    double h_nu_erg;        /* photon energy of the field */
    double rate;            /* absorbed photons per molecule per second (sigma F / h_nu) */
    double t_top;           /* levels reach E(t_top) + h_nu (0: 2500 K) */
} rt_pah_pt_case;
rt_status rt_pah_temperature_distribution(const rt_pah_pt_case *cases, int n_cases,
                                          const double *nu_edges, int n_bins,
                                          const double *sigma, int n_levels, double t_sub,
                                          double *P_out, double *T_out, double *p_above_out,
                                          double *emission_out, void *stream);

/* Training pairs for the surrogate, PAH number `pah`, cells first_cell ..: features
 * X [n][n_coarse+2] (x_k = ln(a_k + 1e-4)/4.6 + 1 for the fraction a_k of absorbed
 * photons in coarse bin k; (log10(P_abs/N_molecules) + 12)/4; log10(N_C) - 2), exact
 * targets Y [n][n_bins] = ln(J_b/P_abs + 1e-6)/7 + 1, and p_abs [n] (erg/s; 0 where
 * the PAH absorbed nothing -- such rows carry no information). Device buffers. */
rt_status rt_pah_training_pairs(rt_grid *g, int pah, int64_t first_cell, int64_t n_cells,
                                float *X, float *Y, float *p_abs, void *stream);

/* ---------------------------------------------------------------------------
 * Multilayer perceptron of the PAH emission surrogate (the learned stand-in for the
 * transient-heating computation; BF16 GEMMs on the 5th-generation tensor cores
 * (tcgen05) with FP32 accumulation in tensor memory,
 * FP32 master weights and Adam). Hidden layers use silu(z) = z / (1 + e^-z), the
 * output layer is linear, the loss is the mean squared error over rows and outputs.
 * Parameters are exchanged as FP32 host arrays in the layout: for each layer
 * W [n_out][n_in] row-major, then b [n_out]. A handle is used by one host thread at
 * a time on the device current at creation.
 * ------------------------------------------------------------------------- */
/* n_layers hidden layers of n_hidden units (1..7), He-uniform weights from `seed`. */
rt_status rt_mlp_create(int n_in, int n_hidden, int n_layers, int n_out, uint64_t seed,
                        rt_mlp **out);
rt_status rt_mlp_destroy(rt_mlp *m);
rt_status rt_mlp_n_params(const rt_mlp *m, int64_t *n);
rt_status rt_mlp_dims(const rt_mlp *m, int *n_in, int *n_out);
/* Admissible range of input n_in - 2 (the absorbed power per molecule of the PAH
 * features); rt_pah_emission in RT_PAH_AUTO sends cells outside it to the exact
 * solution. Default: unbounded. */
rt_status rt_mlp_set_range(rt_mlp *m, float lo, float hi);
rt_status rt_mlp_get_range(const rt_mlp *m, float *lo, float *hi);
/* host [n_params]; RT_ERR_TIMEOUT when a tensor-core forward pass gave up waiting for
 * its MMAs since the handle was created (its outputs were set to NaN) */
rt_status rt_mlp_get_params(rt_mlp *m, float *out);
rt_status rt_mlp_set_params(rt_mlp *m, const float *in);  /* host [n_params] */

/* y [M][n_out] = network(x [M][n_in]); device FP32 buffers; asynchronous. When the
 * padded input and hidden widths are at most 256 (and the output width at most 4096)
 * the whole network runs per 128-row tile in one kernel on the 5th-generation tensor
 * cores (tcgen05.mma, FP32 accumulators in tensor memory, BF16 operands in shared
 * memory; an output layer wider than 256 in chunks of 256 columns); otherwise layer
 * by layer (one tcgen05 GEMM of 128 x 128 output tiles per layer, as in training). */
rt_status rt_mlp_forward(rt_mlp *m, const float *x, float *y, int64_t M, void *stream);

/* Loss and gradients of a batch (device x [M][n_in], targets t [M][n_out]) into the
 * handle's gradient buffer; loss_out / grad_out (host, may be NULL) receive the loss
 * and a copy of the gradients (synchronising when either is given). */
rt_status rt_mlp_loss_grad(rt_mlp *m, const float *x, const float *t, int64_t M,
                           float *loss_out, float *grad_out, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the last gradients. */
rt_status rt_mlp_adam_step(rt_mlp *m, float lr, void *stream);

const char *rt_status_string(rt_status s);

/* Cell temperatures for callers that cannot allocate device memory. The paper has
 * no counterpart; this is a service of the library.
 *
 * Who needs it: code that owns all of its device memory and may not call
 * cudaMalloc at the point where temperatures are wanted -- a framework that hands
 * out memory only from its own pool (a stray cudaMalloc would synchronise the
 * device and fragment the pool), or a host process whose memory budget on the
 * GPU is fixed up front. Such a caller passes every input and the output as its
 * own device buffers; this entry point then allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *
 * It computes what rt_cell_temperatures computes: T from
 * n eps = rho V 4 pi sum_b kappa_abs(b) P_b(T), inverted in FP64, 0 where n = 0 or
 * rho = 0, t_max (counted in *n_clamped) where the energy lies beyond the table.
 * The FP64 emission table it needs lives in one fixed array in device memory that
 * the library reserves statically: 147,712 bytes, held on every GPU that loads the
 * library until the process exits. Hence the limits: n_species <= 8,
 * n_temp <= 2048 table rows, n_bins <= 1024; larger requests return
 * RT_ERR_TOO_LARGE.
 *
 * count   device, [n_species][n_cells] absorption counts
 * rho     device, [n_species][n_cells] densities, g cm^-3
 * volume  device, [n_cells] cell volumes, cm^3
 * kabs    device, [n_species][n_bins] absorption opacities, cm^2 g^-1
 * nu_edges device, [n_bins+1] bin edges, Hz, ascending
 * eps     package energy, erg/s; t_min, t_max, n_temp as in rt_grid_desc (0: defaults)
 * T_out   device, [n_species][n_cells], K
 * n_clamped device, one uint64 (may be NULL): cells set to t_max
 * stream  cudaStream_t; the call is asynchronous on it.
 *
 * Every call looks up the array's address in the current context with
 * cudaGetSymbolAddress (which allocates nothing); the first call in a context may
 * load the library's device code there, so make that first call before any stream
 * capture. Every call reuses the same array and finds
 * there whatever the previous call left, so calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller. */
rt_status rt_cell_temperatures_noalloc(const uint64_t *count, const double *rho,
                                       const double *volume, const double *kabs,
                                       const double *nu_edges, int n_species,
                                       int64_t n_cells, int n_bins, double eps,
                                       double t_min, double t_max, int n_temp,
                                       float *T_out, uint64_t *n_clamped, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RT_GB300_H */
