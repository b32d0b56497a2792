// rt_internal.h -- structures shared by the host side and the kernels of
// librt_gb300. Not part of the public ABI (include/rt.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rt {

constexpr int kMaxSpecies = 8;
constexpr int kMaxLevels = 8;     // levels 0 .. 7
constexpr int kMaxBins = 1024;
constexpr int kMaxPah = 4;        // PAH species per grid
constexpr int kMaxModeGroups = 4; // vibrational mode groups per PAH

// Device status bits.
constexpr unsigned kStatusTree = 1u;     // a package met a malformed tree
constexpr unsigned kStatusTimeout = 2u;  // a launch ran past its time budget

// Indices into the device counter array.
enum Counter {
  kCEmitted = 0, kCEscaped, kCCapped, kCAbsorptions, kCScatters, kCCrossings,
  kCErrors, kCClamped, kCLevels, kCPeelEvents, kCPeelCrossings, kCPeelDropped, kNumCounters
};

// Face links of a leaf (record of 8 int32 per leaf: faces -x,+x,-y,+y,-z,+z, then
// the densities of species 0 and 1 as float bits when S <= 2). A link is
//   kLinkEscape                the face is the domain boundary;
//   id | (level << 28)         the neighbouring leaf (same size or coarser);
//   -(block + 1)               the same-size neighbour is split: descend into block.
constexpr int32_t kLinkEscape = (int32_t)0x80000000;
constexpr int32_t kLinkLeafMask = 0x0FFFFFFF;
constexpr long long kMaxLinkedLeaves = 1ll << 28;

// Geometry and densities (device pointers), passed by value.
struct DevGrid {
  const int32_t* base;     // [n^3]
  const int32_t* child;    // [n_blocks*8]
  const float* rho;        // [n_leaves][S]: density times the base-cube edge, g cm^-2
  const int8_t* level;     // [n_leaves] refinement level of every leaf
  const int32_t* links;    // [n_leaves][8] face links (+ densities when S <= 2)
  // densities by tree slot for the path walk: [n_base^3 + 8 n_blocks][S], slot i < n^3
  // the base cell i, slot n^3 + 8 b + o the child o of block b; zeros where refined
  const float* rho_slot;
  long long n_leaves, n_blocks;
  int n_base, max_level, S, B, n_dir, n_T;
  int n_base3;             // n_base^3, the first block slot
};

// Face-link record of a leaf, 8 words (32 bytes): links of faces -x,+x,-y,+y,-z,+z,
// then the densities of species 0 and 1 when S <= 2 (zero otherwise).
constexpr int kRec = 8;

// Per-bin opacity record for one species, kept in shared memory during transport.
struct Kappa {
  float kext, ksca, kabs, g;  // cm^2 g^-1, cm^2 g^-1, cm^2 g^-1, HG asymmetry
};

// Tables built in FP64 on the device and stored for transport.
struct DevTables {
  const Kappa* kap;           // [B][S]
  const float* star_cdf;      // [B] normalised cumulative stellar spectrum
  const float* S32;           // [S][n_T] emitted power per gram at the table rows
  const double* S64;          // [S][n_T]
  const double* Tgrid;        // [n_T], Tgrid[0] = 0
  const float* dcdf;          // [S][n_T-1][B] normalised cumulative of row differences
  const unsigned short* cdf_guide;  // [S][n_T-1][B]: first bin whose cdf exceeds k/B
  const int* u_guide;         // [S][n_T]: interval holding exp(u_ln0 + k / u_inv)
  float u_ln0[kMaxSpecies];   // ln S_s(T_1)
  float u_inv[kMaxSpecies];   // (n_T - 1) / (ln S_s(T_last) - ln S_s(T_1))
  const float* u_frozen;      // [S][n_leaves] (frozen mode) or null
  const float* pah_cdf;       // [n_pah][B] template re-emission spectrum of each PAH
  const float* pah_cell_cdf;  // [n_pah][n_leaves][B] per-cell PAH re-emission spectra
                              // (normalised cumulative; last entry 0: the template), or null
  int pah_of[kMaxSpecies];    // PAH number of each species, -1 for grains
  int n_coarse;               // coarse bins of the PAH absorbed spectrum
  float u_tmin[kMaxSpecies];  // S_s(t_min)
  float eps_d0_over_V[kMaxLevels];   // eps * d0 / V(level), erg s^-1 cm^-2 (FP32)
  double eps_over_V[kMaxLevels];     // eps / V(level) (FP64, temperatures)
  double d0;                  // base-cube edge, cm
};

// One transport launch.
struct DevRun {
  unsigned long long seed, first_id, n_packages, max_events;
  unsigned long long* next;       // pool: packages handed out so far
  unsigned long long* count;      // [S][n_leaves]
  unsigned long long* sed;        // [2][n_dir][B]
  unsigned long long* counters;   // [kNumCounters]
  unsigned int* status;
  unsigned* pahabs;               // [n_pah][n_leaves][n_coarse] PAH absorptions
  unsigned* pah_flag;             // [n_leaves] bit p set: PAH p absorbed in the cell
  float* pathabs;                 // [S][n_leaves] path-length tallies, or null
  float src[3];                   // source position, base-cube units
  float beam[3];
  double src64[3];
  double beam64[3];
  int source_kind, mode, refill_period;
  int interaction_batch;          // pool: waiting lanes that trigger an interaction phase
  float count_scale;              // BW / no-correction: temperature index = scale x count
  int sed_in_smem;                // pool: escaped-spectrum histogram in shared memory
  unsigned long long budget_ns;
};

// Peel-off images toward a distant observer. Every scattering and re-emission at a
// bin that has an image plane sends the share w of the package's energy per
// steradian toward the observer (HG phase function value, or 1/(4 pi)), attenuated
// by exp(-tau) along the sight line to the boundary, into the pixel its position
// projects to. The transport launch only records these events (position, w, bin);
// a second kernel traces their sight lines. Emissions by a point source are counted
// per bin and peeled once per bin after the launch (they all start at the source).
struct DevPeel {
  const int* plane_of_bin;       // [B] image plane of each bin, -1 for none
  double* image;                 // [n_planes][ny][nx] sums of w exp(-tau) (times eps: erg/s/sr)
  unsigned long long* n_emit;    // [B] point-source emissions since the last source peel
  float4* ev;                    // [capacity] recorded events: position (base units), w
  int* ev_bin;                   // [capacity] their bins
  unsigned long long* n_ev;      // events recorded by the current launch
  unsigned long long capacity;
  float o[3];                    // unit vector toward the observer
  float e1[3], e2[3];            // image axes: e1 = normalise(z x o) (x when o ~ z), e2 = o x e1
  float centre;                  // model centre, base-cube units
  float sx, sy;                  // pixels per base-cube unit along e1, e2
  int nx, ny, n_planes;
  float tau_max;                 // sight lines stop (contribute nothing) beyond this depth
};

constexpr int kMaxImageSide = 16384;
constexpr unsigned long long kPeelCapacityDefault = 1ull << 24;
constexpr unsigned long long kPeelCapacityMax = 1ull << 31;
constexpr size_t kMaxImagePixels = (size_t)1 << 28;  // all planes together (2 GiB of FP64)

// One model of a batched launch, and one chunk of its packages.
struct ModelDesc {
  DevGrid g;
  DevTables t;
  DevRun r;
};

struct BatchChunk {
  int model;
  int pad;
  unsigned long long first, count;  // package indices [first, first + count)
};

// Kernel launchers (rt_transport.cu, rt_tables.cu).
// s_fixed: the species count all models share (2 has a walk compiled for it,
// without the path-length tally), 0 otherwise
cudaError_t launch_transport_batch(const ModelDesc* models, const BatchChunk* chunks,
                                   long long n_chunks, unsigned long long* next_chunk,
                                   int blocks_per_sm, int s_fixed, int threads,
                                   cudaStream_t s);
cudaError_t launch_transport_pool(const DevGrid& g, const DevTables& t, const DevRun& r,
                                  int blocks_per_sm, int threads, cudaStream_t s,
                                  const DevPeel* peel = nullptr, bool path = false);
cudaError_t launch_peel_source(const DevGrid& g, const DevTables& t, const DevRun& r,
                               const DevPeel& peel, cudaStream_t s);
cudaError_t launch_peel_trace(const DevGrid& g, const DevTables& t, const DevRun& r,
                              const DevPeel& peel, cudaStream_t s);
cudaError_t launch_image_out(const double* image, long long n, double scale, double* out,
                             cudaStream_t s);
cudaError_t launch_image_profile(const double* image, int nx, int ny, int plane_a,
                                 int plane_b, int half_rows, double scale, double* out,
                                 cudaStream_t s);
cudaError_t launch_transport_plain(const DevGrid& g, const DevTables& t, const DevRun& r,
                                   bool fp64, int threads, cudaStream_t s);
// One event of a replayed history (rt_trace_events): kind 0 emission, 1 scattering,
// 2 absorption, 3 escape, 4 capped; position in base-cube units.
struct TraceEvent {
  int kind, species, leaf, bin;
  float pos[3];
  int pad;
};
cudaError_t launch_trace(const DevGrid& g, const DevTables& t, const DevRun& r,
                         const unsigned long long* ids, long long n, long long* out,
                         cudaStream_t s, TraceEvent* ev = nullptr, long long ev_cap = 0,
                         long long* ev_n = nullptr);
cudaError_t launch_build_links(const DevGrid& g, const int32_t* leaf_ijk, int32_t* links,
                               cudaStream_t s);
cudaError_t launch_build_rho_slot(const DevGrid& g, float* rho_slot, cudaStream_t s);

// Device walk of the tree (rt_grid.cu): inputs, outputs and work arrays.
struct TreeBuild {
  const int32_t* base;     // [n^3]
  const int32_t* child;    // [n_blocks][8]
  long long n_leaves, n_blocks;
  int n_base, max_level;
  int8_t* level;           // [n_leaves] out
  int32_t* ijk;            // [n_leaves][3] out: integer corner at the leaf's level
  int8_t* blk_level;       // [n_blocks] work
  int32_t* blk_ijk;        // [n_blocks][3] work
  unsigned* leaf_seen;     // [(n_leaves + 31) / 32] work bitmap
  unsigned* blk_seen;      // [(n_blocks + 31) / 32] work bitmap
  unsigned* err;           // nonzero: malformed tree (bit 0) or bad density (bit 1)
  int* max_seen;           // deepest level reached
};
cudaError_t launch_tree_walk(const TreeBuild& tb, cudaStream_t s);
cudaError_t launch_rho_convert(const double* src, long long N, int S, double d0, float* dst,
                               unsigned* err, cudaStream_t s);
cudaError_t launch_philox(const unsigned long long* ids, long long n, unsigned event,
                          unsigned block, unsigned long long seed, unsigned* out,
                          cudaStream_t s);

struct TableBuild {
  int S, B, n_T;
  const double* nu;          // [B+1]
  const double* kabs;        // [S][B]
  const double* ksca;        // [S][B]
  const double* ghg;         // [S][B]
  double T_star, t_min, t_max;
  // outputs
  double* Tgrid;             // [n_T]
  double* P;                 // scratch [n_T][B]
  double* S64;               // [S][n_T]
  float* S32;                // [S][n_T]
  float* dcdf;               // [S][n_T-1][B]
  unsigned short* cdf_guide; // [S][n_T-1][B]
  int* u_guide;              // [S][n_T]
  Kappa* kap;                // [B][S]
  float* star_cdf;           // [B]
  double* star_frac;         // [1] in-range fraction of the stellar blackbody
};
cudaError_t launch_build_tables(const TableBuild& tb, cudaStream_t s);

// PAH molecular data: vibrational mode groups (count, characteristic temperature)
struct PahSpec {
  int n_groups;
  double n_modes[kMaxModeGroups];
  double theta[kMaxModeGroups];
};

struct PahBuild {
  int n_pah, M, K, B;
  const double* nu;          // [B+1]
  const double* sigma;       // [n_pah][B] cross section per molecule, cm^2
  PahSpec spec[kMaxPah];
  double dE[kMaxPah];        // level spacing, erg
  double T_star, f_ref;      // template heating: source blackbody at bolometric flux f_ref
  float* s;                  // [n_pah][M][B] emission per level and bin, erg/s
  double* L;                 // [n_pah][M] cooling rate per level, erg/s
  double* e_k;               // [K] photon energy of each coarse bin, erg
  int* q_k;                  // [n_pah][K] floor(e_k / dE)
  double* w_k;               // [n_pah][K] e_k / dE - q_k
  float* template_cdf;       // [n_pah][B]
  float* c_f;                // [n_pah][M] downward rate L_f / dE, 1/s (FP32 copy)
  float* w_f;                // [n_pah][K] w_k (FP32 copy)
};

struct PahTables {
  int n_pah, M, K;
  const float* s;
  const double* L;
  const double* e_k;
  const int* q_k;
  const double* w_k;
  const float* c_f;          // [n_pah][M] L_f / dE in FP32
  const float* w_f;          // [n_pah][K] w_k in FP32
  double dE[kMaxPah];
  double mol_mass[kMaxPah];  // g per molecule
  int species[kMaxPah];      // species index of each PAH
  int n_carbon[kMaxPah];     // C atoms of each PAH
};

cudaError_t launch_pah_tables(const PahBuild& pb, const PahTables& t, cudaStream_t s);
cudaError_t launch_pah_exact(const DevGrid& g, const PahTables& t, const unsigned* pahabs,
                             double eps, double d0, long long first, long long n,
                             float* j_out, const unsigned char* want, int pah_only,
                             cudaStream_t s, const int* list = nullptr,
                             const int* cell_of_row = nullptr);
cudaError_t launch_pah_features(const DevGrid& g, const PahTables& t, const unsigned* pahabs,
                                double eps, double d0, int p, long long first, long long n,
                                float* X, float* p_abs, cudaStream_t s,
                                const int* list = nullptr);
cudaError_t launch_pah_encode(const float* J, const float* p_abs, long long n, int B, float* Y,
                              cudaStream_t s);
cudaError_t launch_surrogate_check(const float* Y, const float* X, const float* p_abs,
                                   long long n, int B, int F, float tol, float x_lo, float x_hi,
                                   unsigned char* flag, cudaStream_t s);
cudaError_t launch_surrogate_add(const float* Y, const float* p_abs, long long n, int B,
                                 const unsigned char* flag, float* j_out, cudaStream_t s,
                                 const int* list = nullptr);
cudaError_t launch_pah_clear(const unsigned* pah_flag, long long N, int K, int n_pah,
                             unsigned* pahabs, unsigned* pah_flag_out, cudaStream_t s);
cudaError_t launch_compact(const PahTables& t, const unsigned* pah_flag, long long N, int pah,
                           long long first, long long n, const unsigned char* flag,
                           const int* list, int* out, unsigned* count, cudaStream_t s,
                           int off = 0);
cudaError_t launch_count_flags(const unsigned char* flag, long long n, unsigned long long* out,
                               cudaStream_t s);
cudaError_t launch_pah_cell_cdf(const float* J, long long n, int B, float* out, cudaStream_t s);

// One P(T) problem: a PAH in a monochromatic field.
struct PtCase {
  PahSpec spec;
  double h_nu;   // photon energy, erg
  double rate;   // absorbed photons per molecule per second
  double t_top;  // levels span 0 .. E(t_top) + h_nu
};
cudaError_t launch_pah_pt(const PtCase* cases, int n_cases, const double* nu, int B,
                          const double* sigma, int M, double t_sub, double* P_out,
                          double* T_out, double* p_above, double* em_out, cudaStream_t s);

cudaError_t launch_frozen_u(const DevGrid& g, const DevTables& t, const float* T_frozen,
                            float* u_frozen, float t_min, cudaStream_t s);
cudaError_t launch_temperatures(const DevGrid& g, const DevTables& t,
                                const unsigned long long* count, float* T_out,
                                unsigned long long* counters, cudaStream_t s,
                                const float* pathabs = nullptr);

}  // namespace rt
