// rt_api.cu -- host side of librt_gb300: the C ABI declared in include/rt.h.
// Validates inputs, owns the device memory of a grid handle, builds the FP64
// tables on the device and launches the transport and temperature kernels.

#include "../../include/rt.h"
#include "rt_internal.h"

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <thread>
#include <utility>
#include <vector>

using namespace rt;

struct rt_grid {
  int dev = 0;
  rt_grid_desc desc{};
  double d0 = 0;  // base-cube edge, cm
  DevGrid g{};
  // device memory owned by the handle
  int32_t* d_base = nullptr;
  int32_t* d_child = nullptr;
  float* d_rho = nullptr;
  int8_t* d_level = nullptr;
  int32_t* d_links = nullptr;
  float* d_rho_slot = nullptr;  // densities by tree slot (path walk)
  unsigned long long* d_count = nullptr;
  unsigned long long* d_sed = nullptr;
  unsigned long long* d_counters = nullptr;
  unsigned long long* d_next = nullptr;
  unsigned int* d_status = nullptr;
  // tables
  double* d_nu = nullptr;
  double* d_kabs = nullptr;
  double* d_ksca = nullptr;
  double* d_ghg = nullptr;
  double* d_Tgrid = nullptr;
  double* d_P = nullptr;
  double* d_S64 = nullptr;
  float* d_S32 = nullptr;
  float* d_dcdf = nullptr;
  unsigned short* d_cdf_guide = nullptr;
  int* d_u_guide = nullptr;
  Kappa* d_kap = nullptr;
  float* d_star_cdf = nullptr;
  double* d_star_frac = nullptr;
  float* d_Tfrozen = nullptr;
  float* d_ufrozen = nullptr;
  float* d_Tscratch = nullptr;
  // PAH tables and tallies
  double* d_pah_sigma = nullptr;
  float* d_pah_s = nullptr;
  double* d_pah_L = nullptr;
  double* d_pah_ek = nullptr;
  int* d_pah_qk = nullptr;
  double* d_pah_wk = nullptr;
  float* d_pah_cf = nullptr;
  float* d_pah_wf = nullptr;
  float* d_pah_cdf = nullptr;
  float* d_pah_cell_cdf = nullptr;  // [n_pah][N][B] per-cell re-emission spectra
  unsigned* d_pahabs = nullptr;
  unsigned* d_pah_flag = nullptr;  // [N] PAH-active bits per cell (bit p: PAH p)
  float* d_pathabs = nullptr;  // path-length tallies [S][N]
  // peel-off images
  int* d_plane_of_bin = nullptr;         // [B]
  double* d_image = nullptr;             // [n_planes][ny][nx]
  unsigned long long* d_nemit = nullptr; // [B]
  float4* d_ev = nullptr;                // [capacity] recorded peel-off events
  int* d_ev_bin = nullptr;               // [capacity]
  unsigned long long* d_nev = nullptr;   // [1]
  double* d_iscratch = nullptr;          // [max(n_planes*ny*nx, nx)] readout (host copies)
  size_t iscratch_n = 0;
  DevPeel peel{};
  bool images = false;
  float* d_jscratch = nullptr;
  size_t jscratch_n = 0;
  int32_t* d_cells_scratch = nullptr;  // cell list of a host-output active-cell emission
  int64_t cells_scratch_n = 0;
  // surrogate scratch (rows per batch of active cells) and cell lists (per call)
  long long sur_cap = 0, list_cap = 0;
  float* d_sx = nullptr;       // [batch][K+2]
  float* d_sy = nullptr;       // [n_pah][batch][B]
  float* d_spabs = nullptr;    // [n_pah][batch]
  unsigned char* d_sflag = nullptr;  // [batch]
  unsigned long long* d_scount = nullptr;
  int* d_list = nullptr;       // [cells] PAH-active cells of the call
  int* d_list2 = nullptr;      // [cells] cells sent to the exact solution
  unsigned* d_ucount = nullptr;  // [2]
  // host state
  std::vector<double> nu, kabs, ksca, ghg;   // [S][B]
  std::vector<char> dust_set;
  std::vector<int> is_pah, n_carbon;
  std::vector<char> pah_set;
  std::vector<PahSpec> pah_spec;
  std::vector<double> pah_mass;
  int pah_levels = 400;
  double pah_t_top = 2500.0;
  int n_pah = 0;
  PahTables ptab{};
  bool star_set = false;
  double T_star = 0, L_star = 0, pos[3] = {0, 0, 0}, beam[3] = {0, 0, 1};
  int source_kind = 0;
  unsigned long long n_total = 0;
  bool tables_ready = false;
  bool frozen_ready = false;
  double eps = 0, star_frac = 0;
  DevTables tab{};
  int n_levels_used = 0;
};

namespace {

rt_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RT_OK : RT_ERR_CUDA; }

#define RT_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return RT_ERR_CUDA;         \
  } while (0)

template <typename T>
rt_status dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RT_ERR_OOM;
  }
  return cuda_status(e);
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_tables(rt_grid* g) {
  dfree(g->d_nu);
  dfree(g->d_kabs);
  dfree(g->d_ksca);
  dfree(g->d_ghg);
  dfree(g->d_Tgrid);
  dfree(g->d_P);
  dfree(g->d_S64);
  dfree(g->d_S32);
  dfree(g->d_dcdf);
  dfree(g->d_cdf_guide);
  dfree(g->d_u_guide);
  dfree(g->d_kap);
  dfree(g->d_star_cdf);
  dfree(g->d_star_frac);
  dfree(g->d_pah_sigma);
  dfree(g->d_pah_s);
  dfree(g->d_pah_L);
  dfree(g->d_pah_ek);
  dfree(g->d_pah_qk);
  dfree(g->d_pah_wk);
  dfree(g->d_pah_cf);
  dfree(g->d_pah_wf);
  dfree(g->d_pah_cdf);
  g->tables_ready = false;
}

// The path walk serves grids of at most four levels whose tree slots (base cells and
// block children) an int indexes.
static bool path_walk_fits(const rt_grid_desc* d) {
  const double nb = (double)d->n_base * d->n_base * d->n_base;
  return d->max_level <= 4 && nb + 8.0 * (double)d->n_blocks < 2147483647.0;
}

void free_all(rt_grid* g) {
  free_tables(g);
  dfree(g->d_base);
  dfree(g->d_child);
  dfree(g->d_rho);
  dfree(g->d_level);
  dfree(g->d_links);
  dfree(g->d_rho_slot);
  dfree(g->d_count);
  dfree(g->d_sed);
  dfree(g->d_counters);
  dfree(g->d_next);
  dfree(g->d_status);
  dfree(g->d_Tfrozen);
  dfree(g->d_ufrozen);
  dfree(g->d_Tscratch);
  dfree(g->d_pahabs);
  dfree(g->d_pah_flag);
  dfree(g->d_pathabs);
  dfree(g->d_plane_of_bin);
  dfree(g->d_image);
  dfree(g->d_nemit);
  dfree(g->d_ev);
  dfree(g->d_ev_bin);
  dfree(g->d_nev);
  dfree(g->d_iscratch);
  dfree(g->d_pah_cell_cdf);
  dfree(g->d_jscratch);
  dfree(g->d_cells_scratch);
  dfree(g->d_sx);
  dfree(g->d_sy);
  dfree(g->d_spabs);
  dfree(g->d_sflag);
  dfree(g->d_scount);
  dfree(g->d_list);
  dfree(g->d_list2);
  dfree(g->d_ucount);
}

rt_status sync_status(rt_grid* g, cudaStream_t s) {
  RT_CUDA(cudaStreamSynchronize(s));
  unsigned st = 0;
  RT_CUDA(cudaMemcpy(&st, g->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st & kStatusTree) return RT_ERR_DEVICE;
  if (st & kStatusTimeout) return RT_ERR_TIMEOUT;
  return RT_OK;
}

double heat_content_host(double T, const PahSpec& sp) {
  const double kB = 1.380649e-16;
  double e = 0.0;
  for (int i = 0; i < sp.n_groups; ++i) {
    double x = sp.theta[i] / T;
    if (x < 700.0) e += sp.n_modes[i] * kB * sp.theta[i] / std::expm1(x);
  }
  return e;
}

// Level tables, coarse photon energies and template spectra of the PAH species.
rt_status build_pah_tables(rt_grid* g, cudaStream_t s) {
  const int S = g->desc.n_species, B = g->desc.n_bins, N = (int)0;
  (void)N;
  std::vector<int> pahs;
  for (int i = 0; i < S; ++i)
    if (g->is_pah[(size_t)i]) {
      if (!g->pah_set[(size_t)i]) return RT_ERR_STATE;
      pahs.push_back(i);
    }
  g->n_pah = (int)pahs.size();
  if (g->n_pah == 0) return RT_OK;
  if (g->n_pah > kMaxPah) return RT_ERR_ARG;
  const int P = g->n_pah, M = g->pah_levels, K = g->tab.n_coarse;
  rt_status st;
  if ((st = dalloc(&g->d_pah_sigma, (size_t)P * B)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_s, (size_t)P * M * B)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_L, (size_t)P * M)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_ek, (size_t)K)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_qk, (size_t)P * K)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_wk, (size_t)P * K)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_cf, (size_t)P * M)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_wf, (size_t)P * K)) != RT_OK) return st;
  if ((st = dalloc(&g->d_pah_cdf, (size_t)P * B)) != RT_OK) return st;
  if (!g->d_pahabs) {
    if ((st = dalloc(&g->d_pahabs, (size_t)P * g->desc.n_leaves * K)) != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(g->d_pahabs, 0, sizeof(unsigned) * P * g->desc.n_leaves * K, s));
    if ((st = dalloc(&g->d_pah_flag, (size_t)g->desc.n_leaves)) != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(g->d_pah_flag, 0, sizeof(unsigned) * g->desc.n_leaves, s));
  }
  std::vector<double> sigma((size_t)P * B);
  PahBuild pb{};
  PahTables& pt = g->ptab;
  pt = PahTables{};
  pb.n_pah = pt.n_pah = P;
  pb.M = pt.M = M;
  pb.K = pt.K = K;
  pb.B = B;
  const double h = 6.62607015e-27;
  for (int p = 0; p < P; ++p) {
    int sp = pahs[(size_t)p];
    for (int b = 0; b < B; ++b)
      sigma[(size_t)p * B + b] = g->kabs[(size_t)sp * B + b] * g->pah_mass[(size_t)sp];
    pb.spec[p] = g->pah_spec[(size_t)sp];
    double e_max = heat_content_host(g->pah_t_top, pb.spec[p]) + h * g->nu[(size_t)B];
    pb.dE[p] = pt.dE[p] = e_max / (M - 1);
    pt.mol_mass[p] = g->pah_mass[(size_t)sp];
    pt.species[p] = sp;
    pt.n_carbon[p] = g->n_carbon[(size_t)sp];
    g->tab.pah_of[sp] = p;
  }
  RT_CUDA(cudaMemcpyAsync(g->d_pah_sigma, sigma.data(), sizeof(double) * P * B,
                          cudaMemcpyHostToDevice, s));
  pb.nu = g->d_nu;
  pb.sigma = g->d_pah_sigma;
  pb.T_star = g->T_star;
  pb.f_ref = 1.0e4;  // erg s^-1 cm^-2, the heating bath of the paper's Fig. 3
  pb.s = g->d_pah_s;
  pb.L = g->d_pah_L;
  pb.e_k = g->d_pah_ek;
  pb.q_k = g->d_pah_qk;
  pb.w_k = g->d_pah_wk;
  pb.template_cdf = g->d_pah_cdf;
  pb.c_f = g->d_pah_cf;
  pb.w_f = g->d_pah_wf;
  pt.s = g->d_pah_s;
  pt.L = g->d_pah_L;
  pt.e_k = g->d_pah_ek;
  pt.q_k = g->d_pah_qk;
  pt.w_k = g->d_pah_wk;
  pt.c_f = g->d_pah_cf;
  pt.w_f = g->d_pah_wf;
  RT_CUDA(launch_pah_tables(pb, pt, s));
  RT_CUDA(cudaStreamSynchronize(s));
  g->tab.pah_cdf = g->d_pah_cdf;
  return RT_OK;
}

rt_status build_tables(rt_grid* g, cudaStream_t s) {
  if (g->tables_ready) return RT_OK;
  const int S = g->desc.n_species, B = g->desc.n_bins, nT = g->desc.n_temp;
  for (int i = 0; i < S; ++i)
    if (!g->dust_set[i]) return RT_ERR_STATE;
  if (!g->star_set) return RT_ERR_STATE;
  free_tables(g);
  rt_status st;
#define ALLOC(p, n) if ((st = dalloc(&(p), (n))) != RT_OK) { free_tables(g); return st; }
  ALLOC(g->d_nu, (size_t)B + 1);
  ALLOC(g->d_kabs, (size_t)S * B);
  ALLOC(g->d_ksca, (size_t)S * B);
  ALLOC(g->d_ghg, (size_t)S * B);
  ALLOC(g->d_Tgrid, (size_t)nT);
  ALLOC(g->d_P, (size_t)nT * B);
  ALLOC(g->d_S64, (size_t)S * nT);
  ALLOC(g->d_S32, (size_t)S * nT);
  ALLOC(g->d_dcdf, (size_t)S * (nT - 1) * B);
  ALLOC(g->d_cdf_guide, (size_t)S * (nT - 1) * B);
  ALLOC(g->d_u_guide, (size_t)S * nT);
  ALLOC(g->d_kap, (size_t)S * B);
  ALLOC(g->d_star_cdf, (size_t)B);
  ALLOC(g->d_star_frac, 1);
#undef ALLOC
  RT_CUDA(cudaMemcpyAsync(g->d_nu, g->nu.data(), sizeof(double) * (B + 1),
                          cudaMemcpyHostToDevice, s));
  RT_CUDA(cudaMemcpyAsync(g->d_kabs, g->kabs.data(), sizeof(double) * S * B,
                          cudaMemcpyHostToDevice, s));
  RT_CUDA(cudaMemcpyAsync(g->d_ksca, g->ksca.data(), sizeof(double) * S * B,
                          cudaMemcpyHostToDevice, s));
  RT_CUDA(cudaMemcpyAsync(g->d_ghg, g->ghg.data(), sizeof(double) * S * B,
                          cudaMemcpyHostToDevice, s));
  TableBuild tb{};
  tb.S = S;
  tb.B = B;
  tb.n_T = nT;
  tb.nu = g->d_nu;
  tb.kabs = g->d_kabs;
  tb.ksca = g->d_ksca;
  tb.ghg = g->d_ghg;
  tb.T_star = g->T_star;
  tb.t_min = g->desc.t_min;
  tb.t_max = g->desc.t_max;
  tb.Tgrid = g->d_Tgrid;
  tb.P = g->d_P;
  tb.S64 = g->d_S64;
  tb.S32 = g->d_S32;
  tb.dcdf = g->d_dcdf;
  tb.cdf_guide = g->d_cdf_guide;
  tb.u_guide = g->d_u_guide;
  tb.kap = g->d_kap;
  tb.star_cdf = g->d_star_cdf;
  tb.star_frac = g->d_star_frac;
  RT_CUDA(launch_build_tables(tb, s));
  // S(t_min) per species: table row 1 is exactly t_min
  std::vector<double> S64((size_t)S * nT);
  RT_CUDA(cudaMemcpyAsync(S64.data(), g->d_S64, sizeof(double) * S * nT,
                          cudaMemcpyDeviceToHost, s));
  RT_CUDA(cudaMemcpyAsync(&g->star_frac, g->d_star_frac, sizeof(double),
                          cudaMemcpyDeviceToHost, s));
  RT_CUDA(cudaStreamSynchronize(s));
  dfree(g->d_P);
  g->eps = g->L_star * g->star_frac / (double)g->n_total;
  DevTables& t = g->tab;
  t = DevTables{};
  t.kap = g->d_kap;
  t.star_cdf = g->d_star_cdf;
  t.S32 = g->d_S32;
  t.S64 = g->d_S64;
  t.Tgrid = g->d_Tgrid;
  t.dcdf = g->d_dcdf;
  t.cdf_guide = g->d_cdf_guide;
  t.u_guide = g->d_u_guide;
  t.u_frozen = nullptr;
  for (int i = 0; i < S; ++i) {
    t.u_tmin[i] = (float)S64[(size_t)i * nT + 1];
    double l0 = std::log(S64[(size_t)i * nT + 1]), l1 = std::log(S64[(size_t)i * nT + nT - 1]);
    t.u_ln0[i] = (float)l0;
    t.u_inv[i] = (float)((nT - 1) / (l1 - l0));
  }
  for (int l = 0; l < kMaxLevels; ++l) {
    double V = std::pow(g->d0 * std::ldexp(1.0, -l), 3.0);
    t.eps_over_V[l] = g->eps / V;
    t.eps_d0_over_V[l] = (float)(g->eps * g->d0 / V);
  }
  t.d0 = g->d0;
  for (int i = 0; i < kMaxSpecies; ++i) t.pah_of[i] = -1;
  t.pah_cdf = nullptr;
  t.n_coarse = B < 64 ? B : 64;
  if ((st = build_pah_tables(g, s)) != RT_OK) {
    free_tables(g);
    return st;
  }
  g->tables_ready = true;
  g->frozen_ready = false;
  return RT_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool finite3(const double* v) {
  return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

}  // namespace

extern "C" {

const char* rt_status_string(rt_status s) {
  switch (s) {
    case RT_OK: return "ok";
    case RT_ERR_ARG: return "invalid argument";
    case RT_ERR_OOM: return "out of memory";
    case RT_ERR_CUDA: return "CUDA runtime error";
    case RT_ERR_TIMEOUT: return "kernel stopped at its time budget";
    case RT_ERR_STATE: return "call out of order";
    case RT_ERR_RANGE: return "package ids beyond the planned total";
    case RT_ERR_DEVICE: return "malformed grid met on the device";
    case RT_ERR_TOO_LARGE: return "request exceeds a fixed maximum";
  }
  return "unknown status";
}

rt_status rt_grid_create(const rt_grid_desc* d, rt_grid** out) {
  if (!d || !out) return RT_ERR_ARG;
  *out = nullptr;
  if (!(d->half_size_cm > 0) || !std::isfinite(d->half_size_cm)) return RT_ERR_ARG;
  if (d->n_base < 1 || d->n_base > 2048 || d->max_level < 0 || d->max_level >= kMaxLevels)
    return RT_ERR_ARG;
  if ((long long)d->n_base << d->max_level > (1ll << 24)) return RT_ERR_ARG;
  if (d->n_species < 1 || d->n_species > kMaxSpecies) return RT_ERR_ARG;
  if (d->n_bins < 1 || d->n_bins > kMaxBins || d->n_sed_dirs < 1 || d->n_sed_dirs > 1024)
    return RT_ERR_ARG;
  if (d->n_leaves < 1 || d->n_leaves > 0x7fffffffll || d->n_blocks < 0 ||
      d->n_blocks > 0x7fffffffll)
    return RT_ERR_ARG;
  if (!d->base || !d->rho || !d->nu_edges || (d->n_blocks > 0 && !d->child))
    return RT_ERR_ARG;
  for (int b = 0; b <= d->n_bins; ++b)
    if (!(d->nu_edges[b] > 0) || !std::isfinite(d->nu_edges[b]) ||
        (b > 0 && !(d->nu_edges[b] > d->nu_edges[b - 1])))
      return RT_ERR_ARG;
  const long long S = d->n_species, N = d->n_leaves;
  rt_grid* g = new (std::nothrow) rt_grid();
  if (!g) return RT_ERR_OOM;
  g->desc = *d;
  g->desc.base = nullptr;
  g->desc.child = nullptr;
  g->desc.rho = nullptr;
  g->desc.nu_edges = nullptr;
  if (g->desc.n_temp == 0) g->desc.n_temp = 1024;
  if (g->desc.t_min == 0) g->desc.t_min = 1.0;
  if (g->desc.t_max == 0) g->desc.t_max = 3000.0;
  if (g->desc.n_temp < 3 || g->desc.n_temp > 65536 || !(g->desc.t_min > 0) ||
      !(g->desc.t_max > g->desc.t_min) || d->n_leaves >= kMaxLinkedLeaves) {
    delete g;
    return RT_ERR_ARG;
  }
  g->d0 = 2.0 * d->half_size_cm / d->n_base;
  g->nu.assign(d->nu_edges, d->nu_edges + d->n_bins + 1);
  g->kabs.assign((size_t)S * d->n_bins, 0.0);
  g->ksca.assign((size_t)S * d->n_bins, 0.0);
  g->ghg.assign((size_t)S * d->n_bins, 0.0);
  g->dust_set.assign((size_t)S, 0);
  g->is_pah.assign((size_t)S, 0);
  g->n_carbon.assign((size_t)S, 0);
  g->pah_set.assign((size_t)S, 0);
  g->pah_spec.assign((size_t)S, PahSpec{});
  g->pah_mass.assign((size_t)S, 0.0);
  if (cudaGetDevice(&g->dev) != cudaSuccess) {
    delete g;
    return RT_ERR_CUDA;
  }
  const long long nb = (long long)d->n_base * d->n_base * d->n_base;
  const int B = d->n_bins;
  rt_status st;
#define ALLOC(p, n) if ((st = dalloc(&(p), (n))) != RT_OK) { free_all(g); delete g; return st; }
  ALLOC(g->d_base, (size_t)nb);
  ALLOC(g->d_child, (size_t)d->n_blocks * 8);
  ALLOC(g->d_rho, (size_t)S * N);
  ALLOC(g->d_level, (size_t)N);
  // face links only where the automatic walk reads them (built below); otherwise on
  // the first call that needs them (ensure_links). The path walk's densities by tree
  // slot likewise: now where it is the automatic walk, else on first use.
  const bool path_auto = path_walk_fits(d) && (S == 4 || 4.0 * kRec * (double)N > 4.0e9);
  const bool links_now = !path_auto;
  if (links_now) ALLOC(g->d_links, (size_t)N * kRec);
  if (path_auto) ALLOC(g->d_rho_slot, (size_t)S * (nb + 8 * d->n_blocks));
  ALLOC(g->d_count, (size_t)S * N);
  ALLOC(g->d_sed, (size_t)2 * d->n_sed_dirs * B);
  ALLOC(g->d_counters, (size_t)kNumCounters);
  ALLOC(g->d_next, 1);
  ALLOC(g->d_status, 1);
#undef ALLOC
  // work arrays of the device tree walk and the density conversion
  int32_t *d_ijk = nullptr, *d_blk_ijk = nullptr;
  int8_t* d_blk_level = nullptr;
  unsigned *d_leaf_seen = nullptr, *d_blk_seen = nullptr, *d_err = nullptr;
  double* d_rho64 = nullptr;
  auto free_work = [&]() {
    dfree(d_ijk);
    dfree(d_blk_ijk);
    dfree(d_blk_level);
    dfree(d_leaf_seen);
    dfree(d_blk_seen);
    dfree(d_err);
    dfree(d_rho64);
  };
  const long long nbk = d->n_blocks > 0 ? d->n_blocks : 1;
  if ((st = dalloc(&d_ijk, (size_t)N * 3)) != RT_OK ||
      (st = dalloc(&d_blk_ijk, (size_t)nbk * 3)) != RT_OK ||
      (st = dalloc(&d_blk_level, (size_t)nbk)) != RT_OK ||
      (st = dalloc(&d_leaf_seen, (size_t)((N + 31) >> 5))) != RT_OK ||
      (st = dalloc(&d_blk_seen, (size_t)((nbk + 31) >> 5))) != RT_OK ||
      (st = dalloc(&d_err, 2)) != RT_OK || (st = dalloc(&d_rho64, (size_t)S * N)) != RT_OK) {
    free_work();
    free_all(g);
    delete g;
    return st;
  }
  cudaError_t e = cudaMemcpy(g->d_base, d->base, sizeof(int32_t) * nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d->n_blocks > 0)
    e = cudaMemcpy(g->d_child, d->child, sizeof(int32_t) * 8 * d->n_blocks, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(d_rho64, d->rho, sizeof(double) * S * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, 2 * sizeof(unsigned));
  TreeBuild tb{};
  tb.base = g->d_base;
  tb.child = g->d_child;
  tb.n_leaves = N;
  tb.n_blocks = d->n_blocks;
  tb.n_base = d->n_base;
  tb.max_level = d->max_level;
  tb.level = g->d_level;
  tb.ijk = d_ijk;
  tb.blk_level = d_blk_level;
  tb.blk_ijk = d_blk_ijk;
  tb.leaf_seen = d_leaf_seen;
  tb.blk_seen = d_blk_seen;
  tb.err = d_err;
  tb.max_seen = reinterpret_cast<int*>(d_err + 1);
  if (e == cudaSuccess) e = launch_tree_walk(tb, nullptr);
  if (e == cudaSuccess) e = launch_rho_convert(d_rho64, N, (int)S, g->d0, g->d_rho, d_err, nullptr);
  unsigned host_err[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpy(host_err, d_err, sizeof(host_err), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->d_count, 0, sizeof(unsigned long long) * S * N);
  if (e == cudaSuccess) e = cudaMemset(g->d_sed, 0, sizeof(unsigned long long) * 2 * d->n_sed_dirs * B);
  if (e == cudaSuccess) e = cudaMemset(g->d_counters, 0, sizeof(unsigned long long) * kNumCounters);
  if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(unsigned));
  if (e != cudaSuccess || host_err[0] != 0) {
    free_work();
    free_all(g);
    delete g;
    return e != cudaSuccess ? RT_ERR_CUDA : RT_ERR_ARG;
  }
  g->n_levels_used = (int)host_err[1] + 1;
  g->g.base = g->d_base;
  g->g.child = g->d_child;
  g->g.rho = g->d_rho;
  g->g.level = g->d_level;
  g->g.links = g->d_links;
  g->g.rho_slot = g->d_rho_slot;
  g->g.n_base3 = (int)nb;
  g->g.n_leaves = N;
  g->g.n_blocks = d->n_blocks;
  g->g.n_base = d->n_base;
  g->g.max_level = d->max_level;
  g->g.S = (int)S;
  g->g.B = B;
  g->g.n_dir = d->n_sed_dirs;
  g->g.n_T = g->desc.n_temp;
  // face links of every leaf, built on the device from the leaf corners
  if (links_now) e = launch_build_links(g->g, d_ijk, g->d_links, nullptr);
  if (path_auto && e == cudaSuccess) e = launch_build_rho_slot(g->g, g->d_rho_slot, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  free_work();
  if (e != cudaSuccess) {
    free_all(g);
    delete g;
    return RT_ERR_CUDA;
  }
  *out = g;
  return RT_OK;
}

// The face links, built when a call first needs them (a linked-walk transport,
// peel-off sight lines, a replay, a batch): the tree is walked again for the leaf
// corners, then the links are built from them. Synchronises.
static rt_status ensure_links(rt_grid* g) {
  if (g->d_links) return RT_OK;
  const long long N = g->desc.n_leaves;
  const long long nbk = g->desc.n_blocks > 0 ? g->desc.n_blocks : 1;
  int32_t *d_ijk = nullptr, *d_blk_ijk = nullptr;
  int8_t* d_blk_level = nullptr;
  unsigned *d_leaf_seen = nullptr, *d_blk_seen = nullptr, *d_err = nullptr;
  rt_status st = dalloc(&g->d_links, (size_t)N * kRec);
  if (st == RT_OK) st = dalloc(&d_ijk, (size_t)N * 3);
  if (st == RT_OK) st = dalloc(&d_blk_ijk, (size_t)nbk * 3);
  if (st == RT_OK) st = dalloc(&d_blk_level, (size_t)nbk);
  if (st == RT_OK) st = dalloc(&d_leaf_seen, (size_t)((N + 31) >> 5));
  if (st == RT_OK) st = dalloc(&d_blk_seen, (size_t)((nbk + 31) >> 5));
  if (st == RT_OK) st = dalloc(&d_err, 2);
  cudaError_t e = cudaSuccess;
  if (st == RT_OK) {
    TreeBuild tb{};
    tb.base = g->d_base;
    tb.child = g->d_child;
    tb.n_leaves = N;
    tb.n_blocks = g->desc.n_blocks;
    tb.n_base = g->desc.n_base;
    tb.max_level = g->desc.max_level;
    tb.level = g->d_level;
    tb.ijk = d_ijk;
    tb.blk_level = d_blk_level;
    tb.blk_ijk = d_blk_ijk;
    tb.leaf_seen = d_leaf_seen;
    tb.blk_seen = d_blk_seen;
    tb.err = d_err;
    tb.max_seen = reinterpret_cast<int*>(d_err + 1);
    e = cudaMemset(d_err, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = launch_tree_walk(tb, nullptr);
    if (e == cudaSuccess) e = launch_build_links(g->g, d_ijk, g->d_links, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = RT_ERR_CUDA;
  }
  dfree(d_ijk);
  dfree(d_blk_ijk);
  dfree(d_blk_level);
  dfree(d_leaf_seen);
  dfree(d_blk_seen);
  dfree(d_err);
  if (st != RT_OK) {
    dfree(g->d_links);
    g->d_links = nullptr;
    return st;
  }
  g->g.links = g->d_links;
  return RT_OK;
}

// The path walk's densities by tree slot, built when a path-walk transport first
// needs them. Synchronises.
static rt_status ensure_rho_slot(rt_grid* g) {
  if (g->d_rho_slot) return RT_OK;
  const long long n_slots = (long long)g->g.n_base3 + 8 * g->desc.n_blocks;
  rt_status st = dalloc(&g->d_rho_slot, (size_t)g->desc.n_species * n_slots);
  if (st != RT_OK) return st;
  g->g.rho_slot = g->d_rho_slot;
  cudaError_t e = launch_build_rho_slot(g->g, g->d_rho_slot, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    dfree(g->d_rho_slot);
    g->d_rho_slot = nullptr;
    g->g.rho_slot = nullptr;
    return RT_ERR_CUDA;
  }
  return RT_OK;
}

rt_status rt_grid_destroy(rt_grid* g) {
  if (!g) return RT_OK;
  cudaSetDevice(g->dev);
  free_all(g);
  delete g;
  return RT_OK;
}

rt_status rt_set_dust(rt_grid* g, int species, const double* kabs, const double* ksca,
                      const double* g_hg, int n_bins, int is_pah, int n_carbon) {
  if (!g || !kabs || !ksca || !g_hg) return RT_ERR_ARG;
  if (species < 0 || species >= g->desc.n_species || n_bins != g->desc.n_bins)
    return RT_ERR_ARG;
  double tot_abs = 0;
  for (int b = 0; b < n_bins; ++b) {
    if (!(kabs[b] >= 0) || !(ksca[b] >= 0) || !std::isfinite(kabs[b]) ||
        !std::isfinite(ksca[b]) || !(g_hg[b] > -1) || !(g_hg[b] < 1))
      return RT_ERR_ARG;
    tot_abs += kabs[b];
  }
  if (!(tot_abs > 0)) return RT_ERR_ARG;  // a species must be able to emit
  size_t o = (size_t)species * n_bins;
  std::memcpy(&g->kabs[o], kabs, sizeof(double) * n_bins);
  std::memcpy(&g->ksca[o], ksca, sizeof(double) * n_bins);
  std::memcpy(&g->ghg[o], g_hg, sizeof(double) * n_bins);
  g->dust_set[(size_t)species] = 1;
  g->is_pah[(size_t)species] = is_pah;
  g->n_carbon[(size_t)species] = n_carbon;
  g->tables_ready = false;
  return RT_OK;
}

rt_status rt_emit_star(rt_grid* g, double T_star, double L_star, const double pos_cm[3],
                       int source_kind, const double beam_dir[3],
                       uint64_t n_packages_total) {
  if (!g || !pos_cm) return RT_ERR_ARG;
  if (!(T_star > 0) || !(L_star > 0) || !std::isfinite(T_star) || !std::isfinite(L_star))
    return RT_ERR_ARG;
  if (n_packages_total == 0 || !finite3(pos_cm)) return RT_ERR_ARG;
  double H = g->desc.half_size_cm;
  for (int a = 0; a < 3; ++a)
    if (pos_cm[a] < -H || pos_cm[a] > H) return RT_ERR_ARG;
  if (source_kind != RT_SOURCE_POINT && source_kind != RT_SOURCE_BEAM) return RT_ERR_ARG;
  double bd[3] = {0, 0, 1};
  if (source_kind == RT_SOURCE_BEAM) {
    if (!beam_dir || !finite3(beam_dir)) return RT_ERR_ARG;
    double nrm = std::sqrt(beam_dir[0] * beam_dir[0] + beam_dir[1] * beam_dir[1] +
                           beam_dir[2] * beam_dir[2]);
    if (!(nrm > 0)) return RT_ERR_ARG;
    for (int a = 0; a < 3; ++a) bd[a] = beam_dir[a] / nrm;
  }
  g->T_star = T_star;
  g->L_star = L_star;
  for (int a = 0; a < 3; ++a) {
    g->pos[a] = pos_cm[a];
    g->beam[a] = bd[a];
  }
  g->source_kind = source_kind;
  g->n_total = n_packages_total;
  g->star_set = true;
  g->tables_ready = false;
  return RT_OK;
}

rt_status rt_set_frozen_temperatures(rt_grid* g, const float* T, int mem, void* stream) {
  if (!g || !T) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  if (!g->d_Tfrozen && (st = dalloc(&g->d_Tfrozen, n)) != RT_OK) return st;
  if (!g->d_ufrozen && (st = dalloc(&g->d_ufrozen, n)) != RT_OK) return st;
  RT_CUDA(cudaMemcpyAsync(g->d_Tfrozen, T, sizeof(float) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyHostToDevice,
                          s));
  RT_CUDA(launch_frozen_u(g->g, g->tab, g->d_Tfrozen, g->d_ufrozen, (float)g->desc.t_min, s));
  if (mem != RT_MEM_DEVICE) RT_CUDA(cudaStreamSynchronize(s));
  g->frozen_ready = true;
  return RT_OK;
}

rt_status rt_reset(rt_grid* g, void* stream) {
  if (!g) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  const size_t S = g->desc.n_species, N = g->desc.n_leaves;
  RT_CUDA(cudaMemsetAsync(g->d_count, 0, sizeof(unsigned long long) * S * N, s));
  RT_CUDA(cudaMemsetAsync(g->d_sed, 0,
                          sizeof(unsigned long long) * 2 * g->desc.n_sed_dirs * g->desc.n_bins,
                          s));
  RT_CUDA(cudaMemsetAsync(g->d_counters, 0, sizeof(unsigned long long) * kNumCounters, s));
  RT_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(unsigned), s));
  // only the rows of PAH-active cells hold counts: clear those and their flags
  if (g->d_pahabs)
    RT_CUDA(launch_pah_clear(g->d_pah_flag, (long long)N, g->tab.n_coarse, g->n_pah,
                             g->d_pahabs, g->d_pah_flag, s));
  if (g->d_pathabs) RT_CUDA(cudaMemsetAsync(g->d_pathabs, 0, sizeof(float) * S * N, s));
  if (g->images) {
    const size_t n = (size_t)g->peel.n_planes * g->peel.ny * g->peel.nx;
    RT_CUDA(cudaMemsetAsync(g->d_image, 0, sizeof(double) * n, s));
    RT_CUDA(cudaMemsetAsync(g->d_nemit, 0, sizeof(unsigned long long) * g->desc.n_bins, s));
  }
  return RT_OK;
}

// The path-length tallies are allocated (and zeroed) the first time a launch asks
// for them.
static rt_status ensure_pathabs(rt_grid* g, const rt_run_opts* o, cudaStream_t s) {
  if (!o || !(o->estimators & RT_EST_PATHLENGTH) || g->d_pathabs) return RT_OK;
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  rt_status st = dalloc(&g->d_pathabs, n);
  if (st != RT_OK) return st;
  RT_CUDA(cudaMemsetAsync(g->d_pathabs, 0, sizeof(float) * n, s));
  return RT_OK;
}

static rt_status fill_run(rt_grid* g, uint64_t n_packages, uint64_t seed, uint64_t first,
                          const rt_run_opts* o, DevRun* r) {
  int mode = o ? o->mode : RT_REEMIT_BW;
  if (mode < 0 || mode > 2) return RT_ERR_ARG;
  if (o && o->count_scale < 0) return RT_ERR_ARG;
  if (mode == RT_REEMIT_FROZEN && !g->frozen_ready) return RT_ERR_STATE;
  *r = DevRun{};
  r->seed = seed;
  r->first_id = first;
  r->n_packages = n_packages;
  r->max_events = (o && o->max_events) ? o->max_events : 10000000ull;
  if (r->max_events > 0xffffffffull - 1) r->max_events = 0xffffffffull - 1;
  r->next = g->d_next;
  r->count = g->d_count;
  r->sed = g->d_sed;
  r->counters = g->d_counters;
  r->status = g->d_status;
  r->pahabs = g->d_pahabs;
  r->pah_flag = g->d_pah_flag;
  r->pathabs = (o && (o->estimators & RT_EST_PATHLENGTH)) ? g->d_pathabs : nullptr;
  for (int a = 0; a < 3; ++a) {
    double p = (g->pos[a] + g->desc.half_size_cm) / g->d0;
    r->src64[a] = p;
    r->src[a] = (float)p;
    r->beam64[a] = g->beam[a];
    r->beam[a] = (float)g->beam[a];
  }
  r->source_kind = g->source_kind;
  r->mode = mode;
  r->refill_period = (o && o->refill_period > 0) ? o->refill_period : 32;
  r->interaction_batch = (o && o->interaction_batch > 0) ? o->interaction_batch : 8;
  r->count_scale = (o && o->count_scale > 1) ? (float)o->count_scale : 1.0f;
  double budget = (o && o->budget_s > 0) ? o->budget_s : 120.0;
  r->budget_ns = (unsigned long long)(budget * 1e9);
  return RT_OK;
}

// The pool walk for this grid: the path walk when asked for, or (automatic) for four
// species (the link record holds no densities then, and the path walk measured faster
// from 1.9e7 to 1.7e8 cells) and whenever the face-link records exceed 4 GB; grids
// deeper than the path walk serves keep the links.
static bool use_path_walk(const rt_grid* g, const rt_run_opts* o) {
  if (!path_walk_fits(&g->desc)) return false;
  const int w = o ? o->walk : RT_WALK_AUTO;
  if (w == RT_WALK_PATH) return true;
  if (w == RT_WALK_LINKED) return false;
  const double rec_bytes = 4.0 * kRec * (double)g->desc.n_leaves;
  return g->desc.n_species == 4 || rec_bytes > 4.0e9;
}

rt_status rt_transport(rt_grid* g, uint64_t n_packages, uint64_t seed,
                       uint64_t first_package_id, const rt_run_opts* o, void* stream) {
  if (!g) return RT_ERR_ARG;
  int kernel = o ? o->kernel : RT_KERNEL_POOL;
  int threads = (o && o->threads > 0) ? o->threads : 256;
  if (kernel < 0 || kernel > 2 || threads % 32 != 0 || threads > 256) return RT_ERR_ARG;
  if (o && (o->walk < RT_WALK_AUTO || o->walk > RT_WALK_PATH)) return RT_ERR_ARG;
  if (o && (o->blocks_per_sm < 0 || o->blocks_per_sm > 32 || o->refill_period < 0 ||
            o->interaction_batch < 0 || o->interaction_batch > 32 ||
            (o->estimators & ~RT_EST_PATHLENGTH)))
    return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  if ((st = ensure_pathabs(g, o, s)) != RT_OK) return st;
  if (first_package_id > g->n_total || n_packages > g->n_total - first_package_id)
    return RT_ERR_RANGE;
  if (n_packages == 0) return RT_OK;
  DevRun r;
  if ((st = fill_run(g, n_packages, seed, first_package_id, o, &r)) != RT_OK) return st;
  DevTables t = g->tab;
  t.u_frozen = g->d_ufrozen;
  t.pah_cell_cdf = g->d_pah_cell_cdf;
  if (g->images && kernel != RT_KERNEL_POOL) return RT_ERR_STATE;
  if (kernel == RT_KERNEL_POOL) {
    // the path walk runs without images and without the path-length tally
    const bool path = !g->images && !r.pathabs && use_path_walk(g, o);
    if (!path && (st = ensure_links(g)) != RT_OK) return st;
    if (path && (st = ensure_rho_slot(g)) != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(g->d_next, 0, sizeof(unsigned long long), s));
    RT_CUDA(launch_transport_pool(g->g, t, r, o ? o->blocks_per_sm : 0, threads, s,
                                  g->images ? &g->peel : nullptr, path));
    if (g->images) {
      RT_CUDA(launch_peel_source(g->g, t, r, g->peel, s));
      RT_CUDA(launch_peel_trace(g->g, t, r, g->peel, s));
      RT_CUDA(cudaMemsetAsync(g->d_nev, 0, sizeof(unsigned long long), s));
    }
  } else {
    RT_CUDA(launch_transport_plain(g->g, t, r, kernel == RT_KERNEL_PLAIN_F64, threads, s));
  }
  return RT_OK;
}

rt_status rt_cell_temperatures(rt_grid* g, float* T_out, int mem, void* stream) {
  if (!g || !T_out) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  float* dst = T_out;
  if (mem != RT_MEM_DEVICE) {
    if (!g->d_Tscratch && (st = dalloc(&g->d_Tscratch, n)) != RT_OK) return st;
    dst = g->d_Tscratch;
  }
  RT_CUDA(launch_temperatures(g->g, g->tab, g->d_count, dst, g->d_counters, s));
  if (mem != RT_MEM_DEVICE) {
    RT_CUDA(cudaMemcpyAsync(T_out, dst, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    return sync_status(g, s);
  }
  return RT_OK;
}

rt_status rt_cell_temperatures_pathlength(rt_grid* g, float* T_out, int mem, void* stream) {
  if (!g || !T_out) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  if (!g->d_pathabs) return RT_ERR_STATE;
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  float* dst = T_out;
  if (mem != RT_MEM_DEVICE) {
    if (!g->d_Tscratch && (st = dalloc(&g->d_Tscratch, n)) != RT_OK) return st;
    dst = g->d_Tscratch;
  }
  RT_CUDA(launch_temperatures(g->g, g->tab, g->d_count, dst, g->d_counters, s, g->d_pathabs));
  if (mem != RT_MEM_DEVICE) {
    RT_CUDA(cudaMemcpyAsync(T_out, dst, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    return sync_status(g, s);
  }
  return RT_OK;
}

rt_status rt_pathlength(rt_grid* g, float* out, int mem, void* stream) {
  if (!g || !out) return RT_ERR_ARG;
  if (!g->d_pathabs) return RT_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  RT_CUDA(cudaMemcpyAsync(out, g->d_pathabs, sizeof(float) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyDeviceToHost,
                          s));
  if (mem != RT_MEM_DEVICE) return sync_status(g, s);
  return RT_OK;
}

rt_status rt_sed(rt_grid* g, uint64_t* counts_out, int mem, double* eps_out, void* stream) {
  if (!g || !counts_out) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  const size_t n = (size_t)2 * g->desc.n_sed_dirs * g->desc.n_bins;
  RT_CUDA(cudaMemcpyAsync(counts_out, g->d_sed, sizeof(unsigned long long) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyDeviceToHost,
                          s));
  if (eps_out) *eps_out = g->eps;
  if (mem != RT_MEM_DEVICE) return sync_status(g, s);
  return RT_OK;
}

rt_status rt_counts(rt_grid* g, uint64_t* out, int mem, void* stream) {
  if (!g || !out) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  RT_CUDA(cudaMemcpyAsync(out, g->d_count, sizeof(unsigned long long) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyDeviceToHost,
                          s));
  if (mem != RT_MEM_DEVICE) return sync_status(g, s);
  return RT_OK;
}

rt_status rt_set_counts(rt_grid* g, const uint64_t* in, int mem, void* stream) {
  if (!g || !in) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  RT_CUDA(cudaMemcpyAsync(g->d_count, in, sizeof(unsigned long long) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyHostToDevice,
                          s));
  if (mem != RT_MEM_DEVICE) RT_CUDA(cudaStreamSynchronize(s));
  return RT_OK;
}

rt_status rt_get_counters(rt_grid* g, rt_counters* out) {
  if (!g || !out) return RT_ERR_ARG;
  RT_CUDA(cudaSetDevice(g->dev));
  RT_CUDA(cudaDeviceSynchronize());
  unsigned long long c[kNumCounters];
  RT_CUDA(cudaMemcpy(c, g->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
  out->emitted = c[kCEmitted];
  out->escaped = c[kCEscaped];
  out->capped = c[kCCapped];
  out->absorptions = c[kCAbsorptions];
  out->scatters = c[kCScatters];
  out->crossings = c[kCCrossings];
  out->errors = c[kCErrors];
  out->clamped = c[kCClamped];
  out->levels = c[kCLevels];
  out->peel_events = c[kCPeelEvents];
  out->peel_crossings = c[kCPeelCrossings];
  out->peel_dropped = c[kCPeelDropped];
  return sync_status(g, nullptr);
}

rt_status rt_set_images(rt_grid* g, const rt_image_desc* d, const int32_t* plane_of_bin) {
  if (!g) return RT_ERR_ARG;
  RT_CUDA(cudaSetDevice(g->dev));
  if (!d) {  // images off
    RT_CUDA(cudaDeviceSynchronize());
    dfree(g->d_plane_of_bin);
    dfree(g->d_image);
    dfree(g->d_nemit);
    dfree(g->d_ev);
    dfree(g->d_ev_bin);
    dfree(g->d_nev);
    dfree(g->d_iscratch);
    g->iscratch_n = 0;
    g->images = false;
    g->peel = DevPeel{};
    return RT_OK;
  }
  const int B = g->desc.n_bins;
  if (!plane_of_bin || !finite3(d->obs_dir) || d->nx < 1 || d->ny < 1 ||
      d->nx > kMaxImageSide || d->ny > kMaxImageSide || !(d->half_width_cm > 0) ||
      !std::isfinite(d->half_width_cm) || !(d->tau_max >= 0) || !std::isfinite(d->tau_max))
    return RT_ERR_ARG;
  double on = std::sqrt(d->obs_dir[0] * d->obs_dir[0] + d->obs_dir[1] * d->obs_dir[1] +
                        d->obs_dir[2] * d->obs_dir[2]);
  if (!(on > 0)) return RT_ERR_ARG;
  int n_planes = 0;
  for (int b = 0; b < B; ++b) {
    if (plane_of_bin[b] < -1 || plane_of_bin[b] >= B) return RT_ERR_ARG;
    if (plane_of_bin[b] + 1 > n_planes) n_planes = plane_of_bin[b] + 1;
  }
  if (n_planes == 0) return RT_ERR_ARG;
  const size_t n_img = (size_t)n_planes * d->ny * d->nx;
  if (n_img > kMaxImagePixels) return RT_ERR_TOO_LARGE;
  const unsigned long long cap = d->event_capacity ? d->event_capacity : kPeelCapacityDefault;
  if (cap > kPeelCapacityMax) return RT_ERR_TOO_LARGE;
  RT_CUDA(cudaDeviceSynchronize());
  dfree(g->d_plane_of_bin);
  dfree(g->d_image);
  dfree(g->d_nemit);
  dfree(g->d_ev);
  dfree(g->d_ev_bin);
  dfree(g->d_nev);
  dfree(g->d_iscratch);
  g->iscratch_n = 0;
  g->images = false;
  rt_status st;
  if ((st = dalloc(&g->d_plane_of_bin, (size_t)B)) != RT_OK ||
      (st = dalloc(&g->d_image, n_img)) != RT_OK || (st = dalloc(&g->d_nemit, (size_t)B)) != RT_OK ||
      (st = dalloc(&g->d_ev, (size_t)cap)) != RT_OK ||
      (st = dalloc(&g->d_ev_bin, (size_t)cap)) != RT_OK || (st = dalloc(&g->d_nev, 1)) != RT_OK)
    return st;
  RT_CUDA(cudaMemset(g->d_nev, 0, sizeof(unsigned long long)));
  RT_CUDA(cudaMemcpy(g->d_plane_of_bin, plane_of_bin, sizeof(int) * B, cudaMemcpyHostToDevice));
  RT_CUDA(cudaMemset(g->d_image, 0, sizeof(double) * n_img));
  RT_CUDA(cudaMemset(g->d_nemit, 0, sizeof(unsigned long long) * B));
  // image axes: e1 = normalise(z x o) (x when o lies along z), e2 = o x e1
  double o[3] = {d->obs_dir[0] / on, d->obs_dir[1] / on, d->obs_dir[2] / on};
  double e1[3] = {1, 0, 0};
  if (std::fabs(o[2]) < 0.999999) {
    double nn = std::sqrt(o[0] * o[0] + o[1] * o[1]);
    e1[0] = -o[1] / nn;
    e1[1] = o[0] / nn;
    e1[2] = 0;
  }
  double e2[3] = {o[1] * e1[2] - o[2] * e1[1], o[2] * e1[0] - o[0] * e1[2],
                  o[0] * e1[1] - o[1] * e1[0]};
  DevPeel& pe = g->peel;
  pe = DevPeel{};
  pe.plane_of_bin = g->d_plane_of_bin;
  pe.image = g->d_image;
  pe.n_emit = g->d_nemit;
  pe.ev = g->d_ev;
  pe.ev_bin = g->d_ev_bin;
  pe.n_ev = g->d_nev;
  pe.capacity = cap;
  for (int a = 0; a < 3; ++a) {
    pe.o[a] = (float)o[a];
    pe.e1[a] = (float)e1[a];
    pe.e2[a] = (float)e2[a];
  }
  pe.centre = (float)(0.5 * g->desc.n_base);
  pe.sx = (float)(g->d0 * d->nx / (2.0 * d->half_width_cm));
  pe.sy = (float)(g->d0 * d->ny / (2.0 * d->half_width_cm));
  pe.nx = d->nx;
  pe.ny = d->ny;
  pe.n_planes = n_planes;
  pe.tau_max = d->tau_max > 0 ? (float)d->tau_max : 40.0f;
  g->images = true;
  return RT_OK;
}

// Device output of n doubles: the caller's buffer, or the handle's scratch for a host copy.
static double* image_buffer(rt_grid* g, double* out, int mem, size_t n, rt_status* st) {
  *st = RT_OK;
  if (mem == RT_MEM_DEVICE) return out;
  if (g->iscratch_n < n) {
    dfree(g->d_iscratch);
    g->iscratch_n = 0;
    if ((*st = dalloc(&g->d_iscratch, n)) != RT_OK) return nullptr;
    g->iscratch_n = n;
  }
  return g->d_iscratch;
}

rt_status rt_images(rt_grid* g, double* out, int mem, void* stream) {
  if (!g || !out) return RT_ERR_ARG;
  if (!g->images) return RT_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  const size_t n = (size_t)g->peel.n_planes * g->peel.ny * g->peel.nx;
  double* dst = image_buffer(g, out, mem, n, &st);
  if (!dst) return st;
  RT_CUDA(launch_image_out(g->d_image, (long long)n, g->eps, dst, s));
  if (mem != RT_MEM_DEVICE) {
    RT_CUDA(cudaMemcpyAsync(out, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if ((st = sync_status(g, s)) != RT_OK) return st;
    unsigned long long dropped = 0;
    RT_CUDA(cudaMemcpy(&dropped, g->d_counters + kCPeelDropped, sizeof(dropped),
                       cudaMemcpyDeviceToHost));
    return dropped ? RT_ERR_RANGE : RT_OK;
  }
  return RT_OK;
}

rt_status rt_image_profile(rt_grid* g, int plane_a, int plane_b, int half_rows, double* out,
                           int mem, void* stream) {
  if (!g || !out) return RT_ERR_ARG;
  if (!g->images) return RT_ERR_STATE;
  const DevPeel& pe = g->peel;
  if (plane_a < 0 || plane_a >= pe.n_planes || plane_b < -1 || plane_b >= pe.n_planes ||
      half_rows < 0)
    return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  double* dst = image_buffer(g, out, mem, (size_t)pe.nx, &st);
  if (!dst) return st;
  RT_CUDA(launch_image_profile(g->d_image, pe.nx, pe.ny, plane_a, plane_b, half_rows, g->eps,
                               dst, s));
  if (mem != RT_MEM_DEVICE) {
    RT_CUDA(cudaMemcpyAsync(out, dst, sizeof(double) * pe.nx, cudaMemcpyDeviceToHost, s));
    return sync_status(g, s);
  }
  return RT_OK;
}

rt_status rt_trace(rt_grid* g, const uint64_t* ids, int64_t n, uint64_t seed,
                   uint64_t max_events, int64_t* out) {
  if (!g || (n > 0 && (!ids || !out)) || n < 0) return RT_ERR_ARG;
  if (n == 0) return RT_OK;
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, nullptr);
  if (st != RT_OK) return st;
  if ((st = ensure_links(g)) != RT_OK) return st;
  if (!g->frozen_ready) return RT_ERR_STATE;
  rt_run_opts o{};
  o.mode = RT_REEMIT_FROZEN;
  o.max_events = max_events;
  DevRun r;
  if ((st = fill_run(g, 0, seed, 0, &o, &r)) != RT_OK) return st;
  DevTables t = g->tab;
  t.u_frozen = g->d_ufrozen;
  t.pah_cell_cdf = g->d_pah_cell_cdf;
  unsigned long long* d_ids = nullptr;
  long long* d_out = nullptr;
  if ((st = dalloc(&d_ids, (size_t)n)) != RT_OK) return st;
  if ((st = dalloc(&d_out, (size_t)n * 9)) != RT_OK) {
    dfree(d_ids);
    return st;
  }
  cudaError_t e = cudaMemcpy(d_ids, ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_trace(g->g, t, r, d_ids, n, d_out, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(int64_t) * 9 * n, cudaMemcpyDeviceToHost);
  dfree(d_ids);
  dfree(d_out);
  if (e != cudaSuccess) return RT_ERR_CUDA;
  return sync_status(g, nullptr);
}

rt_status rt_trace_events(rt_grid* g, const uint64_t* ids, int64_t n, uint64_t seed,
                          uint64_t max_events, int64_t max_out, rt_event* out,
                          int64_t* n_out) {
  static_assert(sizeof(rt_event) == sizeof(TraceEvent), "event record layouts differ");
  if (!g || n < 0 || max_out < 0 || (n > 0 && (!ids || !n_out || (max_out > 0 && !out))))
    return RT_ERR_ARG;
  if (n == 0) return RT_OK;
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, nullptr);
  if (st != RT_OK) return st;
  if ((st = ensure_links(g)) != RT_OK) return st;
  if (!g->frozen_ready) return RT_ERR_STATE;
  rt_run_opts o{};
  o.mode = RT_REEMIT_FROZEN;
  o.max_events = max_events;
  DevRun r;
  if ((st = fill_run(g, 0, seed, 0, &o, &r)) != RT_OK) return st;
  DevTables t = g->tab;
  t.u_frozen = g->d_ufrozen;
  t.pah_cell_cdf = g->d_pah_cell_cdf;
  unsigned long long* d_ids = nullptr;
  long long *d_rec = nullptr, *d_n = nullptr;
  TraceEvent* d_ev = nullptr;
  const size_t n_ev = (size_t)n * (size_t)max_out;
  if ((st = dalloc(&d_ids, (size_t)n)) == RT_OK && (st = dalloc(&d_rec, (size_t)n * 9)) == RT_OK &&
      (st = dalloc(&d_n, (size_t)n)) == RT_OK && (n_ev == 0 || (st = dalloc(&d_ev, n_ev)) == RT_OK)) {
    cudaError_t e = cudaMemcpy(d_ids, ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = launch_trace(g->g, t, r, d_ids, n, d_rec, nullptr, d_ev, max_out, d_n);
    if (e == cudaSuccess && n_ev)
      e = cudaMemcpy(out, d_ev, sizeof(TraceEvent) * n_ev, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(n_out, d_n, sizeof(int64_t) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = RT_ERR_CUDA;
  }
  dfree(d_ids);
  dfree(d_rec);
  dfree(d_n);
  dfree(d_ev);
  if (st != RT_OK) return st;
  return sync_status(g, nullptr);
}

rt_status rt_set_pah(rt_grid* g, int species, int n_carbon, int n_hydrogen, double mol_mass_g,
                     const double* modes, int n_groups, int n_levels, double t_top) {
  if (!g || !modes) return RT_ERR_ARG;
  if (species < 0 || species >= g->desc.n_species || !g->is_pah[(size_t)species])
    return RT_ERR_ARG;
  if (n_carbon < 1 || n_hydrogen < 0 || !(mol_mass_g > 0) || n_groups < 1 ||
      n_groups > kMaxModeGroups)
    return RT_ERR_ARG;
  if (n_levels == 0) n_levels = 400;
  if (t_top == 0) t_top = 2500.0;
  if (n_levels < 16 || n_levels > 2048 || !(t_top > 0) || !std::isfinite(t_top))
    return RT_ERR_ARG;
  PahSpec sp{};
  sp.n_groups = n_groups;
  for (int i = 0; i < n_groups; ++i) {
    if (!(modes[2 * i] > 0) || !(modes[2 * i + 1] > 0)) return RT_ERR_ARG;
    sp.n_modes[i] = modes[2 * i];
    sp.theta[i] = modes[2 * i + 1];
  }
  g->pah_spec[(size_t)species] = sp;
  g->pah_mass[(size_t)species] = mol_mass_g;
  g->n_carbon[(size_t)species] = n_carbon;
  g->pah_set[(size_t)species] = 1;
  g->pah_levels = n_levels;
  g->pah_t_top = t_top;
  g->tables_ready = false;
  (void)n_hydrogen;
  return RT_OK;
}

rt_status rt_pah_absorbed(rt_grid* g, uint32_t* out, int mem, void* stream) {
  if (!g || !out) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  if (g->n_pah == 0) return RT_ERR_STATE;
  const size_t n = (size_t)g->n_pah * g->desc.n_leaves * g->tab.n_coarse;
  RT_CUDA(cudaMemcpyAsync(out, g->d_pahabs, sizeof(unsigned) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyDeviceToHost,
                          s));
  if (mem != RT_MEM_DEVICE) return sync_status(g, s);
  return RT_OK;
}

rt_status rt_set_pah_spectra(rt_grid* g, int pah, int64_t first_cell, int64_t n_cells,
                             const float* J, int mem, void* stream) {
  if (!g) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  if (!J) {  // back to the templates everywhere
    if (g->d_pah_cell_cdf) {
      RT_CUDA(cudaStreamSynchronize(s));
      RT_CUDA(cudaDeviceSynchronize());
      dfree(g->d_pah_cell_cdf);
    }
    return RT_OK;
  }
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  const long long N = g->desc.n_leaves;
  const int B = g->desc.n_bins;
  if (g->n_pah == 0) return RT_ERR_STATE;
  if (pah < 0 || pah >= g->n_pah || first_cell < 0 || n_cells < 0 || first_cell > N ||
      n_cells > N - first_cell)
    return RT_ERR_ARG;
  if (!g->d_pah_cell_cdf) {
    const size_t n = (size_t)g->n_pah * N * B;
    if ((st = dalloc(&g->d_pah_cell_cdf, n)) != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(g->d_pah_cell_cdf, 0, sizeof(float) * n, s));
  }
  float* dst = g->d_pah_cell_cdf + ((size_t)pah * N + first_cell) * B;
  if (mem == RT_MEM_DEVICE) {
    RT_CUDA(launch_pah_cell_cdf(J, n_cells, B, dst, s));
    return RT_OK;
  }
  // host rows: through the handle's scratch, a chunk at a time
  const long long chunk = n_cells < (1ll << 18) ? n_cells : (1ll << 18);
  if (g->jscratch_n < (size_t)chunk * B) {
    RT_CUDA(cudaStreamSynchronize(s));
    dfree(g->d_jscratch);
    g->jscratch_n = 0;
    if ((st = dalloc(&g->d_jscratch, (size_t)chunk * B)) != RT_OK) return st;
    g->jscratch_n = (size_t)chunk * B;
  }
  for (long long c0 = 0; c0 < n_cells; c0 += chunk) {
    const long long nc = n_cells - c0 < chunk ? n_cells - c0 : chunk;
    RT_CUDA(cudaMemcpyAsync(g->d_jscratch, J + (size_t)c0 * B, sizeof(float) * nc * B,
                            cudaMemcpyHostToDevice, s));
    RT_CUDA(launch_pah_cell_cdf(g->d_jscratch, nc, B, dst + (size_t)c0 * B, s));
  }
  return sync_status(g, s);
}

rt_status rt_pah_temperature_distribution(const rt_pah_pt_case* cases, int n_cases,
                                           const double* nu_edges, int n_bins,
                                           const double* sigma, int n_levels, double t_sub,
                                           double* P_out, double* T_out, double* p_above_out,
                                           double* emission_out, void* stream) {
  if (!cases || !nu_edges || !sigma || !P_out || !T_out || !p_above_out || !emission_out)
    return RT_ERR_ARG;
  if (n_cases < 1 || n_cases > 65535 || n_bins < 1 || n_bins > kMaxBins || n_levels < 16 ||
      n_levels > 4096 || !(t_sub >= 0) || !std::isfinite(t_sub))
    return RT_ERR_ARG;
  for (int b = 0; b <= n_bins; ++b)
    if (!(nu_edges[b] > 0) || !std::isfinite(nu_edges[b]) || (b > 0 && !(nu_edges[b] > nu_edges[b - 1])))
      return RT_ERR_ARG;
  std::vector<PtCase> pc((size_t)n_cases);
  for (int i = 0; i < n_cases; ++i) {
    const rt_pah_pt_case& c = cases[i];
    if (c.n_groups < 1 || c.n_groups > kMaxModeGroups || !(c.h_nu_erg > 0) ||
        !std::isfinite(c.h_nu_erg) || !(c.rate >= 0) || !std::isfinite(c.rate) ||
        !(c.t_top >= 0) || !std::isfinite(c.t_top))
      return RT_ERR_ARG;
    PtCase& d = pc[(size_t)i];
    d = PtCase{};
    d.spec.n_groups = c.n_groups;
    for (int k = 0; k < c.n_groups; ++k) {
      if (!(c.modes[k][0] > 0) || !(c.modes[k][1] > 0)) return RT_ERR_ARG;
      d.spec.n_modes[k] = c.modes[k][0];
      d.spec.theta[k] = c.modes[k][1];
    }
    d.h_nu = c.h_nu_erg;
    d.rate = c.rate;
    d.t_top = c.t_top > 0 ? c.t_top : 2500.0;
  }
  for (size_t i = 0; i < (size_t)n_cases * n_bins; ++i)
    if (!(sigma[i] >= 0) || !std::isfinite(sigma[i])) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  const size_t nP = (size_t)n_cases * n_levels, nE = (size_t)n_cases * n_bins;
  PtCase* d_cases = nullptr;
  double *d_nu = nullptr, *d_sig = nullptr, *d_P = nullptr, *d_T = nullptr, *d_a = nullptr,
         *d_em = nullptr;
  rt_status st = RT_OK;
  if ((st = dalloc(&d_cases, (size_t)n_cases)) == RT_OK &&
      (st = dalloc(&d_nu, (size_t)n_bins + 1)) == RT_OK && (st = dalloc(&d_sig, nE)) == RT_OK &&
      (st = dalloc(&d_P, nP)) == RT_OK && (st = dalloc(&d_T, nP)) == RT_OK &&
      (st = dalloc(&d_a, (size_t)n_cases)) == RT_OK && (st = dalloc(&d_em, nE)) == RT_OK) {
    cudaError_t e = cudaMemcpyAsync(d_cases, pc.data(), sizeof(PtCase) * n_cases,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_nu, nu_edges, sizeof(double) * (n_bins + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_sig, sigma, sizeof(double) * nE, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_pah_pt(d_cases, n_cases, d_nu, n_bins, d_sig, n_levels, t_sub, d_P, d_T, d_a,
                        d_em, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P_out, d_P, sizeof(double) * nP, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(T_out, d_T, sizeof(double) * nP, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p_above_out, d_a, sizeof(double) * n_cases, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(emission_out, d_em, sizeof(double) * nE, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = cuda_status(e);
  }
  dfree(d_cases);
  dfree(d_nu);
  dfree(d_sig);
  dfree(d_P);
  dfree(d_T);
  dfree(d_a);
  dfree(d_em);
  return st;
}

// Work arrays of rt_pah_emission: cell lists for `cells` cells; the network's
// inputs, outputs and flags for `batch` rows only when a surrogate is used.
static rt_status surrogate_scratch(rt_grid* g, long long cells, long long batch, bool with_net) {
  const int K = g->tab.n_coarse, B = g->desc.n_bins, P = g->n_pah;
  rt_status st;
  if (cells > g->list_cap) {
    dfree(g->d_list);
    dfree(g->d_list2);
    g->list_cap = 0;
    if ((st = dalloc(&g->d_list, (size_t)cells)) != RT_OK) return st;
    if ((st = dalloc(&g->d_list2, (size_t)cells)) != RT_OK) return st;
    g->list_cap = cells;
  }
  if (with_net && batch > g->sur_cap) {
    dfree(g->d_sx);
    dfree(g->d_sy);
    dfree(g->d_spabs);
    dfree(g->d_sflag);
    g->sur_cap = 0;
    if ((st = dalloc(&g->d_sflag, (size_t)batch)) != RT_OK) return st;
    if ((st = dalloc(&g->d_sx, (size_t)batch * (K + 2))) != RT_OK) return st;
    if ((st = dalloc(&g->d_sy, (size_t)P * batch * B)) != RT_OK) return st;
    if ((st = dalloc(&g->d_spabs, (size_t)P * batch)) != RT_OK) return st;
    g->sur_cap = batch;
  }
  if (!g->d_scount && (st = dalloc(&g->d_scount, 1)) != RT_OK) return st;
  if (!g->d_ucount && (st = dalloc(&g->d_ucount, 2)) != RT_OK) return st;
  return RT_OK;
}

static float* output_buffer(rt_grid* g, float* j_out, int mem, size_t n, rt_status* st) {
  *st = RT_OK;
  if (mem == RT_MEM_DEVICE) return j_out;
  if (g->jscratch_n < n) {
    dfree(g->d_jscratch);
    g->jscratch_n = 0;
    if ((*st = dalloc(&g->d_jscratch, n)) != RT_OK) return nullptr;
    g->jscratch_n = n;
  }
  return g->d_jscratch;
}

// Shared part of rt_pah_emission (rows = the cells of a range) and
// rt_pah_emission_active (rows = a compact list of the PAH-active cells).
// Range form: dst [n_cells][B] row c is cell first_cell + c. Compact form
// (cells_dev != nullptr): the PAH-active cells of the whole grid are listed, row i of
// dst is cell list[i], copied to cells_dev; at most max_rows rows.
static rt_status pah_emission_impl(rt_grid* g, int64_t first_cell, int64_t n_cells, int pah,
                                   int mode, const rt_mlp* surrogate, float tol,
                                   float* (*get_dst)(rt_grid*, void*, size_t, rt_status*),
                                   void* dst_ctx, int32_t* cells_dev, int64_t max_rows,
                                   int64_t* n_rows_out, uint64_t* n_fallback_out,
                                   float** dst_out, cudaStream_t s) {
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  if (g->n_pah == 0) return RT_ERR_STATE;
  if (pah < -1 || pah >= g->n_pah) return RT_ERR_ARG;
  const int B = g->desc.n_bins, K = g->tab.n_coarse, F = K + 2;
  (void)K;
  if (mode != RT_PAH_EXACT) {
    int ni = 0, no = 0;
    if (rt_mlp_dims(surrogate, &ni, &no) != RT_OK || ni != F || no != B) return RT_ERR_ARG;
  }
  const bool compact = cells_dev != nullptr;
  if (n_fallback_out) *n_fallback_out = 0;
  if (n_rows_out) *n_rows_out = 0;
  *dst_out = nullptr;
  if (n_cells == 0) return RT_OK;
  rt_mlp* m = const_cast<rt_mlp*>(surrogate);
  float x_lo = -1e30f, x_hi = 1e30f;
  if (m) rt_mlp_get_range(m, &x_lo, &x_hi);
  if ((st = surrogate_scratch(g, n_cells, 0, false)) != RT_OK) return st;
  const float t = mode == RT_PAH_AUTO ? tol : 1e30f;
  unsigned long long n_fallback = 0;
  float* dst = nullptr;
  if (!compact) {
    dst = get_dst(g, dst_ctx, (size_t)n_cells * B, &st);
    if (st != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(dst, 0, sizeof(float) * (size_t)n_cells * B, s));
  }
  // the cells where a PAH absorbed anything, in one list for the whole range
  RT_CUDA(cudaMemsetAsync(g->d_ucount, 0, 2 * sizeof(unsigned), s));
  RT_CUDA(launch_compact(g->ptab, g->d_pah_flag, g->desc.n_leaves, pah, first_cell, n_cells,
                         nullptr, nullptr, g->d_list, g->d_ucount, s));
  unsigned na = 0;
  RT_CUDA(cudaMemcpyAsync(&na, g->d_ucount, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RT_CUDA(cudaStreamSynchronize(s));
  if (n_rows_out) *n_rows_out = compact ? (int64_t)na : n_cells;
  if (compact) {
    if ((int64_t)na > max_rows) return RT_ERR_RANGE;
    if (na == 0) return RT_OK;
    dst = get_dst(g, dst_ctx, (size_t)na * B, &st);
    if (st != RT_OK) return st;
    RT_CUDA(cudaMemsetAsync(dst, 0, sizeof(float) * (size_t)na * B, s));
    RT_CUDA(cudaMemcpyAsync(cells_dev, g->d_list, sizeof(int32_t) * na, cudaMemcpyDeviceToDevice,
                            s));
  }
  *dst_out = dst;
  // compact rows: row i is cell d_list[i]; range rows: the list holds the rows
  const int* row_cells = compact ? g->d_list : nullptr;
  if (na > 0 && mode == RT_PAH_EXACT)
    RT_CUDA(launch_pah_exact(g->g, g->ptab, g->d_pahabs, g->eps, g->d0, first_cell, na, dst,
                             nullptr, pah, s, compact ? nullptr : g->d_list, row_cells));
  if (na > 0 && mode != RT_PAH_EXACT) {
    // the surrogate over batches of active cells; cells whose prediction fails its
    // checks are appended to one fallback list, solved exactly in one launch
    const long long batch = na < (1u << 20) ? (long long)na : (1ll << 20);
    if ((st = surrogate_scratch(g, n_cells, batch, true)) != RT_OK) return st;
    for (long long b0 = 0; b0 < (long long)na; b0 += batch) {
      const long long nb = (long long)na - b0 < batch ? (long long)na - b0 : batch;
      const int* lst = g->d_list + b0;
      RT_CUDA(cudaMemsetAsync(g->d_sflag, 0, (size_t)nb, s));
      for (int p = 0; p < g->n_pah; ++p) {
        if (pah >= 0 && p != pah) continue;
        float* Y = g->d_sy + (size_t)p * batch * B;
        float* pa = g->d_spabs + (size_t)p * batch;
        RT_CUDA(launch_pah_features(g->g, g->ptab, g->d_pahabs, g->eps, g->d0, p, first_cell,
                                    nb, g->d_sx, pa, s, lst));
        if ((st = rt_mlp_forward(m, g->d_sx, Y, nb, s)) != RT_OK) return st;
        RT_CUDA(launch_surrogate_check(Y, g->d_sx, pa, nb, B, F, t, x_lo, x_hi, g->d_sflag, s));
      }
      for (int p = 0; p < g->n_pah; ++p) {
        if (pah >= 0 && p != pah) continue;
        RT_CUDA(launch_surrogate_add(g->d_sy + (size_t)p * batch * B,
                                     g->d_spabs + (size_t)p * batch, nb, B,
                                     mode == RT_PAH_AUTO ? g->d_sflag : nullptr,
                                     compact ? dst + (size_t)b0 * B : dst, s,
                                     compact ? nullptr : lst));
      }
      RT_CUDA(launch_compact(g->ptab, g->d_pah_flag, g->desc.n_leaves, pah, first_cell, nb,
                             g->d_sflag, compact ? nullptr : lst, g->d_list2, g->d_ucount + 1,
                             s, (int)b0));
    }
    unsigned nf = 0;
    RT_CUDA(cudaMemcpyAsync(&nf, g->d_ucount + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaStreamSynchronize(s));
    n_fallback = nf;
    if (mode == RT_PAH_AUTO && nf > 0)
      RT_CUDA(launch_pah_exact(g->g, g->ptab, g->d_pahabs, g->eps, g->d0, first_cell, nf, dst,
                               nullptr, pah, s, g->d_list2, row_cells));
  }
  if (n_fallback_out) *n_fallback_out = n_fallback;
  return RT_OK;
}

static float* emission_dst(rt_grid* g, void* ctx, size_t n, rt_status* st) {
  const auto* o = static_cast<const std::pair<float*, int>*>(ctx);
  return output_buffer(g, o->first, o->second, n, st);
}

static rt_status check_pah_mode(int mode, const rt_mlp* surrogate) {
  if (mode != RT_PAH_EXACT && mode != RT_PAH_SURROGATE && mode != RT_PAH_AUTO) return RT_ERR_ARG;
  if (mode != RT_PAH_EXACT && !surrogate) return RT_ERR_ARG;
  return RT_OK;
}

rt_status rt_pah_emission(rt_grid* g, int64_t first_cell, int64_t n_cells, int pah, int mode,
                          const rt_mlp* surrogate, float tol, float* j_out, int mem,
                          uint64_t* n_fallback_out, void* stream) {
  if (!g || !j_out || first_cell < 0 || n_cells < 0) return RT_ERR_ARG;
  if (first_cell > g->desc.n_leaves || n_cells > g->desc.n_leaves - first_cell)
    return RT_ERR_ARG;
  rt_status st = check_pah_mode(mode, surrogate);
  if (st != RT_OK) return st;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  std::pair<float*, int> out{j_out, mem};
  float* dst = nullptr;
  st = pah_emission_impl(g, first_cell, n_cells, pah, mode, surrogate, tol, emission_dst, &out,
                         nullptr, 0, nullptr, n_fallback_out, &dst, s);
  if (st != RT_OK) return st;
  if (mem != RT_MEM_DEVICE && dst) {
    RT_CUDA(cudaMemcpyAsync(j_out, dst, sizeof(float) * (size_t)n_cells * g->desc.n_bins,
                            cudaMemcpyDeviceToHost, s));
    return sync_status(g, s);
  }
  return RT_OK;
}

rt_status rt_pah_emission_active(rt_grid* g, int pah, int mode, const rt_mlp* surrogate,
                                 float tol, int64_t max_cells, int32_t* cells_out,
                                 float* j_out, int mem, int64_t* n_active_out,
                                 uint64_t* n_fallback_out, void* stream) {
  if (!g || !j_out || !cells_out || !n_active_out || max_cells < 0) return RT_ERR_ARG;
  rt_status st = check_pah_mode(mode, surrogate);
  if (st != RT_OK) return st;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  // the cell list goes to the caller's buffer, or through the handle's scratch
  int32_t* cells_dev = cells_out;
  if (mem != RT_MEM_DEVICE) {
    if (g->cells_scratch_n < g->desc.n_leaves) {
      dfree(g->d_cells_scratch);
      g->cells_scratch_n = 0;
      if ((st = dalloc(&g->d_cells_scratch, (size_t)g->desc.n_leaves)) != RT_OK) return st;
      g->cells_scratch_n = g->desc.n_leaves;
    }
    cells_dev = g->d_cells_scratch;
  }
  std::pair<float*, int> out{j_out, mem};
  float* dst = nullptr;
  int64_t na = 0;
  st = pah_emission_impl(g, 0, g->desc.n_leaves, pah, mode, surrogate, tol, emission_dst, &out,
                         cells_dev, max_cells, &na, n_fallback_out, &dst, s);
  *n_active_out = na;
  if (st != RT_OK) return st;
  if (mem != RT_MEM_DEVICE && na > 0) {
    RT_CUDA(cudaMemcpyAsync(j_out, dst, sizeof(float) * (size_t)na * g->desc.n_bins,
                            cudaMemcpyDeviceToHost, s));
    RT_CUDA(cudaMemcpyAsync(cells_out, cells_dev, sizeof(int32_t) * (size_t)na,
                            cudaMemcpyDeviceToHost, s));
    return sync_status(g, s);
  }
  return RT_OK;
}

rt_status rt_pah_training_pairs(rt_grid* g, int pah, int64_t first_cell, int64_t n_cells,
                                float* X, float* Y, float* p_abs, void* stream) {
  if (!g || !X || !Y || !p_abs || first_cell < 0 || n_cells < 0) return RT_ERR_ARG;
  if (first_cell > g->desc.n_leaves || n_cells > g->desc.n_leaves - first_cell)
    return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(g->dev));
  rt_status st = build_tables(g, s);
  if (st != RT_OK) return st;
  if (pah < 0 || pah >= g->n_pah) return RT_ERR_ARG;
  if (n_cells == 0) return RT_OK;
  RT_CUDA(launch_pah_features(g->g, g->ptab, g->d_pahabs, g->eps, g->d0, pah, first_cell,
                              n_cells, X, p_abs, s));
  RT_CUDA(launch_pah_exact(g->g, g->ptab, g->d_pahabs, g->eps, g->d0, first_cell, n_cells, Y,
                           nullptr, pah, s));
  RT_CUDA(launch_pah_encode(Y, p_abs, n_cells, g->desc.n_bins, Y, s));
  return RT_OK;
}

}  // extern "C"

struct rt_batch {
  int dev = 0;
  std::vector<rt_grid*> grids;
  std::vector<unsigned long long> n_pk;
  ModelDesc* d_models = nullptr;
  BatchChunk* d_chunks = nullptr;
  unsigned long long* d_next = nullptr;
  long long n_chunks = 0;
  int blocks_per_sm = 0;
  int threads = 256;  // threads per block of the batched launch
  int s_fixed = 0;  // the species count every model shares (walk compiled for it), else 0
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

extern "C" {

rt_status rt_batch_destroy(rt_batch* b) {
  if (!b) return RT_OK;
  cudaSetDevice(b->dev);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  dfree(b->d_models);
  dfree(b->d_chunks);
  dfree(b->d_next);
  delete b;
  return RT_OK;
}

rt_status rt_batch_create(rt_grid* const* grids, int n, const uint64_t* n_packages, uint64_t seed,
                          const rt_run_opts* o, uint64_t chunk, rt_batch** out) {
  if (!grids || !n_packages || !out || n < 1) return RT_ERR_ARG;
  *out = nullptr;
  if (chunk == 0) chunk = 4096;
  if (o && (o->kernel != RT_KERNEL_POOL || o->blocks_per_sm < 0 || o->blocks_per_sm > 32 ||
            o->refill_period < 0 || o->interaction_batch < 0 || o->interaction_batch > 32 ||
            o->threads < 0 || o->threads % 32 != 0 || o->threads > 256))
    return RT_ERR_ARG;
  rt_batch* b = new (std::nothrow) rt_batch();
  if (!b) return RT_ERR_OOM;
  if (cudaGetDevice(&b->dev) != cudaSuccess) {
    delete b;
    return RT_ERR_CUDA;
  }
  std::vector<ModelDesc> desc((size_t)n);
  std::vector<std::vector<BatchChunk>> per((size_t)n);
  rt_status st = RT_OK;
  for (int m = 0; m < n && st == RT_OK; ++m) {
    rt_grid* g = grids[m];
    if (!g || g->dev != b->dev) { st = RT_ERR_ARG; break; }
    if (g->images) { st = RT_ERR_STATE; break; }  // images need the single-model pool
    if ((st = build_tables(g, nullptr)) != RT_OK) break;
    if ((st = ensure_links(g)) != RT_OK) break;  // the batched launch walks the links
    if ((st = ensure_pathabs(g, o, nullptr)) != RT_OK) break;
    if (n_packages[m] > g->n_total) { st = RT_ERR_RANGE; break; }
    DevRun r;
    if ((st = fill_run(g, n_packages[m], seed + (uint64_t)m, 0, o, &r)) != RT_OK) break;
    const size_t nT = (size_t)g->desc.n_species * g->desc.n_leaves;
    if (!g->d_Tscratch && (st = dalloc(&g->d_Tscratch, nT)) != RT_OK) break;
    desc[(size_t)m].g = g->g;
    desc[(size_t)m].t = g->tab;
    desc[(size_t)m].t.u_frozen = g->d_ufrozen;
    desc[(size_t)m].t.pah_cell_cdf = g->d_pah_cell_cdf;
    desc[(size_t)m].r = r;
    b->grids.push_back(g);
    b->n_pk.push_back(n_packages[m]);
    for (unsigned long long f = 0; f < n_packages[m]; f += chunk) {
      BatchChunk c{m, 0, f, n_packages[m] - f < chunk ? n_packages[m] - f : chunk};
      per[(size_t)m].push_back(c);
    }
  }
  if (st != RT_OK) {
    rt_batch_destroy(b);
    return st;
  }
  // interleave the models' chunks round-robin so every model is in flight early
  std::vector<BatchChunk> chunks;
  for (size_t k = 0;; ++k) {
    bool any = false;
    for (int m = 0; m < n; ++m)
      if (k < per[(size_t)m].size()) {
        chunks.push_back(per[(size_t)m][k]);
        any = true;
      }
    if (!any) break;
  }
  b->n_chunks = (long long)chunks.size();
  b->blocks_per_sm = o ? o->blocks_per_sm : 0;
  b->threads = (o && o->threads > 0) ? o->threads : 256;
  b->s_fixed = grids[0]->desc.n_species;
  for (int m = 0; m < n; ++m)  // the fixed-count walk runs without the path-length tally
    if (grids[m]->desc.n_species != b->s_fixed || desc[(size_t)m].r.pathabs) b->s_fixed = 0;
  if ((st = dalloc(&b->d_models, (size_t)n)) != RT_OK ||
      (st = dalloc(&b->d_chunks, chunks.size())) != RT_OK ||
      (st = dalloc(&b->d_next, 1)) != RT_OK) {
    rt_batch_destroy(b);
    return st;
  }
  cudaError_t e = cudaMemcpy(b->d_models, desc.data(), sizeof(ModelDesc) * n,
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !chunks.empty())
    e = cudaMemcpy(b->d_chunks, chunks.data(), sizeof(BatchChunk) * chunks.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    rt_batch_destroy(b);
    return RT_ERR_CUDA;
  }
  *out = b;
  return RT_OK;
}

rt_status rt_batch_run(rt_batch* b, int reset, int temperatures, void* stream) {
  if (!b) return RT_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(b->dev));
  if (reset)
    for (rt_grid* g : b->grids) {
      rt_status st = rt_reset(g, stream);
      if (st != RT_OK) return st;
    }
  RT_CUDA(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s));
  if (b->n_chunks > 0)
    RT_CUDA(launch_transport_batch(b->d_models, b->d_chunks, b->n_chunks, b->d_next,
                                   b->blocks_per_sm, b->s_fixed, b->threads, s));
  if (temperatures)
    for (rt_grid* g : b->grids)
      RT_CUDA(launch_temperatures(g->g, g->tab, g->d_count, g->d_Tscratch, g->d_counters, s));
  return RT_OK;
}

rt_status rt_batch_run_graph(rt_batch* b, void* stream) {
  if (!b) return RT_ERR_ARG;
  RT_CUDA(cudaSetDevice(b->dev));
  if (!b->exec) {
    if (!b->capture_stream)
      RT_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    RT_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    rt_status st = rt_batch_run(b, 1, 1, b->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
    if (st != RT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return RT_ERR_CUDA;
    b->graph = graph;
    RT_CUDA(cudaGraphInstantiate(&b->exec, graph, 0));
  }
  RT_CUDA(cudaGraphLaunch(b->exec, as_stream(stream)));
  return RT_OK;
}

rt_status rt_batch_temperatures(rt_batch* b, int model, float* T_out, int mem, void* stream) {
  if (!b || model < 0 || model >= (int)b->grids.size() || !T_out) return RT_ERR_ARG;
  rt_grid* g = b->grids[(size_t)model];
  cudaStream_t s = as_stream(stream);
  RT_CUDA(cudaSetDevice(b->dev));
  const size_t n = (size_t)g->desc.n_species * g->desc.n_leaves;
  RT_CUDA(cudaMemcpyAsync(T_out, g->d_Tscratch, sizeof(float) * n,
                          mem == RT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                               : cudaMemcpyDeviceToHost,
                          s));
  if (mem != RT_MEM_DEVICE) return sync_status(g, s);
  return RT_OK;
}

rt_status rt_philox(const uint64_t* ids, int64_t n, uint32_t event, uint32_t block,
                    uint64_t seed, uint32_t* out) {
  if (n < 0 || (n > 0 && (!ids || !out))) return RT_ERR_ARG;
  if (n == 0) return RT_OK;
  unsigned long long* d_ids = nullptr;
  unsigned* d_out = nullptr;
  rt_status st;
  if ((st = dalloc(&d_ids, (size_t)n)) != RT_OK) return st;
  if ((st = dalloc(&d_out, (size_t)n * 4)) != RT_OK) {
    dfree(d_ids);
    return st;
  }
  cudaError_t e = cudaMemcpy(d_ids, ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox(d_ids, n, event, block, seed, d_out, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
  dfree(d_ids);
  dfree(d_out);
  return cuda_status(e);
}

}  // extern "C"
