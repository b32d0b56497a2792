// rt_pah.cu -- transiently heated PAH molecules on the device: FP64 level tables,
// template re-emission spectra, and the exact steady-state emission per cell.
//
// Thermal-discrete steady state (Guhathakurta & Draine 1989): internal-energy
// levels E_f = f dE, f = 0 .. M-1; absorbing a photon of energy e moves a molecule
// from E_i up to E_i + e, split between the two levels around it so the energy is
// kept (uniform levels: e/dE = q + w gives levels i+q and i+q+1 with weights 1-w and
// w); cooling is continuous at L(E) = 4 pi sum_b sigma_b P_b(T(E)), a step to the
// level below at rate C_f = L_f / dE. The upward probability flux across each level
// boundary equals C_f P_f, so the populations follow level by level. The molecule
// then emits sum_f P_f 4 pi sigma_b P_b(T_f) in bin b.

#include "rt_internal.h"
#include "rt_planck.cuh"

#include <math.h>

namespace rt {
namespace {

using namespace planck;

constexpr double kHh = 6.62607015e-27;

__device__ double heat_content(double T, const PahSpec& sp) {
  if (!(T > 0.0)) return 0.0;
  double e = 0.0;
  for (int i = 0; i < sp.n_groups; ++i) {
    double x = sp.theta[i] / T;
    if (x < 700.0) e += sp.n_modes[i] * kK * sp.theta[i] / expm1(x);
  }
  return e;
}

__device__ double temperature_of(double E, const PahSpec& sp) {
  if (!(E > 0.0)) return 0.0;
  double lo = 1e-3, hi = 10.0;
  while (heat_content(hi, sp) < E && hi < 1e9) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    double mid = sqrt(lo * hi);
    if (heat_content(mid, sp) < E) lo = mid; else hi = mid;
    if (hi / lo - 1.0 < 1e-14) break;
  }
  return sqrt(lo * hi);
}

// one thread per (PAH, level): temperature, cooling rate (FP64) and emission
// spectrum per bin (stored FP32)
__global__ void k_pah_levels(PahBuild pb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pb.n_pah * pb.M) return;
  int p = idx / pb.M, f = idx % pb.M;
  const PahSpec& sp = pb.spec[p];
  double T = temperature_of(f * pb.dE[p], sp);
  const double* sig = pb.sigma + (size_t)p * pb.B;
  float* s = pb.s + ((size_t)p * pb.M + f) * pb.B;
  double L = 0.0;
  for (int b = 0; b < pb.B; ++b) {
    double v = 4.0 * kPi * sig[b] * planck_bin(pb.nu[b], pb.nu[b + 1], T);
    s[b] = (float)v;
    L += v;
  }
  pb.L[idx] = L;
}

// coarse photon energies e_k = h sqrt(nu_lo nu_hi) over each coarse bin's range,
// and their split q_k + w_k = e_k / dE for every PAH
__global__ void k_pah_coarse(PahBuild pb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pb.n_pah * pb.K) return;
  int p = idx / pb.K, k = idx % pb.K;
  int b0 = (k * pb.B + pb.K - 1) / pb.K;          // first fine bin with floor(b K/B) == k
  int b1 = ((k + 1) * pb.B + pb.K - 1) / pb.K - 1;  // last one
  double e = kHh * sqrt(pb.nu[b0] * pb.nu[b1 + 1]);
  if (p == 0) pb.e_k[k] = e;
  double x = e / pb.dE[p];
  double q = floor(x);
  pb.q_k[idx] = (int)q;
  pb.w_k[idx] = x - q;
}

// FP32 copies for the per-cell solution: c_f = L_f / dE and w_k
__global__ void k_pah_f32(PahBuild pb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < pb.n_pah * pb.M) pb.c_f[idx] = (float)(pb.L[idx] / pb.dE[idx / pb.M]);
  if (idx < pb.n_pah * pb.K) pb.w_f[idx] = (float)pb.w_k[idx];
}

// Level populations of PAH p for absorption rates R[k] (smem, per molecule per
// second), one warp; P and D are this warp's shared-memory arrays of M doubles.
// Returns the emitted power sum_f P_f L_f of the normalised populations in P.
__device__ double solve_levels(const PahTables& t, int p, const double* R, double* P,
                               double* D) {
  const int lane = threadIdx.x & 31;
  const int M = t.M, K = t.K;
  const double dE = t.dE[p];
  const int* q = t.q_k + p * K;
  const double* w = t.w_k + p * K;
  const double* L = t.L + (size_t)p * M;
  for (int i = lane; i < M; i += 32) {
    D[i] = 0.0;
    P[i] = 0.0;
  }
  __syncwarp();
  double up = 0.0;
  // scatter level i's absorptions into D; returns this lane's upward rate
  auto scatter = [&](int i, double Pi) {
    double u = 0.0;
    for (int k = lane; k < K; k += 32) {
      double r = R[k];
      if (!(r > 0.0)) continue;
      int f = i + q[k];
      double wk = w[k];
      if (f >= M - 1) {
        f = M - 1;
        wk = 0.0;
      }
      if (f > i) {
        atomicAdd(&D[f], Pi * r * (1.0 - wk));
        u += r * (1.0 - wk);
      }
      if (wk > 0.0 && f + 1 < M) {
        atomicAdd(&D[f + 1], Pi * r * wk);
        u += r * wk;
      }
    }
    return u;
  };
  double P0 = 1.0;
  if (lane == 0) P[0] = P0;
  up = scatter(0, P0);
  for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(0xffffffffu, up, o);
  double F = P0 * up;
  for (int f = 1; f < M; ++f) {
    __syncwarp();
    double C = L[f] / dE;
    double Pf = C > 0.0 ? F / C : 0.0;
    if (lane == 0) P[f] = Pf;
    double u = scatter(f, Pf);
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    __syncwarp();
    F = fmax(F - D[f] + Pf * u, 0.0);
    if (Pf > 1e250) {  // keep the numbers finite
      __syncwarp();
      for (int i = lane; i < M; i += 32) {
        P[i] *= 1e-250;
        D[i] *= 1e-250;
      }
      F *= 1e-250;
    }
  }
  __syncwarp();
  double tot = 0.0, em = 0.0;
  for (int i = lane; i < M; i += 32) tot += P[i];
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  __syncwarp();
  for (int i = lane; i < M; i += 32) {
    P[i] /= tot;
    em += P[i] * L[i];
  }
  for (int o = 16; o > 0; o >>= 1) em += __shfl_xor_sync(0xffffffffu, em, o);
  __syncwarp();
  return em;
}

// Template re-emission spectra: one warp per PAH, heated by the source's blackbody
// at bolometric flux pb.f_ref inside the frequency grid.
__global__ void k_pah_template(PahTables t, PahBuild pb) {
  extern __shared__ double sm[];
  const int p = blockIdx.x;
  const int lane = threadIdx.x;
  double* R = sm;            // [K]
  double* P = R + t.K;       // [M]
  double* D = P + t.M;       // [M]
  const double* sig = pb.sigma + (size_t)p * pb.B;
  // stellar flux per fine bin, summed into coarse photon rates
  double tot = 0.0;
  for (int b = lane; b < pb.B; b += 32) tot += planck_bin(pb.nu[b], pb.nu[b + 1], pb.T_star);
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  for (int k = lane; k < t.K; k += 32) R[k] = 0.0;
  __syncwarp();
  for (int b = lane; b < pb.B; b += 32) {
    double fb = pb.f_ref * planck_bin(pb.nu[b], pb.nu[b + 1], pb.T_star) / tot;
    int k = (int)(((long long)b * t.K) / pb.B);
    atomicAdd(&R[k], fb * sig[b] / t.e_k[k]);
  }
  __syncwarp();
  solve_levels(t, p, R, P, D);
  // J_b = sum_f P_f s_fb, then its normalised cumulative
  float* cdf = pb.template_cdf + (size_t)p * pb.B;
  double run = 0.0;
  for (int b0 = 0; b0 < pb.B; b0 += 32) {
    int b = b0 + lane;
    double j = 0.0;
    if (b < pb.B)
      for (int f = 0; f < t.M; ++f) j += P[f] * (double)t.s[((size_t)p * t.M + f) * pb.B + b];
    // inclusive scan over the 32 lanes
    double x = j;
    for (int o = 1; o < 32; o <<= 1) {
      double y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (b < pb.B) cdf[b] = (float)(run + x);  // unnormalised for now
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  __syncwarp();
  for (int b = lane; b < pb.B; b += 32) cdf[b] = run > 0.0 ? (float)((double)cdf[b] / run) : 1.0f;
  __syncwarp();
  if (lane == 0) cdf[pb.B - 1] = 1.0f;
}

// Sum over the 4 lanes of a quad (lanes 4q .. 4q+3 of the warp).
__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

// The same steady state in FP32, for the per-cell solutions: one quad of 4 lanes
// per cell (the 8 quads of a warp run in lockstep; a quad without a cell solves a
// zero rate vector). R, P, G are the cell's shared-memory arrays (K rates, M
// levels). The levels are uniform, so the rate from level i to the levels at or
// above f depends on f - i alone: G(d) = sum over coarse bins of the rate landing d
// or more levels up (an absorption split between i + q_k and i + q_k + 1, or cut at
// the top level, counts alike for every f <= M - 1). The upward flux across the
// boundary below f is then F_f = sum_{d >= 1} G(d) P_{f-d} -- the quantity the
// carried recursion forms, here as a dot product of positive terms, with no
// cancellation in FP32 (about 1e-7 relative on every level that matters) and no
// scatter. P_f = F_f / C_f. Populations are kept below 1e20 by rescaling (the
// normalised result is unchanged). Leaves the unnormalised populations in P and
// returns their sum (in every lane of the quad).
__device__ float solve_levels_f32(const PahTables& t, int p, const float* R, float* P, float* G) {
  const int j = threadIdx.x & 3;  // lane within the quad
  const int M = t.M, K = t.K;
  const int* q = t.q_k + p * K;
  const float* wf = t.w_f + p * K;
  const float* cf = t.c_f + (size_t)p * M;
  for (int i = j; i < M; i += 4) {
    G[i] = 0.0f;
    P[i] = 0.0f;
  }
  __syncwarp();
  // rate landing exactly d levels up, then its suffix sums G(d), d = 1 .. dmax
  int dmax = 0;
  for (int k = j; k < K; k += 4) {
    const float r = R[k];
    if (!(r > 0.0f)) continue;
    const int qq = min(q[k], M - 1);
    const float w = wf[k];
    if (qq >= 1) atomicAdd(&G[qq], r * (1.0f - w));
    if (w > 0.0f) atomicAdd(&G[min(qq + 1, M - 1)], r * w);
    dmax = max(dmax, min(qq + 1, M - 1));
  }
  dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, 1));
  dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, 2));
  __syncwarp();
  {  // suffix sums over d = 1 .. dmax: four contiguous chunks, one per lane
    const int len = (dmax + 3) >> 2;
    const int lo = 1 + j * len, hi = min(dmax, lo + len - 1);
    float part = 0.0f;
    for (int d = lo; d <= hi; ++d) part += G[d];
    // the sum of the chunks above this lane's
    const float p1 = __shfl_down_sync(0xffffffffu, part, 1);
    const float p2 = __shfl_down_sync(0xffffffffu, part, 2);
    const float p3 = __shfl_down_sync(0xffffffffu, part, 3);
    float above = (j < 3 ? p1 : 0.0f) + (j < 2 ? p2 : 0.0f) + (j < 1 ? p3 : 0.0f);
    __syncwarp();
    for (int d = hi; d >= lo; --d) {
      above += G[d];
      G[d] = above;
    }
  }
  if (j == 0) P[0] = 1.0f;
  __syncwarp();
  for (int f = 1; f < M; ++f) {
    const int hi = min(f, dmax);
    float F0 = 0.0f, F1 = 0.0f;  // two chains
    int d = 1 + j;
    for (; d + 4 <= hi; d += 8) {
      F0 = fmaf(G[d], P[f - d], F0);
      F1 = fmaf(G[d + 4], P[f - d - 4], F1);
    }
    if (d <= hi) F0 = fmaf(G[d], P[f - d], F0);
    const float F = quad_sum(F0 + F1);
    const float C = cf[f];
    float Pf = C > 0.0f ? F / C : 0.0f;
    if (!(Pf <= 1e20f)) {  // rescale the levels so far so that P_f = 1e20
      const float sc = (1e20f * C) / F;
      for (int i = j; i < f; i += 4) P[i] *= sc;
      Pf = 1e20f;
    }
    if (j == 0) P[f] = Pf;
    __syncwarp();
  }
  float tot = 0.0f;
  for (int i = j; i < M; i += 4) tot += P[i];
  return quad_sum(tot);
}

// Exact emission of cells [first, first + n): a quad of 4 lanes per cell solves
// the level populations (all PAH species in turn); the block's cells (8 per warp)
// then form their emission together, J_cb = sum_f P_cf s_fb, one thread per bin,
// so that each row of the level table s (read from L2) serves every cell of the
// block. j_out[c][b] = sum over PAH of N_mol sum_f P_f s_fb (erg/s per bin). N_mol
// and the final scaling stay in FP64 (N_mol can exceed the FP32 range).
constexpr int kExactCellsMax = 16;  // two warps of 8 quads

__device__ __forceinline__ int exact_cell_stride(int K, int M) {
  // 16-byte aligned arrays, and a stride of 4 (mod 32) words: the 8 quads of a warp
  // reading the same offset in their own arrays hit 8 different groups of 4 banks
  const int w = ((K + 3) & ~3) + 2 * ((M + 3) & ~3);
  return ((w + 31) & ~31) + 4;
}

__global__ void __launch_bounds__(32 * kExactCellsMax / 8)
    k_pah_exact(DevGrid g, PahTables t, const unsigned* pahabs, double eps, double d0,
                long long first, long long n, float* j_out, const unsigned char* want,
                int pah_only, const int* list, const int* cell_of_row) {
  extern __shared__ __align__(16) float smf[];
  __shared__ double s_norm[kExactCellsMax];   // N_mol / sum_f P_f, 0 without a solution
  __shared__ long long s_row[kExactCellsMax];  // row of j_out
  const int n_cells = blockDim.x >> 2;         // 8 per warp
  const int slot = threadIdx.x >> 2, j = threadIdx.x & 3;
  const int Kp = (t.K + 3) & ~3, Mp = (t.M + 3) & ~3;
  const int CS = exact_cell_stride(t.K, t.M);
  float* R = smf + (size_t)slot * CS;
  float* P = R + Kp;
  float* G = P + Mp;
  const long long i = (long long)blockIdx.x * n_cells + slot;
  const bool active = i < n && !(want && !want[i]);
  // row of j_out; the cell is first + row, or first + cell_of_row[row] when the
  // output rows are a compact list of cells
  const long long c = active ? (list ? (long long)list[i] : i) : -1;
  const long long cell = active ? first + (cell_of_row ? (long long)cell_of_row[c] : c) : -1;
  if (j == 0) s_row[slot] = c;
  if (active)
    for (int b = j; b < g.B; b += 4) j_out[(size_t)c * g.B + b] = 0.0f;
  const double V = active ? d0 * d0 * d0 / (double)(1ll << (3 * g.level[cell])) : 0.0;
  for (int p = 0; p < t.n_pah; ++p) {
    if (pah_only >= 0 && p != pah_only) continue;
    double norm = 0.0, n_mol = 0.0;
    unsigned any = 0;
    if (active) {
      const unsigned* cnt = pahabs + ((size_t)p * g.n_leaves + cell) * t.K;
      const int s = t.species[p];
      const double rho = (double)g.rho[cell * g.S + s] / d0;
      n_mol = rho * V / t.mol_mass[p];
      // absorption rate per molecule: count * eps / (e_k N_mol)
      const float scale = n_mol > 0.0 ? (float)(eps / n_mol) : 0.0f;
      for (int k = j; k < t.K; k += 4) {
        const unsigned v = cnt[k];
        any |= v;
        R[k] = (float)v * scale / (float)t.e_k[k];
      }
    } else {
      for (int k = j; k < t.K; k += 4) R[k] = 0.0f;
    }
    any |= __shfl_xor_sync(0xffffffffu, any, 1);
    any |= __shfl_xor_sync(0xffffffffu, any, 2);
    __syncwarp();
    // every quad of the warp solves (a zero rate vector where there is nothing to
    // solve), so the warp stays converged for its shuffles
    const bool work = __any_sync(0xffffffffu, any != 0 && n_mol > 0.0);
    if (work) {
      const float tot = solve_levels_f32(t, p, R, P, G);
      if (any != 0 && n_mol > 0.0) norm = n_mol / (double)tot;
    }
    if (j == 0) s_norm[slot] = norm;
    __syncthreads();
    bool some = false;
    for (int w = 0; w < n_cells; ++w) some |= s_norm[w] > 0.0;
    if (some) {
      const float* Pc = smf + Kp;  // P of cell w at Pc + w * CS
      for (int b = threadIdx.x; b < g.B; b += blockDim.x) {
        float acc[kExactCellsMax];
#pragma unroll
        for (int w = 0; w < kExactCellsMax; ++w) acc[w] = 0.0f;
        const float* sp = t.s + (size_t)p * t.M * g.B + b;
        for (int f = 0; f < t.M; ++f) {
          const float sf = __ldg(sp + (size_t)f * g.B);
#pragma unroll
          for (int w = 0; w < kExactCellsMax; ++w)
            if (w < n_cells) acc[w] = fmaf(Pc[(size_t)w * CS + f], sf, acc[w]);
        }
#pragma unroll
        for (int w = 0; w < kExactCellsMax; ++w)
          if (w < n_cells && s_norm[w] > 0.0)
            j_out[(size_t)s_row[w] * g.B + b] += (float)(s_norm[w] * (double)acc[w]);
      }
    }
    __syncthreads();
  }
}

// Surrogate features of PAH p in cells [first, first + n): the shape of the absorbed
// spectrum, x_k = ln(a_k + 1e-4)/4.6 + 1 with a_k the fraction of the absorbed
// photons in coarse bin k; the absorbed power per molecule,
// x_K = (log10(P_abs / N_mol) + 12) / 4; the size, x_K+1 = log10(N_C) - 2.
// p_abs[c] = absorbed power of the cell's PAH p (erg/s), 0 without absorptions.
__global__ void k_pah_features(DevGrid g, PahTables t, const unsigned* pahabs, double eps,
                               double d0, int p, long long first, long long n, float* X,
                               float* p_abs, const int* list) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const long long cell = first + (list ? (long long)list[c] : c);
  const int F = t.K + 2;
  const unsigned* cnt = pahabs + ((size_t)p * g.n_leaves + cell) * t.K;
  float* x = X + (size_t)c * F;
  unsigned long long tot = 0;
  for (int k = 0; k < t.K; ++k) tot += cnt[k];
  const int s = t.species[p];
  const double rho = (double)g.rho[cell * g.S + s] / d0;
  const int lev = g.level[cell];
  const double V = d0 * d0 * d0 / (double)(1ll << (3 * lev));
  const double n_mol = rho * V / t.mol_mass[p];
  if (tot == 0 || !(n_mol > 0.0)) {
    for (int k = 0; k < F; ++k) x[k] = 0.0f;
    p_abs[c] = 0.0f;
    return;
  }
  // the shape features in FP32 (they enter a BF16 network)
  const float inv_tot = 1.0f / (float)tot;
  for (int k = 0; k < t.K; ++k) x[k] = logf((float)cnt[k] * inv_tot + 1e-4f) * (1.0f / 4.6f) + 1.0f;
  const double pw = (double)tot * eps;
  x[t.K] = (float)((log10(pw / n_mol) + 12.0) / 4.0);
  x[t.K + 1] = (float)(log10(t.n_carbon[p]) - 2.0);
  p_abs[c] = (float)pw;
}

// Training targets: y_b = ln(J_b / P_abs + 1e-6) / 7 + 1 from the exact emission (bins
// below 1e-6 of the cell's power carry no energy worth learning).
__global__ void k_pah_encode(const float* J, const float* p_abs, long long n, int B, float* Y) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * B) return;
  long long c = idx / B;
  float pa = p_abs[c];
  Y[idx] = pa > 0.0f ? logf(J[idx] / pa + 1e-6f) * (1.0f / 7.0f) + 1.0f : 0.0f;
}

// decoded surrogate output of one bin: q = max(exp(7 (y - 1)) - 1e-6, 0), FP32
__device__ __forceinline__ float decode_q(float y) {
  return fmaxf(expf(7.0f * (y - 1.0f)) - 1e-6f, 0.0f);
}

// Decoded surrogate emission: q_b = max(exp(7 (y_b - 1)) - 1e-6, 0); the energy
// residual |sum_b q_b - 1| (before renormalising) and an out-of-range guard on the
// absorbed power flag a cell for the exact solution. One warp per cell.
__global__ void k_surrogate_check(const float* Y, const float* X, const float* p_abs,
                                  long long n, int B, int F, float tol, float x_lo, float x_hi,
                                  unsigned char* flag) {
  const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n) return;
  if (!(p_abs[c] > 0.0f)) return;
  float sum = 0.0f;
  for (int b = lane; b < B; b += 32) sum += decode_q(Y[c * B + b]);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    const float xp = X[c * F + F - 2];
    if (!(fabsf(sum - 1.0f) <= tol) || xp < x_lo || xp > x_hi) flag[c] = 1;
  }
}

// j_out[c] += P_abs q_b / sum q for cells not flagged. One warp per cell.
__global__ void k_surrogate_add(const float* Y, const float* p_abs, long long n, int B,
                                const unsigned char* flag, float* j_out, const int* list) {
  const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n) return;
  const float pa = p_abs[c];
  if (!(pa > 0.0f) || (flag && flag[c])) return;
  float sum = 0.0f;
  for (int b = lane; b < B; b += 32) sum += decode_q(Y[c * B + b]);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (!(sum > 0.0f)) return;
  const long long row = list ? (long long)list[c] : c;
  const float f = pa / sum;
  for (int b = lane; b < B; b += 32) j_out[row * B + b] += f * decode_q(Y[c * B + b]);
}

// Compaction: rows i < n with sel(i) true are appended to out (order not kept);
// *count receives their number. sel = a PAH absorption in cell first + i (any PAH
// or only `pah`: the cell's flag word), or flag[i] when flag is given (then out
// receives list[i], or off + i without a list).
__global__ void k_compact(const unsigned* pah_flag, int pah, long long first, long long n,
                          const unsigned char* flag, const int* list, int off, int* out,
                          unsigned* count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool sel = false;
  if (i < n) {
    if (flag)
      sel = flag[i] != 0;
    else
      sel = (pah_flag[first + i] & (pah >= 0 ? 1u << pah : ~0u)) != 0u;
  }
  const unsigned m = __ballot_sync(0xffffffffu, sel);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (sel)
    out[base + __popc(m & ((1u << lane) - 1u))] =
        flag ? (list ? list[i] : off + (int)i) : (int)i;
}

// Zero the absorbed spectra of the PAH-active cells and their flags (the other
// rows are zero already). Each lane reads one cell's flag word (coalesced); the warp
// then clears the rows of its flagged cells one after another, a coalesced row of K
// words per PAH.
__global__ void k_pah_clear(const unsigned* pah_flag, long long N, int K, int n_pah,
                            unsigned* pahabs, unsigned* flag_out) {
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  for (long long base = w0 * 32; base < N; base += warps * 32) {
    const long long c = base + lane;
    const unsigned f = c < N ? pah_flag[c] : 0u;
    unsigned m = __ballot_sync(0xffffffffu, f != 0u);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const unsigned fc = __shfl_sync(0xffffffffu, f, src);
      const long long cc = base + src;
      for (int p = 0; p < n_pah; ++p)
        if (fc & (1u << p))
          for (int k = lane; k < K; k += 32) pahabs[((size_t)p * N + cc) * K + k] = 0u;
    }
    if (f) flag_out[c] = 0u;
  }
}

__global__ void k_count_flags(const unsigned char* flag, long long n, unsigned long long* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool f = i < n && flag[i];
  unsigned m = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(out, (unsigned long long)__popc(m));
}

}  // namespace

cudaError_t launch_pah_tables(const PahBuild& pb, const PahTables& t, cudaStream_t s) {
  int n = pb.n_pah * pb.M;
  k_pah_levels<<<(n + 63) / 64, 64, 0, s>>>(pb);
  int nk = pb.n_pah * pb.K;
  k_pah_coarse<<<(nk + 63) / 64, 64, 0, s>>>(pb);
  const int nf = n > nk ? n : nk;
  k_pah_f32<<<(nf + 63) / 64, 64, 0, s>>>(pb);
  size_t smem = sizeof(double) * (t.K + 2 * t.M);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_pah_template,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_pah_template<<<pb.n_pah, 32, smem, s>>>(t, pb);
  return cudaGetLastError();
}

cudaError_t launch_pah_exact(const DevGrid& g, const PahTables& t, const unsigned* pahabs,
                             double eps, double d0, long long first, long long n,
                             float* j_out, const unsigned char* want, int pah_only,
                             cudaStream_t s, const int* list, const int* cell_of_row) {
  if (n <= 0) return cudaSuccess;
  const int w = ((t.K + 3) & ~3) + 2 * ((t.M + 3) & ~3);
  const size_t per_cell = sizeof(float) * (size_t)(((w + 31) & ~31) + 4);
  // 16 cells (two warps) per block when their arrays fit, else 8
  int cells = kExactCellsMax;
  if (per_cell * cells > 200 * 1024) cells = 8;
  const size_t smem = per_cell * cells;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_pah_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  long long blocks = (n + cells - 1) / cells;
  k_pah_exact<<<(unsigned)blocks, 4 * cells, smem, s>>>(g, t, pahabs, eps, d0, first, n,
                                                       j_out, want, pah_only, list,
                                                       cell_of_row);
  return cudaGetLastError();
}

}  // namespace rt

namespace rt {

cudaError_t launch_pah_features(const DevGrid& g, const PahTables& t, const unsigned* pahabs,
                                double eps, double d0, int p, long long first, long long n,
                                float* X, float* p_abs, cudaStream_t s, const int* list) {
  if (n <= 0) return cudaSuccess;
  k_pah_features<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, t, pahabs, eps, d0, p, first, n,
                                                              X, p_abs, list);
  return cudaGetLastError();
}

cudaError_t launch_pah_encode(const float* J, const float* p_abs, long long n, int B, float* Y,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long m = n * B;
  k_pah_encode<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(J, p_abs, n, B, Y);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_check(const float* Y, const float* X, const float* p_abs,
                                   long long n, int B, int F, float tol, float x_lo, float x_hi,
                                   unsigned char* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_surrogate_check<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(Y, X, p_abs, n, B, F, tol,
                                                                       x_lo, x_hi, flag);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_add(const float* Y, const float* p_abs, long long n, int B,
                                 const unsigned char* flag, float* j_out, cudaStream_t s,
                                 const int* list) {
  if (n <= 0) return cudaSuccess;
  k_surrogate_add<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(Y, p_abs, n, B, flag, j_out,
                                                                     list);
  return cudaGetLastError();
}

// P(T) of a PAH in a monochromatic field (Fig. 3), one block per case: levels
// E_f = f dE up to E(t_top) + h nu with their temperatures and cooling rates
// (threads over levels), populations by the level-by-level flux balance for the
// single photon energy (one thread), then the time fraction above t_sub and the
// emission per bin (threads over bins). Shared memory: T, L, D [M] doubles.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

__global__ void k_pah_pt(const PtCase* cases, const double* nu, int B, const double* sigma,
                         int M, double t_sub, double* P_out, double* T_out, double* p_above,
                         double* em_out) {
  extern __shared__ double sm[];
  double* T = sm;
  double* L = T + M;
  double* D = L + M;
  double* red = D + M;  // [32]
  const PtCase c = cases[blockIdx.x];
  const double* sig = sigma + (size_t)blockIdx.x * B;
  double* P = P_out + (size_t)blockIdx.x * M;
  const double dE = (heat_content(c.t_top, c.spec) + c.h_nu) / (double)(M - 1);
  for (int f = threadIdx.x; f < M; f += blockDim.x) {
    const double Tf = f == 0 ? 0.0 : temperature_of(f * dE, c.spec);
    double l = 0.0;
    if (f > 0)
      for (int b = 0; b < B; ++b) l += sig[b] * planck_bin(nu[b], nu[b + 1], Tf);
    T[f] = Tf;
    L[f] = 4.0 * kPi * l;
    D[f] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double x = c.h_nu / dE;
    const int q = (int)floor(x);
    const double w = x - floor(x);
    const double R = c.rate;
    // arrivals from level i: level i + q (weight 1 - w) and i + q + 1 (weight w),
    // both cut at the top level; returns the upward rate out of level i
    auto scatter = [&](int i, double Pi) {
      int f = i + q;
      double wk = w;
      if (f >= M - 1) {
        f = M - 1;
        wk = 0.0;
      }
      double up = 0.0;
      if (f > i) {
        D[f] += Pi * R * (1.0 - wk);
        up += R * (1.0 - wk);
      }
      if (wk > 0.0 && f + 1 < M) {
        D[f + 1] += Pi * R * wk;
        up += R * wk;
      }
      return up;
    };
    P[0] = 1.0;
    double F = scatter(0, 1.0);
    for (int f = 1; f < M; ++f) {
      const double C = L[f] / dE;
      const double Pf = C > 0.0 ? F / C : 0.0;
      P[f] = Pf;
      const double u = scatter(f, Pf);
      F = fmax(F - D[f] + Pf * u, 0.0);
      if (Pf > 1e250) {  // keep the numbers finite
        for (int i = 0; i <= f; ++i) P[i] *= 1e-250;
        for (int i = 0; i < M; ++i) D[i] *= 1e-250;
        F *= 1e-250;
      }
    }
  }
  __syncthreads();
  double s = 0.0, a = 0.0;
  for (int f = threadIdx.x; f < M; f += blockDim.x) s += P[f];
  const double tot = block_sum(s, red);
  for (int f = threadIdx.x; f < M; f += blockDim.x) {
    const double v = P[f] / tot;
    P[f] = v;
    T_out[(size_t)blockIdx.x * M + f] = T[f];
    if (T[f] > t_sub) a += v;
  }
  a = block_sum(a, red);
  if (threadIdx.x == 0) p_above[blockIdx.x] = a;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double e = 0.0;
    for (int f = 1; f < M; ++f) e += P[f] * planck_bin(nu[b], nu[b + 1], T[f]);
    em_out[(size_t)blockIdx.x * B + b] = 4.0 * kPi * sig[b] * e;
  }
}

cudaError_t launch_pah_pt(const PtCase* cases, int n_cases, const double* nu, int B,
                          const double* sigma, int M, double t_sub, double* P_out,
                          double* T_out, double* p_above, double* em_out, cudaStream_t s) {
  const size_t smem = sizeof(double) * (3 * (size_t)M + 32);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_pah_pt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_pah_pt<<<n_cases, 256, smem, s>>>(cases, nu, B, sigma, M, t_sub, P_out, T_out, p_above,
                                      em_out);
  return cudaGetLastError();
}

// Per-cell re-emission spectra: each row of J [n][B] (erg/s per bin; negative or NaN
// entries count as 0) becomes its normalised cumulative sum, the last entry exactly
// 1; a row with nothing positive becomes zeros (the transport then uses the
// template). One warp per row, FP64 sums, a 32-wide inclusive scan per chunk.
__global__ void k_pah_cell_cdf(const float* J, long long n, int B, float* out) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
       row += warps) {
    const float* j = J + row * B;
    float* o = out + row * B;
    double tot = 0.0;
    for (int b = lane; b < B; b += 32) tot += (double)fmaxf(j[b], 0.f);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, s);
    if (!(tot > 0.0)) {
      for (int b = lane; b < B; b += 32) o[b] = 0.f;
      continue;
    }
    double carry = 0.0;
    for (int base = 0; base < B; base += 32) {
      const int b = base + lane;
      double v = b < B ? (double)fmaxf(j[b], 0.f) : 0.0;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, s);
        if (lane >= s) v += u;
      }
      if (b < B) o[b] = b == B - 1 ? 1.f : (float)((carry + v) / tot);
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
}

cudaError_t launch_pah_cell_cdf(const float* J, long long n, int B, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 7) / 8;
  if (blocks > 65536) blocks = 65536;
  k_pah_cell_cdf<<<(unsigned)blocks, 256, 0, s>>>(J, n, B, out);
  return cudaGetLastError();
}

cudaError_t launch_compact(const PahTables& t, const unsigned* pah_flag, long long N, int pah,
                           long long first, long long n, const unsigned char* flag,
                           const int* list, int* out, unsigned* count, cudaStream_t s,
                           int off) {
  (void)t;
  (void)N;
  if (n <= 0) return cudaSuccess;
  k_compact<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pah_flag, pah, first, n, flag, list,
                                                         off, out, count);
  return cudaGetLastError();
}

cudaError_t launch_pah_clear(const unsigned* pah_flag, long long N, int K, int n_pah,
                             unsigned* pahabs, unsigned* flag_out, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (N + 255) / 256;  // a lane per cell
  const long long cap = (long long)(sms > 0 ? sms : 152) * 8;
  if (blocks > cap) blocks = cap;
  k_pah_clear<<<(unsigned)blocks, 256, 0, s>>>(pah_flag, N, K, n_pah, pahabs, flag_out);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(const unsigned char* flag, long long n, unsigned long long* out,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_count_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flag, n, out);
  return cudaGetLastError();
}

}  // namespace rt
