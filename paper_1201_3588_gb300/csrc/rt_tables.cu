// rt_tables.cu -- FP64 table builders, frozen-temperature energies and the
// per-cell temperature update of librt_gb300 (Planck integrals: rt_planck.cuh).

#include "rt_internal.h"
#include "rt_planck.cuh"

#include <math.h>

namespace rt {
namespace {

using namespace planck;

__global__ void k_planck_rows(TableBuild tb) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)tb.n_T * tb.B;
  if (idx >= tot) return;
  int i = (int)(idx / tb.B), b = (int)(idx % tb.B);
  double T = table_T(i, tb.n_T, tb.t_min, tb.t_max);
  if (b == 0) tb.Tgrid[i] = T;
  tb.P[idx] = planck_bin(tb.nu[b], tb.nu[b + 1], T);
}

// one thread per (species, row): S(T_i) = 4 pi sum_b kappa_abs P_b(T_i)
__global__ void k_emission_rows(TableBuild tb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= tb.S * tb.n_T) return;
  int s = idx / tb.n_T, i = idx % tb.n_T;
  const double* ka = tb.kabs + (size_t)s * tb.B;
  const double* P = tb.P + (size_t)i * tb.B;
  double acc = 0.0;
  for (int b = 0; b < tb.B; ++b) acc += ka[b] * P[b];
  acc *= 4.0 * kPi;
  tb.S64[idx] = acc;
  tb.S32[idx] = (float)acc;
}

// one thread per (species, interval): normalised cumulative of
// kappa_abs(b) [P_b(T_{i+1}) - P_b(T_i)] over the bins
__global__ void k_difference_cdfs(TableBuild tb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nI = tb.n_T - 1;
  if (idx >= tb.S * nI) return;
  int s = idx / nI, i = idx % nI;
  const double* ka = tb.kabs + (size_t)s * tb.B;
  const double* P0 = tb.P + (size_t)i * tb.B;
  const double* P1 = P0 + tb.B;
  float* out = tb.dcdf + (size_t)idx * tb.B;
  double tot = 0.0;
  for (int b = 0; b < tb.B; ++b) {
    double d = ka[b] * (P1[b] - P0[b]);
    tot += d > 0.0 ? d : 0.0;
  }
  double cum = 0.0;
  for (int b = 0; b < tb.B; ++b) {
    double d = ka[b] * (P1[b] - P0[b]);
    cum += d > 0.0 ? d : 0.0;
    out[b] = tot > 0.0 ? (float)(cum / tot) : 1.0f;
  }
  out[tb.B - 1] = 1.0f;
}

// Search accelerators (results identical to a binary search; they only give the
// search a starting point). Per difference-CDF row: the first bin whose cumulative
// value exceeds k/B, k = 0..B-1. One thread per row.
__global__ void k_cdf_guides(TableBuild tb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int nI = tb.n_T - 1;
  if (idx >= tb.S * nI) return;
  const float* cdf = tb.dcdf + (size_t)idx * tb.B;
  unsigned short* gd = tb.cdf_guide + (size_t)idx * tb.B;
  int b = 0;
  for (int k = 0; k < tb.B; ++k) {
    float thr = (float)k / (float)tb.B;
    while (b < tb.B - 1 && cdf[b] <= thr) ++b;
    gd[k] = (unsigned short)b;
  }
}

// Per species: for u_k = exp(ln S(T_1) + k (ln S(T_last) - ln S(T_1)) / (n_T - 1)),
// the largest interval i <= n_T - 2 with S(T_i) <= u_k. One thread per (s, k).
__global__ void k_u_guides(TableBuild tb) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= tb.S * tb.n_T) return;
  int s = idx / tb.n_T, k = idx % tb.n_T;
  const double* S = tb.S64 + (size_t)s * tb.n_T;
  int nI = tb.n_T - 1;
  double l0 = log(S[1]), l1 = log(S[nI]);
  double u = exp(l0 + (l1 - l0) * (double)k / (double)nI);
  int lo = 0, hi = nI;  // S[lo] <= u < S[hi] (clamped at the last interval)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (S[mid] <= u) lo = mid; else hi = mid;
  }
  tb.u_guide[idx] = lo;
}

__global__ void k_opacity(TableBuild tb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < tb.B) {
    for (int s = 0; s < tb.S; ++s) {
      size_t j = (size_t)s * tb.B + b;
      Kappa k;
      k.kabs = (float)tb.kabs[j];
      k.ksca = (float)tb.ksca[j];
      k.kext = (float)(tb.kabs[j] + tb.ksca[j]);
      k.g = (float)tb.ghg[j];
      tb.kap[(size_t)b * tb.S + s] = k;
    }
  }
}

// Stellar CDF and the in-range fraction of the blackbody: the bins' Planck
// integrals in parallel (one block of 1024 threads), the sums by one thread in bin
// order.
__global__ void __launch_bounds__(1024) k_star_cdf(TableBuild tb) {
  __shared__ double P[kMaxBins];
  for (int i = threadIdx.x; i < tb.B; i += blockDim.x)
    P[i] = planck_bin(tb.nu[i], tb.nu[i + 1], tb.T_star);
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < tb.B; ++i) tot += P[i];
    double cum = 0.0;
    for (int i = 0; i < tb.B; ++i) {
      cum += P[i];
      tb.star_cdf[i] = tot > 0.0 ? (float)(cum / tot) : 1.0f;
    }
    tb.star_cdf[tb.B - 1] = 1.0f;
    // sigma = 2 pi^5 k^4 / (15 c^2 h^3)
    double sigma = 2.0 * pow(kPi, 5.0) * pow(kK, 4.0) / (15.0 * kC * kC * pow(kH, 3.0));
    double T4 = pow(tb.T_star, 4.0);
    tb.star_frac[0] = kPi * tot / (sigma * T4);
  }
}

// S at temperature T by linear interpolation in T between table rows (the same
// piecewise-linear model the transport samples from).
__global__ void k_frozen_u(DevGrid g, DevTables t, const float* T_frozen, float* u_frozen,
                           float t_min) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)g.S * g.n_leaves;
  if (idx >= tot) return;
  int s = (int)(idx / g.n_leaves);
  double T = fmax((double)T_frozen[idx], (double)t_min);
  const double* Tg = t.Tgrid;
  const double* S = t.S64 + (size_t)s * g.n_T;
  int n_T = g.n_T;
  double u;
  if (T >= Tg[n_T - 1]) {
    u = S[n_T - 1];
  } else {
    int lo = 0, hi = n_T - 1;  // Tg[lo] <= T < Tg[hi]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (Tg[mid] <= T) lo = mid; else hi = mid;
    }
    double w = (T - Tg[lo]) / (Tg[hi] - Tg[lo]);
    u = S[lo] + w * (S[hi] - S[lo]);
  }
  u_frozen[idx] = (float)u;
}

// T from n eps = M S(T): the FP64 S table's interval (guide + scan), then power-law
// (log-log) interpolation between rows; linear from T = 0 in the first interval.
__global__ void k_temperatures(DevGrid g, DevTables t, const unsigned long long* count,
                               float* T_out, unsigned long long* counters,
                               const float* pathabs) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)g.S * g.n_leaves;
  bool clamped = false;
  if (idx < tot) {
    int s = (int)(idx / g.n_leaves);
    long long c = idx - (long long)s * g.n_leaves;
    // absorbed energy in units of eps: the count, or the path-length tally
    const double n = pathabs ? (double)pathabs[idx] : (double)count[idx];
    float rho_d0 = g.rho[c * g.S + s];
    float Tv = 0.0f;
    if (n > 0.0 && rho_d0 > 0.0f) {
      int lev = g.level[c];
      double rho = (double)rho_d0 / t.d0;
      double u = n * t.eps_over_V[lev] / rho;
      const double* S = t.S64 + (size_t)s * g.n_T;
      const double* Tg = t.Tgrid;
      int n_T = g.n_T;
      if (u >= S[n_T - 1]) {
        Tv = (float)Tg[n_T - 1];
        clamped = true;
      } else {
        // interval i with S[i] <= u < S[i+1]: start from the guide of ln S (the
        // re-emission draws use the same one), finish by scanning
        const int nI = n_T - 1;
        float kf = (__logf(fmaxf((float)u, 1e-30f)) - t.u_ln0[s]) * t.u_inv[s];
        int kk = (int)fminf(fmaxf(kf, 0.0f), (float)nI);
        int i = t.u_guide[s * n_T + kk];
        while (i > 0 && S[i] > u) --i;
        while (i + 1 < nI && S[i + 1] <= u) ++i;
        double T;
        if (i == 0 || !(S[i] > 0.0)) {
          T = Tg[i + 1] * u / S[i + 1];
        } else {
          // power law between the rows: ln(T/T_i) = ln(u/S_i) ln(T_i+1/T_i) / ln(S_i+1/S_i);
          // the ratios are formed in FP64, their logarithms (of numbers near 1) in FP32
          const double inv = 1.0 / S[i];
          const float a = log1pf((float)(u * inv - 1.0)) / log1pf((float)(S[i + 1] * inv - 1.0));
          T = Tg[i] * (double)expf(a * logf((float)(Tg[i + 1] / Tg[i])));
        }
        Tv = (float)T;
      }
    }
    T_out[idx] = Tv;
  }
  unsigned m = __ballot_sync(0xffffffffu, clamped);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(&counters[kCClamped], (unsigned long long)__popc(m));
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_build_tables(const TableBuild& tb, cudaStream_t s) {
  k_planck_rows<<<nblk((long long)tb.n_T * tb.B, 256), 256, 0, s>>>(tb);
  k_emission_rows<<<nblk((long long)tb.S * tb.n_T, 128), 128, 0, s>>>(tb);
  k_difference_cdfs<<<nblk((long long)tb.S * (tb.n_T - 1), 128), 128, 0, s>>>(tb);
  k_cdf_guides<<<nblk((long long)tb.S * (tb.n_T - 1), 128), 128, 0, s>>>(tb);
  k_u_guides<<<nblk((long long)tb.S * tb.n_T, 128), 128, 0, s>>>(tb);
  k_opacity<<<nblk(tb.B, 128), 128, 0, s>>>(tb);
  k_star_cdf<<<1, 1024, 0, s>>>(tb);
  return cudaGetLastError();
}

cudaError_t launch_frozen_u(const DevGrid& g, const DevTables& t, const float* T_frozen,
                            float* u_frozen, float t_min, cudaStream_t s) {
  long long n = (long long)g.S * g.n_leaves;
  k_frozen_u<<<nblk(n, 256), 256, 0, s>>>(g, t, T_frozen, u_frozen, t_min);
  return cudaGetLastError();
}

cudaError_t launch_temperatures(const DevGrid& g, const DevTables& t,
                                const unsigned long long* count, float* T_out,
                                unsigned long long* counters, cudaStream_t s,
                                const float* pathabs) {
  long long n = (long long)g.S * g.n_leaves;
  k_temperatures<<<nblk(n, 256), 256, 0, s>>>(g, t, count, T_out, counters, pathabs);
  return cudaGetLastError();
}

}  // namespace rt
