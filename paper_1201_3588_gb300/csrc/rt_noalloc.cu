// rt_noalloc.cu -- cell temperatures from caller-owned device buffers, with no
// device memory allocated by the library.
//
// The FP64 emission table S_s(T_i) that the temperature inversion needs is built
// into a fixed file-scope device array instead of memory from cudaMalloc. Host
// code may not pass that array's name to a kernel (in host code it is only a
// stand-in object, not a device address); every call asks the runtime for the
// array's address in the current context with cudaGetSymbolAddress, which
// allocates nothing. No address is cached: after cudaDeviceReset, or in another
// context, the module is loaded again at another address.

#include "../../include/rt.h"
#include "rt_internal.h"
#include "rt_planck.cuh"

#include <cuda_runtime.h>

#include <cmath>

namespace {

constexpr int kNoAllocMaxSpecies = 8;
constexpr int kNoAllocMaxRows = 2048;
constexpr int kNoAllocMaxBins = 1024;

// Layout: [0, 256) clamped counter (uint64) | T grid (double [rows]) |
// emission table (double [species][rows]).
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes =
    kCounterBytes + sizeof(double) * (size_t)kNoAllocMaxRows * (1 + kNoAllocMaxSpecies);

// 147,712 bytes, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array in the current context. The first call in
// a context may load the library's device code there.
rt_status scratch_in_current_context(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) return RT_ERR_CUDA;
  *out = static_cast<unsigned char*>(p);
  return RT_OK;
}

using namespace rt::planck;

// T grid and S_s(T_i) = 4 pi sum_b kappa_abs,s(b) P_b(T_i), one thread per row
__global__ void k_noalloc_rows(const double* kabs, const double* nu, int S, int B, int n_T,
                               double t_min, double t_max, double* Tgrid, double* S64) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n_T) {
    Tgrid[idx] = table_T(idx, n_T, t_min, t_max);
    return;
  }
  idx -= n_T;
  if (idx >= S * n_T) return;
  int s = idx / n_T, i = idx % n_T;
  double T = table_T(i, n_T, t_min, t_max);
  const double* ka = kabs + (size_t)s * B;
  double acc = 0.0;
  for (int b = 0; b < B; ++b) acc += ka[b] * planck_bin(nu[b], nu[b + 1], T);
  S64[idx] = acc * (4.0 * kPi);
}

// n eps = rho V S_s(T): binary search in S_s, log-log interpolation between rows,
// linear from T = 0 in the first interval; beyond the last row T = t_max (counted)
__global__ void k_noalloc_temperatures(const unsigned long long* count, const double* rho,
                                       const double* volume, long long N, int S, int n_T,
                                       double eps, const double* Tgrid, const double* S64,
                                       float* T_out, unsigned long long* clamped_count) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool clamped = false;
  if (idx < (long long)S * N) {
    int s = (int)(idx / N);
    long long c = idx - (long long)s * N;
    unsigned long long n = count[idx];
    double r = rho[idx];
    float Tv = 0.0f;
    if (n > 0 && r > 0.0) {
      double u = (double)n * eps / (r * volume[c]);
      const double* Sr = S64 + (size_t)s * n_T;
      if (u >= Sr[n_T - 1]) {
        Tv = (float)Tgrid[n_T - 1];
        clamped = true;
      } else {
        int lo = 0, hi = n_T - 1;
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (Sr[mid] <= u) lo = mid; else hi = mid;
        }
        double T;
        if (lo == 0 || !(Sr[lo] > 0.0)) {
          T = Tgrid[hi] * u / Sr[hi];
        } else {
          double a = log(u / Sr[lo]) / log(Sr[hi] / Sr[lo]);
          T = Tgrid[lo] * exp(a * log(Tgrid[hi] / Tgrid[lo]));
        }
        Tv = (float)T;
      }
    }
    T_out[idx] = Tv;
  }
  unsigned m = __ballot_sync(0xffffffffu, clamped);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(clamped_count, (unsigned long long)__popc(m));
}

}  // namespace

extern "C" rt_status rt_cell_temperatures_noalloc(
    const uint64_t* count, const double* rho, const double* volume, const double* kabs,
    const double* nu_edges, int n_species, int64_t n_cells, int n_bins, double eps,
    double t_min, double t_max, int n_temp, float* T_out, uint64_t* n_clamped,
    void* stream) {
  if (!count || !rho || !volume || !kabs || !nu_edges || !T_out) return RT_ERR_ARG;
  if (n_species < 1 || n_cells < 0 || n_bins < 1 || n_temp < 0) return RT_ERR_ARG;
  if (!(eps > 0) || !std::isfinite(eps)) return RT_ERR_ARG;
  if (n_temp == 0) n_temp = 1024;
  if (t_min == 0) t_min = 1.0;
  if (t_max == 0) t_max = 3000.0;
  if (!(t_min > 0) || !(t_max > t_min) || !std::isfinite(t_max) || n_temp < 3)
    return RT_ERR_ARG;
  if (n_species > kNoAllocMaxSpecies || n_temp > kNoAllocMaxRows || n_bins > kNoAllocMaxBins ||
      n_cells * (int64_t)n_species > 0x7fffffffll * 32)
    return RT_ERR_TOO_LARGE;
  unsigned char* base = nullptr;
  rt_status st = scratch_in_current_context(&base);
  if (st != RT_OK) return st;
  unsigned long long* clamped = reinterpret_cast<unsigned long long*>(base);
  double* Tgrid = reinterpret_cast<double*>(base + kCounterBytes);
  double* S64 = Tgrid + n_temp;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the counter must start at zero,
  // the table rows are all rewritten below
  if (cudaMemsetAsync(clamped, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return RT_ERR_CUDA;
  int rows = n_temp * (1 + n_species);
  k_noalloc_rows<<<(rows + 127) / 128, 128, 0, s>>>(kabs, nu_edges, n_species, n_bins, n_temp,
                                                    t_min, t_max, Tgrid, S64);
  if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
  long long n = (long long)n_species * n_cells;
  if (n > 0) {
    k_noalloc_temperatures<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const unsigned long long*>(count), rho, volume, n_cells, n_species,
        n_temp, eps, Tgrid, S64, T_out, clamped);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
  }
  if (n_clamped && cudaMemcpyAsync(n_clamped, clamped, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RT_ERR_CUDA;
  return RT_OK;
}
