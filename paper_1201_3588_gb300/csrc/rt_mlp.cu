// rt_mlp.cu -- the multilayer perceptron of the PAH emission surrogate: forward
// pass, mean-squared-error gradients and Adam, on the 5th-generation tensor cores
// (tcgen05.mma, FP32 accumulators in tensor memory) in BF16 with FP32 accumulation.
// Inference runs the whole network per 128-row tile in one kernel; training runs
// layer by layer, each GEMM on 128 x 128 output tiles.
//
// Network: a_0 = x; z_l = a_{l-1} W_l^T + b_l; a_l = silu(z_l) for the hidden layers,
// linear output. Loss = mean over rows and outputs of (y - t)^2. Master weights,
// gradients and Adam moments are FP32; the GEMM operands are BF16 copies.
// Internally every dimension is padded to a multiple of 16 (zero weights, zero
// inputs); the exported parameter layout is the unpadded one: per layer W [out][in]
// row-major, then b [out].

#include "../../include/rt.h"
#include "rt_internal.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

typedef __nv_bfloat16 bf16;

namespace {

constexpr int kTile = 64;     // rows are padded to a multiple of this
constexpr int kMaxLayers = 8;

inline int pad16(int x) { return (x + 15) / 16 * 16; }

struct Layer {
  int n_in, n_out;    // unpadded
  int in_p, out_p;    // padded to 16
  size_t w_off, b_off;  // offsets in the padded parameter arrays (floats)
};

}  // namespace

struct rt_mlp {
  int dev = 0;
  int n_layers_total = 0;
  Layer layer[kMaxLayers];
  int n_in = 0, n_out = 0;
  size_t n_padded = 0;     // padded parameter count
  int64_t n_params = 0;    // unpadded
  float* d_param = nullptr;  // padded FP32 master
  float* d_grad = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  bf16* d_wbf = nullptr;     // padded BF16 weights
  bf16* d_wpk = nullptr;     // the same weights in the tensor-core operand layout
  bool pk_stale = true;      // d_wpk lags behind d_wbf
  unsigned* d_err = nullptr; // fused forward: nonzero after a wait ran out
  float* d_loss = nullptr;
  long long step = 0;
  float x_lo = -1e30f, x_hi = 1e30f;  // admissible range of the second-to-last input
  // activations for up to cap rows (padded to 64)
  long long cap = 0;
  bf16* d_a[kMaxLayers + 1] = {};   // a_l in BF16 [cap][dim_p]
  float* d_z[kMaxLayers] = {};      // z_l in FP32 [cap][out_p]
  float* d_dz = nullptr;            // FP32 scratch [cap][max_p]
  bf16* d_dzb = nullptr;            // BF16 of dz
  int max_p = 0;
};

namespace {

// ---------------------------------------------------------------- kernels
// x [M][n_in] FP32 -> a0 [Mp][in_p] BF16, zero padding
__global__ void k_pack_input(const float* x, long long M, int n_in, long long Mp, int in_p,
                             bf16* a0) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Mp * in_p) return;
  long long r = idx / in_p;
  int c = (int)(idx % in_p);
  float v = (r < M && c < n_in) ? x[r * n_in + c] : 0.0f;
  a0[idx] = __float2bfloat16(v);
}

// logistic sigmoid as 1/2 + tanh(z/2)/2, with the hardware tanh approximation
// (relative error about 2^-11, below the BF16 rounding of the activations); both the
// layer-by-layer path and the fused forward use it, so their activations agree
__device__ __forceinline__ float sigmoid_fast(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return fmaf(0.5f, t, 0.5f);
}

__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
  return fmaf(h, t, h);
}

// z += b; a = silu(z) (hidden) or copy (output); padded columns forced to zero
__global__ void k_bias_act(float* z, const float* b, long long Mp, int out_p, int n_out,
                           int hidden, bf16* a) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Mp * out_p) return;
  int c = (int)(idx % out_p);
  float v = c < n_out ? z[idx] + b[c] : 0.0f;
  z[idx] = v;
  if (a) {
    float y = hidden ? silu_fast(v) : v;
    a[idx] = __float2bfloat16(y);
  }
}

// dz = 2 (y - t) / (M n_out) on valid rows/columns; loss accumulated
__global__ void k_mse_grad(const float* y, const float* t, long long M, int n_out, long long Mp,
                           int out_p, float* dz, bf16* dzb, float* loss) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (idx < Mp * out_p) {
    long long r = idx / out_p;
    int c = (int)(idx % out_p);
    float d = 0.0f;
    if (r < M && c < n_out) {
      float e = y[idx] - t[r * n_out + c];
      l = e * e;
      d = 2.0f * e / ((float)M * (float)n_out);
    }
    dz[idx] = d;
    dzb[idx] = __float2bfloat16(d);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l / ((float)M * (float)n_out));
}

// dz = da * silu'(z) (da in dz, in place) and its BF16 copy
__global__ void k_act_back(float* dz, const float* z, long long Mp, int p, int n_valid, bf16* dzb) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Mp * p) return;
  int c = (int)(idx % p);
  float v = 0.0f;
  if (c < n_valid) {
    float zz = z[idx];
    float s = sigmoid_fast(zz);
    v = dz[idx] * s * (1.0f + zz * (1.0f - s));
  }
  dz[idx] = v;
  dzb[idx] = __float2bfloat16(v);
}

// db[c] += sum over rows of dz[r][c]
__global__ void k_col_sums(const float* dz, long long Mp, int p, float* db) {
  int c = blockIdx.x * 32 + (threadIdx.x & 31);
  int r0 = threadIdx.x >> 5;
  float s = 0.0f;
  if (c < p)
    for (long long r = r0 + (long long)blockIdx.y * 8; r < Mp; r += 8ll * gridDim.y) s += dz[r * p + c];
  __shared__ float red[8][32];
  red[r0][threadIdx.x & 31] = s;
  __syncthreads();
  if (r0 == 0 && c < p) {
    float t = 0.0f;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x & 31];
    atomicAdd(&db[c], t);
  }
}

__global__ void k_to_bf16(const float* p, bf16* q, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) q[i] = __float2bfloat16(p[i]);
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, size_t n, float lr,
                       float b1, float b2, float c1, float c2, float eps) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.0f - b1) * gi;
  float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// y [M][n_out] <- z_last [Mp][out_p]
__global__ void k_unpack_output(const float* z, long long M, int n_out, int out_p, float* y) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= M * n_out) return;
  long long r = idx / n_out;
  int c = (int)(idx % n_out);
  y[idx] = z[r * out_p + c];
}


// ---------------------------------------------------------------- fused forward
// The whole forward pass of a 128-row tile in one CTA on the 5th-generation tensor
// cores: per layer, the activations (BF16, shared memory) times the layer's weights
// (BF16, shared memory) accumulate in FP32 in tensor memory (tcgen05.mma, issued by
// one thread), then 32 warps read the accumulators back (tcgen05.ld), add the
// bias, apply silu and write the next layer's activations. Every padded input and
// hidden width must be at most 256 (one MMA of M = 128, N = width per 16-wide K
// step); a wider output layer runs in chunks of 256 output columns, each its own
// weight copy, MMAs and epilogue.
//
// Operand layout in shared memory (no swizzle, K-major): 8-row x 16-byte core
// matrices; the core holding (row r, column k) starts at (r/8)*SBO + (k/8)*128 bytes,
// with SBO = (K/8)*128; inside it row r%8 is 16 bytes at (r%8)*16.
constexpr int kTcRows = 128;
constexpr int kTcThreads = 1024;  // 32 warps: each reads its lane quarter of the
                                  // accumulators, the column chunks shared by 8 warps
constexpr int kTcMaxWidth = 256;
constexpr int kTcMaxOut = 4096;  // output layer: up to 16 chunks of 256 columns
constexpr unsigned long long kTcWaitNs = 2000000000ull;  // give up a wait after 2 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// element offset of (r, k) in a [rows][K] operand in the core-matrix layout
__device__ __forceinline__ int core_off(int r, int k, int K) {
  return (r >> 3) * (K << 3) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: start, LBO (K direction) and SBO (row direction)
// in 16-byte units, the fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ unsigned long long tc_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = tc_now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return true;
    if (tc_now_ns() - t0 > kTcWaitNs) return false;
  }
}

// one thread: the next phase of `bar` completes once `bytes` have arrived from the
// bulk copy of [src, src + bytes) into shared memory at dst (16-byte aligned, size a
// multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(
          bar),
      "r"(bytes)
      : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
      "[%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// ---------------------------------------------------------------- training GEMM
// C[M][N] (=|+=) A[M][K] . B[K][N] on the 5th-generation tensor cores, for the
// layer-by-layer passes of training: A row-major (lda) or column-major, B row-major
// (ldb) or column-major; BF16 operands, FP32 accumulation in tensor memory. A CTA of
// 4 warps owns a 128 x 128 tile of C. The contraction runs in chunks of 64: all
// threads pack the chunk's A and B tiles from global memory (any layout) into the
// K-major core-matrix layout in one of two shared-memory buffers, one thread issues
// the chunk's four MMAs (K = 16 each) and commits them to that buffer's mbarrier, and
// the packing of the next chunk overlaps them. gridDim.z splits K into chunks of
// k_chunk (atomic adds). Every wait is bounded: after 2 s the tile's outputs are left
// untouched and *err is set.
constexpr int kGemmRows = 128, kGemmCols = 128, kGemmK = 64, kGemmThreads = 128;

template <bool kAcol, bool kBcol>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tc(const bf16* A, int lda, const bf16* B,
                                                          int ldb, float* C, int ldc, int M, int N,
                                                          int K, int k_chunk, int atomic_out,
                                                          unsigned* err) {
  extern __shared__ __align__(128) unsigned char gemm_smem[];
  bf16* sA0 = reinterpret_cast<bf16*>(gemm_smem);          // [2][128 x 64]: 2 x 16 KB
  bf16* sB0 = sA0 + 2 * kGemmRows * kGemmK;                 // [2][128 x 64]: 2 x 16 KB
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kGemmRows, n0 = blockIdx.y * kGemmCols;
  const int k_begin = blockIdx.z * k_chunk;
  const int k_end = min(K, k_begin + k_chunk);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kGemmCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc_idesc(kGemmRows, kGemmCols);
  bool ok = true;
  int n_chunks = 0;
  for (int k0 = k_begin; k0 < k_end && ok; k0 += kGemmK, ++n_chunks) {
    const int buf = n_chunks & 1;
    // the buffer was last read by the MMAs of chunk n_chunks - 2
    if (n_chunks >= 2) {
      const bool got = mbar_wait(smem_addr(&bar[buf]), (uint32_t)(((n_chunks - 2) >> 1) & 1));
      if (!__syncthreads_and(got)) {
        if (tid == 0) atomicOr(err, 1u);
        ok = false;
        break;
      }
    }
    const int kc = min(kGemmK, k_end - k0);  // a multiple of 16
    // A tile: element (r, k) = A[m0 + r][k0 + k], zero outside; 8 k per item
    bf16* a = sA0 + buf * kGemmRows * kGemmK;
    for (int i = tid; i < kGemmRows * (kGemmK / 8); i += kGemmThreads) {
      const int r = i / (kGemmK / 8), k8 = (i % (kGemmK / 8)) * 8;
      const int m = m0 + r;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (m < M && k8 < kc) {
        if (!kAcol) {
          v = *reinterpret_cast<const uint4*>(A + (size_t)m * lda + k0 + k8);
        } else {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            w[j] = (uint32_t)__bfloat16_as_ushort(A[(size_t)(k0 + k8 + 2 * j) * lda + m]) |
                   ((uint32_t)__bfloat16_as_ushort(A[(size_t)(k0 + k8 + 2 * j + 1) * lda + m])
                    << 16);
          v = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      *reinterpret_cast<uint4*>(&a[core_off(r, k8, kGemmK)]) = v;
    }
    // B tile as the MMA's [N][K] operand: element (n, k) = B[k0 + k][n0 + n]
    bf16* b = sB0 + buf * kGemmCols * kGemmK;
    for (int i = tid; i < kGemmCols * (kGemmK / 8); i += kGemmThreads) {
      const int c = i / (kGemmK / 8), k8 = (i % (kGemmK / 8)) * 8;
      const int n = n0 + c;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (n < N && k8 < kc) {
        if (kBcol) {
          v = *reinterpret_cast<const uint4*>(B + (size_t)n * ldb + k0 + k8);
        } else {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            w[j] = (uint32_t)__bfloat16_as_ushort(B[(size_t)(k0 + k8 + 2 * j) * ldb + n]) |
                   ((uint32_t)__bfloat16_as_ushort(B[(size_t)(k0 + k8 + 2 * j + 1) * ldb + n])
                    << 16);
          v = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      *reinterpret_cast<uint4*>(&b[core_off(c, k8, kGemmK)]) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_addr(a), b0 = smem_addr(b);
      const uint32_t sbo = (uint32_t)kGemmK * 16u;
      for (int kk = 0; kk < kc / 16; ++kk)
        tc_mma(tmem, tc_desc(a0 + kk * 256u, 128u, sbo), tc_desc(b0 + kk * 256u, 128u, sbo), idesc,
               (n_chunks > 0 || kk > 0) ? 1u : 0u);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_addr(&bar[buf]))
          : "memory");
    }
  }
  // the last chunk's MMAs (and with them all earlier ones) done
  if (ok && n_chunks > 0) {
    const int last = n_chunks - 1;
    const bool got = mbar_wait(smem_addr(&bar[last & 1]), (uint32_t)((last >> 1) & 1));
    if (!__syncthreads_and(got)) {
      if (tid == 0) atomicOr(err, 1u);
      ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok && n_chunks > 0) {
    // warp w holds rows 32 w .. 32 w + 31 of the tile (tensor-memory lanes)
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kGemmCols; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m >= M || n0 + c0 >= N) continue;
      float* cr = C + (size_t)m * ldc + n0 + c0;
      const int nv = min(16, N - n0 - c0);
      if (atomic_out) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j < nv) atomicAdd(&cr[j], v[j]);
      } else if (nv == 16 && ((reinterpret_cast<uintptr_t>(cr) & 15) == 0)) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(&cr[j]) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j < nv) cr[j] = v[j];
      }
    }
  } else if (!ok && n_chunks > 0 && warp == 0) {
    // a wait ran out: let the MMAs still in flight land before releasing tensor memory
    const int last = n_chunks - 1;
    mbar_wait(smem_addr(&bar[last & 1]), (uint32_t)((last >> 1) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kGemmCols));
  }
}

struct TcNet {
  int n_layers, n_in, n_out;
  int in_p[kMaxLayers], out_p[kMaxLayers], n_valid[kMaxLayers];
  const bf16* w[kMaxLayers];    // packed weights of each layer
  const float* b[kMaxLayers];   // padded biases
};

// weights [out_p][in_p] row-major -> the core-matrix layout (one thread per element)
__global__ void k_pack_weights(const bf16* w, int out_p, int in_p, bf16* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)out_p * in_p) return;
  const int r = (int)(i / in_p), k = (int)(i % in_p);
  out[core_off(r, k, in_p)] = w[i];
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_forward_tc(const __grid_constant__ TcNet net,
                                                           const float* x, long long M,
                                                           float* y, unsigned* err) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  bf16* sA = reinterpret_cast<bf16*>(tc_smem);                       // [128][256]
  bf16* sB = sA + kTcRows * kTcMaxWidth;                             // [256][256]
  float* sBias = reinterpret_cast<float*>(sB + kTcMaxWidth * kTcMaxWidth);  // [layers][256]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sBias + kMaxLayers * kTcMaxWidth);  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // biases of every layer, zero in the padding columns
  for (int i = tid; i < net.n_layers * kTcMaxWidth; i += kTcThreads) {
    const int l = i / kTcMaxWidth, c = i % kTcMaxWidth;
    sBias[i] = c < net.n_valid[l] ? net.b[l][c] : 0.0f;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(kTcMaxWidth));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t bar_a = smem_addr(bar);      // MMAs done
  const uint32_t bar_w = smem_addr(bar + 1);  // weights arrived
  uint32_t parity = 0, wparity = 0;
  bool ok = true;
  uint32_t pend = 0;  // after a wait ran out: the barrier still owed a completion
  const long long n_tiles = (M + kTcRows - 1) / kTcRows;
  for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const long long r0 = tile * kTcRows;
    // the first layer's weights stream in while the input is converted
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      const int n0 = net.out_p[0] < kTcMaxWidth ? net.out_p[0] : kTcMaxWidth;
      bulk_load(smem_addr(sB), net.w[0], (uint32_t)(n0 * net.in_p[0] * 2), bar_w);
    }
    // input rows -> BF16 activations: the tile's rows are contiguous in x, read
    // coalesced; zero beyond the valid rows and in the padding columns
    {
      const int K = net.in_p[0], F = net.n_in;
      const long long valid = M - r0 < kTcRows ? M - r0 : kTcRows;
      const float* xt = x + r0 * F;
      const int total = kTcRows * F, n_ok = (int)valid * F;
      // row of element i: (i + 1/2)/F lies at least 1/(2F) >= 2^-9 from an integer
      // and i < 2^15, so the FP32 product truncates to floor(i/F) exactly
      const float inv_f = 1.0f / (float)F;
      for (int i0 = tid; i0 < total; i0 += 4 * kTcThreads) {
        float v[4];  // four loads in flight before the stores
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * kTcThreads;
          v[u] = i < n_ok ? __ldg(&xt[i]) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * kTcThreads;
          if (i < total) {
            const int r = (int)(((float)i + 0.5f) * inv_f), k = i - r * F;
            sA[core_off(r, k, K)] = __float2bfloat16(v[u]);
          }
        }
      }
      if (tid < kTcRows)
        for (int k = F; k < K; ++k) sA[core_off(tid, k, K)] = __float2bfloat16(0.0f);
    }
    // stages: (layer, chunk of at most 256 output columns); only the output layer
    // may have more than one chunk (its packed weight rows are contiguous per chunk)
    for (int l = 0; l < net.n_layers && ok; ++l) {
      const int K = net.in_p[l], Np = net.out_p[l];
      const bool hidden = l < net.n_layers - 1;
      const int n_chunks = (Np + kTcMaxWidth - 1) / kTcMaxWidth;
      for (int ch = 0; ch < n_chunks && ok; ++ch) {
        const int col0 = ch * kTcMaxWidth;                    // first output column
        const int N = Np - col0 < kTcMaxWidth ? Np - col0 : kTcMaxWidth;
        // this stage's weights (bulk copy issued earlier)
        const bool got_w = mbar_wait(bar_w, wparity);
        if (!__syncthreads_and(got_w)) {
          if (tid == 0) atomicOr(err, 1u);
          ok = false;
          pend = bar_w;
          const long long gr = r0 + tid;
          if (tid < kTcRows && gr < M)
            for (int c = 0; c < net.n_out; ++c) y[gr * net.n_out + c] = __int_as_float(0x7fc00000);
          break;
        }
        wparity ^= 1u;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t idesc = tc_idesc(kTcRows, N);
          const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
          const uint32_t sbo = (uint32_t)K * 16u;  // (K/8) cores of 128 bytes
          for (int kk = 0; kk < K / 16; ++kk)
            tc_mma(tmem, tc_desc(a0 + kk * 256u, 128u, sbo), tc_desc(b0 + kk * 256u, 128u, sbo),
                   idesc, kk > 0 ? 1u : 0u);
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                  bar_a)
              : "memory");
        }
        const bool waited = mbar_wait(bar_a, parity);
        if (!__syncthreads_and(waited)) {  // the MMAs never signalled completion
          if (tid == 0) atomicOr(err, 1u);
          ok = false;
          pend = bar_a;
          const long long gr = r0 + tid;
          if (tid < kTcRows && gr < M)
            for (int c = 0; c < net.n_out; ++c) y[gr * net.n_out + c] = __int_as_float(0x7fc00000);
          break;
        }
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // the weight buffer is free: the next stage's weights stream in meanwhile
        // (after a single-chunk output layer the buffer stages the outputs instead)
        if (tid == 0) {
          if (ch + 1 < n_chunks) {
            const int n1 = Np - col0 - kTcMaxWidth < kTcMaxWidth ? Np - col0 - kTcMaxWidth
                                                                : kTcMaxWidth;
            bulk_load(smem_addr(sB), net.w[l] + (size_t)(col0 + kTcMaxWidth) * K,
                      (uint32_t)(n1 * K * 2), bar_w);
          } else if (hidden) {
            const int n1 = net.out_p[l + 1] < kTcMaxWidth ? net.out_p[l + 1] : kTcMaxWidth;
            bulk_load(smem_addr(sB), net.w[l + 1], (uint32_t)(n1 * net.in_p[l + 1] * 2), bar_w);
          }
        }
        // accumulators of this warp's 32 rows: bias, activation, next operand or output
        const int quarter = warp & 3;                 // lanes 32 quarter .. of the accumulators
        const int row = quarter * 32 + lane;
        const int group = warp >> 2, n_groups = kTcThreads / 128;
        const float* bias = sBias + l * kTcMaxWidth;
        // a single-chunk output layer is staged over both operand buffers (the last MMA
        // is done) with an odd row stride, so that the 32 rows a warp stores hit 32
        // different banks; wider output layers are stored from registers per chunk
        const int o_stride = net.n_out | 1;
        float* so = reinterpret_cast<float*>(sA);
        const long long grow = r0 + row;
        const bool vec4 = (net.n_out & 3) == 0;
        for (int c0 = 16 * group; c0 < N; c0 += 16 * n_groups) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
          float bv[16];
          if (n_chunks == 1) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(&bv[j]) =
                *reinterpret_cast<const float4*>(&bias[c0 + j]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = col0 + c0 + j;
              bv[j] = c < net.n_valid[l] ? __ldg(&net.b[l][c]) : 0.0f;
            }
          }
          if (hidden) {
            uint32_t h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const __nv_bfloat162 p =
                  __floats2bfloat162_rn(silu_fast(v[2 * j] + bv[2 * j]),
                                        silu_fast(v[2 * j + 1] + bv[2 * j + 1]));
              h[j] = *reinterpret_cast<const uint32_t*>(&p);
            }
            // columns c0..c0+15 of this row: two 16-byte pieces of the next operand
            *reinterpret_cast<uint4*>(&sA[core_off(row, c0, N)]) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(&sA[core_off(row, c0 + 8, N)]) =
                make_uint4(h[4], h[5], h[6], h[7]);
          } else if (n_chunks == 1) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = c0 + j;
              if (c < net.n_out) so[row * o_stride + c] = v[j] + bv[j];
            }
          } else if (grow < M) {
            float* yr = y + grow * net.n_out + col0 + c0;
            if (vec4 && col0 + c0 + 16 <= net.n_out) {
#pragma unroll
              for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(&yr[j]) =
                    make_float4(v[j] + bv[j], v[j + 1] + bv[j + 1], v[j + 2] + bv[j + 2],
                                v[j + 3] + bv[j + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (col0 + c0 + j < net.n_out) yr[j] = v[j] + bv[j];
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (!hidden && n_chunks == 1) {  // the tile's output rows are contiguous in y
          const long long valid = M - r0 < kTcRows ? M - r0 : kTcRows;
          float* yt = y + r0 * net.n_out;
          for (int r = warp; r < (int)valid; r += kTcThreads / 32)
            for (int c = lane; c < net.n_out; c += 32)
              yt[(long long)r * net.n_out + c] = so[r * o_stride + c];
          __syncthreads();
        }
      }
    }
  }
  // after a wait that ran out: let the weight copy or the MMAs still in flight land
  // (again with a time limit) before the shared and tensor memory are released
  if (pend != 0 && warp == 0) mbar_wait(pend, pend == bar_w ? wparity : parity);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcMaxWidth));
  }
}

size_t tc_smem_bytes() {
  return sizeof(bf16) * (size_t)(kTcRows + kTcMaxWidth) * kTcMaxWidth +
         sizeof(float) * kMaxLayers * kTcMaxWidth + 32;
}

inline unsigned nb(long long n, int t);

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- host helpers
template <bool Acol, bool Bcol>
cudaError_t gemm(const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, long long M,
                 int N, int K, bool split, unsigned* err, cudaStream_t s) {
  dim3 grid(nb(M, kGemmRows), nb(N, kGemmCols), 1);
  int chunk = K;
  if (split) {
    // split the contraction so that the grid fills the GPU
    long long tiles = (long long)grid.x * grid.y;
    long long want = (152 * 2 + tiles - 1) / tiles;
    long long ksteps = (K + kGemmK - 1) / kGemmK;
    if (want > ksteps) want = ksteps;
    if (want < 1) want = 1;
    chunk = (int)(((ksteps + want - 1) / want) * kGemmK);
    grid.z = (unsigned)((K + chunk - 1) / chunk);
  }
  const size_t smem = sizeof(bf16) * 2 * (kGemmRows + kGemmCols) * kGemmK;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<Acol, Bcol>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gemm_tc<Acol, Bcol><<<grid, kGemmThreads, smem, s>>>(A, lda, B, ldb, C, ldc, (int)M, N, K,
                                                         chunk, split ? 1 : 0, err);
  return cudaGetLastError();
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
rt_status alloc(T** p, size_t n) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RT_ERR_OOM;
  }
  return e == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

template <typename T>
void release(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_acts(rt_mlp* m) {
  for (int l = 0; l <= kMaxLayers; ++l) release(m->d_a[l]);
  for (int l = 0; l < kMaxLayers; ++l) release(m->d_z[l]);
  release(m->d_dz);
  release(m->d_dzb);
  m->cap = 0;
}

rt_status ensure_rows(rt_mlp* m, long long Mp) {
  if (Mp <= m->cap) return RT_OK;
  free_acts(m);
  rt_status st;
  const int L = m->n_layers_total;
  if ((st = alloc(&m->d_a[0], (size_t)Mp * m->layer[0].in_p)) != RT_OK) return st;
  for (int l = 0; l < L; ++l) {
    if ((st = alloc(&m->d_z[l], (size_t)Mp * m->layer[l].out_p)) != RT_OK) return st;
    if ((st = alloc(&m->d_a[l + 1], (size_t)Mp * m->layer[l].out_p)) != RT_OK) return st;
  }
  if ((st = alloc(&m->d_dz, (size_t)Mp * m->max_p)) != RT_OK) return st;
  if ((st = alloc(&m->d_dzb, (size_t)Mp * m->max_p)) != RT_OK) return st;
  m->cap = Mp;
  return RT_OK;
}

rt_status refresh_bf16(rt_mlp* m, cudaStream_t s) {
  k_to_bf16<<<nb((long long)m->n_padded, 256), 256, 0, s>>>(m->d_param, m->d_wbf, m->n_padded);
  m->pk_stale = true;
  return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

// Every padded width fits one tensor-core MMA (N <= 256): the fused forward applies.
bool tc_eligible(const rt_mlp* m) {
  const int L = m->n_layers_total;
  for (int l = 0; l < L; ++l) {
    if (m->layer[l].in_p > kTcMaxWidth) return false;
    // hidden widths are one MMA; the output layer runs in chunks of 256 columns
    if (m->layer[l].out_p > (l + 1 < L ? kTcMaxWidth : kTcMaxOut)) return false;
  }
  return true;
}

// forward of M rows with the fused tensor-core kernel (weights repacked when stale)
rt_status forward_tc(rt_mlp* m, const float* x, float* y, long long M, cudaStream_t s) {
  if (m->pk_stale) {
    for (int l = 0; l < m->n_layers_total; ++l) {
      const Layer& ly = m->layer[l];
      k_pack_weights<<<nb((long long)ly.out_p * ly.in_p, 256), 256, 0, s>>>(
          m->d_wbf + ly.w_off, ly.out_p, ly.in_p, m->d_wpk + ly.w_off);
    }
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    m->pk_stale = false;
  }
  TcNet net{};
  net.n_layers = m->n_layers_total;
  net.n_in = m->n_in;
  net.n_out = m->n_out;
  for (int l = 0; l < m->n_layers_total; ++l) {
    const Layer& ly = m->layer[l];
    net.in_p[l] = ly.in_p;
    net.out_p[l] = ly.out_p;
    net.n_valid[l] = ly.n_out;
    net.w[l] = m->d_wpk + ly.w_off;
    net.b[l] = m->d_param + ly.b_off;
  }
  const size_t smem = tc_smem_bytes();
  if (cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return RT_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->dev) != cudaSuccess)
    return RT_ERR_CUDA;
  const long long tiles = (M + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  k_mlp_forward_tc<<<grid, kTcThreads, smem, s>>>(net, x, M, y, m->d_err);
  return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

// forward over Mp padded rows of d_a[0]
rt_status forward_rows(rt_mlp* m, long long Mp, cudaStream_t s) {
  const int L = m->n_layers_total;
  for (int l = 0; l < L; ++l) {
    const Layer& ly = m->layer[l];
    if (gemm<false, true>(m->d_a[l], ly.in_p, m->d_wbf + ly.w_off, ly.in_p, m->d_z[l], ly.out_p,
                          Mp, ly.out_p, ly.in_p, false, m->d_err, s) != cudaSuccess)
      return RT_ERR_CUDA;
    k_bias_act<<<nb(Mp * ly.out_p, 256), 256, 0, s>>>(m->d_z[l], m->d_param + ly.b_off, Mp,
                                                      ly.out_p, ly.n_out, l < L - 1,
                                                      m->d_a[l + 1]);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
  }
  return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_mlp_create(int n_in, int n_hidden, int n_layers, int n_out, uint64_t seed,
                        rt_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_layers < 1 || n_layers > kMaxLayers - 1 ||
      n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
    return RT_ERR_ARG;
  *out = nullptr;
  rt_mlp* m = new (std::nothrow) rt_mlp();
  if (!m) return RT_ERR_OOM;
  if (cudaGetDevice(&m->dev) != cudaSuccess) {
    delete m;
    return RT_ERR_CUDA;
  }
  m->n_in = n_in;
  m->n_out = n_out;
  m->n_layers_total = n_layers + 1;
  size_t off = 0;
  int64_t np = 0;
  for (int l = 0; l <= n_layers; ++l) {
    Layer& ly = m->layer[l];
    ly.n_in = l == 0 ? n_in : n_hidden;
    ly.n_out = l == n_layers ? n_out : n_hidden;
    ly.in_p = pad16(ly.n_in);
    ly.out_p = pad16(ly.n_out);
    ly.w_off = off;
    off += (size_t)ly.in_p * ly.out_p;
    ly.b_off = off;
    off += (size_t)ly.out_p;
    np += (int64_t)ly.n_in * ly.n_out + ly.n_out;
    if (ly.in_p > m->max_p) m->max_p = ly.in_p;
    if (ly.out_p > m->max_p) m->max_p = ly.out_p;
  }
  // keep BF16 weight offsets 16-element aligned: offsets are sums of multiples of 16
  m->n_padded = off;
  m->n_params = np;
  rt_status st;
  if ((st = alloc(&m->d_param, off)) != RT_OK || (st = alloc(&m->d_grad, off)) != RT_OK ||
      (st = alloc(&m->d_m, off)) != RT_OK || (st = alloc(&m->d_v, off)) != RT_OK ||
      (st = alloc(&m->d_wbf, off)) != RT_OK || (st = alloc(&m->d_wpk, off)) != RT_OK ||
      (st = alloc(&m->d_err, 1)) != RT_OK || (st = alloc(&m->d_loss, 1)) != RT_OK) {
    rt_mlp_destroy(m);
    return st;
  }
  // He-uniform weights from a seeded splitmix64 stream, zero biases
  std::vector<float> h(off, 0.0f);
  uint64_t x = seed;
  for (int l = 0; l <= n_layers; ++l) {
    const Layer& ly = m->layer[l];
    float lim = std::sqrt(6.0f / (float)ly.n_in);
    for (int r = 0; r < ly.n_out; ++r)
      for (int c = 0; c < ly.n_in; ++c) {
        double u = (double)(splitmix(x) >> 11) * (1.0 / 9007199254740992.0);
        h[ly.w_off + (size_t)r * ly.in_p + c] = (float)((2.0 * u - 1.0) * lim);
      }
  }
  cudaError_t e = cudaMemcpy(m->d_param, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMemset(m->d_grad, 0, sizeof(float) * off);
  if (e == cudaSuccess) e = cudaMemset(m->d_err, 0, sizeof(unsigned));
  if (e != cudaSuccess || refresh_bf16(m, nullptr) != RT_OK) {
    rt_mlp_destroy(m);
    return RT_ERR_CUDA;
  }
  *out = m;
  return RT_OK;
}

rt_status rt_mlp_destroy(rt_mlp* m) {
  if (!m) return RT_OK;
  cudaSetDevice(m->dev);
  free_acts(m);
  release(m->d_param);
  release(m->d_grad);
  release(m->d_m);
  release(m->d_v);
  release(m->d_wbf);
  release(m->d_wpk);
  release(m->d_err);
  release(m->d_loss);
  delete m;
  return RT_OK;
}

rt_status rt_mlp_dims(const rt_mlp* m, int* n_in, int* n_out) {
  if (!m || !n_in || !n_out) return RT_ERR_ARG;
  *n_in = m->n_in;
  *n_out = m->n_out;
  return RT_OK;
}

rt_status rt_mlp_set_range(rt_mlp* m, float lo, float hi) {
  if (!m || !(hi >= lo)) return RT_ERR_ARG;
  m->x_lo = lo;
  m->x_hi = hi;
  return RT_OK;
}

rt_status rt_mlp_get_range(const rt_mlp* m, float* lo, float* hi) {
  if (!m || !lo || !hi) return RT_ERR_ARG;
  *lo = m->x_lo;
  *hi = m->x_hi;
  return RT_OK;
}

rt_status rt_mlp_n_params(const rt_mlp* m, int64_t* n) {
  if (!m || !n) return RT_ERR_ARG;
  *n = m->n_params;
  return RT_OK;
}

static rt_status copy_params(rt_mlp* m, float* host, const float* src_dev) {
  std::vector<float> h(m->n_padded);
  if (cudaMemcpy(h.data(), src_dev, sizeof(float) * m->n_padded, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return RT_ERR_CUDA;
  size_t o = 0;
  for (int l = 0; l < m->n_layers_total; ++l) {
    const Layer& ly = m->layer[l];
    for (int r = 0; r < ly.n_out; ++r)
      for (int c = 0; c < ly.n_in; ++c) host[o++] = h[ly.w_off + (size_t)r * ly.in_p + c];
    for (int r = 0; r < ly.n_out; ++r) host[o++] = h[ly.b_off + r];
  }
  return RT_OK;
}

rt_status rt_mlp_get_params(rt_mlp* m, float* out) {
  if (!m || !out) return RT_ERR_ARG;
  if (cudaSetDevice(m->dev) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return RT_ERR_CUDA;
  unsigned err = 0;
  if (cudaMemcpy(&err, m->d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RT_ERR_CUDA;
  rt_status st = copy_params(m, out, m->d_param);
  return st != RT_OK ? st : (err ? RT_ERR_TIMEOUT : RT_OK);
}

rt_status rt_mlp_set_params(rt_mlp* m, const float* in) {
  if (!m || !in) return RT_ERR_ARG;
  std::vector<float> h(m->n_padded, 0.0f);
  size_t o = 0;
  for (int l = 0; l < m->n_layers_total; ++l) {
    const Layer& ly = m->layer[l];
    for (int r = 0; r < ly.n_out; ++r)
      for (int c = 0; c < ly.n_in; ++c) h[ly.w_off + (size_t)r * ly.in_p + c] = in[o++];
    for (int r = 0; r < ly.n_out; ++r) h[ly.b_off + r] = in[o++];
  }
  if (cudaSetDevice(m->dev) != cudaSuccess) return RT_ERR_CUDA;
  if (cudaMemcpy(m->d_param, h.data(), sizeof(float) * m->n_padded, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return RT_ERR_CUDA;
  return refresh_bf16(m, nullptr);
}

rt_status rt_mlp_forward(rt_mlp* m, const float* x, float* y, int64_t M, void* stream) {
  if (!m || !x || !y || M < 0) return RT_ERR_ARG;
  if (M == 0) return RT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(m->dev) != cudaSuccess) return RT_ERR_CUDA;
  if (tc_eligible(m)) return forward_tc(m, x, y, M, s);
  const long long chunk = 1ll << 18;
  for (long long r0 = 0; r0 < M; r0 += chunk) {
    long long Mc = M - r0 < chunk ? M - r0 : chunk;
    long long Mp = (Mc + kTile - 1) / kTile * kTile;
    rt_status st = ensure_rows(m, Mp);
    if (st != RT_OK) return st;
    const Layer& l0 = m->layer[0];
    k_pack_input<<<nb(Mp * l0.in_p, 256), 256, 0, s>>>(x + r0 * m->n_in, Mc, m->n_in, Mp,
                                                       l0.in_p, m->d_a[0]);
    if ((st = forward_rows(m, Mp, s)) != RT_OK) return st;
    const Layer& ll = m->layer[m->n_layers_total - 1];
    k_unpack_output<<<nb(Mc * m->n_out, 256), 256, 0, s>>>(m->d_z[m->n_layers_total - 1], Mc,
                                                           m->n_out, ll.out_p,
                                                           y + r0 * m->n_out);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
  }
  return RT_OK;
}

rt_status rt_mlp_loss_grad(rt_mlp* m, const float* x, const float* t, int64_t M, float* loss_out,
                           float* grad_out, void* stream) {
  if (!m || !x || !t || M < 1 || M > (1ll << 24)) return RT_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(m->dev) != cudaSuccess) return RT_ERR_CUDA;
  const long long Mp = (M + kTile - 1) / kTile * kTile;
  rt_status st = ensure_rows(m, Mp);
  if (st != RT_OK) return st;
  const int L = m->n_layers_total;
  const Layer& l0 = m->layer[0];
  if (cudaMemsetAsync(m->d_grad, 0, sizeof(float) * m->n_padded, s) != cudaSuccess ||
      cudaMemsetAsync(m->d_loss, 0, sizeof(float), s) != cudaSuccess)
    return RT_ERR_CUDA;
  k_pack_input<<<nb(Mp * l0.in_p, 256), 256, 0, s>>>(x, M, m->n_in, Mp, l0.in_p, m->d_a[0]);
  if ((st = forward_rows(m, Mp, s)) != RT_OK) return st;
  const Layer& lo = m->layer[L - 1];
  k_mse_grad<<<nb(Mp * lo.out_p, 256), 256, 0, s>>>(m->d_z[L - 1], t, M, m->n_out, Mp, lo.out_p,
                                                    m->d_dz, m->d_dzb, m->d_loss);
  for (int l = L - 1; l >= 0; --l) {
    const Layer& ly = m->layer[l];
    // dW_l = dz^T a_{l-1}: [out_p][in_p], contraction over rows (split)
    if (gemm<true, false>(m->d_dzb, ly.out_p, m->d_a[l], ly.in_p, m->d_grad + ly.w_off, ly.in_p,
                          ly.out_p, ly.in_p, (int)Mp, true, m->d_err, s) != cudaSuccess)
      return RT_ERR_CUDA;
    dim3 g2(nb(ly.out_p, 32), 64);
    k_col_sums<<<g2, 256, 0, s>>>(m->d_dz, Mp, ly.out_p, m->d_grad + ly.b_off);
    if (l > 0) {
      // da_{l-1} = dz W_l: [Mp][in_p]; then through silu'
      if (gemm<false, false>(m->d_dzb, ly.out_p, m->d_wbf + ly.w_off, ly.in_p, m->d_dz, ly.in_p,
                             Mp, ly.in_p, ly.out_p, false, m->d_err, s) != cudaSuccess)
        return RT_ERR_CUDA;
      const Layer& lp = m->layer[l - 1];
      k_act_back<<<nb(Mp * ly.in_p, 256), 256, 0, s>>>(m->d_dz, m->d_z[l - 1], Mp, ly.in_p,
                                                       lp.n_out, m->d_dzb);
    }
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
  }
  if (loss_out &&
      cudaMemcpyAsync(loss_out, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return RT_ERR_CUDA;
  if (grad_out || loss_out) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return RT_ERR_CUDA;
  }
  if (grad_out) return copy_params(m, grad_out, m->d_grad);
  return RT_OK;
}

rt_status rt_mlp_adam_step(rt_mlp* m, float lr, void* stream) {
  if (!m || !(lr > 0)) return RT_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(m->dev) != cudaSuccess) return RT_ERR_CUDA;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
  k_adam<<<nb((long long)m->n_padded, 256), 256, 0, s>>>(m->d_param, m->d_grad, m->d_m, m->d_v,
                                                         m->n_padded, lr, b1, b2, c1, c2, 1e-8f);
  if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
  return refresh_bf16(m, s);
}

}  // extern "C"
