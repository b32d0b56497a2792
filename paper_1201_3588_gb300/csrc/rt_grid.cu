// rt_grid.cu -- building a grid handle on the device: the walk of the tree of cubes
// and 2x2x2 subcubes that gives every leaf its level and integer corner (checking
// that every leaf and every block is reached exactly once, within max_level), and
// the densities as [leaf][species] floats times the base-cube edge (checking that
// they are finite and not negative).
//
// The walk goes level by level: the base cubes first, then the children of the
// blocks reached at the level before. A leaf or block reached twice, an id out of
// range or a block below max_level sets the error word; so does any leaf or block
// left unreached.

#include "rt_internal.h"

namespace rt {
namespace {

// claim bit i of a bitmap; true when it was already set
__device__ __forceinline__ bool claim(unsigned* bits, long long i) {
  const unsigned m = 1u << (i & 31);
  return (atomicOr(&bits[i >> 5], m) & m) != 0u;
}

__device__ __forceinline__ void reach(const TreeBuild& tb, int node, int lev, int i, int j,
                                      int k) {
  if (node >= 0) {
    if ((long long)node >= tb.n_leaves || claim(tb.leaf_seen, node)) {
      atomicOr(tb.err, 1u);
      return;
    }
    tb.level[node] = (int8_t)lev;
    tb.ijk[(size_t)node * 3 + 0] = i;
    tb.ijk[(size_t)node * 3 + 1] = j;
    tb.ijk[(size_t)node * 3 + 2] = k;
    atomicMax(tb.max_seen, lev);
  } else {
    const long long blk = -(long long)node - 1;
    if (blk >= tb.n_blocks || lev >= tb.max_level || claim(tb.blk_seen, blk)) {
      atomicOr(tb.err, 1u);
      return;
    }
    tb.blk_level[blk] = (int8_t)lev;
    tb.blk_ijk[(size_t)blk * 3 + 0] = i;
    tb.blk_ijk[(size_t)blk * 3 + 1] = j;
    tb.blk_ijk[(size_t)blk * 3 + 2] = k;
  }
}

__global__ void k_tree_base(TreeBuild tb) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = tb.n_base;
  if (b >= n * n * n) return;
  reach(tb, tb.base[b], 0, (int)(b % n), (int)((b / n) % n), (int)(b / (n * n)));
}

// children of the blocks reached at level lev - 1, one thread per (block, octant)
__global__ void k_tree_level(TreeBuild tb, int lev) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= tb.n_blocks * 8) return;
  const long long blk = idx >> 3;
  const int o = (int)(idx & 7);
  if (tb.blk_level[blk] != lev - 1) return;
  const int* I = tb.blk_ijk + blk * 3;
  reach(tb, tb.child[idx], lev, 2 * I[0] + (o & 1), 2 * I[1] + ((o >> 1) & 1),
        2 * I[2] + ((o >> 2) & 1));
}

// every leaf and block reached
__global__ void k_tree_complete(TreeBuild tb) {
  const long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nl = (tb.n_leaves + 31) >> 5, nb = (tb.n_blocks + 31) >> 5;
  if (w < nl) {
    const long long rest = tb.n_leaves - (w << 5);
    const unsigned want = rest >= 32 ? 0xffffffffu : ((1u << rest) - 1u);
    if ((tb.leaf_seen[w] & want) != want) atomicOr(tb.err, 1u);
  }
  if (w < nb) {
    const long long rest = tb.n_blocks - (w << 5);
    const unsigned want = rest >= 32 ? 0xffffffffu : ((1u << rest) - 1u);
    if ((tb.blk_seen[w] & want) != want) atomicOr(tb.err, 1u);
  }
}

// [S][N] doubles -> [N][S] floats times d0; bad values set the error word
__global__ void k_rho_convert(const double* src, long long N, int S, double d0, float* dst,
                              unsigned* err) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  for (int s = 0; s < S; ++s) {
    const double r = src[(size_t)s * N + c];
    if (!(r >= 0.0) || !isfinite(r)) atomicOr(err, 2u);
    dst[(size_t)c * S + s] = (float)(r * d0);
  }
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_tree_walk(const TreeBuild& tb, cudaStream_t s) {
  const long long nb = (long long)tb.n_base * tb.n_base * tb.n_base;
  cudaError_t e = cudaMemsetAsync(tb.leaf_seen, 0, sizeof(unsigned) * ((tb.n_leaves + 31) >> 5), s);
  if (e == cudaSuccess && tb.n_blocks > 0)
    e = cudaMemsetAsync(tb.blk_seen, 0, sizeof(unsigned) * ((tb.n_blocks + 31) >> 5), s);
  if (e == cudaSuccess && tb.n_blocks > 0)
    e = cudaMemsetAsync(tb.blk_level, 0xff, (size_t)tb.n_blocks, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tb.level, 0xff, (size_t)tb.n_leaves, s);
  if (e != cudaSuccess) return e;
  k_tree_base<<<nblk(nb, 256), 256, 0, s>>>(tb);
  for (int lev = 1; lev <= tb.max_level && tb.n_blocks > 0; ++lev)
    k_tree_level<<<nblk(tb.n_blocks * 8, 256), 256, 0, s>>>(tb, lev);
  const long long words = ((tb.n_leaves > tb.n_blocks ? tb.n_leaves : tb.n_blocks) + 31) >> 5;
  k_tree_complete<<<nblk(words, 256), 256, 0, s>>>(tb);
  return cudaGetLastError();
}

cudaError_t launch_rho_convert(const double* src, long long N, int S, double d0, float* dst,
                               unsigned* err, cudaStream_t s) {
  k_rho_convert<<<nblk(N, 256), 256, 0, s>>>(src, N, S, d0, dst, err);
  return cudaGetLastError();
}

}  // namespace rt
