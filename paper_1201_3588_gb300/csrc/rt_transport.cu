// rt_transport.cu -- photon-package transport kernels of librt_gb300.
//
// A package (Sec. 2) leaves the star with constant energy eps at a frequency bin
// drawn from the stellar spectrum, samples an optical depth tau = -ln(xi), and
// walks the grid of cubes and subcubes cell by cell, spending
// rho * kappa_ext * path of its tau in each cell. Where tau runs out it
// interacts: with probability kappa_sca / kappa_ext it scatters by the
// Henyey-Greenstein phase function, otherwise it is absorbed -- the cell's count
// of absorptions rises by one (an exact integer; eps is constant) and a package
// of the same energy leaves the absorption spot isotropically at a frequency
// drawn from the re-emission spectrum. A package that leaves the domain is binned
// into the escaped spectrum.
//
// Random numbers: Philox4x32-10 (Salmon et al. 2011), key = seed, counter =
// (package id lo, id hi, event index, block). Event 0 is the emission and uses
// one block: {bin, mu, phi, tau}. Interaction k uses block 0 = {albedo test,
// species, mu, phi} and block 1 = {tau, energy position, bin, -}. Each 32-bit word
// maps to the midpoint of one of 2^23 equal sub-intervals of (0,1).
//
// Re-emission bin: the three rules of Sec. 2 (the Bjorkman & Wood difference
// spectrum, its omission, a frozen temperature) are all mixtures over the
// temperature-table intervals: an energy per gram u is drawn uniformly in
// [u_lo, u_hi] (BW: [n, n+1] eps/M; no correction: [0, max(n eps/M, S(t_min))];
// frozen: [0, S(T_frozen)]), the table interval holding u is found in S(T), and
// the bin is drawn from that interval's normalised cumulative difference
// kappa_abs [P_b(T_{i+1}) - P_b(T_i)].
//
// Geometry: positions are in base-cube units. A point on a face belongs to the
// cell ahead of the direction of motion. After a face crossing the position is
// set exactly onto the face (exactly representable) and the other coordinates are
// clamped into the cell, so every crossing advances the cell index.

#include "rt_internal.h"

#include <math.h>

#include <type_traits>

namespace rt {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 draw(unsigned long long seed, unsigned long long id,
                                      unsigned event, unsigned block) {
  return philox10(make_uint4((unsigned)id, (unsigned)(id >> 32), event, block),
                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

template <typename R>
__device__ __forceinline__ R unit(unsigned x) {
  return ((R)(x >> 9) + (R)0.5) * (R)(1.0 / 8388608.0);
}

// ---------------------------------------------------------------- math helpers
template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ void sincos2pi(R xi, R* s, R* c);
template <> __device__ __forceinline__ void sincos2pi(float xi, float* s, float* c) {
  sincospif(2.0f * xi, s, c);
}
template <> __device__ __forceinline__ void sincos2pi(double xi, double* s, double* c) {
  sincospi(2.0 * xi, s, c);
}

template <typename R> __device__ __forceinline__ R log_(R x);
template <> __device__ __forceinline__ float log_(float x) { return logf(x); }
template <> __device__ __forceinline__ double log_(double x) { return log(x); }

// isotropic direction from two deviates
template <typename R>
__device__ __forceinline__ void isotropic(R xmu, R xphi, R d[3]) {
  R mu = (R)2 * xmu - (R)1;
  R s = sqrt(fmax((R)0, (R)1 - mu * mu));
  R sp, cp;
  sincos2pi(xphi, &sp, &cp);
  d[0] = s * cp;
  d[1] = s * sp;
  d[2] = mu;
}

// Henyey-Greenstein cos(theta) by inversion of its cumulative distribution
template <typename R>
__device__ __forceinline__ R hg_mu(R g, R xi) {
  if (fabs(g) < (R)1e-6) return (R)2 * xi - (R)1;
  R f = ((R)1 - g * g) / ((R)1 - g + (R)2 * g * xi);
  R mu = ((R)1 + g * g - f * f) / ((R)2 * g);
  return fmin((R)1, fmax((R)-1, mu));
}

// turn d by polar cosine mu and azimuth 2 pi xphi, azimuth counted from
// (dx dz, dy dz, -(1-dz^2))/sqrt(1-dz^2) towards (-dy, dx, 0)/sqrt(1-dz^2)
template <typename R>
__device__ __forceinline__ void turn(R d[3], R mu, R xphi) {
  R s = sqrt(fmax((R)0, (R)1 - mu * mu));
  R sp, cp;
  sincos2pi(xphi, &sp, &cp);
  R ux = d[0], uy = d[1], uz = d[2], nx, ny, nz;
  if (fabs(uz) > (R)0.99999) {
    nx = s * cp;
    ny = s * sp;
    nz = (uz > (R)0 ? mu : -mu);
  } else {
    R r2 = (R)1 - uz * uz;
    R ir = rsqrt_(r2);
    R r = r2 * ir;
    nx = mu * ux + s * (ux * uz * cp - uy * sp) * ir;
    ny = mu * uy + s * (uy * uz * cp + ux * sp) * ir;
    nz = mu * uz - s * r * cp;
  }
  R in = rsqrt_(nx * nx + ny * ny + nz * nz);
  d[0] = nx * in;
  d[1] = ny * in;
  d[2] = nz * in;
}

// first index whose normalised cumulative value exceeds xi (cdf[n-1] == 1)
__device__ __forceinline__ int search_cdf(const float* cdf, int n, float xi) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > xi) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// ---------------------------------------------------------------- grid
template <typename R>
__device__ __forceinline__ int cell_index(R q, R d) {
  R f = floor(q);
  int i = (int)f;
  if (d < (R)0 && f == q) --i;
  return i;
}

// Leaf holding p when moving along d. Returns 0 inside, 1 outside, -1 malformed.
template <typename R>
__device__ __forceinline__ int locate(const DevGrid& g, const R p[3], const R d[3],
                                      int& leaf, int& level, int I[3]) {
  const int n = g.n_base;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    I[a] = cell_index(p[a], d[a]);
    if (I[a] < 0 || I[a] >= n) return 1;
  }
  int node = __ldg(&g.base[I[0] + n * (I[1] + n * I[2])]);
  int lev = 0;
  while (node < 0) {
    long long blk = -(long long)node - 1;
    if (blk >= g.n_blocks || lev >= g.max_level) return -1;
    ++lev;
    R sc = (R)(1 << lev);
    int oct = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int j = cell_index(p[a] * sc, d[a]);
      int o = j - 2 * I[a];
      if ((unsigned)o > 1u) return -1;
      oct |= o << a;
      I[a] = j;
    }
    node = __ldg(&g.child[blk * 8 + oct]);
  }
  if ((long long)node >= g.n_leaves) return -1;
  leaf = node;
  level = lev;
  return 0;
}

// ---------------------------------------------------------------- package
template <typename R>
struct Pkg {
  R p[3], d[3];
  R inv[3];  // 1/d; +inf where d == 0 (of either sign)
  R tau;
  int bin;
  unsigned event;
  unsigned long long id;
  bool touched;  // interacted at least once
};

struct Tally {  // per-thread counters, flushed to the 64-bit device totals
  unsigned emitted, escaped, capped, absorptions, scatters, crossings, errors, clamped;
  unsigned levels;  // child-table reads of the walk
  unsigned peel_events, peel_crossings;  // peel-off sight lines and the cells they cross
};

// a flush is forced before any per-thread counter could pass 2^31
constexpr unsigned kTallyFlushAt = 1u << 31;

enum Adv { kCrossed = 0, kInteract = 1, kEscaped = 2, kError = 3 };

template <typename R>
__device__ __forceinline__ void set_inverse(Pkg<R>& k) {
#pragma unroll
  for (int a = 0; a < 3; ++a) k.inv[a] = k.d[a] == (R)0 ? (R)INFINITY : (R)1 / k.d[a];
}

template <typename R>
__device__ __forceinline__ void emit(Pkg<R>& k, unsigned long long id, const DevRun& r,
                                     const float* star_cdf, int B) {
  uint4 w = draw(r.seed, id, 0u, 0u);
  k.id = id;
  k.event = 0;
  k.touched = false;
  k.bin = search_cdf(star_cdf, B, unit<float>(w.x));
  if (r.source_kind == 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) k.d[a] = sizeof(R) == 8 ? (R)r.beam64[a] : (R)r.beam[a];
  } else {
    isotropic<R>(unit<R>(w.y), unit<R>(w.z), k.d);
  }
  k.tau = -log_(unit<R>(w.w));
#pragma unroll
  for (int a = 0; a < 3; ++a) k.p[a] = sizeof(R) == 8 ? (R)r.src64[a] : (R)r.src[a];
  set_inverse(k);
}

// One cell: cross it, or move to the interaction point inside it (the leaf is found
// from the base cube each time: the plain walk).
template <typename R>
__device__ __forceinline__ int advance(Pkg<R>& k, const DevGrid& g, const Kappa* kap,
                                       int& leaf, int& level, float* pathabs) {
  int I[3];
  int rc = locate(g, k.p, k.d, leaf, level, I);
  if (rc == 1) return kEscaped;
  if (rc < 0) return kError;
  const R sz = (R)1 / (R)(1 << level);
  const R lo0 = (R)I[0] * sz, lo1 = (R)I[1] * sz, lo2 = (R)I[2] * sz;
  const R hi0 = lo0 + sz, hi1 = lo1 + sz, hi2 = lo2 + sz;
  const R d0 = k.d[0], d1 = k.d[1], d2 = k.d[2];
  const R inf = (R)INFINITY;
  const R t0 = d0 > (R)0 ? (hi0 - k.p[0]) * k.inv[0] : (d0 < (R)0 ? (lo0 - k.p[0]) * k.inv[0] : inf);
  const R t1 = d1 > (R)0 ? (hi1 - k.p[1]) * k.inv[1] : (d1 < (R)0 ? (lo1 - k.p[1]) * k.inv[1] : inf);
  const R t2 = d2 > (R)0 ? (hi2 - k.p[2]) * k.inv[2] : (d2 < (R)0 ? (lo2 - k.p[2]) * k.inv[2] : inf);
  int ax;
  R tex;
  if (t0 <= t1 && t0 <= t2) {
    ax = 0;
    tex = t0;
  } else if (t1 <= t2) {
    ax = 1;
    tex = t1;
  } else {
    ax = 2;
    tex = t2;
  }
  tex = fmax(tex, (R)0);
  // extinction per base-cube unit of path: sum_s (rho_s d0) kappa_ext,s(bin)
  const float* rho = g.rho + (size_t)leaf * g.S;
  const Kappa* kb = kap + k.bin * g.S;
  R kx = (R)0;
  for (int s = 0; s < g.S; ++s) kx += (R)__ldg(&rho[s]) * (R)kb[s].kext;
  const R dtau = kx * tex;
  if (pathabs) {  // path-length tally of the segment inside this cell
    const R seg = (kx > (R)0 && dtau > k.tau) ? k.tau / kx : tex;
    for (int s = 0; s < g.S; ++s) {
      const float v = (float)((R)__ldg(&rho[s]) * (R)kb[s].kabs * seg);
      if (v > 0.f) atomicAdd(&pathabs[(size_t)s * g.n_leaves + leaf], v);
    }
  }
  if (kx > (R)0 && dtau > k.tau) {
    const R sd = k.tau / kx;
    k.p[0] = fmin(hi0, fmax(lo0, k.p[0] + sd * d0));
    k.p[1] = fmin(hi1, fmax(lo1, k.p[1] + sd * d1));
    k.p[2] = fmin(hi2, fmax(lo2, k.p[2] + sd * d2));
    return kInteract;
  }
  k.tau -= dtau;
  const R f0 = d0 > (R)0 ? hi0 : lo0, f1 = d1 > (R)0 ? hi1 : lo1, f2 = d2 > (R)0 ? hi2 : lo2;
  k.p[0] = ax == 0 ? f0 : fmin(hi0, fmax(lo0, k.p[0] + tex * d0));
  k.p[1] = ax == 1 ? f1 : fmin(hi1, fmax(lo1, k.p[1] + tex * d1));
  k.p[2] = ax == 2 ? f2 : fmin(hi2, fmax(lo2, k.p[2] + tex * d2));
  return kCrossed;
}

// ---------------------------------------------------------------- linked walk
// The leaf a package is in, with its level, its lower corner and its edge (base-cube
// units; both exact in FP32: multiples of 2^-level below 2^13).
struct Cell {
  int leaf;
  float lo[3];
  float sz;  // 2^-level
  __device__ __forceinline__ int level() const { return 127 - (__float_as_int(sz) >> 23); }
};

__device__ __forceinline__ void set_corner(Cell& c, const int I[3], int level) {
  c.sz = __int_as_float((127 - level) << 23);
#pragma unroll
  for (int a = 0; a < 3; ++a) c.lo[a] = (float)I[a] * c.sz;
}

// Enter the grid at the package's position (full descent from the base cube).
__device__ __forceinline__ int enter(const Pkg<float>& k, const DevGrid& g, Cell& c,
                                     unsigned& child_reads) {
  int I[3], level;
  int rc = locate<float>(g, k.p, k.d, c.leaf, level, I);
  if (rc == 0) {
    child_reads += level;
    set_corner(c, I, level);
  }
  return rc;
}

// One cell of the walk using the face links: the exit face follows from the
// geometry alone, so the face link and the densities come from one record read;
// the next leaf is the linked one (same size or coarser), or is found by a short
// descent when the neighbouring region is finer. kLos: a sight line, which never
// interacts and adds the cell's optical depth to *tau_los instead.
template <bool kLos = false, int kS = 0>
__device__ __forceinline__ int advance_linked(Pkg<float>& k, Cell& c, const DevGrid& g,
                                              const Kappa* kap,
                                              unsigned& child_reads, float* pathabs,
                                              float* tau_los = nullptr) {
  // every array below is indexed with constants only, so it stays in registers
  const float sz = c.sz;
  const float lo0 = c.lo[0], lo1 = c.lo[1], lo2 = c.lo[2];
  const float hi0 = lo0 + sz, hi1 = lo1 + sz, hi2 = lo2 + sz;
  const float d0 = k.d[0], d1 = k.d[1], d2 = k.d[2];
  // distance to the face ahead on each axis; an axis with d == 0 has inv = +inf and
  // gives +inf, or NaN on its upper face, which the minimum below never picks
  const float t0 = ((k.inv[0] > 0.f ? hi0 : lo0) - k.p[0]) * k.inv[0];
  const float t1 = ((k.inv[1] > 0.f ? hi1 : lo1) - k.p[1]) * k.inv[1];
  const float t2 = ((k.inv[2] > 0.f ? hi2 : lo2) - k.p[2]) * k.inv[2];
  // exit axis: the nearest face, the lowest axis on ties
  const float tmin = fminf(fminf(t0, t1), t2);
  const int ax = t0 == tmin ? 0 : (t1 == tmin ? 1 : 2);
  const float tex = fmaxf(tmin, 0.f);
  const float dax = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
  const bool up = dax > 0.f;
  const int* rec = g.links + (size_t)c.leaf * kRec;
  const int link = __ldg(rec + 2 * ax + (up ? 1 : 0));
  // kS: the species count when fixed at compile time (2: both densities in the
  // record), 0 when read from the grid
  const Kappa* kb = kap + k.bin * (kS > 0 ? kS : g.S);
  float kx;
  if (kS == 2 || (kS == 0 && g.S <= 2)) {
    kx = __int_as_float(__ldg(rec + 6)) * kb[0].kext;
    if (kS == 2 || g.S == 2) kx += __int_as_float(__ldg(rec + 7)) * kb[1].kext;
  } else {
    const float* rho = g.rho + (size_t)c.leaf * g.S;
    kx = 0.f;
    for (int s = 0; s < g.S; ++s) kx += __ldg(&rho[s]) * kb[s].kext;
  }
  const float dtau = kx * tex;
  bool hit;
  if constexpr (kLos) {
    *tau_los += dtau;
    hit = false;
  } else {
    hit = kx > 0.f && dtau > k.tau;
  }
  if (!kLos && pathabs) {  // path-length tally of the segment inside this cell
    const float seg = hit ? k.tau / kx : tex;
    const float* rho = g.rho + (size_t)c.leaf * g.S;
    for (int s = 0; s < g.S; ++s) {
      const float v = __ldg(&rho[s]) * kb[s].kabs * seg;
      if (v > 0.f) atomicAdd(&pathabs[(size_t)s * g.n_leaves + c.leaf], v);
    }
  }
  if (hit) {
    const float sd = k.tau / kx;
    k.p[0] = fminf(hi0, fmaxf(lo0, k.p[0] + sd * d0));
    k.p[1] = fminf(hi1, fmaxf(lo1, k.p[1] + sd * d1));
    k.p[2] = fminf(hi2, fmaxf(lo2, k.p[2] + sd * d2));
    return kInteract;
  }
  if constexpr (!kLos) k.tau -= dtau;
  const float f0 = d0 > 0.f ? hi0 : lo0, f1 = d1 > 0.f ? hi1 : lo1, f2 = d2 > 0.f ? hi2 : lo2;
  k.p[0] = ax == 0 ? f0 : fminf(hi0, fmaxf(lo0, k.p[0] + tex * d0));
  k.p[1] = ax == 1 ? f1 : fminf(hi1, fmaxf(lo1, k.p[1] + tex * d1));
  k.p[2] = ax == 2 ? f2 : fminf(hi2, fmaxf(lo2, k.p[2] + tex * d2));
  if (link == kLinkEscape) return kEscaped;
  // the same-size neighbour's corner
  const float step = up ? sz : -sz;
  const float n0 = ax == 0 ? lo0 + step : lo0;
  const float n1 = ax == 1 ? lo1 + step : lo1;
  const float n2 = ax == 2 ? lo2 + step : lo2;
  if (link >= 0) {
    const int nl = link >> 28;
    const float nsz = __int_as_float((127 - nl) << 23);
    c.leaf = link & kLinkLeafMask;
    if (nsz == sz) {
      c.lo[0] = n0;
      c.lo[1] = n1;
      c.lo[2] = n2;
    } else {  // a coarser leaf: round the corner down to its edge (exact)
      c.sz = nsz;
      const float isz = __int_as_float((127 + nl) << 23);
      c.lo[0] = floorf(n0 * isz) * c.sz;
      c.lo[1] = floorf(n1 * isz) * c.sz;
      c.lo[2] = floorf(n2 * isz) * c.sz;
    }
    return kCrossed;
  }
  // the same-size neighbour is split: descend, staying inside that node
  int lev = c.level();
  const float iz = __int_as_float((127 + lev) << 23);  // 2^level
  int J0 = (int)(n0 * iz), J1 = (int)(n1 * iz), J2 = (int)(n2 * iz);
  long long blk = -(long long)link - 1;
  for (;;) {
    if (blk >= g.n_blocks || lev >= g.max_level) return kError;
    ++lev;
    ++child_reads;
    const float sc = (float)(1 << lev);
    const int j0 = min(max(cell_index(k.p[0] * sc, d0), 2 * J0), 2 * J0 + 1);
    const int j1 = min(max(cell_index(k.p[1] * sc, d1), 2 * J1), 2 * J1 + 1);
    const int j2 = min(max(cell_index(k.p[2] * sc, d2), 2 * J2), 2 * J2 + 1);
    const int oct = (j0 - 2 * J0) | ((j1 - 2 * J1) << 1) | ((j2 - 2 * J2) << 2);
    J0 = j0;
    J1 = j1;
    J2 = j2;
    const int node = __ldg(&g.child[blk * 8 + oct]);
    if (node >= 0) {
      if ((long long)node >= g.n_leaves) return kError;
      c.leaf = node;
      const int I[3] = {J0, J1, J2};
      set_corner(c, I, lev);
      return kCrossed;
    }
    blk = -(long long)node - 1;
  }
}

// ---------------------------------------------------------------- path walk
// The walk without face links. A package keeps the ids of the child blocks on the
// path from its base cube to its leaf (blk(l): the block holding the path's node at
// level l). Crossing a face, it climbs to the deepest common ancestor of its leaf and
// of the neighbouring position -- the highest bit in which their integer coordinates
// differ gives the number of levels to climb -- and descends from there: a neighbour
// in the same block costs one child read, in the sector the leaf's own read left in
// L1. Its random reads go to the densities and the child table (3.5 GB for the large
// disk's 1.7e8 cells) instead of the face-link records and densities (8.3 GB), whose
// address translation misses cost more than the extra reads on grids that large. The
// geometry is the linked walk's, and so is every neighbour it finds: both walks give
// the same histories.
constexpr int kPathLevels = 4;  // the path walk serves grids of at most 4 levels

struct PathCell {
  int slot;  // tree slot of the leaf: its row in rho_slot
  float kx;  // the leaf's extinction at the package's bin, or -1 when not yet read
  int J[3];  // integer coordinates of the leaf's lower corner at its level
  float sz;  // 2^-level
  int b1, b2, b3, b4;
  __device__ __forceinline__ int level() const { return 127 - (__float_as_int(sz) >> 23); }
  __device__ __forceinline__ int blk(int l) const {
    return l == 1 ? b1 : (l == 2 ? b2 : (l == 3 ? b3 : b4));
  }
  __device__ __forceinline__ void set_blk(int l, int b) {
    if (l == 1) b1 = b;
    else if (l == 2) b2 = b;
    else if (l == 3) b3 = b;
    else b4 = b;
  }
};

// Enter the grid at the package's position: descent from the base cube, recording
// the blocks on the path. 0 inside, 1 outside, -1 malformed (or deeper than the
// walk serves).
__device__ __forceinline__ int enter_path(const Pkg<float>& k, const DevGrid& g, PathCell& c,
                                          unsigned& child_reads) {
  const int n = g.n_base;
  int I[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    I[a] = cell_index(k.p[a], k.d[a]);
    if (I[a] < 0 || I[a] >= n) return 1;
  }
  int slot = I[0] + n * (I[1] + n * I[2]);
  int node = __ldg(&g.base[slot]);
  int lev = 0;
  while (node < 0) {
    const long long blk = -(long long)node - 1;
    if (blk >= g.n_blocks || lev >= g.max_level || lev >= kPathLevels) return -1;
    ++lev;
    c.set_blk(lev, (int)blk);
    const float sc = (float)(1 << lev);
    int oct = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int j = cell_index(k.p[a] * sc, k.d[a]);
      const int o = j - 2 * I[a];
      if ((unsigned)o > 1u) return -1;
      oct |= o << a;
      I[a] = j;
    }
    slot = g.n_base3 + (int)blk * 8 + oct;
    node = __ldg(&g.child[blk * 8 + oct]);
    ++child_reads;
  }
  if ((long long)node >= g.n_leaves) return -1;
  c.slot = slot;
  c.kx = -1.f;
  c.sz = __int_as_float((127 - lev) << 23);
#pragma unroll
  for (int a = 0; a < 3; ++a) c.J[a] = I[a];
  return 0;
}

// The row of a tree slot as one vector (kS = 4 or 2 species; the generic form reads
// the first word here and the rest in slot_ext): a leaf's densities, or for a refined
// slot the child block's code -(block + 1) in the first word (densities are >= +0, so
// the sign bit tells them apart); and the extinction sum over species at the bin's
// opacities kb.
template <int kS>
__device__ __forceinline__ float4 slot_row(const DevGrid& g, int slot) {
  if constexpr (kS == 4) {
    return __ldg(reinterpret_cast<const float4*>(g.rho_slot) + slot);
  } else if constexpr (kS == 2) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(g.rho_slot) + slot);
    return make_float4(v.x, v.y, 0.f, 0.f);
  } else {
    return make_float4(__ldg(&g.rho_slot[(size_t)slot * g.S]), 0.f, 0.f, 0.f);
  }
}

// The leaf id of a leaf's tree slot (from the tree arrays; the walk itself reads only
// the rows), or -1 if the slot holds no leaf.
__device__ __forceinline__ int path_leaf(const DevGrid& g, int slot) {
  const int node = slot < g.n_base3 ? __ldg(&g.base[slot]) : __ldg(&g.child[slot - g.n_base3]);
  return node >= 0 && (long long)node < g.n_leaves ? node : -1;
}

// The extinction opacities of a bin as one vector (kS = 4 or 2: from the block's
// shared-memory copy, one 16- or 8-byte read; zeros for the generic form, which reads
// them from the opacity records kb in slot_ext).
template <int kS>
__device__ __forceinline__ float4 bin_ext(const float* kext, int bin) {
  if constexpr (kS == 4) {
    return reinterpret_cast<const float4*>(kext)[bin];
  } else if constexpr (kS == 2) {
    const float2 e = reinterpret_cast<const float2*>(kext)[bin];
    return make_float4(e.x, e.y, 0.f, 0.f);
  } else {
    return make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int kS>
__device__ __forceinline__ float slot_ext(const DevGrid& g, float4 v, int slot, float4 e,
                                          const Kappa* kb) {
  if constexpr (kS == 4) {
    return v.x * e.x + v.y * e.y + v.z * e.z + v.w * e.w;
  } else if constexpr (kS == 2) {
    return v.x * e.x + v.y * e.y;
  } else {
    const float* rho = g.rho_slot + (size_t)slot * g.S;
    float kx = 0.f;
    for (int s = 0; s < g.S; ++s) kx += __ldg(&rho[s]) * kb[s].kext;
    return kx;
  }
}

// One cell of the path walk (kS: 2 or 4 species read as one vector, 0 the generic
// loop). The next cell is found from the rows alone: the slot of the first node off
// the package's path is known from the block ids it carries, and that slot's row is
// either the leaf's densities or the code of the block to descend into -- one read
// per crossing (one more per level descended). The extinction at the package's bin
// is kept in the cell for the next step.
template <int kS>
__device__ __forceinline__ int advance_path(Pkg<float>& k, PathCell& c, const DevGrid& g,
                                            const Kappa* kap, const float* kext,
                                            unsigned& child_reads) {
  const float sz = c.sz;
  int J0 = c.J[0], J1 = c.J[1], J2 = c.J[2];
  const float lo0 = (float)J0 * sz, lo1 = (float)J1 * sz, lo2 = (float)J2 * sz;
  const float hi0 = lo0 + sz, hi1 = lo1 + sz, hi2 = lo2 + sz;
  const float d0 = k.d[0], d1 = k.d[1], d2 = k.d[2];
  const float t0 = ((k.inv[0] > 0.f ? hi0 : lo0) - k.p[0]) * k.inv[0];
  const float t1 = ((k.inv[1] > 0.f ? hi1 : lo1) - k.p[1]) * k.inv[1];
  const float t2 = ((k.inv[2] > 0.f ? hi2 : lo2) - k.p[2]) * k.inv[2];
  const float tmin = fminf(fminf(t0, t1), t2);
  const int ax = t0 == tmin ? 0 : (t1 == tmin ? 1 : 2);
  const float tex = fmaxf(tmin, 0.f);
  const float dax = ax == 0 ? d0 : (ax == 1 ? d1 : d2);
  const bool up = dax > 0.f;
  const Kappa* kb = kap + k.bin * (kS > 0 ? kS : g.S);
  float kx = c.kx;
  if (kx < 0.f) kx = slot_ext<kS>(g, slot_row<kS>(g, c.slot), c.slot, bin_ext<kS>(kext, k.bin), kb);
  const float dtau = kx * tex;
  if (kx > 0.f && dtau > k.tau) {
    const float sd = k.tau / kx;
    k.p[0] = fminf(hi0, fmaxf(lo0, k.p[0] + sd * d0));
    k.p[1] = fminf(hi1, fmaxf(lo1, k.p[1] + sd * d1));
    k.p[2] = fminf(hi2, fmaxf(lo2, k.p[2] + sd * d2));
    return kInteract;
  }
  k.tau -= dtau;
  const float f0 = d0 > 0.f ? hi0 : lo0, f1 = d1 > 0.f ? hi1 : lo1, f2 = d2 > 0.f ? hi2 : lo2;
  k.p[0] = ax == 0 ? f0 : fminf(hi0, fmaxf(lo0, k.p[0] + tex * d0));
  k.p[1] = ax == 1 ? f1 : fminf(hi1, fmaxf(lo1, k.p[1] + tex * d1));
  k.p[2] = ax == 2 ? f2 : fminf(hi2, fmaxf(lo2, k.p[2] + tex * d2));
  // integer coordinates of the same-size neighbour across face ax
  const int L = c.level();
  const int Iax = ax == 0 ? J0 : (ax == 1 ? J1 : J2);
  const int Jax = up ? Iax + 1 : Iax - 1;
  if (Jax < 0 || Jax >= (g.n_base << L)) return kEscaped;
  if (ax == 0) J0 = Jax;
  else if (ax == 1) J1 = Jax;
  else J2 = Jax;
  const int u = 32 - __clz(Iax ^ Jax);  // levels up to the common ancestor
  int lev, slot;
  if (u > L) {  // another base cube
    lev = 0;
    const int n = g.n_base;
    slot = (J0 >> L) + n * ((J1 >> L) + n * (J2 >> L));
  } else {      // the common ancestor's block holds the first node off the path
    lev = L - u + 1;
    const int sh = L - lev;
    const int oct = ((J0 >> sh) & 1) | (((J1 >> sh) & 1) << 1) | (((J2 >> sh) & 1) << 2);
    slot = g.n_base3 + c.blk(lev) * 8 + oct;
  }
  float4 row = slot_row<kS>(g, slot);
  int K0 = J0 >> (L - lev), K1 = J1 >> (L - lev), K2 = J2 >> (L - lev);
  int code = __float_as_int(row.x);
  while (code < 0) {
    const long long blk = -(long long)code - 1;
    if (blk >= g.n_blocks || lev >= g.max_level || lev >= kPathLevels) return kError;
    ++lev;
    c.set_blk(lev, (int)blk);
    if (lev <= L) {
      const int sh = L - lev;
      K0 = J0 >> sh;
      K1 = J1 >> sh;
      K2 = J2 >> sh;
    } else {  // a finer neighbour: the child holding the crossing point
      const float sc = (float)(1 << lev);
      K0 = min(max(cell_index(k.p[0] * sc, d0), 2 * K0), 2 * K0 + 1);
      K1 = min(max(cell_index(k.p[1] * sc, d1), 2 * K1), 2 * K1 + 1);
      K2 = min(max(cell_index(k.p[2] * sc, d2), 2 * K2), 2 * K2 + 1);
    }
    const int oct = (K0 & 1) | ((K1 & 1) << 1) | ((K2 & 1) << 2);
    slot = g.n_base3 + (int)blk * 8 + oct;
    row = slot_row<kS>(g, slot);
    code = __float_as_int(row.x);
    ++child_reads;
  }
  c.slot = slot;
  c.kx = slot_ext<kS>(g, row, slot, bin_ext<kS>(kext, k.bin), kb);
  c.sz = __int_as_float((127 - lev) << 23);
  c.J[0] = K0;
  c.J[1] = K1;
  c.J[2] = K2;
  return kCrossed;
}

constexpr float kInv4Pi = 0.0795774715459476679f;  // 1 / (4 pi)

// Henyey-Greenstein phase function per steradian at cos(angle) = mu.
__device__ __forceinline__ float hg_per_sr(float g, float mu) {
  const float den = fmaxf(1.f + g * g - 2.f * g * mu, 1e-30f);
  return (1.f - g * g) * kInv4Pi / (den * sqrtf(den));
}

// Interaction part 1: draw the event's numbers; scatter completely, or pick the
// absorbing species. Returns the species (>= 0) for an absorption, -1 for a scatter.
// peel_o / peel_w (peel-off): for a scattering, *peel_w receives the phase function
// per steradian toward the unit vector peel_o, at the direction before the turn.
// kS: the species count when fixed at compile time (2: the densities come from the
// cell's face-link record, which the linked walk has just read; -2 or -4: from the
// slot row, which the path walk has just read), 0 when read from the grid. `row` is
// the leaf id, or for the path walk (kS < 0) the leaf's tree slot.
template <int kS>
__device__ __forceinline__ float cell_rho(const DevGrid& g, int row, int s) {
  if (kS == 2) return __int_as_float(__ldg(g.links + (size_t)row * kRec + 6 + s));
  if (kS < 0) return __ldg(&g.rho_slot[(size_t)row * (size_t)(kS < 0 ? -kS : 1) + s]);
  return __ldg(&g.rho[(size_t)row * g.S + s]);
}

template <typename R, int kS = 0>
__device__ __forceinline__ int interact(Pkg<R>& k, const DevGrid& g, const Kappa* kap,
                                        int row, const DevRun& r, uint4& w1,
                                        const float* peel_o = nullptr,
                                        float* peel_w = nullptr) {
  uint4 w0 = draw(r.seed, k.id, k.event, 0u);
  w1 = draw(r.seed, k.id, k.event, 1u);
  const int S = kS > 0 ? kS : (kS < 0 ? -kS : g.S);
  const Kappa* kb = kap + k.bin * S;
  float ksca = 0.f, kext = 0.f, kabs = 0.f;
  for (int s = 0; s < S; ++s) {
    const float rs = cell_rho<kS>(g, row, s);
    ksca += rs * kb[s].ksca;
    kext += rs * kb[s].kext;
    kabs += rs * kb[s].kabs;
  }
  k.touched = true;
  const float xs = unit<float>(w0.y);
  int sp = S - 1;
  if (unit<float>(w0.x) * kext < ksca) {
    const float target = xs * ksca;
    float cum = 0.f;
    for (int s = 0; s < S; ++s) {
      cum += cell_rho<kS>(g, row, s) * kb[s].ksca;
      if (cum > target) { sp = s; break; }
    }
    if (peel_w)
      *peel_w = hg_per_sr(kb[sp].g, (float)k.d[0] * peel_o[0] + (float)k.d[1] * peel_o[1] +
                                        (float)k.d[2] * peel_o[2]);
    R mu = hg_mu<R>((R)kb[sp].g, unit<R>(w0.z));
    turn<R>(k.d, mu, unit<R>(w0.w));
    set_inverse(k);
    k.tau = -log_(unit<R>(w1.x));
    return -1;
  }
  const float target = xs * kabs;
  float cum = 0.f;
  for (int s = 0; s < S; ++s) {
    cum += cell_rho<kS>(g, row, s) * kb[s].kabs;
    if (cum > target) { sp = s; break; }
  }
  isotropic<R>(unit<R>(w0.z), unit<R>(w0.w), k.d);
  set_inverse(k);
  k.tau = -log_(unit<R>(w1.x));
  return sp;
}

// Interaction part 2 (absorption): n is this package's place in the cell's
// absorption count (the count before it); draw the new bin.
template <typename R, int kS = 0>
__device__ __forceinline__ void reemit(Pkg<R>& k, const DevGrid& g, const DevTables& t,
                                       const DevRun& r, int s, int leaf, int row, int level,
                                       unsigned long long n, const uint4& w1,
                                       Tally& tl) {
  float xu = unit<float>(w1.y), xb = unit<float>(w1.z);
  float rho = cell_rho<kS>(g, row, s);
  float u;
  if (r.mode == 0) {
    float e = r.count_scale * t.eps_d0_over_V[level] / rho;
    u = ((float)n + xu) * e;
  } else if (r.mode == 1) {
    float e = r.count_scale * t.eps_d0_over_V[level] / rho;
    u = xu * fmaxf((float)n * e, t.u_tmin[s]);
  } else {
    u = xu * __ldg(&t.u_frozen[(size_t)s * g.n_leaves + leaf]);
  }
  const float* S = t.S32 + (size_t)s * g.n_T;
  int nI = g.n_T - 1;
  int i;
  if (u >= __ldg(&S[nI])) {
    i = nI - 1;
    ++tl.clamped;
  } else {
    // interval i with S[i] <= u < S[i+1]: start from the guide, finish by scanning
    float kf = (__logf(fmaxf(u, 1e-30f)) - t.u_ln0[s]) * t.u_inv[s];
    int kk = (int)fminf(fmaxf(kf, 0.0f), (float)nI);
    i = __ldg(&t.u_guide[s * g.n_T + kk]);
    while (i > 0 && __ldg(&S[i]) > u) --i;
    while (i + 1 < nI && __ldg(&S[i + 1]) <= u) ++i;
  }
  // first bin whose cumulative value exceeds xb: guide start, then scan
  const size_t cdf_row = ((size_t)s * nI + i) * g.B;
  const float* cdf = t.dcdf + cdf_row;
  int b = __ldg(&t.cdf_guide[cdf_row + min((int)(xb * (float)g.B), g.B - 1)]);
  while (b > 0 && __ldg(&cdf[b - 1]) > xb) --b;
  while (__ldg(&cdf[b]) <= xb) ++b;
  k.bin = b;
}

// New bin after an absorption by PAH number p: drawn from the PAH's emission
// spectrum in this cell (its template unless a per-cell spectrum is set).
template <typename R>
__device__ __forceinline__ void pah_bin(Pkg<R>& k, const DevGrid& g, const DevTables& t, int p,
                                        int leaf, const uint4& w1) {
  const float xb = unit<float>(w1.z);
  const float* cdf = t.pah_cdf + (size_t)p * g.B;
  if (t.pah_cell_cdf) {
    const float* cc = t.pah_cell_cdf + ((size_t)p * g.n_leaves + leaf) * g.B;
    if (__ldg(&cc[g.B - 1]) > 0.f) cdf = cc;
  }
  int lo = 0, hi = g.B - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(&cdf[mid]) > xb) hi = mid; else lo = mid + 1;
  }
  k.bin = lo;
}

// Absorption by a PAH species: tally the photon in the cell's coarse absorbed
// spectrum and mark the cell as PAH-active for that PAH, then draw the new bin.
template <typename R>
__device__ __forceinline__ void pah_absorb(Pkg<R>& k, const DevGrid& g, const DevTables& t,
                                           const DevRun& r, int p, int leaf, const uint4& w1) {
  const int kc = (k.bin * t.n_coarse) / g.B;
  atomicAdd(&r.pahabs[((size_t)p * g.n_leaves + leaf) * t.n_coarse + kc], 1u);
  atomicOr(&r.pah_flag[leaf], 1u << p);
  pah_bin(k, g, t, p, leaf, w1);
}

__device__ __forceinline__ int dir_bin(float dz, int n_dir) {
  int b = (int)floorf(0.5f * (dz + 1.0f) * (float)n_dir);
  return min(max(b, 0), n_dir - 1);
}

__device__ __forceinline__ void flush_tally(Tally& tl, unsigned long long* c) {
  const unsigned v[kNumCounters] = {tl.emitted,   tl.escaped, tl.capped,
                                    tl.absorptions, tl.scatters, tl.crossings,
                                    tl.errors,    tl.clamped, tl.levels,
                                    tl.peel_events, tl.peel_crossings};
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) {
    unsigned long long x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&c[i], x);
  }
  tl = Tally{};
}

// ---------------------------------------------------------------- peel-off
// Sight line from the point x (base-cube units) toward the observer at bin `bin`:
// the pixel x projects to and the attenuation exp(-tau) to the boundary. Returns
// false when x falls outside the image, tau passes pe.tau_max, or the walk fails
// (then the tree status bit is set).
__device__ __forceinline__ bool sight_line(const DevGrid& g, const Kappa* kap,
                                           const DevPeel& pe, float x0, float x1, float x2,
                                           int bin, float& att, size_t& pix,
                                           unsigned& crossings, unsigned* status) {
  const float r0 = x0 - pe.centre, r1 = x1 - pe.centre, r2 = x2 - pe.centre;
  const float u = r0 * pe.e1[0] + r1 * pe.e1[1] + r2 * pe.e1[2];
  const float v = r0 * pe.e2[0] + r1 * pe.e2[1] + r2 * pe.e2[2];
  const int px = (int)floorf(u * pe.sx + 0.5f * (float)pe.nx);
  const int py = (int)floorf(v * pe.sy + 0.5f * (float)pe.ny);
  const int plane = __ldg(&pe.plane_of_bin[bin]);
  if (plane < 0 || px < 0 || px >= pe.nx || py < 0 || py >= pe.ny) return false;
  Pkg<float> k;
  k.p[0] = x0;
  k.p[1] = x1;
  k.p[2] = x2;
  k.d[0] = pe.o[0];
  k.d[1] = pe.o[1];
  k.d[2] = pe.o[2];
  set_inverse(k);
  k.bin = bin;
  k.tau = 0.f;
  Cell c;
  unsigned lv = 0;
  float tau = 0.f;
  int I0[3], lev0;
  const int rc = locate<float>(g, k.p, k.d, c.leaf, lev0, I0);
  if (rc == 0) set_corner(c, I0, lev0);
  if (rc < 0) {
    atomicOr(status, kStatusTree);
    return false;
  }
  if (rc == 0) {
    // a straight line crosses at most 3 n 2^L finest cells of the n^3 base grid
    const long long cap = 3ll * ((long long)g.n_base << g.max_level) + 8;
    for (long long i = 0;; ++i) {
      const int a = advance_linked<true>(k, c, g, kap, lv, nullptr, &tau);
      ++crossings;
      if (a == kEscaped) break;
      if (a == kError || i >= cap) {
        atomicOr(status, kStatusTree);
        return false;
      }
      if (tau > pe.tau_max) return false;
    }
  }
  att = expf(-tau);
  pix = ((size_t)plane * pe.ny + py) * pe.nx + px;
  return true;
}

// Point-source emissions: all start at the source, so each bin's emissions of the
// launch are peeled together, then its count is cleared.
__global__ void k_peel_source(DevGrid g, DevTables t, DevRun r, DevPeel pe) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.B) return;
  const unsigned long long n = pe.n_emit[b];
  if (n == 0) return;
  pe.n_emit[b] = 0;
  if (r.source_kind == 1) return;
  float att;
  size_t pix;
  unsigned cr = 0;
  if (sight_line(g, t.kap, pe, r.src[0], r.src[1], r.src[2], b, att, pix, cr, r.status))
    atomicAdd(&pe.image[pix], (double)n * (double)kInv4Pi * (double)att);
  if (cr) atomicAdd(&r.counters[kCPeelCrossings], (unsigned long long)cr);
}

// The events a transport launch recorded: one sight line per thread (grid-stride).
// Events beyond the buffer's capacity were not recorded; their number is added to
// the dropped counter.
__global__ void __launch_bounds__(256) k_peel_trace(DevGrid g, DevTables t, DevRun r,
                                                    const __grid_constant__ DevPeel pe) {
  const unsigned long long n_rec = *pe.n_ev;
  const unsigned long long n = n_rec < pe.capacity ? n_rec : pe.capacity;
  if (blockIdx.x == 0 && threadIdx.x == 0 && n_rec > n)
    atomicAdd(&r.counters[kCPeelDropped], n_rec - n);
  unsigned cr = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float4 e = pe.ev[i];
    const int bin = pe.ev_bin[i];
    float att;
    size_t pix;
    if (sight_line(g, t.kap, pe, e.x, e.y, e.z, bin, att, pix, cr, r.status))
      atomicAdd(&pe.image[pix], (double)(e.w * att));
  }
  unsigned long long x = cr;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  if ((threadIdx.x & 31) == 0 && x) atomicAdd(&r.counters[kCPeelCrossings], x);
}

__global__ void k_image_out(const double* image, long long n, double scale, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = image[i] * scale;
}

// Mean over the rows whose centres lie within half_rows pixels of the image's
// centre line (|py + 1/2 - ny/2| <= half_rows) of plane a minus plane b (b < 0:
// none), times scale; one thread per column.
__global__ void k_image_profile(const double* image, int nx, int ny, int plane_a, int plane_b,
                                int half_rows, double scale, double* out) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= nx) return;
  double sum = 0.0;
  int rows = 0;
  for (int py = 0; py < ny; ++py) {
    if (fabs(py + 0.5 - 0.5 * ny) > (double)half_rows) continue;
    double v = image[((size_t)plane_a * ny + py) * nx + px];
    if (plane_b >= 0) v -= image[((size_t)plane_b * ny + py) * nx + px];
    sum += v;
    ++rows;
  }
  out[px] = rows ? sum * scale / rows : 0.0;
}

// ---------------------------------------------------------------- plain kernel
// One thread per package, tables read from global memory, one global atomic per
// absorption and per escape.
template <typename R>
__global__ void __launch_bounds__(256) k_transport_plain(DevGrid g, DevTables t, DevRun r) {
  Tally tl = {};
  unsigned long long idx = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long t0 = global_ns();
  if (idx < r.n_packages) {
    Pkg<R> k;
    emit<R>(k, r.first_id + idx, r, t.star_cdf, g.B);
    ++tl.emitted;
    unsigned steps = 0;
    for (;;) {
      if ((++steps & 1023u) == 0 && global_ns() - t0 > r.budget_ns) {
        atomicOr(r.status, kStatusTimeout);
        break;
      }
      int leaf, level;
      int a = advance<R>(k, g, t.kap, leaf, level, r.pathabs);
      if (a <= kInteract) tl.levels += level;
      if (a == kCrossed) { ++tl.crossings; continue; }
      if (a == kEscaped) {
        ++tl.escaped;
        int db = dir_bin((float)k.d[2], g.n_dir);
        atomicAdd(&r.sed[(size_t)db * g.B + k.bin], 1ull);
        if (!k.touched) atomicAdd(&r.sed[(size_t)(g.n_dir + db) * g.B + k.bin], 1ull);
        break;
      }
      if (a == kError) {
        ++tl.errors;
        atomicOr(r.status, kStatusTree);
        break;
      }
      if (++k.event > r.max_events) { ++tl.capped; break; }
      uint4 w1;
      int s = interact<R>(k, g, t.kap, leaf, r, w1);
      if (s < 0) { ++tl.scatters; continue; }
      unsigned long long n = atomicAdd(&r.count[(size_t)s * g.n_leaves + leaf], 1ull);
      if (t.pah_of[s] >= 0)
        pah_absorb<R>(k, g, t, r, t.pah_of[s], leaf, w1);
      else
        reemit<R>(k, g, t, r, s, leaf, leaf, level, n, w1, tl);
      ++tl.absorptions;
    }
  }
  flush_tally(tl, r.counters);
}

// ---------------------------------------------------------------- pool loop
// Where a warp's package indices come from: one global counter shared by all warps
// (one model), or a range owned by the warp (one chunk of a batch). take() returns
// the first of nd consecutive indices to every lane of the warp.
struct GlobalIds {
  unsigned long long* next;
  __device__ __forceinline__ unsigned long long take(int nd, int lane, int leader) {
    unsigned long long b = 0;
    if (lane == leader) b = atomicAdd(next, (unsigned long long)nd);
    return __shfl_sync(kFull, b, leader);
  }
};

struct RangeIds {
  unsigned long long pos;
  __device__ __forceinline__ unsigned long long take(int nd, int, int) {
    unsigned long long b = pos;
    pos += (unsigned long long)nd;
    return b;
  }
};

// One warp of the packet pool: each lane owns a package slot; dead lanes are refilled
// with indices below n_end every `refill_period` steps. A lane that reaches its
// interaction point waits; the warp runs the (long, divergent) interaction code only
// once `interaction_batch` lanes wait or no lane is left walking, so both phases run
// with most lanes active. Each package's history is unchanged by this schedule.
// Absorptions of lanes hitting the same (species, cell) in one phase are merged into
// one atomic. `sed` is the escaped-spectrum histogram (shared or global memory).
// kPeel: scatterings and re-emissions at image bins are recorded (position, w,
// bin) in the peel-off event buffer, one slot range per warp and phase; point-source
// emissions are counted per bin in s_nemit.
template <bool kPeel, class Ids, int kS = 0, bool kPath = false>
__device__ __forceinline__ void pool_warp(const DevGrid& g, const DevTables& t, const DevRun& r,
                                          const Kappa* kap, const float* star_cdf,
                                          unsigned long long* sed, unsigned long long n_end,
                                          Ids& ids, Tally& tl, unsigned long long t0,
                                          const DevPeel* pe = nullptr,
                                          unsigned long long* s_nemit = nullptr,
                                          const float* kext = nullptr) {
  const int B = g.B;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  Pkg<float> k;
  k.id = 0;
  bool alive = false;
  bool pending = false;  // reached an interaction point, waiting for the batch
  // kPath: the path walk (densities from the density array, kI = -kS for the
  // interaction); otherwise the linked walk
  using CellT = typename std::conditional<kPath, PathCell, Cell>::type;
  constexpr int kI = kPath ? -kS : kS;
  CellT cell{};
  cell.sz = 1.f;
  const int K = r.refill_period > 0 ? r.refill_period : 32;
  const int batch = r.interaction_batch > 0 ? r.interaction_batch : 8;

  for (;;) {
    unsigned dead = __ballot_sync(kFull, !alive);
    if (dead) {
      const int nd = __popc(dead);
      const unsigned long long base = ids.take(nd, lane, __ffs(dead) - 1);
      if (!alive) {
        unsigned long long j = base + __popc(dead & lt_mask);
        if (j < n_end) {
          emit<float>(k, r.first_id + j, r, star_cdf, B);
          ++tl.emitted;
          if constexpr (kPeel) {
            if (r.source_kind != 1) atomicAdd(&s_nemit[k.bin], 1ull);
          }
          int rc;
          if constexpr (kPath)
            rc = enter_path(k, g, cell, tl.levels);
          else
            rc = enter(k, g, cell, tl.levels);
          if (rc == 0) {
            alive = true;
          } else if (rc == 1) {  // source outside the grid, moving away
            ++tl.escaped;
            const int db = dir_bin(k.d[2], g.n_dir);
            atomicAdd(&sed[db * B + k.bin], 1ull);
            atomicAdd(&sed[(g.n_dir + db) * B + k.bin], 1ull);
          } else {
            ++tl.errors;
            atomicOr(r.status, kStatusTree);
          }
        }
      }
    }
    if (!__any_sync(kFull, alive)) break;
    if (__any_sync(kFull, tl.crossings >= kTallyFlushAt || tl.levels >= kTallyFlushAt))
      flush_tally(tl, r.counters);
    bool stop = false;
    if (lane == 0) stop = global_ns() - t0 > r.budget_ns;
    stop = __shfl_sync(kFull, stop, 0);
    if (stop) {
      if (lane == 0) atomicOr(r.status, kStatusTimeout);
      break;
    }
    for (int step = 0; step < K; ++step) {
      // walk phase: lanes not waiting for an interaction cross one cell
      if (alive && !pending) {
        // the two-species form and the path walk run without the path-length tally
        // (launched only then)
        int a;
        if constexpr (kPath)
          a = advance_path<kS>(k, cell, g, kap, kext, tl.levels);
        else
          a = advance_linked<false, kS>(k, cell, g, kap, tl.levels,
                                        kS > 0 ? nullptr : r.pathabs);
        if (a == kCrossed) {
          ++tl.crossings;
        } else if (a == kEscaped) {
          ++tl.crossings;  // the boundary face it left through
          ++tl.escaped;
          int db = dir_bin(k.d[2], g.n_dir);
          atomicAdd(&sed[db * B + k.bin], 1ull);
          if (!k.touched) atomicAdd(&sed[(g.n_dir + db) * B + k.bin], 1ull);
          alive = false;
        } else if (a == kError) {
          ++tl.errors;
          atomicOr(r.status, kStatusTree);
          alive = false;
        } else {
          pending = true;  // at the interaction point inside the cell
        }
      }
      // interaction phase, warp-uniform: once `batch` lanes wait, or nobody walks
      const unsigned pm = __ballot_sync(kFull, pending);
      if (pm == 0u) continue;
      const unsigned walking = __ballot_sync(kFull, alive && !pending);
      if (__popc(pm) < batch && walking != 0u) continue;
      int sp = -1;
      uint4 w1 = make_uint4(0, 0, 0, 0);
      bool absorbing = false;
      bool scattered = false;
      float wv = kInv4Pi;  // peel-off weight per steradian of this lane's event
      int leaf = 0, row = 0;  // the cell's leaf id; its density row (leaf or slot)
      if (pending) {
        pending = false;
        if constexpr (kPath) {
          cell.kx = -1.f;  // the bin may change: read the row again
          leaf = path_leaf(g, cell.slot);
          row = kI < 0 ? cell.slot : leaf;  // slot rows for 2 or 4 species
        } else {
          leaf = cell.leaf;
          row = leaf;
        }
        if (++k.event > r.max_events) {
          ++tl.capped;
          alive = false;
        } else if (leaf < 0) {
          ++tl.errors;
          atomicOr(r.status, kStatusTree);
          alive = false;
        } else {
          sp = interact<float, kI>(k, g, kap, row, r, w1, kPeel ? pe->o : nullptr,
                                   kPeel ? &wv : nullptr);
          if (sp < 0) {
            ++tl.scatters;
            scattered = true;
          } else {
            absorbing = true;
          }
        }
      }
      const unsigned am = __ballot_sync(kFull, absorbing);
      if (absorbing) {
        unsigned long long key = ((unsigned long long)sp << 48) | (unsigned long long)leaf;
        unsigned peers = __match_any_sync(am, key);
        int leader = __ffs(peers) - 1;
        unsigned long long old = 0;
        if (lane == leader)
          old = atomicAdd(&r.count[(size_t)sp * g.n_leaves + leaf],
                          (unsigned long long)__popc(peers));
        old = __shfl_sync(peers, old, leader);
        if (t.pah_of[sp] >= 0)
          pah_absorb<float>(k, g, t, r, t.pah_of[sp], leaf, w1);
        else
          reemit<float, kI>(k, g, t, r, sp, leaf, row, cell.level(), old + __popc(peers & lt_mask),
                            w1, tl);
        ++tl.absorptions;
      }
      if constexpr (kPeel) {
        // the event's share toward the observer, at the bin it leaves with
        const bool ev = (scattered || absorbing) && __ldg(&pe->plane_of_bin[k.bin]) >= 0;
        const unsigned em = __ballot_sync(kFull, ev);
        if (em) {
          const int leader = __ffs(em) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(pe->n_ev, (unsigned long long)__popc(em));
          base = __shfl_sync(kFull, base, leader);
          if (ev) {
            const unsigned long long slot = base + __popc(em & lt_mask);
            if (slot < pe->capacity) {
              pe->ev[slot] = make_float4(k.p[0], k.p[1], k.p[2], wv);
              pe->ev_bin[slot] = k.bin;
            }
            ++tl.peel_events;
          }
        }
      }
    }
  }
}

// Shared-memory words (floats) of the path walk's per-bin extinction vectors: B x kS
// for 2 or 4 species, rounded up to 16 bytes; none otherwise.
template <int kS, bool kPath>
__host__ __device__ constexpr int kext_words(int B) {
  return (kPath && (kS == 2 || kS == 4)) ? (B * kS + 3) / 4 * 4 : 0;
}

// ---------------------------------------------------------------- pool kernel
// Persistent packet pool over one model: all warps draw package indices from one
// global counter; the opacity table, the stellar CDF and (when it fits) the
// escaped-spectrum histogram live in shared memory.
template <int kMinBlocks, bool kPeel, int kS = 0, bool kPath = false>
__global__ void __launch_bounds__(256, kMinBlocks)
    k_transport_pool(DevGrid g, DevTables t, DevRun r, const __grid_constant__ DevPeel pe) {
  extern __shared__ unsigned long long smem_u64[];
  const int S = g.S, B = g.B;
  const int n_sed = 2 * g.n_dir * B;
  const bool sed_local = r.sed_in_smem != 0;
  // the path walk with 2 or 4 species: the extinction opacities [B][S] first, one
  // vector per bin (a multiple of 16 bytes)
  float* s_kext = reinterpret_cast<float*>(smem_u64);
  const int n_kext = kext_words<kS, kPath>(B);
  unsigned long long* s_u64 = smem_u64 + n_kext / 2;
  unsigned long long* s_sed = sed_local ? s_u64 : r.sed;   // [2][n_dir][B]
  Kappa* s_kap = reinterpret_cast<Kappa*>(s_u64 + (sed_local ? n_sed : 0));  // [B][S]
  float* s_cdf = reinterpret_cast<float*>(s_kap + B * S);     // [B]
  if (sed_local)
    for (int i = threadIdx.x; i < n_sed; i += blockDim.x) s_sed[i] = 0ull;
  for (int i = threadIdx.x; i < B * S; i += blockDim.x) s_kap[i] = t.kap[i];
  if (n_kext)
    for (int i = threadIdx.x; i < B * S; i += blockDim.x) s_kext[i] = t.kap[i].kext;
  for (int i = threadIdx.x; i < B; i += blockDim.x) s_cdf[i] = t.star_cdf[i];
  // peel-off: the block's point-source emission counts per bin
  unsigned long long* s_nemit = nullptr;
  if constexpr (kPeel) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(s_cdf + B) + 15) & ~(uintptr_t)15;
    s_nemit = reinterpret_cast<unsigned long long*>(a);
    for (int i = threadIdx.x; i < B; i += blockDim.x) s_nemit[i] = 0ull;
  }
  __syncthreads();
  Tally tl = {};
  GlobalIds ids{r.next};
  pool_warp<kPeel, GlobalIds, kS, kPath>(g, t, r, s_kap, s_cdf, s_sed, r.n_packages, ids, tl,
                                         global_ns(), &pe, s_nemit, s_kext);
  flush_tally(tl, r.counters);
  if (sed_local || kPeel) __syncthreads();
  if (sed_local) {
    for (int i = threadIdx.x; i < n_sed; i += blockDim.x)
      if (s_sed[i]) atomicAdd(&r.sed[i], s_sed[i]);
  }
  if constexpr (kPeel) {
    for (int i = threadIdx.x; i < B; i += blockDim.x)
      if (s_nemit[i]) atomicAdd(&pe.n_emit[i], s_nemit[i]);
  }
}

// ---------------------------------------------------------------- batch kernel
// Many models in one persistent launch: warps take chunks (model, package range)
// from a global queue, stage that model's descriptor in shared memory and run the
// pool loop over the chunk (tables in global memory / L2, spectrum by global
// atomics). Counters are flushed to the chunk's model when the chunk ends.
template <int kS>
__global__ void __launch_bounds__(256) k_transport_batch(const ModelDesc* models,
                                                         const BatchChunk* chunks,
                                                         long long n_chunks,
                                                         unsigned long long* next_chunk) {
  __shared__ ModelDesc sdesc[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(next_chunk, 1ull);
    c = __shfl_sync(kFull, c, 0);
    if ((long long)c >= n_chunks) break;
    const BatchChunk ch = chunks[c];
    const int* src = reinterpret_cast<const int*>(&models[ch.model]);
    int* dst = reinterpret_cast<int*>(&sdesc[warp]);
    for (int i = lane; i < (int)(sizeof(ModelDesc) / sizeof(int)); i += 32) dst[i] = src[i];
    __syncwarp();
    const ModelDesc& md = sdesc[warp];
    Tally tl = {};
    RangeIds ids{ch.first};
    pool_warp<false, RangeIds, kS>(md.g, md.t, md.r, md.t.kap, md.t.star_cdf, md.r.sed,
                                    ch.first + ch.count, ids, tl, t0);
    flush_tally(tl, md.r.counters);
    __syncwarp();
  }
}

// ---------------------------------------------------------------- replay
// Frozen mode only: counts do not steer the path, so each listed package is
// followed alone and its history recorded.
// ev (optional): the package's events, at most ev_cap of them at ev + i ev_cap;
// ev_n[i] receives how many the history has.
__device__ __forceinline__ void trace_event(TraceEvent* ev, long long cap, long long& n,
                                            int kind, int species, int leaf, int bin,
                                            const float p[3]) {
  if (ev && n < cap) {
    TraceEvent e;
    e.kind = kind;
    e.species = species;
    e.leaf = leaf;
    e.bin = bin;
    e.pos[0] = p[0];
    e.pos[1] = p[1];
    e.pos[2] = p[2];
    e.pad = 0;
    ev[n] = e;
  }
  ++n;
}

__global__ void k_trace(DevGrid g, DevTables t, DevRun r, const unsigned long long* ids,
                        long long n, long long* out, TraceEvent* ev, long long ev_cap,
                        long long* ev_n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  TraceEvent* my_ev = ev ? ev + i * ev_cap : nullptr;
  long long n_ev = 0;
  Tally tl = {};
  Pkg<float> k;
  emit<float>(k, ids[i], r, t.star_cdf, g.B);
  trace_event(my_ev, ev_cap, n_ev, 0, -1, -1, k.bin, k.p);
  long long rec[9] = {0, 0, 0, 0, 0, 0, 0, 0, -1};
  const unsigned long long t0 = global_ns();
  unsigned steps = 0;
  Cell c{0, {0.f, 0.f, 0.f}, 1.f};
  int rc = enter(k, g, c, tl.levels);
  if (rc == 1) rec[4] = 1;
  if (rc < 0) atomicOr(r.status, kStatusTree);
  while (rc == 0) {
    if ((++steps & 1023u) == 0 && global_ns() - t0 > r.budget_ns) {
      atomicOr(r.status, kStatusTimeout);
      break;
    }
    const int lf = c.leaf;
    const int a = advance_linked(k, c, g, t.kap, tl.levels, nullptr);
    rec[8] = lf;
    if (a == kCrossed) { ++rec[3]; continue; }
    if (a == kEscaped) {
      ++rec[3];
      rec[4] = 1;
      trace_event(my_ev, ev_cap, n_ev, 3, -1, lf, k.bin, k.p);
      break;
    }
    if (a == kError) { atomicOr(r.status, kStatusTree); break; }
    if (++k.event > r.max_events) {
      rec[5] = 1;
      trace_event(my_ev, ev_cap, n_ev, 4, -1, c.leaf, k.bin, k.p);
      break;
    }
    uint4 w1;
    const float pi[3] = {k.p[0], k.p[1], k.p[2]};
    int s = interact<float>(k, g, t.kap, c.leaf, r, w1);
    if (s < 0) {
      ++rec[2];
      trace_event(my_ev, ev_cap, n_ev, 1, -1, c.leaf, k.bin, pi);
      continue;
    }
    if (t.pah_of[s] >= 0) {
      pah_bin(k, g, t, t.pah_of[s], c.leaf, w1);  // replay does not tally
    } else {
      reemit<float>(k, g, t, r, s, c.leaf, c.leaf, c.level(), 0ull, w1, tl);
    }
    trace_event(my_ev, ev_cap, n_ev, 2, s, c.leaf, k.bin, pi);
    ++rec[1];
  }
  if (ev_n) ev_n[i] = n_ev;
  rec[0] = k.event;
  rec[6] = k.bin;
  rec[7] = dir_bin(k.d[2], g.n_dir);
  for (int j = 0; j < 9; ++j) out[i * 9 + j] = rec[j];
}

// Rows by tree slot (the path walk's grid): slot i < n^3 is base cell i, slot
// n^3 + 8 b + o the child o of block b. A leaf's row holds its densities (a -0 made
// +0: the densities are non-negative); a refined slot's row holds the code -(block +
// 1) of its block in the first word, zeros after it.
__global__ void k_build_rho_slot(DevGrid g, long long n_slots, float* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_slots) return;
  const long long nb = g.n_base3;
  const int node = i < nb ? g.base[i] : g.child[i - nb];
  const bool leaf = node >= 0 && node < g.n_leaves;
  for (int s = 0; s < g.S; ++s)
    out[i * g.S + s] = leaf ? fabsf(g.rho[(long long)node * g.S + s])
                            : (s == 0 && node < 0 ? __int_as_float(node) : 0.f);
}

// Face links: for each leaf and face, the neighbour across it at the leaf's level
// (descending from the base cube with integer coordinates).
__global__ void k_build_links(DevGrid g, const int32_t* ijk, int32_t* links) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.n_leaves * 6) return;
  const long long leaf = idx / 6;
  const int f = (int)(idx % 6), a = f >> 1;
  const int lev = g.level[leaf];
  int J[3] = {ijk[leaf * 3], ijk[leaf * 3 + 1], ijk[leaf * 3 + 2]};
  J[a] += (f & 1) ? 1 : -1;
  const long long nl = (long long)g.n_base << lev;
  int32_t link;
  if (J[a] < 0 || J[a] >= nl) {
    link = kLinkEscape;
  } else {
    const int n = g.n_base;
    int node = g.base[(J[0] >> lev) + n * ((J[1] >> lev) + n * (J[2] >> lev))];
    int l = 0;
    while (node < 0 && l < lev) {
      const long long blk = -(long long)node - 1;
      ++l;
      const int sh = lev - l;
      const int oct = ((J[0] >> sh) & 1) | (((J[1] >> sh) & 1) << 1) | (((J[2] >> sh) & 1) << 2);
      node = g.child[blk * 8 + oct];
    }
    link = node >= 0 ? (node | (l << 28)) : node;
  }
  int32_t* rec = links + leaf * kRec;
  rec[f] = link;
  if (f == 0) {
    rec[6] = g.S >= 1 && g.S <= 2 ? __float_as_int(g.rho[leaf * g.S]) : 0;
    rec[7] = g.S == 2 ? __float_as_int(g.rho[leaf * g.S + 1]) : 0;
  }
}

__global__ void k_philox(const unsigned long long* ids, long long n, unsigned event,
                         unsigned block, unsigned long long seed, unsigned* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 w = draw(seed, ids[i], event, block);
  out[4 * i] = w.x;
  out[4 * i + 1] = w.y;
  out[4 * i + 2] = w.z;
  out[4 * i + 3] = w.w;
}

}  // namespace

constexpr size_t kSmemBudget = 200 * 1024;

static size_t table_smem(const DevGrid& g) {
  return sizeof(Kappa) * g.B * g.S + sizeof(float) * g.B;
}

static size_t sed_smem(const DevGrid& g) {
  return sizeof(unsigned long long) * 2 * g.n_dir * g.B;
}

static size_t peel_smem(const DevGrid& g) { return 16 + sizeof(unsigned long long) * g.B; }

template <int kMinBlocks, bool kPeel, int kS = 0, bool kPath = false>
static cudaError_t launch_pool_variant(const DevGrid& g, const DevTables& t, const DevRun& r,
                                       const DevPeel& pe, int blocks_per_sm, int threads,
                                       int sms, cudaStream_t s) {
  DevRun rr = r;
  const size_t extra = (kPeel ? peel_smem(g) : 0) + sizeof(float) * kext_words<kS, kPath>(g.B);
  rr.sed_in_smem = table_smem(g) + extra + sed_smem(g) <= kSmemBudget ? 1 : 0;
  size_t sm = table_smem(g) + extra + (rr.sed_in_smem ? sed_smem(g) : 0);
  cudaError_t e;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(k_transport_pool<kMinBlocks, kPeel, kS, kPath>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ,
                                                    k_transport_pool<kMinBlocks, kPeel, kS, kPath>,
                                                    threads, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  int bps = blocks_per_sm > 0 ? (blocks_per_sm < occ ? blocks_per_sm : occ) : occ;
  k_transport_pool<kMinBlocks, kPeel, kS, kPath><<<sms * bps, threads, sm, s>>>(g, t, rr, pe);
  return cudaGetLastError();
}

// blocks_per_sm selects the register budget: 5 or 6 resident blocks of 256 threads
// use variants compiled for that occupancy (fewer registers, more spills); other
// values use the 4-block variants, capped at their occupancy: the two-species one
// (no spills; used when the path-length tally is off) or the generic one (8 bytes
// of spills). With peel-off images the 4-block variants are used.
cudaError_t launch_transport_pool(const DevGrid& g, const DevTables& t, const DevRun& r,
                                  int blocks_per_sm, int threads, cudaStream_t s,
                                  const DevPeel* peel, bool path) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (peel && g.S == 2 && !r.pathabs)
    return launch_pool_variant<4, true, 2>(g, t, r, *peel, blocks_per_sm, threads, sms, s);
  if (peel) return launch_pool_variant<4, true>(g, t, r, *peel, blocks_per_sm, threads, sms, s);
  const DevPeel none{};
  // the path walk (no face links; grids of at most kPathLevels levels)
  if (path && !r.pathabs && g.max_level <= kPathLevels) {
    if (g.S == 4)
      return launch_pool_variant<4, false, 4, true>(g, t, r, none, blocks_per_sm, threads, sms, s);
    if (g.S == 2)
      return launch_pool_variant<4, false, 2, true>(g, t, r, none, blocks_per_sm, threads, sms, s);
    return launch_pool_variant<4, false, 0, true>(g, t, r, none, blocks_per_sm, threads, sms, s);
  }
  if (threads == 256 && blocks_per_sm == 6)
    return launch_pool_variant<6, false>(g, t, r, none, blocks_per_sm, threads, sms, s);
  if (threads == 256 && blocks_per_sm == 5)
    return launch_pool_variant<5, false>(g, t, r, none, blocks_per_sm, threads, sms, s);
  // two species: a walk compiled for the densities in the face-link record (a
  // variant for four species reading them as one 16-byte load measured 4 % slower)
  if (g.S == 2 && !r.pathabs)
    return launch_pool_variant<4, false, 2>(g, t, r, none, blocks_per_sm, threads, sms, s);
  return launch_pool_variant<4, false>(g, t, r, none, blocks_per_sm, threads, sms, s);
}

cudaError_t launch_peel_source(const DevGrid& g, const DevTables& t, const DevRun& r,
                               const DevPeel& peel, cudaStream_t s) {
  k_peel_source<<<(g.B + 127) / 128, 128, 0, s>>>(g, t, r, peel);
  return cudaGetLastError();
}

cudaError_t launch_peel_trace(const DevGrid& g, const DevTables& t, const DevRun& r,
                              const DevPeel& peel, cudaStream_t s) {
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peel_trace, 256, 0);
  if (e != cudaSuccess) return e;
  k_peel_trace<<<sms * (occ > 0 ? occ : 1), 256, 0, s>>>(g, t, r, peel);
  return cudaGetLastError();
}

cudaError_t launch_image_out(const double* image, long long n, double scale, double* out,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_image_out<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(image, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_image_profile(const double* image, int nx, int ny, int plane_a,
                                 int plane_b, int half_rows, double scale, double* out,
                                 cudaStream_t s) {
  k_image_profile<<<(nx + 127) / 128, 128, 0, s>>>(image, nx, ny, plane_a, plane_b, half_rows,
                                                    scale, out);
  return cudaGetLastError();
}

cudaError_t launch_transport_plain(const DevGrid& g, const DevTables& t, const DevRun& r,
                                   bool fp64, int threads, cudaStream_t s) {
  unsigned long long nb = (r.n_packages + threads - 1) / threads;
  if (nb == 0) return cudaSuccess;
  if (nb > 0x7fffffffull) return cudaErrorInvalidValue;
  if (fp64)
    k_transport_plain<double><<<(unsigned)nb, threads, 0, s>>>(g, t, r);
  else
    k_transport_plain<float><<<(unsigned)nb, threads, 0, s>>>(g, t, r);
  return cudaGetLastError();
}

template <int kS>
static cudaError_t launch_batch_variant(const ModelDesc* models, const BatchChunk* chunks,
                                        long long n_chunks, unsigned long long* next_chunk,
                                        int blocks_per_sm, int threads, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_transport_batch<kS>, threads, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  int bps = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
  k_transport_batch<kS><<<sms * bps, threads, 0, s>>>(models, chunks, n_chunks, next_chunk);
  return cudaGetLastError();
}

cudaError_t launch_transport_batch(const ModelDesc* models, const BatchChunk* chunks,
                                   long long n_chunks, unsigned long long* next_chunk,
                                   int blocks_per_sm, int s_fixed, int threads,
                                   cudaStream_t s) {
  if (threads <= 0) threads = 256;
  if (threads % 32 != 0 || threads > 256) return cudaErrorInvalidValue;
  if (s_fixed == 2)
    return launch_batch_variant<2>(models, chunks, n_chunks, next_chunk, blocks_per_sm,
                                   threads, s);
  return launch_batch_variant<0>(models, chunks, n_chunks, next_chunk, blocks_per_sm, threads,
                                 s);
}

cudaError_t launch_trace(const DevGrid& g, const DevTables& t, const DevRun& r,
                         const unsigned long long* ids, long long n, long long* out,
                         cudaStream_t s, TraceEvent* ev, long long ev_cap, long long* ev_n) {
  if (n <= 0) return cudaSuccess;
  k_trace<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, t, r, ids, n, out, ev, ev_cap,
                                                      ev_n);
  return cudaGetLastError();
}

cudaError_t launch_build_links(const DevGrid& g, const int32_t* leaf_ijk, int32_t* links,
                               cudaStream_t s) {
  long long n = g.n_leaves * 6;
  k_build_links<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, leaf_ijk, links);
  return cudaGetLastError();
}

cudaError_t launch_build_rho_slot(const DevGrid& g, float* rho_slot, cudaStream_t s) {
  const long long n = (long long)g.n_base3 + 8 * g.n_blocks;
  k_build_rho_slot<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, n, rho_slot);
  return cudaGetLastError();
}

cudaError_t launch_philox(const unsigned long long* ids, long long n, unsigned event,
                          unsigned block, unsigned long long seed, unsigned* out,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_philox<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(ids, n, event, block, seed, out);
  return cudaGetLastError();
}

}  // namespace rt
