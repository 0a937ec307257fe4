// Particle kernels: the cell list (counting sort of particles into lattice-cell
// bins) and the coupled particle kernel, which for each particle
//   - interpolates the post-stream moments rho, j of the fluid with the per-axis
//     delta weights (Eq. 4 of the paper, the interpolant being the same kernel
//     as the spreading, Eqs. 10-11),
//   - sums the linear spring-dashpot contact forces over the 3^d neighbouring
//     bins and the walls,
//   - advances U and X (Eq. 13, with the drag implicit or explicit),
//   - forms the force density g = 2 (rho_l U - j_l) of the moving bounce-back
//     (Eqs. 6-7) and spreads A_p g back to the lattice (Eq. 9).
// Particle state is FP64 structure-of-arrays; positions and velocities are
// double-buffered so that every contact reads the state of step n.
#include <limits.h>
#include <math.h>

#include "pibm_internal.cuh"

namespace pibm {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_PER_THREAD;

// ---------------------------------------------------------------------------
// Cell list
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bin_coord(double X, int n) {
  int b = (int)floor(X);
  return b < 0 ? 0 : (b >= n ? n - 1 : b);
}

template <int D>
__device__ __forceinline__ unsigned bin_index(const BinMap& b, int x, int y, int z) {
  using TD = TileDims<D>;
  const int tx = x / TD::TX, ty = y / TD::TY, tz = z / TD::TZ;
  const int lx = x - tx * TD::TX, ly = y - ty * TD::TY, lz = z - tz * TD::TZ;
  return (unsigned)(tx + b.nt[0] * (ty + b.nt[1] * tz)) * (unsigned)TD::TC +
         (unsigned)(lx + TD::TX * (ly + TD::TY * lz));
}

// Bins are lattice cells, numbered tile-major: the cells of one tile form a
// contiguous bin range, so after sorting its particles form one contiguous range.
template <int D>
__global__ void k_bin_key(const double* __restrict__ X, long long np, Geometry g, BinMap bm,
                          const float* __restrict__ radf, unsigned* __restrict__ key,
                          unsigned* __restrict__ rank, unsigned* __restrict__ cnt,
                          float4* __restrict__ xr, int4* __restrict__ cr) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  int b[3] = {0, 0, 0};
  float fr[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double x = X[k * np + p];
    b[k] = bin_coord(x, g.n[k]);
    fr[k] = (float)(x - (double)b[k]);  // position inside its cell, exact to FP32
  }
  xr[p] = make_float4(fr[0], fr[1], fr[2], radf[p]);
  cr[p] = make_int4(b[0], b[1], b[2], (int)p);
  unsigned kk = bin_index<D>(bm, b[0], b[1], b[2]);
  key[p] = kk;
  rank[p] = atomicAdd(&cnt[kk], 1u);
}

// Block-wide exclusive scan of SCAN_CHUNK unsigned values; returns the total.
__device__ unsigned block_scan(unsigned (&v)[SCAN_PER_THREAD], unsigned* sm) {
  unsigned t = 0;
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) {
    unsigned x = v[i];
    v[i] = t;
    t += x;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned incl = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sm[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned w = sm[lane];
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    sm[lane] = wi - w;  // exclusive warp offsets
    if (lane == 31) sm[32] = wi;
  }
  __syncthreads();
  unsigned base = sm[wid] + incl - t;
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) v[i] += base;
  unsigned total = sm[32];
  __syncthreads();
  return total;
}

// Eight consecutive counts per thread; full groups move as two 16-byte vectors
// (the array is 256-byte aligned and every group starts at a multiple of 8).
__device__ __forceinline__ void load8(const unsigned* __restrict__ in, long long base, long long n,
                                      unsigned (&v)[SCAN_PER_THREAD]) {
  if (base + SCAN_PER_THREAD <= n) {
    const uint4 a = *reinterpret_cast<const uint4*>(in + base);
    const uint4 b = *reinterpret_cast<const uint4*>(in + base + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) v[i] = (base + i < n) ? in[base + i] : 0u;
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const unsigned* __restrict__ in,
                                                              long long n,
                                                              unsigned* __restrict__ sums) {
  __shared__ unsigned sm[33];
  long long base = blockIdx.x * (long long)SCAN_CHUNK + threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
  load8(in, base, n, v);
  unsigned total = block_scan(v, sm);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(unsigned* __restrict__ sums, int nb) {
  __shared__ unsigned sm[33];
  long long base = threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) v[i] = (base + i < nb) ? sums[base + i] : 0u;
  block_scan(v, sm);
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i)
    if (base + i < nb) sums[base + i] = v[i];
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(unsigned* __restrict__ data,
                                                            long long n,
                                                            const unsigned* __restrict__ sums) {
  __shared__ unsigned sm[33];
  long long base = blockIdx.x * (long long)SCAN_CHUNK + threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
  load8(data, base, n, v);
  block_scan(v, sm);
  const unsigned off = sums[blockIdx.x];
  if (base + SCAN_PER_THREAD <= n) {
    *reinterpret_cast<uint4*>(data + base) = make_uint4(v[0] + off, v[1] + off, v[2] + off, v[3] + off);
    *reinterpret_cast<uint4*>(data + base + 4) = make_uint4(v[4] + off, v[5] + off, v[6] + off, v[7] + off);
  } else {
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i)
      if (base + i < n) data[base + i] = v[i] + off;
  }
}

// Place each particle at its slot, together with its FP32 in-cell position and
// radius (xs) and its cell and id (cs), which the contact and coupling kernels
// read in slot order.
__global__ void k_bin_scatter(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
                              const unsigned* __restrict__ start, long long np,
                              const float4* __restrict__ xr, const int4* __restrict__ cr,
                              unsigned* __restrict__ perm, float4* __restrict__ xs,
                              int4* __restrict__ cs) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const unsigned sl = start[key[p]] + rank[p];
  perm[sl] = (unsigned)p;
  xs[sl] = xr[p];
  cs[sl] = cr[p];
}

// Deterministic mode: order every bin by particle id so that every sum over a
// bin runs in a fixed order.
__global__ void k_bin_sort(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
                           const unsigned* __restrict__ start, long long np,
                           const float4* __restrict__ xr, const int4* __restrict__ cr,
                           unsigned* __restrict__ perm, float4* __restrict__ xs,
                           int4* __restrict__ cs) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np || rank[p] != 0u) return;
  unsigned b = key[p];
  unsigned lo = start[b], hi = start[b + 1];
  for (unsigned i = lo + 1; i < hi; ++i) {
    unsigned v = perm[i];
    unsigned j = i;
    while (j > lo && perm[j - 1] > v) {
      perm[j] = perm[j - 1];
      --j;
    }
    perm[j] = v;
  }
  for (unsigned i = lo; i < hi; ++i) {
    xs[i] = xr[perm[i]];
    cs[i] = cr[perm[i]];
  }
}

// ---------------------------------------------------------------------------
// Delta weights along one axis (Eqs. 10-11 and the 2-point hat)
// ---------------------------------------------------------------------------
template <int W, typename WT>
struct Taps {
  int first;    // unwrapped index of the first node
  int idx[W];   // wrapped (periodic) or clamped (dropped wall node) index
  WT w[W];
};

__device__ __forceinline__ void sincospi_t(double a, double* s, double* c) { sincospi(a, s, c); }
__device__ __forceinline__ void sincospi_t(float a, float* s, float* c) { sincospif(a, s, c); }

// b = floor(X - 1/2); nodes b..b+1 (W = 2) or b-1..b+2 (W = 4) at distance
// r_t = first + t + 1/2 - X. For the cosine kernel the four values are
// 1/4 (1 + cos th), 1/4 (1 - sin th), 1/4 (1 - cos th), 1/4 (1 + sin th) with
// th = pi r_0 / 2 (cos shifts by a quarter period per node). On a wall axis the
// nodes outside [0, n) are dropped (weight 0) and the kept weights renormalised.
template <int W, typename WT>
__device__ __forceinline__ void axis_taps(double X, int n, int periodic, Taps<W, WT>& t) {
  const int b = (int)floor(X - 0.5);
  t.first = (W == 2) ? b : b - 1;
  const WT r0 = (WT)((double)t.first + 0.5 - X);
  if constexpr (W == 2) {
    t.w[0] = WT(1) + r0;  // 1 - |r0|, r0 in (-1, 0]
    t.w[1] = -r0;         // 1 - |r0 + 1|
  } else {
    WT sn, cs;
    sincospi_t(WT(0.5) * r0, &sn, &cs);
    t.w[0] = WT(0.25) * (WT(1) + cs);
    t.w[1] = WT(0.25) * (WT(1) - sn);
    t.w[2] = WT(0.25) * (WT(1) - cs);
    t.w[3] = WT(0.25) * (WT(1) + sn);
  }
  if (periodic) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = (t.first + i) % n;  // any X (even a non-finite one) maps into [0, n)
      t.idx[i] = k < 0 ? k + n : k;
    }
  } else {
    WT s = WT(0);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = t.first + i;
      bool in = (k >= 0 && k < n);
      // a dropped node keeps the nearest in-domain index: it lies next to the
      // particle, so every field read there is one the step has written
      t.idx[i] = in ? k : (k < 0 ? 0 : n - 1);
      if (!in) t.w[i] = WT(0);
      s += t.w[i];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) t.w[i] /= s;
  }
}

// The same taps from a particle's cell c and FP32 offset f inside it (X = c + f),
// all in FP32 and integer arithmetic: floor(X - 1/2) = c + floor(f - 1/2) and
// r_0 = (first - c) + 1/2 - f.
template <int W>
__device__ __forceinline__ void axis_taps_local(int c, float f, int n, int periodic,
                                                Taps<W, float>& t) {
  const int b = c + (int)floorf(f - 0.5f);
  t.first = (W == 2) ? b : b - 1;
  const float r0 = (float)(t.first - c) + 0.5f - f;
  if constexpr (W == 2) {
    t.w[0] = 1.f + r0;
    t.w[1] = -r0;
  } else {
    float sn, cs;
    sincospif(0.5f * r0, &sn, &cs);
    t.w[0] = 0.25f * (1.f + cs);
    t.w[1] = 0.25f * (1.f - sn);
    t.w[2] = 0.25f * (1.f - cs);
    t.w[3] = 0.25f * (1.f + sn);
  }
  if (periodic) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = (t.first + i) % n;
      t.idx[i] = k < 0 ? k + n : k;
    }
  } else {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = t.first + i;
      bool in = (k >= 0 && k < n);
      t.idx[i] = in ? k : (k < 0 ? 0 : n - 1);
      if (!in) t.w[i] = 0.f;
      s += t.w[i];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) t.w[i] /= s;
  }
}

// 1/d in FP64 from an FP32 seed refined by Newton steps: one step gives about
// 2^-46 relative error, two reach FP64 rounding.
template <int STEPS>
__device__ __forceinline__ double rcp_newton(double d) {
  double r = (double)__frcp_rn((float)d);
  if (!isfinite(r)) return 1.0 / d;
#pragma unroll
  for (int i = 0; i < STEPS; ++i) {
    const double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
  }
  return r;
}

// Bit tests (integer pipe): not finite, and outside [0, n] for a wall axis.
__device__ __forceinline__ bool not_finite_bits(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) ==
         0x7ff0000000000000ull;
}
__device__ __forceinline__ bool outside_bits(double v, double n) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return b > 0x8000000000000000ull ||  // negative and non-zero
         (b < 0x8000000000000000ull && b > (unsigned long long)__double_as_longlong(n));
}

// Wrap a region coordinate onto the lattice: periodic axes wrap, wall axes
// report cells outside [0, n).
__device__ __forceinline__ bool lattice_coord(int& x, int n, int periodic) {
  if (x >= 0 && x < n) return true;
  if (!periodic) return false;
  x %= n;
  if (x < 0) x += n;
  return true;
}

// Post-stream moments at lattice cell (x, y, z), pulled from the stored f*:
// sum of the stored values (rho - S) and the first moment j, in type R.
template <int Q, class St>
__device__ __forceinline__ void pull_moments(const typename St::T* __restrict__ f,
                                             const Geometry& g, int x, int y, int z,
                                             typename St::R& r, typename St::R (&j)[3]) {
  using L = Lattice<Q>;
  using R = typename St::R;
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  R s = R(0), m0 = R(0), m1 = R(0), m2 = R(0);
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    int s0 = x - L::e(a, 0), s1 = y - L::e(a, 1), s2 = z - L::e(a, 2);
    bool bb = false;
    if (L::e(a, 0) != 0) {
      if (s0 < 0) { if (g.periodic[0]) s0 += g.n[0]; else bb = true; }
      else if (s0 >= g.n[0]) { if (g.periodic[0]) s0 -= g.n[0]; else bb = true; }
    }
    if (L::e(a, 1) != 0) {
      if (s1 < 0) { if (g.periodic[1]) s1 += g.n[1]; else bb = true; }
      else if (s1 >= g.n[1]) { if (g.periodic[1]) s1 -= g.n[1]; else bb = true; }
    }
    if (L::e(a, 2) != 0) {
      if (s2 < 0) { if (g.periodic[2]) s2 += g.n[2]; else bb = true; }
      else if (s2 >= g.n[2]) { if (g.periodic[2]) s2 -= g.n[2]; else bb = true; }
    }
    long long src = s0 + (long long)g.n[0] * (s1 + (long long)g.n[1] * s2);
    R v = St::load(bb ? f[opp(a) * g.pitch + c] : f[a * g.pitch + src]);
    s += v;
    if (L::e(a, 0)) m0 += L::e(a, 0) * v;
    if (L::e(a, 1)) m1 += L::e(a, 1) * v;
    if (L::e(a, 2)) m2 += L::e(a, 2) * v;
  }
  r = s;
  j[0] = m0;
  j[1] = m1;
  j[2] = m2;
}

__device__ __forceinline__ double min_image(double s, int n, int periodic) {
  if (periodic) {
    double N = (double)n;
    if (s > 0.5 * N) s -= N;
    if (s < -0.5 * N) s += N;
  }
  return s;
}

struct CoupleArgs {
  Geometry g;
  Physics ph;
  BinMap bm;
  long long np;
  const double* X;   // [d][np], step n
  const double* U;
  double* Xn;        // [d][np], step n + 1
  double* Un;
  const double* rad;
  const double* mass;
  const double* Ap;
  const double* buoy;
  const double* gw;     // wall damping coefficient per particle
  const float* radf;    // radius (FP32)
  const float4* xs;     // [np] FP32 in-cell position and radius of step n, sorted order
  const int4* cs;       // [np] cell (x, y, z) and particle id, sorted order
  float xf_margin;      // bound on the FP32 rounding error of a distance
  double* gout;      // [d][np]
  double* Fcout;     // [d][np]
  const unsigned* perm;
  const unsigned* start;
  const void* f;     // stored populations f*
  const void* mom;   // moment field (k_moments)
  void* F;           // force field
  unsigned* err;
  int spread;        // 1: spread A_p g into F (through the tile's shared-memory copy)
};

// Contact forces (linear spring-dashpot, normal only) on the step-n state, one
// thread per particle in sorted order: the 3^d neighbouring cells through the
// cell list, then the walls. gamma = 2 beta sqrt(m_eff kn) with
// beta = -ln e / sqrt(pi^2 + ln^2 e) fixes the restitution coefficient e.
// Candidates are first screened in FP32 with a margin larger than the FP32
// rounding of the positions (xf_margin), so only pairs that may overlap reach
// the FP64 overlap test; the force itself is FP64.
template <int D>
__global__ void __launch_bounds__(256) k_contacts(CoupleArgs A) {
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (sl >= A.np) return;
  const Geometry& g = A.g;
  const BinMap& bm = A.bm;
  const long long np = A.np;
  const int4 mc = A.cs[sl];
  const unsigned p = (unsigned)mc.w;
  if (p >= (unsigned)np) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
  const float mrg = A.xf_margin;
  const float4 me = A.xs[sl];
  const float xp[3] = {me.x, me.y, me.z};
  const float rpf = me.w;
  const int bc[3] = {mc.x, mc.y, mc.z};
  double Fc[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
  for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
    int cz = bc[2] + oz;
    if (D == 3 && !lattice_coord(cz, g.n[2], g.periodic[2])) continue;
#pragma unroll 1
    for (int oy = -1; oy <= 1; ++oy) {
      int cy = bc[1] + oy;
      if (!lattice_coord(cy, g.n[1], g.periodic[1])) continue;
      // the cells x-1, x, x+1 of this row, as runs of consecutive bins
      unsigned runs[3][2];
      int nrun = 0;
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        int cx = bc[0] + ox;
        if (!lattice_coord(cx, g.n[0], g.periodic[0])) continue;
        const unsigned b = bin_index<D>(bm, cx, cy, cz);
        if (nrun > 0 && runs[nrun - 1][1] == b) {
          runs[nrun - 1][1] = b + 1;
        } else {
          runs[nrun][0] = b;
          runs[nrun][1] = b + 1;
          ++nrun;
        }
      }
#pragma unroll 1
      for (int r = 0; r < nrun; ++r) {
        const unsigned lo = A.start[runs[r][0]], hi = A.start[runs[r][1]];
        if (hi > (unsigned)np || lo > hi) {
          atomicOr(A.err, ERR_INDEX);
          continue;
        }
        for (unsigned s2 = lo; s2 < hi; ++s2) {
          if (s2 == (unsigned)sl) continue;
          const float4 o = A.xs[s2];
          const int4 oc = A.cs[s2];
          const float oq[3] = {o.x, o.y, o.z};
          const int cq[3] = {oc.x, oc.y, oc.z};
          float d2f = 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            // whole cells apart (minimum image on periodic axes) plus the in-cell offsets
            int dc = bc[k] - cq[k];
            if (g.periodic[k]) {
              if (2 * dc > g.n[k]) dc -= g.n[k];
              if (2 * dc < -g.n[k]) dc += g.n[k];
            }
            const float s = (float)dc + (xp[k] - oq[k]);
            d2f += s * s;
          }
          const float reach = rpf + o.w + mrg;
          if (d2f > reach * reach) continue;
          const unsigned q = (unsigned)oc.w;
          // FP64 overlap test and force
          if (q >= (unsigned)np) {
            atomicOr(A.err, ERR_INDEX);
            continue;
          }
          double X[3], s[3], d2 = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            X[k] = A.X[k * np + p];
            s[k] = min_image(X[k] - A.X[k * np + q], g.n[k], g.periodic[k]);
            d2 += s[k] * s[k];
          }
          const double dist = sqrt(d2);
          const double delta = A.rad[p] + A.rad[q] - dist;
          if (!(delta > 0.0) || !(dist > 0.0)) continue;
          const double mi = A.mass[p], mq = A.mass[q];
          const double meff = mi * mq / (mi + mq);
          const double gam = 2.0 * A.ph.beta * sqrt(meff * A.ph.kn);
          const double inv = 1.0 / dist;
          double vn = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) vn += (A.U[k * np + p] - A.U[k * np + q]) * (s[k] * inv);
          const double mag = A.ph.kn * delta - gam * vn;
#pragma unroll
          for (int k = 0; k < D; ++k) Fc[k] += mag * (s[k] * inv);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (g.periodic[k]) continue;
    const float nk = (float)g.n[k];
    const float xabs = (float)bc[k] + xp[k];
    if (xabs < rpf + mrg) {  // near the wall at 0 (normal +e_k)
      const double delta = A.rad[p] - A.X[k * np + p];
      if (delta > 0.0) Fc[k] += A.ph.kn * delta - A.gw[p] * A.U[k * np + p];
    }
    if (xabs > nk - rpf - mrg) {  // near the wall at n (normal -e_k)
      const double delta = A.rad[p] - ((double)g.n[k] - A.X[k * np + p]);
      if (delta > 0.0) Fc[k] -= A.ph.kn * delta + A.gw[p] * A.U[k * np + p];
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) A.Fcout[k * np + p] = Fc[k];
}

// Post-stream moments of every cell of the tiles that hold particles or touch
// a tile that does (the 2-cell delta stencil never reaches further), one CTA per
// tile of TileDims cells: mom[0] = sum of stored values (rho - S), mom[1..d] = j.
// Cells of other tiles are left untouched; no stencil reads them.
template <int Q, class St>
__global__ void __launch_bounds__(256) k_moments(Geometry g, BinMap bm,
                                                 const unsigned* __restrict__ start,
                                                 const typename St::T* __restrict__ f,
                                                 typename St::R* __restrict__ mom) {
  using L = Lattice<Q>;
  using R = typename St::R;
  constexpr int D = L::D;
  using TD = TileDims<D>;
  const int tile = blockIdx.x;
  const int t[3] = {tile % bm.nt[0], (tile / bm.nt[0]) % bm.nt[1], tile / (bm.nt[0] * bm.nt[1])};
  int busy = 0;
  if (threadIdx.x < (D == 3 ? 27 : 9)) {
    const int o[3] = {(int)threadIdx.x % 3 - 1, ((int)threadIdx.x / 3) % 3 - 1,
                      D == 3 ? (int)threadIdx.x / 9 - 1 : 0};
    int nb[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      nb[k] = t[k] + o[k];
      if (nb[k] < 0 || nb[k] >= bm.nt[k]) {
        if (g.periodic[k]) nb[k] = (nb[k] + bm.nt[k]) % bm.nt[k];
        else ok = false;
      }
    }
    if (ok) {
      const unsigned nt = (unsigned)(nb[0] + bm.nt[0] * (nb[1] + bm.nt[1] * nb[2]));
      busy = start[(nt + 1) * (unsigned)TD::TC] != start[nt * (unsigned)TD::TC];
    }
  }
  if (!__syncthreads_or(busy)) return;
  for (int i = threadIdx.x; i < TD::TC; i += blockDim.x) {
    const int x = t[0] * TD::TX + i % TD::TX;
    const int y = t[1] * TD::TY + (i / TD::TX) % TD::TY;
    const int z = t[2] * TD::TZ + i / (TD::TX * TD::TY);
    if (x >= g.n[0] || y >= g.n[1] || z >= g.n[2]) continue;
    R r, j[3];
    pull_moments<Q, St>(f, g, x, y, z, r, j);
    const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
    store_moments<R>(mom, c, r, j);
  }
}

// Particle coupling, one thread per particle in cell-sorted order: interpolate
// rho, j from the moment field with the delta weights (Eq. 4), take the contact
// force (k_contacts), advance U and X (Eq. 13), form g = 2 (rho_l U - j_l)
// (Eqs. 6-7) and spread A_p g w into F (Eq. 9).
// Spreading adds each tap with one vector atomic per cell (FP32) or one atomic
// per component (FP64); the cell-sorted order keeps a warp's taps close together.
template <int Q, int W, class St, typename FT>
__global__ void __launch_bounds__(256) k_couple(CoupleArgs A) {
  using L = Lattice<Q>;
  using R = typename St::R;
  constexpr int D = L::D;
  constexpr int WZ = D == 3 ? W : 1;
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const Geometry& g = A.g;
  const long long np = A.np;
  Taps<W, R> tx, ty, tz;
  FT amp[3] = {FT(0), FT(0), FT(0)};
  bool act = sl < A.np;
  unsigned p = 0;
  int4 mc = make_int4(0, 0, 0, 0);
  float4 mf = make_float4(0.f, 0.f, 0.f, 0.f);
  if (act) {
    mc = A.cs[sl];
    mf = A.xs[sl];
    p = (unsigned)mc.w;
    if (p >= (unsigned)np) {
      atomicOr(A.err, ERR_INDEX);
      act = false;
    }
  }
  if (act) {
    double X[3] = {0.0, 0.0, 0.0}, U[3] = {0.0, 0.0, 0.0}, Fc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) {
      X[k] = A.X[k * np + p];
      U[k] = A.U[k * np + p];
      Fc[k] = A.Fcout[k * np + p];
    }
    const double mi = A.mass[p], Ap = A.Ap[p], bu = A.buoy[p];
    const R* mom = (const R*)A.mom;

    // --- interpolation of rho, j (Eq. 4) ---
    if constexpr (sizeof(R) == 4) {
      axis_taps_local<W>(mc.x, mf.x, g.n[0], g.periodic[0], tx);
      axis_taps_local<W>(mc.y, mf.y, g.n[1], g.periodic[1], ty);
      if constexpr (D == 3) axis_taps_local<W>(mc.z, mf.z, g.n[2], g.periodic[2], tz);
    } else {
      axis_taps<W, R>(X[0], g.n[0], g.periodic[0], tx);
      axis_taps<W, R>(X[1], g.n[1], g.periodic[1], ty);
      if constexpr (D == 3) axis_taps<W, R>(X[2], g.n[2], g.periodic[2], tz);
    }
    R rs = R(0), js[3] = {R(0), R(0), R(0)};
#pragma unroll 1
    for (int iz = 0; iz < WZ; ++iz) {
      R wz = R(1);
      long long zoff = 0;
      if constexpr (D == 3) {
        wz = tz.w[iz];
        zoff = (long long)tz.idx[iz] * g.n[1];
      }
      if (wz == R(0)) continue;
#pragma unroll
      for (int iy = 0; iy < W; ++iy) {
        const R wyz = ty.w[iy] * wz;
        const long long row = (zoff + ty.idx[iy]) * g.n[0];
#pragma unroll
        for (int ix = 0; ix < W; ++ix) {
          const R wt = tx.w[ix] * wyz;
          if (wt == R(0)) continue;
          R m[4];
          if (row + tx.idx[ix] < 0 || row + tx.idx[ix] >= g.ncell) {
            atomicOr(A.err, ERR_INDEX);
            continue;
          }
          load_moments<R>(mom, row + tx.idx[ix], m);
          rs += wt * m[0];
#pragma unroll
          for (int k = 0; k < D; ++k) js[k] += wt * m[k + 1];
        }
      }
    }
    const double rho_l = (double)St::S + (double)rs;
    double j_l[3] = {(double)js[0], (double)js[1], (double)js[2]};

    // --- particle update (Eq. 13) and force density (Eqs. 6-7) ---
    double Un[3], Ub[3], gg[3];
    if (A.ph.implicit_drag) {
      const double inv = rcp_newton<sizeof(R) == 4 ? 1 : 2>(mi + 2.0 * Ap * rho_l);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        Un[k] = (mi * U[k] + 2.0 * Ap * j_l[k] + bu * A.ph.gravity[k] + Fc[k]) * inv;
        Ub[k] = Un[k];
      }
    } else {
      const double invm = 1.0 / mi;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        Un[k] = U[k] + (bu * A.ph.gravity[k] + Fc[k] - Ap * 2.0 * (rho_l * U[k] - j_l[k])) * invm;
        Ub[k] = U[k];
      }
    }
    bool bad = false, esc = false;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      gg[k] = 2.0 * (rho_l * Ub[k] - j_l[k]);
      if constexpr (sizeof(FT) == 4) amp[k] = (float)gg[k] * (float)Ap;
      else amp[k] = (FT)(Ap * gg[k]);
      double xn = X[k] + Un[k];
      if (g.periodic[k]) {
        const double N = (double)g.n[k];
        if (xn < 0.0) xn += N;
        else if (xn >= N) xn -= N;
        if (!(xn >= 0.0 && xn < N)) xn = xn - N * floor(xn / N);  // |U| > N: not physical
        if (!(xn >= 0.0 && xn < N)) xn = 0.0;
      } else if (outside_bits(xn, (double)g.n[k])) {
        esc = true;
      }
      bad |= not_finite_bits(xn) || not_finite_bits(Un[k]);
      A.Xn[k * np + p] = xn;
      A.Un[k * np + p] = Un[k];
      A.gout[k * np + p] = gg[k];
    }
    if (bad) atomicOr(A.err, ERR_PARTICLE_NONFINITE);
    if (esc) atomicOr(A.err, ERR_ESCAPED);
  }

  // --- spreading (Eq. 9) ---
  if (!A.spread || !act) return;
  FT* F = (FT*)A.F;
#pragma unroll 1
  for (int iz = 0; iz < WZ; ++iz) {
    FT wz = FT(1);
    long long zoff = 0;
    if constexpr (D == 3) {
      wz = (FT)tz.w[iz];
      zoff = (long long)tz.idx[iz] * g.n[1];
    }
    if (wz == FT(0)) continue;
#pragma unroll
    for (int iy = 0; iy < W; ++iy) {
      const FT wyz = (FT)ty.w[iy] * wz;
      const long long row = (zoff + ty.idx[iy]) * g.n[0];
#pragma unroll
      for (int ix = 0; ix < W; ++ix) {
        const FT wt = (FT)tx.w[ix] * wyz;
        if (wt == FT(0)) continue;
        FT v[3] = {amp[0] * wt, amp[1] * wt, amp[2] * wt};
        add_force<D, FT>(F, row + tx.idx[ix], v);
      }
    }
  }
}

// Deterministic spreading: every cell gathers, in a fixed order (neighbour cells
// by ascending z, y, x offset; particles by id inside a cell), the A_p g w of
// every particle whose stencil covers it. Writes every cell of F.
template <int D, int W, typename FT>
__global__ void __launch_bounds__(256) k_spread_gather(Geometry g, BinMap bm, long long np,
                                                       const double* __restrict__ X,
                                                       const double* __restrict__ Ap,
                                                       const double* __restrict__ gin,
                                                       const unsigned* __restrict__ perm,
                                                       const unsigned* __restrict__ start,
                                                       FT* __restrict__ F) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.n[0] || y >= g.n[1]) return;
  constexpr int R = (W == 2) ? 1 : 2;
  FT acc[3] = {FT(0), FT(0), FT(0)};
  const int cell[3] = {x, y, z};
#pragma unroll 1
  for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz) {
    int cz = z + oz;
    if (D == 3 && !lattice_coord(cz, g.n[2], g.periodic[2])) continue;
#pragma unroll 1
    for (int oy = -R; oy <= R; ++oy) {
      int cy = y + oy;
      if (!lattice_coord(cy, g.n[1], g.periodic[1])) continue;
#pragma unroll 1
      for (int ox = -R; ox <= R; ++ox) {
        int cx = x + ox;
        if (!lattice_coord(cx, g.n[0], g.periodic[0])) continue;
        const unsigned b = bin_index<D>(bm, cx, cy, cz);
        const unsigned lo = start[b], hi = start[b + 1];
        for (unsigned sl = lo; sl < hi; ++sl) {
          const unsigned p = perm[sl];
          FT wt = FT(1);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            Taps<W, FT> t;
            axis_taps<W, FT>(X[k * np + p], g.n[k], g.periodic[k], t);
            FT wk = FT(0);
#pragma unroll
            for (int i = 0; i < W; ++i)
              if (t.idx[i] == cell[k]) wk += t.w[i];
            wt *= wk;
          }
          if (wt == FT(0)) continue;
          const double a = Ap[p];
#pragma unroll
          for (int k = 0; k < D; ++k) acc[k] += (FT)(a * gin[k * np + p]) * wt;
        }
      }
    }
  }
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  store_force<D, FT>(F, c, acc);
}

__global__ void k_forces(long long np, int d, const double* __restrict__ Ap,
                         const double* __restrict__ gin, const double* __restrict__ Fc,
                         double* __restrict__ f_fpi, double* __restrict__ f_c) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  for (int k = 0; k < d; ++k) {
    if (f_fpi) f_fpi[p * d + k] = -Ap[p] * gin[k * np + p];
    if (f_c) f_c[p * d + k] = Fc[k * np + p];
  }
}

__global__ void k_interleave(long long np, int d, const double* __restrict__ soa,
                             double* __restrict__ aos) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  for (int k = 0; k < d; ++k) aos[p * d + k] = soa[k * np + p];
}


constexpr int PRED_BLOCKS = 256;
constexpr int PRED_THREADS = 256;

__global__ void __launch_bounds__(PRED_THREADS) k_particle_momentum(
    long long np, int d, const double* __restrict__ mass, const double* __restrict__ U,
    double* __restrict__ out) {
  __shared__ double sm[3 * PRED_THREADS];
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long p = blockIdx.x * (long long)PRED_THREADS + threadIdx.x; p < np;
       p += (long long)PRED_BLOCKS * PRED_THREADS)
    for (int k = 0; k < d; ++k) acc[k] += mass[p] * U[k * np + p];
  for (int k = 0; k < 3; ++k) sm[k * PRED_THREADS + threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = PRED_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 3; ++k) sm[k * PRED_THREADS + threadIdx.x] += sm[k * PRED_THREADS + threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) out[k * PRED_BLOCKS + blockIdx.x] = sm[k * PRED_THREADS];
}

__global__ void k_particle_momentum_final(int d, const double* __restrict__ partial,
                                          double* __restrict__ out) {
  // one thread per component, blocks summed in index order
  int k = threadIdx.x;
  if (k >= d) return;
  double s = 0.0;
  for (int b = 0; b < PRED_BLOCKS; ++b) s += partial[k * PRED_BLOCKS + b];
  out[k] = s;
}


// Per-particle constants from the diameter (held in rad on entry) and the
// density ratio (held in buoy on entry): radius, mass (rho_p pi d^2/4 per unit
// depth in 2D, rho_p pi d^3/6 in 3D, rho_f = 1), cross-section A_p = pi d^2/4
// (section 2.2) and the buoyancy-reduced weight factor m (1 - rho_f/rho_p) of
// Eq. (13).
__global__ void k_particle_init(long long np, int d, double kn, double beta,
                                double* __restrict__ rad, double* __restrict__ mass,
                                double* __restrict__ Ap, double* __restrict__ buoy,
                                double* __restrict__ gw, float* __restrict__ radf) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double dia = rad[p], rr = buoy[p];
  const double pi = 3.14159265358979323846;
  const double m = d == 2 ? rr * pi * dia * dia / 4.0 : rr * pi * dia * dia * dia / 6.0;
  rad[p] = 0.5 * dia;
  radf[p] = (float)(0.5 * dia);
  mass[p] = m;
  Ap[p] = pi * dia * dia / 4.0;
  buoy[p] = m * (1.0 - 1.0 / rr);
  gw[p] = 2.0 * beta * sqrt(m * kn);
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_bin(const State& s, cudaStream_t st, int* nk) {
  const Particles& P = s.p;
  if (P.np == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P.bin_cnt, 0, sizeof(unsigned) * (P.nbin + 1), st);
  if (e != cudaSuccess) return e;
  const double* X = P.X[s.cur];
  if (s.geo.d == 2)
    k_bin_key<2><<<blocks_for(P.np, 256), 256, 0, st>>>(X, P.np, s.geo, P.bm, P.radf, P.key,
                                                        P.rank, P.bin_cnt, P.xr, P.cr);
  else
    k_bin_key<3><<<blocks_for(P.np, 256), 256, 0, st>>>(X, P.np, s.geo, P.bm, P.radf, P.key,
                                                        P.rank, P.bin_cnt, P.xr, P.cr);
  const long long n = P.nbin + 1;
  k_scan_reduce<<<P.scan_blocks, SCAN_THREADS, 0, st>>>(P.bin_cnt, n, P.block_sums);
  k_scan_top<<<1, SCAN_THREADS, 0, st>>>(P.block_sums, P.scan_blocks);
  k_scan_down<<<P.scan_blocks, SCAN_THREADS, 0, st>>>(P.bin_cnt, n, P.block_sums);
  k_bin_scatter<<<blocks_for(P.np, 256), 256, 0, st>>>(P.key, P.rank, P.bin_cnt, P.np, P.xr,
                                                       P.cr, P.perm, P.xs, P.cs);
  if (nk) *nk += 5;
  if (s.deterministic) {
    // bins in particle-id order: every sum over a bin then runs in a fixed order
    k_bin_sort<<<blocks_for(P.np, 256), 256, 0, st>>>(P.key, P.rank, P.bin_cnt, P.np, P.xr,
                                                      P.cr, P.perm, P.xs, P.cs);
    if (nk) *nk += 1;
  }
  return cudaGetLastError();
}

namespace {
CoupleArgs couple_args(const State& s) {
  const Particles& P = s.p;
  CoupleArgs A;
  A.g = s.geo;
  A.ph = s.phy;
  A.bm = P.bm;
  A.np = P.np;
  A.X = P.X[s.cur];
  A.U = P.U[s.cur];
  A.Xn = P.X[1 - s.cur];
  A.Un = P.U[1 - s.cur];
  A.rad = P.rad;
  A.mass = P.mass;
  A.Ap = P.Ap;
  A.buoy = P.buoy;
  A.gw = P.gw;
  A.radf = P.radf;
  A.xs = P.xs;
  A.cs = P.cs;
  // in-cell offsets are exact to 2^-24 and whole-cell differences exactly so
  A.xf_margin = 1e-5f;
  A.gout = P.g;
  A.Fcout = P.Fc;
  A.perm = P.perm;
  A.start = P.bin_cnt;
  A.f = s.f[s.cur];
  A.mom = s.mom;
  A.F = s.F;
  A.err = s.err;
  A.spread = s.deterministic ? 0 : 1;
  return A;
}

template <int Q, int W, class St, typename FT>
cudaError_t couple_t(const State& s, cudaStream_t st, int* nk) {
  const Particles& P = s.p;
  constexpr int D = Lattice<Q>::D;
  using T = typename St::T;
  using R = typename St::R;
  CoupleArgs A = couple_args(s);
  const unsigned ntiles = (unsigned)(P.nbin / P.bm.tc);
  k_moments<Q, St><<<ntiles, 256, 0, st>>>(s.geo, P.bm, P.bin_cnt, (const T*)s.f[s.cur],
                                           (R*)s.mom);
  k_couple<Q, W, St, FT><<<blocks_for(P.np, 256), 256, 0, st>>>(A);
  if (nk) *nk += 2;
  if (s.deterministic) {
    const Geometry& g = s.geo;
    int bx = g.n[0] <= 32 ? 32 : (g.n[0] <= 64 ? 64 : 128);
    dim3 blk(bx, 256 / bx, 1);
    dim3 grd((g.n[0] + blk.x - 1) / blk.x, (g.n[1] + blk.y - 1) / blk.y, g.n[2]);
    k_spread_gather<D, W, FT><<<grd, blk, 0, st>>>(g, P.bm, P.np, P.X[s.cur], P.Ap, P.g, P.perm,
                                                   P.bin_cnt, (FT*)s.F);
    if (nk) *nk += 1;
  }
  return cudaGetLastError();
}

template <int Q, class St, typename FT>
cudaError_t couple_w(const State& s, cudaStream_t st, int* nk) {
  return s.phy.width == 2 ? couple_t<Q, 2, St, FT>(s, st, nk) : couple_t<Q, 4, St, FT>(s, st, nk);
}
}  // namespace

cudaError_t launch_contacts(const State& s, cudaStream_t st, int* nk) {
  if (s.p.np == 0) return cudaSuccess;
  CoupleArgs A = couple_args(s);
  if (s.geo.d == 2)
    k_contacts<2><<<blocks_for(s.p.np, 256), 256, 0, st>>>(A);
  else
    k_contacts<3><<<blocks_for(s.p.np, 256), 256, 0, st>>>(A);
  if (nk) *nk += 1;
  return cudaGetLastError();
}

cudaError_t launch_couple(const State& s, cudaStream_t st, int* nk) {
  if (s.p.np == 0) return cudaSuccess;
  const int q = s.geo.q;
  if (s.precision == PIBM_FP64) {
    if (q == 9) return couple_w<9, StoreF64, double>(s, st, nk);
    if (q == 15) return couple_w<15, StoreF64, double>(s, st, nk);
    if (q == 19) return couple_w<19, StoreF64, double>(s, st, nk);
  } else if (s.precision == PIBM_FP32) {
    if (q == 9) return couple_w<9, StoreF32, float>(s, st, nk);
    if (q == 15) return couple_w<15, StoreF32, float>(s, st, nk);
    if (q == 19) return couple_w<19, StoreF32, float>(s, st, nk);
  } else if (s.precision == PIBM_FP16) {
    if (q == 9) return couple_w<9, StoreF16, float>(s, st, nk);
    if (q == 15) return couple_w<15, StoreF16, float>(s, st, nk);
    if (q == 19) return couple_w<19, StoreF16, float>(s, st, nk);
  } else if (s.precision == PIBM_BF16) {
    if (q == 9) return couple_w<9, StoreBF16, float>(s, st, nk);
    if (q == 15) return couple_w<15, StoreBF16, float>(s, st, nk);
    if (q == 19) return couple_w<19, StoreBF16, float>(s, st, nk);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_particle_forces(const State& s, double* f_fpi, double* f_c, cudaStream_t st) {
  if (s.p.np == 0) return cudaSuccess;
  k_forces<<<blocks_for(s.p.np, 256), 256, 0, st>>>(s.p.np, s.geo.d, s.p.Ap, s.p.g, s.p.Fc, f_fpi,
                                                    f_c);
  return cudaGetLastError();
}

cudaError_t launch_interleave(const State& s, const double* soa, double* aos, cudaStream_t st) {
  if (s.p.np == 0) return cudaSuccess;
  k_interleave<<<blocks_for(s.p.np, 256), 256, 0, st>>>(s.p.np, s.geo.d, soa, aos);
  return cudaGetLastError();
}

cudaError_t launch_particle_momentum(const State& s, double* out_dev, cudaStream_t st) {
  // out_dev[0..d) = sum_p m_p U_p; s.red + 3 * PRED_BLOCKS... scratch after the fluid partials
  double* partial = s.red + 4 * 512;
  if (s.p.np == 0) {
    return cudaMemsetAsync(out_dev, 0, sizeof(double) * s.geo.d, st);
  }
  k_particle_momentum<<<PRED_BLOCKS, PRED_THREADS, 0, st>>>(s.p.np, s.geo.d, s.p.mass,
                                                            s.p.U[s.cur], partial);
  k_particle_momentum_final<<<1, 32, 0, st>>>(s.geo.d, partial, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_particle_init(const State& s, cudaStream_t st) {
  if (s.p.np == 0) return cudaSuccess;
  k_particle_init<<<blocks_for(s.p.np, 256), 256, 0, st>>>(s.p.np, s.geo.d, s.phy.kn,
                                                           s.phy.beta, s.p.rad, s.p.mass,
                                                           s.p.Ap, s.p.buoy, s.p.gw, s.p.radf);
  return cudaGetLastError();
}

}  // namespace pibm
