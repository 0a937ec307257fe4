// Device code of the particle phase shared by the single-simulation kernels
// (particles.cu) and the batched persistent kernel (ensemble.cu): the cell list
// (counting sort of particles into lattice-cell bins) with its busy and free tile
// lists, the moment field, the contact forces and the coupled particle update.
// Each kernel is a thin wrapper around a device function that does the work of
// one thread (a particle, a cell) or of one CTA (a block of a scan, a group of
// tiles), so that the persistent kernel runs exactly the same arithmetic.
#pragma once

#include <limits.h>
#include <math.h>

#include <type_traits>

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

// Bins are lattice cells, numbered tile-major: the cells of one tile form a
// contiguous bin range, so after sorting its particles form one contiguous range.
template <int D>
__device__ __forceinline__ void bin_key_at(const double* __restrict__ X, long long np,
                                           const Geometry& g, const BinMap& bm,
                                           const float4* __restrict__ cf,
                                           unsigned* __restrict__ key, unsigned* __restrict__ rank,
                                           unsigned* __restrict__ cnt, float4* __restrict__ xr,
                                           int4* __restrict__ cr, long long p) {
  if (p >= np) return;
  int b[3] = {0, 0, 0};
  float fr[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double x = X[k * np + p];
    b[k] = bin_coord(x, g.n[k]);
    fr[k] = (float)(x - (double)b[k]);  // position inside its cell, exact to FP32
  }
  xr[p] = make_float4(fr[0], fr[1], fr[2], cf[p].w);
  cr[p] = make_int4(b[0], b[1], b[2], (int)p);  // p: storage position
  unsigned kk = bin_index<D>(bm, b[0], b[1], b[2]);
  key[p] = kk;
  rank[p] = atomicAdd(&cnt[kk], 1u);
}

template <int D>
__global__ void k_bin_key(const double* __restrict__ X, long long np, Geometry g, BinMap bm,
                          const float4* __restrict__ cf, unsigned* __restrict__ key,
                          unsigned* __restrict__ rank, unsigned* __restrict__ cnt,
                          float4* __restrict__ xr, int4* __restrict__ cr) {
  bin_key_at<D>(X, np, g, bm, cf, key, rank, cnt, xr, cr,
                blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Block-wide exclusive scan of NT * SCAN_PER_THREAD unsigned values (NT threads,
// a multiple of 32); returns the total. sm: 33 words of shared memory.
template <int NT>
__device__ unsigned block_scan(unsigned (&v)[SCAN_PER_THREAD], unsigned* sm) {
  constexpr int NW = NT / 32;
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
    unsigned w = lane < NW ? sm[lane] : 0u;
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
  unsigned total = block_scan<SCAN_THREADS>(v, sm);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(unsigned* __restrict__ sums, int nb) {
  __shared__ unsigned sm[33];
  long long base = threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) v[i] = (base + i < nb) ? sums[base + i] : 0u;
  block_scan<SCAN_THREADS>(v, sm);
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i)
    if (base + i < nb) sums[base + i] = v[i];
}

// Chunk b of the exclusive scan: the chunk's own scan plus the offset off.
template <int NT>
__device__ __forceinline__ void scan_down_chunk(unsigned* __restrict__ data, long long n,
                                                long long b, unsigned off, unsigned* sm) {
  const long long base = b * (long long)(NT * SCAN_PER_THREAD) + threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
  load8(data, base, n, v);
  block_scan<NT>(v, sm);
  if (base + SCAN_PER_THREAD <= n) {
    *reinterpret_cast<uint4*>(data + base) = make_uint4(v[0] + off, v[1] + off, v[2] + off, v[3] + off);
    *reinterpret_cast<uint4*>(data + base + 4) = make_uint4(v[4] + off, v[5] + off, v[6] + off, v[7] + off);
  } else {
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i)
      if (base + i < n) data[base + i] = v[i] + off;
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(unsigned* __restrict__ data,
                                                            long long n,
                                                            const unsigned* __restrict__ sums) {
  __shared__ unsigned sm[33];
  scan_down_chunk<SCAN_THREADS>(data, n, blockIdx.x, sums[blockIdx.x], sm);
}

// The two passes of the same scan for a CTA of NT threads working on chunk b of
// NT * SCAN_PER_THREAD values: the chunk totals, then each chunk scanned with
// the sum of the totals before it (which the CTA adds up itself, so no pass over
// the totals is needed in between).
template <int NT>
__device__ __forceinline__ void scan_reduce_chunk(const unsigned* __restrict__ in, long long n,
                                                  long long b, unsigned* __restrict__ sums,
                                                  unsigned* sm) {
  const long long base = b * (long long)(NT * SCAN_PER_THREAD) + threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
  load8(in, base, n, v);
  const unsigned total = block_scan<NT>(v, sm);
  if (threadIdx.x == 0) sums[b] = total;
}

template <int NT>
__device__ __forceinline__ void scan_down_chunk_self(unsigned* __restrict__ data, long long n,
                                                     long long b,
                                                     const unsigned* __restrict__ sums,
                                                     unsigned* sm) {
  unsigned before = 0;
  for (long long i = threadIdx.x; i < b; i += NT) before += sums[i];
  for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = before;
  __syncthreads();
  unsigned off = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) off += sm[w];
  __syncthreads();
  scan_down_chunk<NT>(data, n, b, off, sm);
}

// Place each particle at its slot, together with its FP32 in-cell position and
// radius (xs) and its cell and id (cs), which the contact and coupling kernels
// read in slot order.
__device__ __forceinline__ void bin_scatter_at(const unsigned* __restrict__ key,
                                               const unsigned* __restrict__ rank,
                                               const unsigned* __restrict__ start, long long np,
                                               const float4* __restrict__ xr,
                                               const int4* __restrict__ cr,
                                               unsigned* __restrict__ perm, float4* __restrict__ xs,
                                               int4* __restrict__ cs, float4* __restrict__ xs0,
                                               long long p) {
  if (p >= np) return;
  const unsigned sl = start[key[p]] + rank[p];
  perm[sl] = (unsigned)p;
  xs[sl] = xr[p];
  cs[sl] = cr[p];
  if (xs0) xs0[sl] = xr[p];  // kept cell list: the offsets at the rebuild
}

__global__ void k_bin_scatter(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
                              const unsigned* __restrict__ start, long long np,
                              const float4* __restrict__ xr, const int4* __restrict__ cr,
                              unsigned* __restrict__ perm, float4* __restrict__ xs,
                              int4* __restrict__ cs, float4* __restrict__ xs0) {
  bin_scatter_at(key, rank, start, np, xr, cr, perm, xs, cs, xs0,
                 blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Deterministic mode: order every bin by storage position so that every sum over a
// bin runs in a fixed order.
__device__ __forceinline__ void bin_sort_at(const unsigned* __restrict__ key,
                                            const unsigned* __restrict__ rank,
                                            const unsigned* __restrict__ start, long long np,
                                            const float4* __restrict__ xr,
                                            const int4* __restrict__ cr,
                                            unsigned* __restrict__ perm, float4* __restrict__ xs,
                                            int4* __restrict__ cs, float4* __restrict__ xs0,
                                            long long p) {
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
    if (xs0) xs0[i] = xr[perm[i]];
  }
}

__global__ void k_bin_sort(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
                           const unsigned* __restrict__ start, long long np,
                           const float4* __restrict__ xr, const int4* __restrict__ cr,
                           unsigned* __restrict__ perm, float4* __restrict__ xs,
                           int4* __restrict__ cs, float4* __restrict__ xs0) {
  bin_sort_at(key, rank, start, np, xr, cr, perm, xs, cs, xs0,
              blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Tile lists. A tile is busy when a particle's cell lies within two cells of it
// (wrapped on periodic axes). Until the next rebuild every particle stays
// within the skin (< 1/2 cell) of its cell, so each cell of its delta stencil
// (at most two cells to either side) and of its Lagrange block lies in a busy
// tile; the moment and force fields of the free tiles are never touched. Along
// an axis the cells within two of a tile lie in it and its two neighbours,
// except on a periodic axis whose last tile is one cell wide: a stencil can
// then cross that tile and wrap into the next one, so the neighbours two tiles
// away along that axis count too.
// Pass 1: the busy flag of every tile and the number of busy tiles per block.
// (one CTA of TILE_BLOCK threads per block vb of tiles)
template <int D>
__device__ __forceinline__ void tile_flags_block(const unsigned* __restrict__ start,
                                                 const BinMap& bm, const Geometry& g,
                                                 long long ntiles, int* __restrict__ flag,
                                                 unsigned* __restrict__ tblk, int vb) {
  const long long t = vb * (long long)TILE_BLOCK + threadIdx.x;
  int busy = 0;
  if (t < ntiles) {
    const int tt[3] = {(int)(t % bm.nt[0]), (int)((t / bm.nt[0]) % bm.nt[1]),
                       (int)(t / ((long long)bm.nt[0] * bm.nt[1]))};
    int span[3], w[3];  // neighbour tiles to either side along each axis
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      span[a] = (a < D && g.periodic[a] && g.n[a] % bm.T[a] == 1) ? 2 : 1;
      w[a] = 2 * span[a] + 1;
    }
    const int count = w[0] * w[1] * (D == 3 ? w[2] : 1);
#pragma unroll 1
    for (int o = 0; o < count; ++o) {
      const int off[3] = {o % w[0] - span[0], (o / w[0]) % w[1] - span[1],
                          D == 3 ? o / (w[0] * w[1]) - span[2] : 0};
      int nb[3];
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        nb[a] = tt[a] + off[a];
        if (nb[a] < 0 || nb[a] >= bm.nt[a]) {
          if (g.periodic[a]) nb[a] = ((nb[a] % bm.nt[a]) + bm.nt[a]) % bm.nt[a];
          else ok = false;
        }
      }
      if (!ok) continue;
      const unsigned long long n =
          (unsigned long long)nb[0] + bm.nt[0] * ((unsigned long long)nb[1] + bm.nt[1] * (unsigned long long)nb[2]);
      if (start[(n + 1) * bm.tc] != start[n * bm.tc]) {
        busy = 1;
        break;
      }
    }
    flag[t] = busy;
  }
  const int cnt = __syncthreads_count(busy);
  if (threadIdx.x == 0) tblk[vb] = (unsigned)cnt;
}

template <int D>
__global__ void __launch_bounds__(TILE_BLOCK) k_tile_flags(const unsigned* __restrict__ start,
                                                           BinMap bm, Geometry g, long long ntiles,
                                                           int* __restrict__ flag,
                                                           unsigned* __restrict__ tblk) {
  tile_flags_block<D>(start, bm, g, ntiles, flag, tblk, blockIdx.x);
}

// Pass 2: each tile's place in the busy or the free list (block prefix of the
// pass-1 counts plus the rank inside the block), and the two list lengths.
__device__ __forceinline__ void tile_lists_block(const int* __restrict__ flag,
                                                 const unsigned* __restrict__ tblk,
                                                 long long ntiles, int* __restrict__ tbusy,
                                                 int* __restrict__ tfree,
                                                 unsigned* __restrict__ tn, int vb) {
  constexpr int NW = TILE_BLOCK / 32;  // warps
  __shared__ unsigned red[32], wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long t = vb * (long long)TILE_BLOCK + threadIdx.x;
  // busy tiles of the blocks before this one, and of all blocks
  unsigned before = 0, all = 0;
  const int nblk = (int)((ntiles + TILE_BLOCK - 1) / TILE_BLOCK);
  for (int b = threadIdx.x; b < nblk; b += TILE_BLOCK) {
    const unsigned c = tblk[b];
    all += c;
    if (b < vb) before += c;
  }
  for (int o = 16; o > 0; o >>= 1) {
    before += __shfl_xor_sync(0xffffffffu, before, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if (lane == 0) {
    red[wid] = before;
    wsum[wid] = all;
  }
  const bool busy = t < ntiles && flag[t] != 0;
  __syncthreads();
  if (wid == 0) {
    unsigned a = lane < NW ? red[lane] : 0u, b = lane < NW ? wsum[lane] : 0u;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      red[0] = a;
      wsum[0] = b;
    }
  }
  __syncthreads();
  const unsigned base = red[0], total = wsum[0];
  // rank among the busy tiles of this block
  const unsigned m = __ballot_sync(0xffffffffu, busy);
  __syncthreads();
  if (lane == 0) red[wid] = __popc(m);
  __syncthreads();
  if (wid == 0) {
    const unsigned v = lane < NW ? red[lane] : 0u;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    red[lane] = incl - v;  // exclusive prefix over warps
  }
  __syncthreads();
  const unsigned rank = base + red[wid] + __popc(m & ((1u << lane) - 1u));
  if (t < ntiles) {
    if (busy) tbusy[rank] = (int)t;
    else tfree[t - rank] = (int)t;
  }
  if (t == 0) {
    tn[0] = total;
    tn[1] = (unsigned)(ntiles - total);
  }
  __syncthreads();  // red and wsum are reused by the next block of the same CTA
}

__global__ void __launch_bounds__(TILE_BLOCK) k_tile_lists(const int* __restrict__ flag,
                                                           const unsigned* __restrict__ tblk,
                                                           long long ntiles, int* __restrict__ tbusy,
                                                           int* __restrict__ tfree,
                                                           unsigned* __restrict__ tn) {
  tile_lists_block(flag, tblk, ntiles, tbusy, tfree, tn, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Delta weights along one axis (Eqs. 10-11 and the 2-point hat)
// ---------------------------------------------------------------------------
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

// The stored values that stream into lattice cell (x, y, z): f*(x - e_a, a), or
// f*(x, opp a) (halfway bounce-back) where x - e_a lies beyond a wall.
template <int Q, class St>
__device__ __forceinline__ void pull_load(const typename St::T* __restrict__ f, const Geometry& g,
                                          int x, int y, int z, typename St::T (&v)[Q]) {
  using L = Lattice<Q>;
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
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
    const long long src = s0 + (long long)g.n[0] * (s1 + (long long)g.n[1] * s2);
    v[a] = bb ? f[opp(a) * g.pitch + c] : f[a * g.pitch + src];
  }
}

// Zeroth and first moments of pulled values: sum of the stored values (rho - S)
// and j, in type R.
template <int Q, class St>
__device__ __forceinline__ void sum_moments(const typename St::T (&v)[Q], typename St::R& r,
                                            typename St::R (&j)[3]) {
  using L = Lattice<Q>;
  using R = typename St::R;
  R s = R(0), m0 = R(0), m1 = R(0), m2 = R(0);
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const R x = St::load(v[a]);
    s += x;
    if (L::e(a, 0)) m0 += L::e(a, 0) * x;
    if (L::e(a, 1)) m1 += L::e(a, 1) * x;
    if (L::e(a, 2)) m2 += L::e(a, 2) * x;
  }
  r = s;
  j[0] = m0;
  j[1] = m1;
  j[2] = m2;
}

struct CoupleArgs {
  Geometry g;
  Physics ph;
  BinMap bm;
  long long np;
  const double* X;   // [d][np], step n, by storage position
  const double* U;
  double* Xn;        // [d][np], step n + 1, by slot (also the sub-step state)
  double* Un;
  // per-particle constants of step n by storage position, and their copies for
  // step n + 1 by slot (written by the coupled kernel)
  const double* rad;
  const double* mass;
  const double* Ap;
  const double* buoy;
  const double* gw;     // wall damping coefficient per particle (linear law)
  const float4* cf;     // FP32 {mass, A_p, buoy, radius}
  const unsigned* pid;  // user index
  double* radn;
  double* massn;
  double* Apn;
  double* buoyn;
  double* gwn;
  float4* cfn;
  unsigned* pidn;
  const float4* xs;     // [np] FP32 in-cell position and radius of step n, sorted order
  const int4* cs;       // [np] cell (x, y, z) and storage position, sorted order
  float4* xsn;          // the same records for step n + 1 when the cell list is kept
  int4* csn;
  int keep_cells;       // 1: the next step keeps the cell list (write xsn, csn; skin check)
  const float4* xs0;    // in-cell offsets at the last rebuild, by slot (kept cell list)
  int nb_mode;          // contact candidates: 0 traverse, 1 traverse and record, 2 use the record
  int move_consts;      // 0: the other buffer already holds the constants in this order
  int nb_max;           // capacity of the candidate record per particle
  unsigned* nb;         // [nb_max][np] candidate slots recorded at the last rebuild
  int* nbn;             // [np] their number, -1 when they did not fit
  float xf_margin;      // bound on the FP32 rounding error of a distance
  double* gout;      // [d][np] by slot
  double* Fcout;     // [d][np] by slot
  float* Fcf;        // [d][np] by slot, FP32 copy of Fcout (32- and 16-bit storage), or null
  double* rl;        // sub-cycling: [np] rho_l by slot
  double* jl;        // sub-cycling: [d][np] j_l by slot
  double* Fs;        // sub-cycling: [d][np] contact force of the sub-step by slot
  int* ti;           // ordered spreading: [np][3][4] spreading tap cells by slot
  double* tw;        // ordered spreading: [np][3][4] spreading tap weights by slot
  const unsigned* perm;
  const unsigned* start;
  long long nbin;    // bins of the cell list (tiles * cells per tile)
  const void* f;     // stored populations f*
  const void* mom;   // moment field (k_moments)
  void* F;           // force field
  unsigned* err;
  int spread;        // 1: spread A_p g into F with atomics (0: ordered gather kernel)
};

// Magnitude of the normal contact force (positive = repulsive) for an overlap
// delta > 0 and normal relative velocity vn (positive = separating), reduced
// mass meff. Linear: k_n delta - gamma vn with gamma = 2 beta sqrt(meff k_n).
// Hertz (Eq. 15): (4/3) E* sqrt(R*) delta^{3/2} - gamma vn with the
// Hertz-Mindlin damping gamma = 2 sqrt(5/6) beta sqrt(S_n meff),
// S_n = 2 E* sqrt(R* delta).
template <bool HZ>
__device__ __forceinline__ double normal_force(const Physics& ph, double delta, double vn,
                                               double meff, double Rs, double Es) {
  if constexpr (HZ) {
    const double sd = sqrt(delta), sR = sqrt(Rs);
    const double gam = ph.hz_damp * sqrt(2.0 * Es * sR * sd * meff);
    return (4.0 / 3.0) * Es * sR * delta * sd - gam * vn;
  }
  const double gam = 2.0 * ph.beta * sqrt(meff * ph.kn);
  return ph.kn * delta - gam * vn;
}

// Contact forces (normal only, linear spring-dashpot or Hertz) on the step-n
// state (SUB = false) or on the sub-step state (SUB = true: positions and
// velocities by slot in Xn, Un), one thread per particle in sorted order,
// written by slot: the 3^d neighbouring cells through the cell list of the step
// start, then the walls. beta = -ln e / sqrt(pi^2 + ln^2 e) fixes the
// restitution coefficient e. Candidates are first screened in FP32 with a
// margin larger than the FP32 rounding of the positions (xf_margin), plus twice
// the largest sub-step displacement, so only pairs that may overlap reach the
// FP64 overlap test; the force itself is FP64. HZ selects the Hertz law. With a
// kept cell list the traversal of a rebuild step records each particle's
// candidates and the following steps take them from the record: the same
// candidates in the same order, so the same sums.
// In 3D the kernel is held to 80 registers (three CTAs of 256 per SM): the
// traversal and the recorded-candidate pass are latency-bound, and the extra
// warps in flight took them from 2.13 to 1.43 ms and from 0.32 to 0.20 ms on the
// 256^3 workload; in 2D the unbounded kernel measured faster.
// HS (half shell; atomic spreading, no sub-cycling): each pair is handled once, by
// the particle whose neighbour cell lies in the forward half of the 3^d block (the
// own cell: the later slot), which adds the equal and opposite force to its partner
// with an FP64 atomic; the contact force array is zeroed before the launch and
// every particle adds its own sum atomically at the end. The forces on the two
// particles of a pair are exact negatives of each other (the separation and the
// relative velocity flip sign exactly), so only the summation order differs from
// the full shell; the recorded candidates are halved too.
template <int D, bool SUB, bool HZ, int NB, bool HS = false>
__device__ __forceinline__ void contacts_at(const CoupleArgs& A, long long sl) {
  static_assert(!(HS && SUB), "the half shell is for the plain step");
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
  // positions and velocities: step n by storage position, or the sub-step state by slot
  auto Xat = [&](int k, unsigned i) { return SUB ? A.Xn[k * np + i] : A.X[k * np + i]; };
  auto Uat = [&](int k, unsigned i) { return SUB ? A.Un[k * np + i] : A.U[k * np + i]; };
  const unsigned me_i = SUB ? (unsigned)sl : p;
  const float mrg = A.xf_margin + (SUB ? 2.f * A.ph.skinf : 0.f);
  const float4 me = A.xs[sl];
  const float xp[3] = {me.x, me.y, me.z};
  const float rpf = me.w;
  const int bc[3] = {mc.x, mc.y, mc.z};
  double Fc[3] = {0.0, 0.0, 0.0};
  // FP32 screen of the candidate at slot s2 (positions of the step start, so the
  // same answer at every sub-step)
  auto screen = [&](unsigned s2, unsigned& q) {
    const float4 o = A.xs[s2];
    const int4 oc = A.cs[s2];
    q = (unsigned)oc.w;
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
    return d2f <= reach * reach;
  };
  // the contact force of the candidate at slot s2
  auto consider = [&](unsigned s2) {
    unsigned q;
    if (!screen(s2, q)) return;
    // FP64 overlap test and force
    if (q >= (unsigned)np) {
      atomicOr(A.err, ERR_INDEX);
      return;
    }
    const unsigned ot_i = SUB ? s2 : q;
    double s[3], d2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      s[k] = min_image(Xat(k, me_i) - Xat(k, ot_i), g.n[k], g.periodic[k]);
      d2 += s[k] * s[k];
    }
    const double dist = sqrt(d2);
    const double rp = A.rad[p], rq = A.rad[q];
    const double delta = rp + rq - dist;
    if (!(delta > 0.0) || !(dist > 0.0)) return;
    const double mp = A.mass[p], mq = A.mass[q];
    const double meff = mp * mq / (mp + mq);
    const double inv = 1.0 / dist;
    double vn = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) vn += (Uat(k, me_i) - Uat(k, ot_i)) * (s[k] * inv);
    const double mag =
        normal_force<HZ>(A.ph, delta, vn, meff, HZ ? rp * rq / (rp + rq) : 0.0, A.ph.Epp);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double f = mag * (s[k] * inv);
      Fc[k] += f;
      if constexpr (HS) atomicAdd(A.Fcout + k * np + s2, -f);
    }
  };
  // At a rebuild, the candidates that can touch before the next one: every
  // particle stays within disp_skin of its rebuild position on each axis, so a
  // pair farther apart than r_i + r_j + 2 disp_skin sqrt(d) never touches.
  auto near_at_rebuild = [&](unsigned s2) {
    const float4 o = A.xs[s2];
    const int4 oc = A.cs[s2];
    const float oq[3] = {o.x, o.y, o.z};
    const int cq[3] = {oc.x, oc.y, oc.z};
    float d2f = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      int dc = bc[k] - cq[k];
      if (g.periodic[k]) {
        if (2 * dc > g.n[k]) dc -= g.n[k];
        if (2 * dc < -g.n[k]) dc += g.n[k];
      }
      const float s = (float)dc + (xp[k] - oq[k]);
      d2f += s * s;
    }
    const float reach = rpf + o.w + 2.f * A.ph.disp_skinf * sqrtf((float)D) + mrg;
    return d2f <= reach * reach;
  };
  // NB: 0 traverse the cells, 1 traverse and record the candidates, 2 take the
  // recorded candidates (traversing when they did not fit). Kept cell list: the
  // record of a rebuild holds the pairs that can touch before the next rebuild.
  // Sub-cycling (SUB): the record of the first sub-step holds the pairs that pass
  // the FP32 screen, whose answer does not change over the step's sub-steps, so
  // every later sub-step sees the same candidates in the same order.
  if (NB == 2 && A.nbn[sl] >= 0) {
    // the candidates the traversal of the last rebuild recorded, in its order
    const int cnt = A.nbn[sl];
    for (int i = 0; i < cnt; ++i) consider(A.nb[(long long)i * np + sl]);
  } else {
    const bool rec = NB == 1;
    int nrec = 0;
#pragma unroll 1
    for (int oz = (D == 3 && !HS ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
      int cz = bc[2] + oz;
      if (D == 3 && !lattice_coord(cz, g.n[2], g.periodic[2])) continue;
#pragma unroll 1
      for (int oy = (HS && oz == 0 ? 0 : -1); oy <= 1; ++oy) {
        int cy = bc[1] + oy;
        if (!lattice_coord(cy, g.n[1], g.periodic[1])) continue;
        // half shell, own row: the own cell (later slots only) and x + 1
        const bool own_row = HS && oz == 0 && oy == 0;
        // the cells x-1, x, x+1 of this row: one run of consecutive bins in the
        // common case, else each in-domain cell on its own
        unsigned b[3];
        bool ok[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          int cx = bc[0] + i - 1;
          ok[i] = !(own_row && i == 0) && lattice_coord(cx, g.n[0], g.periodic[0]);
          b[i] = ok[i] ? bin_index<D>(bm, cx, cy, cz) : 0u;
        }
        const bool one = ok[0] && ok[1] && ok[2] && b[1] == b[0] + 1 && b[2] == b[1] + 1;
#pragma unroll 1
        for (int r = 0; r < (one ? 1 : 3); ++r) {
          const bool okr = one || (r == 0 ? ok[0] : (r == 1 ? ok[1] : ok[2]));
          if (!okr) continue;
          const unsigned br = r == 0 ? b[0] : (r == 1 ? b[1] : b[2]);
          const unsigned lo = A.start[br], hi = A.start[one ? b[2] + 1 : br + 1];
          if (hi > (unsigned)np || lo > hi) {
            atomicOr(A.err, ERR_INDEX);
            continue;
          }
          for (unsigned s2 = lo; s2 < hi; ++s2) {
            if (s2 == (unsigned)sl || (own_row && r == 1 && s2 < (unsigned)sl)) continue;
            unsigned q_;
            if (rec && (SUB ? screen(s2, q_) : near_at_rebuild(s2))) {
              if (nrec < A.nb_max) A.nb[(long long)nrec * np + sl] = s2;
              ++nrec;
            }
            consider(s2);
          }
        }
      }
    }
    if (rec) A.nbn[sl] = nrec <= A.nb_max ? nrec : -1;  // -1: traverse again
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (g.periodic[k]) continue;
    const float nk = (float)g.n[k];
    const float xabs = (float)bc[k] + xp[k];
    // walls are bodies at rest: m_eff = m, R* = R, the wall's E in E*
    if (xabs < rpf + mrg) {  // near the wall at 0 (normal +e_k)
      const double delta = A.rad[p] - Xat(k, me_i);
      if (delta > 0.0) {
        const double vn = Uat(k, me_i);
        Fc[k] += HZ ? normal_force<true>(A.ph, delta, vn, A.mass[p], A.rad[p], A.ph.Epw)
                    : A.ph.kn * delta - A.gw[p] * vn;
      }
    }
    if (xabs > nk - rpf - mrg) {  // near the wall at n (normal -e_k)
      const double delta = A.rad[p] - ((double)g.n[k] - Xat(k, me_i));
      if (delta > 0.0) {
        const double vn = -Uat(k, me_i);
        Fc[k] -= HZ ? normal_force<true>(A.ph, delta, vn, A.mass[p], A.rad[p], A.ph.Epw)
                    : A.ph.kn * delta - A.gw[p] * vn;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if constexpr (HS) atomicAdd(A.Fcout + k * np + sl, Fc[k]);
    else (SUB ? A.Fs : A.Fcout)[k * np + sl] = Fc[k];
  }
  if (!SUB && !HS && A.Fcf) {
    // most particles touch nothing: their zero needs no FP64 conversion (the
    // test is on the bit pattern, so it costs no FP64 operation either)
#pragma unroll
    for (int k = 0; k < D; ++k)
      A.Fcf[k * np + sl] = __double_as_longlong(Fc[k]) != 0 ? (float)Fc[k] : 0.f;
  }
}

// 3D half shell: 64 registers (four CTAs per SM) measured 0.192 ms/step of contacts
// on the 256^3 workload, against 0.233 at 80 and 0.333 at 128.
template <int D, bool SUB, bool HZ, int NB, bool HS = false>
__global__ void __launch_bounds__(256, D == 3 ? (HS ? 4 : 3) : 1) k_contacts(CoupleArgs A) {
  contacts_at<D, SUB, HZ, NB, HS>(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Shape of the moment kernel: cells per thread (as many loads in flight as the
// registers allow) and tiles per CTA of 256 threads.
template <int Q, class St>
struct MomentsShape {
  static constexpr int D = Lattice<Q>::D;
  static constexpr int TC = TileDims<D>::TC;
  static constexpr int CPT = (D == 3 || sizeof(typename St::T) == 8) ? 2 : 4;
  static constexpr int MINB = sizeof(typename St::T) == 8 ? 2 : 4;  // CTAs per SM
  static constexpr int KT = CPT * 256 / TC;
};

// Post-stream moments of every cell of the busy tiles (k_tile_lists), KT tiles
// of TileDims cells per CTA: mom[0] = sum of stored values (rho - S),
// mom[1..d] = j. Each thread issues the loads of all its cells before it sums
// any of them. A cell whose neighbours all lie inside the lattice (no wall, no
// wrap) reads its sources at fixed 32-bit offsets; only cells on the lattice
// faces take the general path. Cells of free tiles are left untouched; no
// stencil reads them.
// (one CTA of 256 threads per group vb of KT busy tiles)
template <int Q, class St>
__device__ __forceinline__ void moments_block(const Geometry& g, const BinMap& bm,
                                              const int* __restrict__ tbusy,
                                              const unsigned* __restrict__ tn,
                                              const typename St::T* __restrict__ f,
                                              typename St::R* __restrict__ mom, int vb) {
  using Sh = MomentsShape<Q, St>;
  using L = Lattice<Q>;
  using T = typename St::T;
  using R = typename St::R;
  constexpr int D = Sh::D;
  using TD = TileDims<D>;
  __shared__ int busy[Sh::KT];
  __shared__ int corner[Sh::KT][3];  // first cell of each tile
  const int nbusy = (int)tn[0];
  const int i0 = vb * Sh::KT;
  if (i0 >= nbusy) return;  // the list is shorter than the grid
  __syncthreads();  // busy and corner may still be read for the CTA's previous group
  if (threadIdx.x < Sh::KT) {
    const int i = i0 + threadIdx.x;
    const int tile = i < nbusy ? tbusy[i] : 0;
    const int r = tile / bm.nt[0];
    busy[threadIdx.x] = i < nbusy;
    corner[threadIdx.x][0] = (tile - r * bm.nt[0]) * TD::TX;
    corner[threadIdx.x][1] = (r % bm.nt[1]) * TD::TY;
    corner[threadIdx.x][2] = (r / bm.nt[1]) * TD::TZ;
  }
  __syncthreads();
  const int n0 = g.n[0], n01 = g.n[0] * g.n[1];
  T v[Sh::CPT][Q];
  int cell[Sh::CPT];
  bool on[Sh::CPT];
#pragma unroll
  for (int c = 0; c < Sh::CPT; ++c) {
    const int lin = c * 256 + (int)threadIdx.x;
    const int k = lin / TD::TC, i = lin % TD::TC;
    const int x = corner[k][0] + i % TD::TX;
    const int y = corner[k][1] + (i / TD::TX) % TD::TY;
    const int z = corner[k][2] + i / (TD::TX * TD::TY);
    on[c] = busy[k] && x < g.n[0] && y < g.n[1] && z < g.n[2];
    cell[c] = x + n0 * y + n01 * z;
    if (!on[c]) continue;
    const bool inner = x >= 1 && x <= g.n[0] - 2 && y >= 1 && y <= g.n[1] - 2 &&
                       (D == 2 || (z >= 1 && z <= g.n[2] - 2));
    if (inner) {
      const T* fa = f;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        v[c][a] = fa[cell[c] - (L::e(a, 0) + n0 * L::e(a, 1) + n01 * L::e(a, 2))];
        fa += g.pitch;
      }
    } else {
      pull_load<Q, St>(f, g, x, y, z, v[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < Sh::CPT; ++c) {
    if (!on[c]) continue;
    R r, j[3];
    sum_moments<Q, St>(v[c], r, j);
    store_moments<R>(mom, cell[c], r, j);
  }
}

template <int Q, class St>
__global__ void __launch_bounds__(256, MomentsShape<Q, St>::MINB) k_moments(Geometry g, BinMap bm,
                                                 const int* __restrict__ tbusy,
                                                 const unsigned* __restrict__ tn,
                                                 const typename St::T* __restrict__ f,
                                                 typename St::R* __restrict__ mom) {
  moments_block<Q, St>(g, bm, tbusy, tn, f, mom, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Interpolation (Eq. 4 with the spreading kernel, or Eq. 5) and spreading
// (Eq. 9) of one particle
// ---------------------------------------------------------------------------
// Cubic Lagrange basis on the nodes 0, 1, 2, 3 at coordinate t (Eq. 5 with
// unit node spacing): w_i = prod_{l != i} (t - l) / (i - l).
template <typename WT>
__device__ __forceinline__ void lagrange_weights(WT t, WT (&w)[4]) {
  const WT t1 = t - WT(1), t2 = t - WT(2), t3 = t - WT(3);
  const WT sixth = WT(1) / WT(6);
  w[0] = -(t1 * t2 * t3) * sixth;
  w[1] = WT(0.5) * (t * t2 * t3);
  w[2] = -WT(0.5) * (t * t1 * t3);
  w[3] = (t * t1 * t2) * sixth;
}

// The 4-node block of Eq. (5) along one axis: first = floor(X - 1/2) - 1,
// shifted into [0, n - 4] on a wall axis (one-sided next to the wall), wrapped
// on a periodic axis; t = X - (first + 1/2).
template <typename WT>
__device__ __forceinline__ void lagrange_block(int first, int n, int periodic, Taps<4, WT>& t) {
  t.first = first;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int k = first + i;
    if (periodic) {
      k %= n;
      if (k < 0) k += n;
    }
    t.idx[i] = k;
  }
}

template <typename WT>
__device__ __forceinline__ void axis_lagrange(double X, int n, int periodic, Taps<4, WT>& t) {
  int first = (int)floor(X - 0.5) - 1;
  if (!periodic) first = first < 0 ? 0 : (first > n - 4 ? n - 4 : first);
  lagrange_block<WT>(first, n, periodic, t);
  lagrange_weights<WT>((WT)(X - ((double)first + 0.5)), t.w);
}

// The same from the cell c and the FP32 offset f inside it (X = c + f).
__device__ __forceinline__ void axis_lagrange_local(int c, float f, int n, int periodic,
                                                    Taps<4, float>& t) {
  int first = c + (int)floorf(f - 0.5f) - 1;
  if (!periodic) first = first < 0 ? 0 : (first > n - 4 ? n - 4 : first);
  lagrange_block<float>(first, n, periodic, t);
  lagrange_weights<float>((float)(c - first) - 0.5f + f, t.w);
}

// Per-axis taps of one particle: LAG selects Eq. (5) (WI = 4), else the delta
// kernel of width WI. FP32 modes work from the cell and in-cell offset, FP64
// from the FP64 position.
template <int D, int WI, bool LAG, typename R>
__device__ __forceinline__ void particle_taps(const Geometry& g, const int4& mc, const float4& mf,
                                              const double (&X)[3], Taps<WI, R>& tx,
                                              Taps<WI, R>& ty, Taps<WI, R>& tz) {
  static_assert(!LAG || WI == 4, "the Lagrange block has four nodes");
  if constexpr (sizeof(R) == 4) {
    if constexpr (LAG) {
      axis_lagrange_local(mc.x, mf.x, g.n[0], g.periodic[0], tx);
      axis_lagrange_local(mc.y, mf.y, g.n[1], g.periodic[1], ty);
      if constexpr (D == 3) axis_lagrange_local(mc.z, mf.z, g.n[2], g.periodic[2], tz);
    } else {
      axis_taps_local<WI>(mc.x, mf.x, g.n[0], g.periodic[0], tx);
      axis_taps_local<WI>(mc.y, mf.y, g.n[1], g.periodic[1], ty);
      if constexpr (D == 3) axis_taps_local<WI>(mc.z, mf.z, g.n[2], g.periodic[2], tz);
    }
  } else {
    if constexpr (LAG) {
      axis_lagrange<R>(X[0], g.n[0], g.periodic[0], tx);
      axis_lagrange<R>(X[1], g.n[1], g.periodic[1], ty);
      if constexpr (D == 3) axis_lagrange<R>(X[2], g.n[2], g.periodic[2], tz);
    } else {
      axis_taps<WI, R>(X[0], g.n[0], g.periodic[0], tx);
      axis_taps<WI, R>(X[1], g.n[1], g.periodic[1], ty);
      if constexpr (D == 3) axis_taps<WI, R>(X[2], g.n[2], g.periodic[2], tz);
    }
  }
}

// a[i] for a loop index the compiler does not unroll, by selects (the array
// stays in registers instead of local memory).
template <typename T, int W>
__device__ __forceinline__ T pick(const T (&a)[W], int i) {
  T v = a[0];
#pragma unroll
  for (int k = 1; k < W; ++k) v = i == k ? a[k] : v;
  return v;
}

// Every per-axis tap index inside [0, n) (then every tap cell lies in the
// lattice). The tap builders wrap or clamp each index, so this holds for any
// position; it is checked once per particle instead of at every tap.
template <int D, int WI, typename R>
__device__ __forceinline__ bool taps_in_lattice(const Geometry& g, const Taps<WI, R>& tx,
                                                const Taps<WI, R>& ty, const Taps<WI, R>& tz) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < WI; ++i) {
    ok &= (unsigned)tx.idx[i] < (unsigned)g.n[0];
    ok &= (unsigned)ty.idx[i] < (unsigned)g.n[1];
    if constexpr (D == 3) ok &= (unsigned)tz.idx[i] < (unsigned)g.n[2];
  }
  return ok;
}

// Eq. (4) on the moments: rs = sum w (rho - S), js = sum w j over the taps.
// The loads of one stencil row are all issued before any of them is summed;
// a dropped wall node repeats an in-lattice index with weight 0 and is summed
// like the others (it adds zero).
template <int D, int WI, typename R, bool NC = true>
__device__ __forceinline__ void gather_moments(const CoupleArgs& A, const Taps<WI, R>& tx,
                                               const Taps<WI, R>& ty, const Taps<WI, R>& tz,
                                               R& rs, R (&js)[3]) {
  constexpr int WZ = D == 3 ? WI : 1;
  const Geometry& g = A.g;
  const R* mom = (const R*)A.mom;
  rs = R(0);
  js[0] = js[1] = js[2] = R(0);
  if (!taps_in_lattice<D, WI, R>(g, tx, ty, tz)) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
#pragma unroll 1
  for (int iz = 0; iz < WZ; ++iz) {
    R wz = R(1);
    long long zoff = 0;
    if constexpr (D == 3) {
      wz = pick(tz.w, iz);
      zoff = (long long)pick(tz.idx, iz) * g.n[1];
    }
    if (wz == R(0)) continue;
    // 2D: the whole stencil unrolled; 3D: one row at a time (registers)
#pragma unroll(D == 2 ? WI : 1)
    for (int iy = 0; iy < WI; ++iy) {
      const R wyz = pick(ty.w, iy) * wz;
      const long long row = (zoff + pick(ty.idx, iy)) * g.n[0];
      R m[WI][4];
#pragma unroll
      for (int ix = 0; ix < WI; ++ix) load_moments<R, NC>(mom, row + tx.idx[ix], m[ix]);
#pragma unroll
      for (int ix = 0; ix < WI; ++ix) {
        const R wt = tx.w[ix] * wyz;
        rs += wt * m[ix][0];
#pragma unroll
        for (int k = 0; k < D; ++k) js[k] += wt * m[ix][k + 1];
      }
    }
  }
}

// One row of a 2D FP32 stencil whose W cells are consecutive (no wall drop, no
// wrap): the force of two neighbouring cells (Fx, Fy, Fx, Fy) is one 16-byte
// vector atomic when the first of them has an even index, so a row takes W/2
// atomics (aligned) or W/2 + 1 (one lone cell at each end), and so fewer L1
// sector requests than one atomic per cell.
template <int W>
__device__ __forceinline__ void spread_row_pairs(float* __restrict__ F, long long c0,
                                                 const float (&wt)[W], float ax, float ay) {
  float2* F2 = reinterpret_cast<float2*>(F);
  float4* F4 = reinterpret_cast<float4*>(F);
  int i = 0;
  if (c0 & 1) {
    atomicAdd(F2 + c0, make_float2(ax * wt[0], ay * wt[0]));
    i = 1;
  }
#pragma unroll
  for (int k = 0; k < W / 2; ++k) {
    const int j = i + 2 * k;
    if (j + 1 < W)
      atomicAdd(F4 + ((c0 + j) >> 1),
                make_float4(ax * wt[j], ay * wt[j], ax * wt[j + 1], ay * wt[j + 1]));
  }
  if (c0 & 1) atomicAdd(F2 + c0 + W - 1, make_float2(ax * wt[W - 1], ay * wt[W - 1]));
}

// Eq. (9): add amp * w to F at every tap (one vector atomic per cell in FP32,
// one atomic per component in FP64; in 2D FP32, rows of consecutive cells by
// pairs of cells).
template <int D, int W, typename TW, typename FT>
__device__ __forceinline__ void spread_amp(const CoupleArgs& A, const Taps<W, TW>& tx,
                                           const Taps<W, TW>& ty, const Taps<W, TW>& tz,
                                           const FT (&amp)[3]) {
  constexpr int WZ = D == 3 ? W : 1;
  const Geometry& g = A.g;
  FT* F = (FT*)A.F;
  if constexpr (D == 2 && sizeof(FT) == 4) {
    if (tx.idx[W - 1] == tx.idx[0] + (W - 1)) {  // consecutive: no dropped node, no wrap
#pragma unroll
      for (int iy = 0; iy < W; ++iy) {
        const FT wyz = (FT)ty.w[iy];
        if (wyz == FT(0)) continue;
        float wt[W];
#pragma unroll
        for (int ix = 0; ix < W; ++ix) wt[ix] = (FT)tx.w[ix] * wyz;
        spread_row_pairs<W>((float*)F, (long long)ty.idx[iy] * g.n[0] + tx.idx[0], wt, amp[0],
                            amp[1]);
      }
      return;
    }
  }
#pragma unroll 1
  for (int iz = 0; iz < WZ; ++iz) {
    FT wz = FT(1);
    long long zoff = 0;
    if constexpr (D == 3) {
      wz = (FT)pick(tz.w, iz);
      zoff = (long long)pick(tz.idx, iz) * g.n[1];
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

// Position update along one axis: periodic axes wrap, wall axes report a
// particle outside [0, n].
__device__ __forceinline__ double advance_axis(double x, int n, int periodic, bool& esc) {
  if (periodic) {
    const double N = (double)n;
    if (x < 0.0) x += N;
    else if (x >= N) x -= N;
    if (!(x >= 0.0 && x < N)) x = x - N * floor(x / N);  // |U| > N: not physical
    if (!(x >= 0.0 && x < N)) x = 0.0;
  } else if (outside_bits(x, (double)n)) {
    esc = true;
  }
  return x;
}

// Ordered spreading: keep the particle's spreading taps at its slot for the
// gather kernel, which then applies exactly the weights the atomic path would.
// One axis at a time, with no pointer to the taps: taking their address would
// move them (and every gather that reads them) to local memory.
template <int W, typename TW>
__device__ __forceinline__ void keep_axis(const CoupleArgs& A, long long sl, int k, bool on,
                                          const Taps<W, TW>& t) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int idx = -1;
    double w = 0.0;
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (on && j == i) {
        idx = t.idx[j];
        w = (double)t.w[j];
      }
    A.ti[(sl * 3 + k) * 4 + i] = idx;
    A.tw[(sl * 3 + k) * 4 + i] = w;
  }
}

template <int D, int W, typename TW>
__device__ __forceinline__ void keep_taps(const CoupleArgs& A, long long sl, const Taps<W, TW>& tx,
                                          const Taps<W, TW>& ty, const Taps<W, TW>& tz) {
  keep_axis<W, TW>(A, sl, 0, true, tx);
  keep_axis<W, TW>(A, sl, 1, true, ty);
  keep_axis<W, TW>(A, sl, 2, D == 3, tz);
}

// The particle's constants move with it to its slot.
__device__ __forceinline__ void move_constants(const CoupleArgs& A, unsigned p, long long sl) {
  A.radn[sl] = A.rad[p];
  A.massn[sl] = A.mass[p];
  A.Apn[sl] = A.Ap[p];
  A.buoyn[sl] = A.buoy[p];
  A.gwn[sl] = A.gw[p];
  A.cfn[sl] = A.cf[p];
  A.pidn[sl] = A.pid[p];
}

// Particle update (Eq. 13) and force density (Eqs. 6-7) of the particle at slot
// sl (storage position p), from the interpolated rs = sum w (rho - S) and js and
// the contact force: writes X', U', g and the particle's constants at the slot
// and returns A_p g in amp. FP64 mode solves the update in FP64. The
// FP32-storage modes (whose rho_l, j_l come from FP32 moments) form the velocity
// increment U' - U and g in FP32 and add the increment to the FP64 state.
// When the next step keeps the cell list, also writes the particle's sorted
// record for it (same cell, offset of the new position from that cell) and
// checks that the particle stays within the skin of that cell.
// P64: 32- and 16-bit storage with the update formed in FP64 (the FP64 branch,
// with rho_l, j_l widened from FP32 and the FP64 contact force FCT = double).
template <int D, class St, typename FT, bool P64 = false, typename FCT = typename St::R>
__device__ __forceinline__ void advance_particle(const CoupleArgs& A, long long sl, unsigned p,
                                                 const int4& mc, const float4& mf,
                                                 const double (&X)[3], const double (&U)[3],
                                                 const FCT (&Fc)[3], typename St::R rs,
                                                 const typename St::R (&js)[3], FT (&amp)[3]) {
  using R = typename St::R;
  const Geometry& g = A.g;
  const long long np = A.np;
  double Un[3];
  bool bad = false, esc = false;
  if constexpr (sizeof(R) == 8 || P64) {
    const double mi = A.mass[p], Ap = A.Ap[p], bu = A.buoy[p];
    const double rho_l = (double)St::S + rs;
    double Ub[3];
    if (A.ph.implicit_drag) {
      const double inv = rcp_newton<2>(mi + 2.0 * Ap * rho_l);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        Un[k] = (mi * U[k] + 2.0 * Ap * js[k] + bu * A.ph.gravity[k] + Fc[k]) * inv;
        Ub[k] = Un[k];
      }
    } else {
      const double invm = 1.0 / mi;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        Un[k] = U[k] + (bu * A.ph.gravity[k] + Fc[k] - Ap * 2.0 * (rho_l * U[k] - js[k])) * invm;
        Ub[k] = U[k];
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double gg = 2.0 * (rho_l * Ub[k] - js[k]);
      amp[k] = (FT)(Ap * gg);
      A.gout[k * np + sl] = gg;
    }
  } else {
    const float4 cc = A.cf[p];  // mass, A_p, buoy, radius
    const float rho = (float)St::S + rs;
    float Uf[3], dU[3], Ub[3];
#pragma unroll
    for (int k = 0; k < D; ++k) Uf[k] = (float)U[k];
    if (A.ph.implicit_drag) {
      // U' - U = (2 A_p (j_l - rho_l U) + buoy g + F_c) / (m + 2 A_p rho_l)
      const float inv = 1.f / (cc.x + 2.f * cc.y * rho);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dU[k] = (2.f * cc.y * (js[k] - rho * Uf[k]) + cc.z * A.ph.gravityf[k] + Fc[k]) * inv;
        Ub[k] = Uf[k] + dU[k];
      }
    } else {
      const float invm = 1.f / cc.x;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dU[k] = (cc.z * A.ph.gravityf[k] + Fc[k] - 2.f * cc.y * (rho * Uf[k] - js[k])) * invm;
        Ub[k] = Uf[k];
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Un[k] = U[k] + (double)dU[k];
      const float gg = 2.f * (rho * Ub[k] - js[k]);
      amp[k] = (FT)(gg * cc.y);
      A.gout[k * np + sl] = (double)gg;
    }
  }
  const int cell[3] = {mc.x, mc.y, mc.z};
  float off[3] = {0.f, 0.f, 0.f};
  bool far = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double xn = advance_axis(X[k] + Un[k], g.n[k], g.periodic[k], esc);
    bad |= not_finite_bits(xn) || not_finite_bits(Un[k]);
    A.Xn[k * np + sl] = xn;
    A.Un[k * np + sl] = Un[k];
    if (A.keep_cells) {
      if constexpr (sizeof(R) == 8) {
        // distance from the cell centre, minimum image on periodic axes
        const double dc = min_image(xn - ((double)cell[k] + 0.5), g.n[k], g.periodic[k]);
        far |= !(fabs(dc) <= 0.5 + A.ph.skin);
        off[k] = (float)(dc + 0.5);
      } else {
        // the same from the offset to the cell's lower face, tested in FP32 (the
        // rounding moves the bound by about 1e-7 of a cell)
        off[k] = (float)min_image(xn - (double)cell[k], g.n[k], g.periodic[k]);
        far |= !(fabsf(off[k] - 0.5f) <= 0.5f + A.ph.skinf);
      }
    }
  }
  if (bad) atomicOr(A.err, ERR_PARTICLE_NONFINITE);
  if (esc) atomicOr(A.err, ERR_ESCAPED);
  if (A.keep_cells) {
    // and within disp_skin of its position at the rebuild (the recorded candidates)
    const float4 o0 = A.xs0[sl];
    const float q0[3] = {o0.x, o0.y, o0.z};
#pragma unroll
    for (int k = 0; k < D; ++k) far |= !(fabsf(off[k] - q0[k]) <= A.ph.disp_skinf);
    if (far) atomicOr(A.err, ERR_SKIN);
    // the cell and slot change only at a rebuild (written then and on the step after)
    if (A.move_consts) A.csn[sl] = make_int4(mc.x, mc.y, mc.z, (int)sl);
    A.xsn[sl] = make_float4(off[0], off[1], off[2], mf.w);
  }
  if (A.move_consts) move_constants(A, p, sl);
}

// Particle coupling, one thread per particle in cell-sorted order: interpolate
// rho, j from the moment field (Eq. 4; the delta kernel, or Eq. 5 when LAG),
// take the contact force (k_contacts), advance U and X (Eq. 13), form
// g = 2 (rho_l U_b - j_l) (Eqs. 6-7) and spread A_p g w into F (Eq. 9) with the
// delta kernel of width W. The new state, g and the particle's constants are
// written at its slot, which becomes its storage position for the next step.
// NC: the moment field is read through the read-only path (it was written by an
// earlier kernel).
template <int Q, int W, class St, typename FT, bool LAG, bool NC = true, bool P64 = false>
__device__ __forceinline__ void couple_at(const CoupleArgs& A, long long sl) {
  using L = Lattice<Q>;
  using R = typename St::R;
  constexpr int D = L::D;
  constexpr int WI = LAG ? 4 : W;
  const Geometry& g = A.g;
  const long long np = A.np;
  Taps<WI, R> tx, ty, tz;
  FT amp[3] = {FT(0), FT(0), FT(0)};
  bool act = sl < A.np;
  unsigned p = 0;
  int4 mc = make_int4(0, 0, 0, 0);
  float4 mf = make_float4(0.f, 0.f, 0.f, 0.f);
  double X[3] = {0.0, 0.0, 0.0};
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
    // The 2D FP32-storage taps come from the cell record alone; loading the
    // particle state after the gathers keeps it out of their registers.
    constexpr bool LATE = D == 2 && sizeof(R) == 4;
    double U[3] = {0.0, 0.0, 0.0};
    using FCT = typename std::conditional<P64, double, R>::type;
    FCT Fc[3] = {FCT(0), FCT(0), FCT(0)};
    auto load_state = [&]() {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        X[k] = A.X[k * np + p];
        U[k] = A.U[k * np + p];
        if constexpr (sizeof(R) == 8 || P64) Fc[k] = A.Fcout[k * np + sl];
        else Fc[k] = A.Fcf ? A.Fcf[k * np + sl] : (R)A.Fcout[k * np + sl];
      }
    };
    if constexpr (!LATE) load_state();
    // --- interpolation of rho, j (Eq. 4) ---
    particle_taps<D, WI, LAG, R>(g, mc, mf, X, tx, ty, tz);
    R rs, js[3];
    gather_moments<D, WI, R, NC>(A, tx, ty, tz, rs, js);
    if constexpr (LATE) load_state();

    // --- particle update (Eq. 13) and force density (Eqs. 6-7) ---
    advance_particle<D, St, FT, P64, FCT>(A, sl, p, mc, mf, X, U, Fc, rs, js, amp);
  }

  // --- spreading (Eq. 9) with the delta kernel ---
  if (!act) return;
  if constexpr (LAG) {
    Taps<W, R> sx, sy, sz;
    particle_taps<D, W, false, R>(g, mc, mf, X, sx, sy, sz);
    if (A.spread) spread_amp<D, W, R, FT>(A, sx, sy, sz, amp);
    else keep_taps<D, W, R>(A, sl, sx, sy, sz);
  } else if constexpr (sizeof(R) == 4) {
    // FP32 taps come from the sorted record alone: recomputing them after the
    // update (from a fresh read of the record, which the stores above may alias)
    // costs a few FP32 operations and keeps them out of the registers the update
    // needs
    const float4 mf2 = A.xs[sl];
    Taps<W, R> sx, sy, sz;
    particle_taps<D, W, false, R>(g, mc, mf2, X, sx, sy, sz);
    if (A.spread) spread_amp<D, W, R, FT>(A, sx, sy, sz, amp);
    else keep_taps<D, W, R>(A, sl, sx, sy, sz);
  } else {
    if (A.spread) spread_amp<D, W, R, FT>(A, tx, ty, tz, amp);
    else keep_taps<D, W, R>(A, sl, tx, ty, tz);
  }
}

template <int Q, int W, class St, typename FT, bool LAG, bool P64 = false>
__global__ void __launch_bounds__(256, sizeof(typename St::R) == 4 ? (Lattice<Q>::D == 2 ? 5 : 3) : 2)
    k_couple(CoupleArgs A) {
  couple_at<Q, W, St, FT, LAG, true, P64>(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Coupling by tiles (32- and 16-bit storage, delta interpolation, atomic
// spreading). The scattered moment gathers and force atomics of k_couple (W^d of
// each per particle) are bound by L1 sector requests. Here one CTA takes up to 256
// particles of a group of cell-list tiles (one tile in 3D, four consecutive tiles
// of a tile row in 2D; chunk `blockIdx.x % TILE_CHUNKS` of group
// `blockIdx.x / TILE_CHUNKS`; the particles of consecutive tiles are contiguous in
// the sorted order) and works in a shared-memory window of the lattice that
// covers every stencil node of its particles (the box of their unwrapped tap
// indices):
//   1. the window is filled with the moment field by coalesced loads (periodic
//      axes wrap; nodes beyond a wall read zero and carry weight zero);
//   2. each particle interpolates from the window in the order of
//      gather_moments, so rho_l and j_l equal the direct path's bit for bit, and
//      advances as in k_couple;
//   3. the window is cleared and each particle adds A_p g w into it (the weights
//      of spread_amp), in fixed point: shared-memory atomic adds of 32-bit
//      integers are native, those of floats are not. Each component k has a
//      power-of-two scale chosen per CTA so that no sum can overflow: 2^30 over
//      the sum, over the CTA's particles, of |A_p g_k| times the particle's
//      largest weight product, which bounds every node's sum of that component.
//      A contribution is then resolved to about 1e-9 of that bound (for the
//      cosine kernel away from walls the largest weight product is about 1/8 in
//      3D and 1/4 in 2D, so the bound is some tens of contributions), and the
//      sums are exact (independent of their order);
//   4. every window node with a non-zero force is added to the force field by
//      one vector atomic, converted back to FP32.
// The last chunk of a group takes every remaining particle; beyond 256 of them,
// or if the box exceeds the window (a 2D group that wraps to the next tile row),
// the CTA falls back to the direct path.
// The step launches it in 3D only. On the 256^3 workload it took the coupling
// kernel from 1.53 to 1.42 ms; on the 2048^2 workload (about 200 particles per
// CTA, 16 taps each) the phases of each CTA in sequence outweighed the saved
// sectors: 0.200 ms/step against 0.154 with k_couple.
constexpr int TILE_CHUNKS = 2;

template <int D, int W>
struct CoupleWindow {
  using TD = TileDims<D>;
  static constexpr int TPC = D == 2 ? 4 : 1;  // tiles per group, along x
  // the taps of a particle lie within W + 1 cells of its tile along each axis
  static constexpr int VMAX = (TPC * TD::TX + W + 1) * (TD::TY + W + 1) *
                              (D == 3 ? TD::TZ + W + 1 : 1);
};

template <int Q, int W, class St, typename FT, bool P64 = false>
__global__ void __launch_bounds__(256, Lattice<Q>::D == 3 ? 3 : 4) k_couple_tiles(CoupleArgs A) {
  using R = typename St::R;
  constexpr int D = Lattice<Q>::D;
  using Win = CoupleWindow<D, W>;
  static_assert(sizeof(R) == 4 && sizeof(FT) == 4, "FP32 arithmetic");
  __shared__ float4 win[Win::VMAX];
  __shared__ int box[6];
  __shared__ float amp_bound[8][3];  // per warp and component: sum of |A_p g_k| w_max
  const Geometry& g = A.g;
  const long long np = A.np;
  const long long ntiles = A.nbin / A.bm.tc;
  const long long grp = blockIdx.x / TILE_CHUNKS;
  const int chunk = blockIdx.x % TILE_CHUNKS;
  const long long t0 = grp * Win::TPC, t1 = min(t0 + Win::TPC, ntiles);
  const unsigned t_lo = A.start[t0 * A.bm.tc], t_hi = A.start[t1 * A.bm.tc];
  const unsigned lo = t_lo + 256u * chunk;
  if (lo >= t_hi) return;  // uniform across the CTA
  const unsigned hi = chunk == TILE_CHUNKS - 1 ? t_hi : min(t_hi, lo + 256u);
  if (hi > (unsigned)np || t_lo > t_hi) {
    if (threadIdx.x == 0) atomicOr(A.err, ERR_INDEX);
    return;
  }
  if (threadIdx.x < 3) {
    box[threadIdx.x] = D == 3 || threadIdx.x < 2 ? INT_MAX : 0;
    box[3 + threadIdx.x] = D == 3 || threadIdx.x < 2 ? INT_MIN : 0;
  }
  __syncthreads();
  const bool windowed0 = hi - lo <= 256u;
  // --- each thread's particle: record and taps (FP32 from the record) ---
  const unsigned sl = lo + threadIdx.x;
  bool act = windowed0 && sl < hi;
  int4 mc = make_int4(0, 0, 0, 0);
  float4 mf = make_float4(0.f, 0.f, 0.f, 0.f);
  unsigned p = 0;
  double X[3] = {0.0, 0.0, 0.0};
  Taps<W, R> tx, ty, tz;
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
    particle_taps<D, W, false, R>(g, mc, mf, X, tx, ty, tz);
    atomicMin(&box[0], tx.first);
    atomicMin(&box[1], ty.first);
    atomicMax(&box[3], tx.first + W - 1);
    atomicMax(&box[4], ty.first + W - 1);
    if constexpr (D == 3) {
      atomicMin(&box[2], tz.first);
      atomicMax(&box[5], tz.first + W - 1);
    }
  }
  __syncthreads();
  const int bx = box[0], by = box[1], bz = box[2];
  // extents in 64 bits: a box that no particle set stays empty (max < min)
  const long long wxl = (long long)box[3] - bx + 1, wyl = (long long)box[4] - by + 1,
                  wzl = (long long)box[5] - bz + 1;
  const bool windowed = windowed0 && wxl > 0 && wyl > 0 && wzl > 0 &&
                        wxl * wyl * wzl <= Win::VMAX;
  const int wx = (int)wxl, wy = (int)wyl, wz = (int)wzl;
  if (!windowed) {
    // the direct path, one particle at a time per thread
    for (unsigned s2 = lo + threadIdx.x; s2 < hi; s2 += blockDim.x) {
      const int4 c2 = A.cs[s2];
      const float4 f2 = A.xs[s2];
      const unsigned p2 = (unsigned)c2.w;
      if (p2 >= (unsigned)np) {
        atomicOr(A.err, ERR_INDEX);
        continue;
      }
      double X2[3] = {0.0, 0.0, 0.0}, U2[3] = {0.0, 0.0, 0.0};
      using FCT = typename std::conditional<P64, double, R>::type;
      FCT Fc2[3] = {FCT(0), FCT(0), FCT(0)};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        X2[k] = A.X[k * np + p2];
        U2[k] = A.U[k * np + p2];
        if constexpr (P64) Fc2[k] = A.Fcout[k * np + s2];
        else Fc2[k] = A.Fcf ? A.Fcf[k * np + s2] : (R)A.Fcout[k * np + s2];
      }
      Taps<W, R> ax, ay, az;
      particle_taps<D, W, false, R>(g, c2, f2, X2, ax, ay, az);
      R rs2, js2[3];
      gather_moments<D, W, R>(A, ax, ay, az, rs2, js2);
      FT amp2[3] = {FT(0), FT(0), FT(0)};
      advance_particle<D, St, FT, P64, FCT>(A, s2, p2, c2, f2, X2, U2, Fc2, rs2, js2, amp2);
      spread_amp<D, W, R, FT>(A, ax, ay, az, amp2);
    }
    return;
  }
  const int V = wx * wy * wz;
  constexpr int WZ = D == 3 ? W : 1;
  // --- 1. the moment field over the window ---
  {
    const float4* mom = (const float4*)A.mom;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      int cx = bx + v % wx, cy = by + (v / wx) % wy, cz = bz + v / (wx * wy);
      const bool in = lattice_coord(cx, g.n[0], g.periodic[0]) &&
                      lattice_coord(cy, g.n[1], g.periodic[1]) &&
                      (D == 2 || lattice_coord(cz, g.n[2], g.periodic[2]));
      win[v] = in ? __ldg(mom + cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  __syncthreads();
  // --- 2. interpolation (Eq. 4) and the particle update (Eq. 13) ---
  FT amp[3] = {FT(0), FT(0), FT(0)};
  if (act) {
    double U[3] = {0.0, 0.0, 0.0};
    using FCT = typename std::conditional<P64, double, R>::type;
    FCT Fc[3] = {FCT(0), FCT(0), FCT(0)};
#pragma unroll
    for (int k = 0; k < D; ++k) {
      X[k] = A.X[k * np + p];
      U[k] = A.U[k * np + p];
      if constexpr (P64) Fc[k] = A.Fcout[k * np + sl];
      else Fc[k] = A.Fcf ? A.Fcf[k * np + sl] : (R)A.Fcout[k * np + sl];
    }
    R rs = R(0), js[3] = {R(0), R(0), R(0)};
#pragma unroll 1
    for (int iz = 0; iz < WZ; ++iz) {
      R wzz = R(1);
      int oz = 0;
      if constexpr (D == 3) {
        wzz = pick(tz.w, iz);
        oz = (tz.first + iz - bz) * wy;
      }
      if (wzz == R(0)) continue;
#pragma unroll
      for (int iy = 0; iy < W; ++iy) {
        const R wyz = ty.w[iy] * wzz;
        const int row = (oz + ty.first + iy - by) * wx + tx.first - bx;
#pragma unroll
        for (int ix = 0; ix < W; ++ix) {
          const float4 m = win[row + ix];
          const R wt = tx.w[ix] * wyz;
          rs += wt * m.x;
          js[0] += wt * m.y;
          js[1] += wt * m.z;
          if constexpr (D == 3) js[2] += wt * m.w;
        }
      }
    }
    advance_particle<D, St, FT, P64, FCT>(A, sl, p, mc, mf, X, U, Fc, rs, js, amp);
  }
  // the fixed-point scales: per component, a bound on every node's |sum|
  {
    float wm = 0.f;
    if (act) {
      float mx = 0.f, my = 0.f, mz = 1.f;
#pragma unroll
      for (int i = 0; i < W; ++i) {
        mx = fmaxf(mx, tx.w[i]);
        my = fmaxf(my, ty.w[i]);
      }
      if constexpr (D == 3) {
        mz = 0.f;
#pragma unroll
        for (int i = 0; i < W; ++i) mz = fmaxf(mz, tz.w[i]);
      }
      wm = mx * my * mz;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float b = fabsf(amp[k]) * wm;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
      if ((threadIdx.x & 31) == 0) amp_bound[threadIdx.x >> 5][k] = b;
    }
  }
  __syncthreads();  // every particle has read the window
  // per component: the largest power of two with bound * scale <= 2^30 (1 if the
  // bound is zero or not finite: the step is then flagged unstable anyway); the
  // bound is rounded up a little so that FP32 rounding of the sums cannot
  // undercut it
  float scale[3] = {1.f, 1.f, 1.f}, inv_scale[3] = {1.f, 1.f, 1.f};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    float bound = 0.f;
#pragma unroll
    for (int w8 = 0; w8 < 8; ++w8) bound += amp_bound[w8][k];
    bound *= 1.0001f;
    if (bound > 0.f && bound < 3.0e38f)
      scale[k] = exp2f(fminf(floorf(log2f(1073741824.f / bound)), 126.f));
    inv_scale[k] = 1.f / scale[k];  // exact: a power of two
  }
  // --- 3. A_p g w into the window (Eq. 9) ---
  int4* wi = reinterpret_cast<int4*>(win);
  for (int v = threadIdx.x; v < V; v += blockDim.x) wi[v] = make_int4(0, 0, 0, 0);
  __syncthreads();
  if (act) {
#pragma unroll 1
    for (int iz = 0; iz < WZ; ++iz) {
      FT wzz = FT(1);
      int oz = 0;
      if constexpr (D == 3) {
        wzz = (FT)pick(tz.w, iz);
        oz = (tz.first + iz - bz) * wy;
      }
      if (wzz == FT(0)) continue;
#pragma unroll
      for (int iy = 0; iy < W; ++iy) {
        const FT wyz = (FT)ty.w[iy] * wzz;
        const int row = (oz + ty.first + iy - by) * wx + tx.first - bx;
#pragma unroll
        for (int ix = 0; ix < W; ++ix) {
          const FT wt = (FT)tx.w[ix] * wyz;
          if (wt == FT(0)) continue;
          int* c = reinterpret_cast<int*>(wi + row + ix);
#pragma unroll
          for (int k = 0; k < D; ++k) atomicAdd(c + k, __float2int_rn(amp[k] * wt * scale[k]));
        }
      }
    }
  }
  __syncthreads();
  // --- 4. the window's force into the force field ---
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const int4 q = wi[v];
    if (q.x == 0 && q.y == 0 && (D == 2 || q.z == 0)) continue;
    int cx = bx + v % wx, cy = by + (v / wx) % wy, cz = bz + v / (wx * wy);
    if (!(lattice_coord(cx, g.n[0], g.periodic[0]) && lattice_coord(cy, g.n[1], g.periodic[1]) &&
          (D == 2 || lattice_coord(cz, g.n[2], g.periodic[2])))) {
      atomicOr(A.err, ERR_INDEX);  // only zero weights fall beyond a wall
      continue;
    }
    const long long c = cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
    if constexpr (D == 2)
      atomicAdd(reinterpret_cast<float2*>(A.F) + c,
                make_float2((float)q.x * inv_scale[0], (float)q.y * inv_scale[1]));
    else
      atomicAdd(reinterpret_cast<float4*>(A.F) + c,
                make_float4((float)q.x * inv_scale[0], (float)q.y * inv_scale[1],
                            (float)q.z * inv_scale[2], 0.f));
  }
}

// DEM sub-cycling, step start: interpolate rho_l, j_l once (Eq. 4 / Eq. 5) and
// store them by slot, copy the step-n state to the slot-ordered buffers Xn, Un
// (the sub-step state), clear the accumulated force density and contact force,
// and move the constants to their slots.
template <int Q, int W, class St, bool LAG>
__global__ void __launch_bounds__(256) k_sub_init(CoupleArgs A) {
  using R = typename St::R;
  constexpr int D = Lattice<Q>::D;
  constexpr int WI = LAG ? 4 : W;
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (sl >= A.np) return;
  const long long np = A.np;
  const int4 mc = A.cs[sl];
  const float4 mf = A.xs[sl];
  const unsigned p = (unsigned)mc.w;
  if (p >= (unsigned)np) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
  double X[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    X[k] = A.X[k * np + p];
    A.Xn[k * np + sl] = X[k];
    A.Un[k * np + sl] = A.U[k * np + p];
    A.gout[k * np + sl] = 0.0;
    A.Fcout[k * np + sl] = 0.0;
  }
  Taps<WI, R> tx, ty, tz;
  particle_taps<D, WI, LAG, R>(A.g, mc, mf, X, tx, ty, tz);
  R rs, js[3];
  gather_moments<D, WI, R>(A, tx, ty, tz, rs, js);
  if (!A.spread) {  // ordered spreading at the end of the step: keep the taps
    if constexpr (LAG) {
      Taps<W, R> sx, sy, sz;
      particle_taps<D, W, false, R>(A.g, mc, mf, X, sx, sy, sz);
      keep_taps<D, W, R>(A, sl, sx, sy, sz);
    } else {
      keep_taps<D, W, R>(A, sl, tx, ty, tz);
    }
  }
  A.rl[sl] = (double)St::S + (double)rs;
#pragma unroll
  for (int k = 0; k < D; ++k) A.jl[k * np + sl] = (double)js[k];
  move_constants(A, p, sl);
}

// One DEM sub-step of length h = 1/S for every particle (by slot), FP64:
//   implicit: U' = (m U + h (2 A_p j_l + buoy g + F_c)) / (m + 2 A_p rho_l h),
//   explicit: U' = U + h (buoy g + F_c - 2 A_p (rho_l U - j_l)) / m,
//   X' = X + h U';
// g and F_c accumulate h 2 (rho_l U_b - j_l) and h F_c. A particle farther than
// the skin from its step-start cell position raises ERR_SKIN: the cell list of
// the step start would no longer hold all its contacts.
template <int D>
__global__ void __launch_bounds__(256) k_substep(CoupleArgs A, double h) {
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (sl >= A.np) return;
  const long long np = A.np;
  const Geometry& g = A.g;
  const double m = A.massn[sl], Ap = A.Apn[sl], bu = A.buoyn[sl], rho = A.rl[sl];
  const int4 mc = A.cs[sl];
  const float4 mf = A.xs[sl];
  const int c0[3] = {mc.x, mc.y, mc.z};
  const float f0[3] = {mf.x, mf.y, mf.z};
  bool bad = false, esc = false, far = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double U = A.Un[k * np + sl], j = A.jl[k * np + sl], Fc = A.Fs[k * np + sl];
    double Un, Ub;
    if (A.ph.implicit_drag) {
      Un = (m * U + h * (2.0 * Ap * j + bu * A.ph.gravity[k] + Fc)) / (m + 2.0 * Ap * rho * h);
      Ub = Un;
    } else {
      Un = U + h * (bu * A.ph.gravity[k] + Fc - Ap * 2.0 * (rho * U - j)) / m;
      Ub = U;
    }
    A.gout[k * np + sl] += h * 2.0 * (rho * Ub - j);
    A.Fcout[k * np + sl] += h * Fc;
    const double xn = advance_axis(A.Xn[k * np + sl] + h * Un, g.n[k], g.periodic[k], esc);
    bad |= not_finite_bits(xn) || not_finite_bits(Un);
    const double moved = min_image(xn - ((double)c0[k] + (double)f0[k]), g.n[k], g.periodic[k]);
    far |= !(fabs(moved) <= A.ph.skin);
    A.Xn[k * np + sl] = xn;
    A.Un[k * np + sl] = Un;
  }
  if (bad) atomicOr(A.err, ERR_PARTICLE_NONFINITE);
  if (esc) atomicOr(A.err, ERR_ESCAPED);
  if (far) atomicOr(A.err, ERR_SKIN);
}

// DEM sub-cycling, step end: spread A_p times the sub-step average of g with the
// delta kernel at the step-start position (Eq. 9), as in the single-step path.
template <int Q, int W, class St, typename FT>
__global__ void __launch_bounds__(256) k_sub_spread(CoupleArgs A) {
  using R = typename St::R;
  constexpr int D = Lattice<Q>::D;
  const long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (sl >= A.np) return;
  const long long np = A.np;
  const int4 mc = A.cs[sl];
  const float4 mf = A.xs[sl];
  const unsigned p = (unsigned)mc.w;
  if (p >= (unsigned)np) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
  double X[3] = {0.0, 0.0, 0.0};
  if constexpr (sizeof(R) == 8) {
#pragma unroll
    for (int k = 0; k < D; ++k) X[k] = A.X[k * np + p];
  }
  const double Ap = A.Apn[sl];
  FT amp[3] = {FT(0), FT(0), FT(0)};
#pragma unroll
  for (int k = 0; k < D; ++k) amp[k] = (FT)(Ap * A.gout[k * np + sl]);
  Taps<W, R> tx, ty, tz;
  particle_taps<D, W, false, R>(A.g, mc, mf, X, tx, ty, tz);
  spread_amp<D, W, R, FT>(A, tx, ty, tz, amp);
}

// Deterministic spreading: every cell gathers, in a fixed order (neighbour cells
// by ascending z, y, x offset; particles by storage position inside a cell), the
// A_p g w of every particle whose stencil covers it, with the taps the coupling
// kernel kept at each slot (A_p, g and taps by slot). R: the search reach in
// cells around each bin, the stencil's (1 for 2 taps, 2 for 4) plus one when the
// cell list is kept across steps (particles within half a cell of their bin).
// Writes every cell of F.
template <int D, int W, int R, typename FT>
__device__ __forceinline__ void spread_gather_at(const Geometry& g, const BinMap& bm, long long np,
                                                 const int* __restrict__ ti,
                                                 const double* __restrict__ tw,
                                                 const double* __restrict__ Ap,
                                                 const double* __restrict__ gin,
                                                 const unsigned* __restrict__ start,
                                                 FT* __restrict__ F, int x, int y, int z) {
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
      // the 2R + 1 cells of this row in ascending x: one run of consecutive bins
      // when they are (the common case), else cell by cell; either way the
      // particles are visited in the same order
      constexpr int NX = 2 * R + 1;
      unsigned b[NX];
      bool ok[NX];
      bool one = true;
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        int cx = x + i - R;
        ok[i] = lattice_coord(cx, g.n[0], g.periodic[0]);
        b[i] = ok[i] ? bin_index<D>(bm, cx, cy, cz) : 0u;
        one = one && ok[i] && (i == 0 || b[i] == b[i - 1] + 1);
      }
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        if (one ? i > 0 : !ok[i]) continue;
        const unsigned lo = start[b[i]], hi = start[one ? b[NX - 1] + 1 : b[i] + 1];
        for (unsigned sl = lo; sl < hi; ++sl) {
          FT wt = FT(1);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            FT wk = FT(0);
#pragma unroll
            for (int j = 0; j < W; ++j)
              if (ti[((long long)sl * 3 + k) * 4 + j] == cell[k])
                wk += (FT)tw[((long long)sl * 3 + k) * 4 + j];
            wt *= wk;
          }
          if (wt == FT(0)) continue;
          const double a = Ap[sl];
#pragma unroll
          for (int k = 0; k < D; ++k) acc[k] += (FT)(a * gin[k * np + sl]) * wt;
        }
      }
    }
  }
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  store_force<D, FT>(F, c, acc);
}

template <int D, int W, int R, typename FT>
__global__ void __launch_bounds__(256) k_spread_gather(Geometry g, BinMap bm, long long np,
                                                       const int* __restrict__ ti,
                                                       const double* __restrict__ tw,
                                                       const double* __restrict__ Ap,
                                                       const double* __restrict__ gin,
                                                       const unsigned* __restrict__ start,
                                                       FT* __restrict__ F) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.n[0] || y >= g.n[1]) return;
  spread_gather_at<D, W, R, FT>(g, bm, np, ti, tw, Ap, gin, start, F, x, y, z);
}

// g and Fc of the last step are stored by that step's slot, which is the storage
// position of the current state: Ap and pid of the current buffer match them.
__global__ void k_forces(long long np, int d, const double* __restrict__ Ap,
                         const double* __restrict__ gin, const double* __restrict__ Fc,
                         const unsigned* __restrict__ pid, double* __restrict__ f_fpi,
                         double* __restrict__ f_c, unsigned* __restrict__ err) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const unsigned p = pid[i];
  if (p >= (unsigned long long)np) {
    atomicOr(err, ERR_INDEX);
    return;
  }
  for (int k = 0; k < d; ++k) {
    if (f_fpi) f_fpi[(long long)p * d + k] = -Ap[i] * gin[k * np + i];
    if (f_c) f_c[(long long)p * d + k] = Fc[k * np + i];
  }
}

// aos[p][k] (user order) -> soa[k][p] (storage order at creation: the same).
__global__ void k_aos_to_soa(long long np, int d, const double* __restrict__ aos,
                             double* __restrict__ soa) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  for (int k = 0; k < d; ++k) soa[k * np + p] = aos[p * d + k];
}

__global__ void k_interleave(long long np, int d, const double* __restrict__ soa,
                             const unsigned* __restrict__ pid, double* __restrict__ aos,
                             unsigned* __restrict__ err) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const unsigned p = pid[i];
  if (p >= (unsigned long long)np) {
    atomicOr(err, ERR_INDEX);
    return;
  }
  for (int k = 0; k < d; ++k) aos[(long long)p * d + k] = soa[k * np + i];
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
// (section 2.2), the buoyancy-reduced weight factor m (1 - rho_f/rho_p) of
// Eq. (13), the linear-law wall damping and their FP32 copies; the particles are
// numbered in user order.
__global__ void k_particle_init(long long np, int d, double kn, double beta,
                                double* __restrict__ rad, double* __restrict__ mass,
                                double* __restrict__ Ap, double* __restrict__ buoy,
                                double* __restrict__ gw, float4* __restrict__ cf,
                                unsigned* __restrict__ pid) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  pid[p] = (unsigned)p;
  const double dia = rad[p], rr = buoy[p];
  const double pi = 3.14159265358979323846;
  const double m = d == 2 ? rr * pi * dia * dia / 4.0 : rr * pi * dia * dia * dia / 6.0;
  const double a = pi * dia * dia / 4.0, b = m * (1.0 - 1.0 / rr);
  rad[p] = 0.5 * dia;
  mass[p] = m;
  Ap[p] = a;
  buoy[p] = b;
  gw[p] = 2.0 * beta * sqrt(m * kn);
  cf[p] = make_float4((float)m, (float)a, (float)b, (float)(0.5 * dia));
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// The 3D contact kernel takes the half shell (each pair once, partner forces added
// atomically) unless the sums must follow a fixed order (deterministic mode) or the
// DEM is sub-cycled. On the 256^3 workload it took the contacts from 0.328 to 0.233
// ms/step; in 2D, where the contact search runs beside the coupling on the second
// stream, the step measured 1 % slower with it, so 2D keeps the full shell.
inline bool contacts_half_shell(const State& s) {
  return s.geo.d == 3 && !s.deterministic && s.phy.substeps <= 1;
}

// Arguments of the particle kernels for the current state of s (host side).
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
  const int c = s.cur, n = 1 - s.cur;
  A.rad = P.rad[c];
  A.mass = P.mass[c];
  A.Ap = P.Ap[c];
  A.buoy = P.buoy[c];
  A.gw = P.gw[c];
  A.cf = P.cf[c];
  A.pid = P.pid[c];
  A.radn = P.rad[n];
  A.massn = P.mass[n];
  A.Apn = P.Ap[n];
  A.buoyn = P.buoy[n];
  A.gwn = P.gw[n];
  A.cfn = P.cf[n];
  A.pidn = P.pid[n];
  A.xs = P.xs[c];
  A.cs = P.cs[c];
  A.xsn = P.xs[n];
  A.csn = P.cs[n];
  A.keep_cells = s.phy.rebin > 1;
  A.xs0 = P.xs0;
  A.nb_mode = s.phy.rebin > 1 ? s.nb_mode : 0;
  A.move_consts = s.phy.rebin > 1 ? s.move_consts : 1;
  A.nb_max = P.nb_max;
  A.nb = P.nb;
  A.nbn = P.nbn;
  // in-cell offsets are exact to 2^-24 and whole-cell differences exactly so
  A.xf_margin = 1e-5f;
  A.gout = P.g;
  A.Fcout = P.Fc;
  // the FP32 copy of the contact force serves only the FP32-formed update of the
  // full-shell (deterministic) contact kernel
  A.Fcf = (s.precision == PIBM_FP64 || s.phy.p64 || contacts_half_shell(s)) ? nullptr : P.Fcf;
  A.rl = P.rl;
  A.jl = P.jl;
  A.Fs = P.Fs;
  A.ti = P.ti;
  A.tw = P.tw;
  A.perm = P.perm;
  A.start = P.bin_cnt;
  A.nbin = P.nbin;
  A.f = s.f[s.cur];
  A.mom = s.mom;
  A.F = s.F;
  A.err = s.err;
  A.spread = s.deterministic ? 0 : 1;
  return A;
}

}  // namespace

}  // namespace pibm
