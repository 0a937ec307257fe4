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
__global__ void k_bin_key(const double* __restrict__ X, long long np, Geometry g,
                          unsigned* __restrict__ key, unsigned* __restrict__ rank,
                          unsigned* __restrict__ cnt) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  int b0 = bin_coord(X[p], g.n[0]);
  int b1 = bin_coord(X[np + p], g.n[1]);
  int b2 = D == 3 ? bin_coord(X[2 * np + p], g.n[2]) : 0;
  unsigned k = (unsigned)(b0 + (long long)g.n[0] * (b1 + (long long)g.n[1] * b2));
  key[p] = k;
  rank[p] = atomicAdd(&cnt[k], 1u);
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

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const unsigned* __restrict__ in,
                                                              long long n,
                                                              unsigned* __restrict__ sums) {
  __shared__ unsigned sm[33];
  long long base = blockIdx.x * (long long)SCAN_CHUNK + threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) v[i] = (base + i < n) ? in[base + i] : 0u;
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
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) v[i] = (base + i < n) ? data[base + i] : 0u;
  block_scan(v, sm);
  unsigned off = sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i)
    if (base + i < n) data[base + i] = v[i] + off;
}

// Place each particle at its slot, then order every bin by particle id so that
// the contact sums run in a fixed order.
__global__ void k_bin_scatter(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
                              const unsigned* __restrict__ start, long long np,
                              unsigned* __restrict__ perm) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  perm[start[key[p]] + rank[p]] = (unsigned)p;
}

__global__ void k_bin_sort(const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
                           const unsigned* __restrict__ start, long long np,
                           unsigned* __restrict__ perm) {
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
}

// ---------------------------------------------------------------------------
// Delta weights along one axis (Eqs. 10-11 and the 2-point hat)
// ---------------------------------------------------------------------------
template <int W>
struct Taps {
  int idx[W];
  double w[W];
};

// b = floor(X - 1/2); nodes b..b+1 (W = 2) or b-1..b+2 (W = 4) at distance
// r_t = first + t + 1/2 - X. For the cosine kernel the four values are
// 1/4 (1 + cos th), 1/4 (1 - sin th), 1/4 (1 - cos th), 1/4 (1 + sin th) with
// th = pi r_0 / 2 (cos shifts by a quarter period per node). On a wall axis the
// nodes outside [0, n) are dropped (weight 0) and the kept weights renormalised.
template <int W>
__device__ __forceinline__ void axis_taps(double X, int n, int periodic, Taps<W>& t) {
  int b = (int)floor(X - 0.5);
  int first = (W == 2) ? b : b - 1;
  double r0 = (double)first + 0.5 - X;
  if constexpr (W == 2) {
    t.w[0] = 1.0 + r0;  // 1 - |r0|, r0 in (-1, 0]
    t.w[1] = -r0;       // 1 - |r0 + 1|
  } else {
    double sn, cs;
    sincospi(0.5 * r0, &sn, &cs);
    t.w[0] = 0.25 * (1.0 + cs);
    t.w[1] = 0.25 * (1.0 - sn);
    t.w[2] = 0.25 * (1.0 - cs);
    t.w[3] = 0.25 * (1.0 + sn);
  }
  if (periodic) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = (first + i) % n;  // any X (even a non-finite one) maps into [0, n)
      t.idx[i] = k < 0 ? k + n : k;
    }
  } else {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = first + i;
      bool in = (k >= 0 && k < n);
      t.idx[i] = in ? k : 0;
      if (!in) t.w[i] = 0.0;
      s += t.w[i];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) t.w[i] /= s;
  }
}

// Post-stream moments (rho, j) at cell (x, y, z) pulled from the stored f*.
template <int Q, class St>
__device__ __forceinline__ void tap_moments(const typename St::T* __restrict__ f,
                                            const Geometry& g, int x, int y, int z, double& rho,
                                            double (&j)[3]) {
  using L = Lattice<Q>;
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  double r = St::S ? 1.0 : 0.0, m0 = 0.0, m1 = 0.0, m2 = 0.0;
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
    double v = (double)(bb ? f[opp(a) * g.pitch + c] : f[a * g.pitch + src]);
    r += v;
    if (L::e(a, 0)) m0 += L::e(a, 0) * v;
    if (L::e(a, 1)) m1 += L::e(a, 1) * v;
    if (L::e(a, 2)) m2 += L::e(a, 2) * v;
  }
  rho = r;
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
  long long np;
  const double* X;   // [d][np], step n
  const double* U;
  double* Xn;        // [d][np], step n + 1
  double* Un;
  const double* rad;
  const double* mass;
  const double* Ap;
  const double* buoy;
  double* gout;      // [d][np]
  double* Fcout;     // [d][np]
  const unsigned* perm;
  const unsigned* start;
  const void* f;     // stored populations f*
  void* F;           // force field
  unsigned* err;
  int spread;        // 1: scatter A_p g into F with atomics
};

__device__ __forceinline__ void atomic_add_f(double* a, double v) { atomicAdd(a, v); }
__device__ __forceinline__ void atomic_add_f(float* a, double v) { atomicAdd(a, (float)v); }

template <int Q, int W, class St, typename FT>
__global__ void __launch_bounds__(128) k_couple(CoupleArgs A) {
  using L = Lattice<Q>;
  using T = typename St::T;
  constexpr int D = L::D;
  const long long slot = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (slot >= A.np) return;
  const Geometry& g = A.g;
  const long long np = A.np;
  const unsigned p = A.perm[slot];

  double X[3] = {0.0, 0.0, 0.0}, U[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    X[k] = A.X[k * np + p];
    U[k] = A.U[k * np + p];
  }

  // --- interpolation of rho, j (Eq. 4) ---
  Taps<W> tx, ty, tz;
  axis_taps<W>(X[0], g.n[0], g.periodic[0], tx);
  axis_taps<W>(X[1], g.n[1], g.periodic[1], ty);
  if (D == 3) axis_taps<W>(X[2], g.n[2], g.periodic[2], tz);
  const T* f = (const T*)A.f;
  double rho_l = 0.0, j_l[3] = {0.0, 0.0, 0.0};
  constexpr int WZ = (D == 3) ? W : 1;
#pragma unroll 1
  for (int iz = 0; iz < WZ; ++iz) {
    const double wz = (D == 3) ? tz.w[iz] : 1.0;
    const int z = (D == 3) ? tz.idx[iz] : 0;
    if (wz == 0.0) continue;
#pragma unroll 1
    for (int iy = 0; iy < W; ++iy) {
      const double wyz = ty.w[iy] * wz;
      if (wyz == 0.0) continue;
#pragma unroll 1
      for (int ix = 0; ix < W; ++ix) {
        const double wt = tx.w[ix] * wyz;
        if (wt == 0.0) continue;
        double r, jj[3];
        tap_moments<Q, St>(f, g, tx.idx[ix], ty.idx[iy], z, r, jj);
        rho_l += wt * r;
#pragma unroll
        for (int k = 0; k < D; ++k) j_l[k] += wt * jj[k];
      }
    }
  }

  // --- contacts over the 3^d neighbouring bins, then the walls ---
  const double ri = A.rad[p], mi = A.mass[p];
  double Fc[3] = {0.0, 0.0, 0.0};
  int bc[3] = {bin_coord(X[0], g.n[0]), bin_coord(X[1], g.n[1]),
               D == 3 ? bin_coord(X[2], g.n[2]) : 0};
  const double kn = A.ph.kn, beta = A.ph.beta;
#pragma unroll 1
  for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
    int cz = bc[2] + oz;
    if (D == 3) {
      if (cz < 0 || cz >= g.n[2]) {
        if (!g.periodic[2]) continue;
        cz = cz < 0 ? cz + g.n[2] : cz - g.n[2];
      }
    }
#pragma unroll 1
    for (int oy = -1; oy <= 1; ++oy) {
      int cy = bc[1] + oy;
      if (cy < 0 || cy >= g.n[1]) {
        if (!g.periodic[1]) continue;
        cy = cy < 0 ? cy + g.n[1] : cy - g.n[1];
      }
#pragma unroll 1
      for (int ox = -1; ox <= 1; ++ox) {
        int cx = bc[0] + ox;
        if (cx < 0 || cx >= g.n[0]) {
          if (!g.periodic[0]) continue;
          cx = cx < 0 ? cx + g.n[0] : cx - g.n[0];
        }
        const long long b = cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
        const unsigned lo = A.start[b], hi = A.start[b + 1];
        for (unsigned sl = lo; sl < hi; ++sl) {
          const unsigned q = A.perm[sl];
          if (q == p) continue;
          double s[3], d2 = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            s[k] = min_image(X[k] - A.X[k * np + q], g.n[k], g.periodic[k]);
            d2 += s[k] * s[k];
          }
          const double dist = sqrt(d2);
          const double delta = ri + A.rad[q] - dist;
          if (!(delta > 0.0) || !(dist > 0.0)) continue;
          const double mq = A.mass[q];
          const double meff = mi * mq / (mi + mq);
          const double gam = 2.0 * beta * sqrt(meff * kn);
          const double inv = 1.0 / dist;
          double vn = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) vn += (U[k] - A.U[k * np + q]) * (s[k] * inv);
          const double mag = kn * delta - gam * vn;
#pragma unroll
          for (int k = 0; k < D; ++k) Fc[k] += mag * (s[k] * inv);
        }
      }
    }
  }
  {
    const double gw = 2.0 * beta * sqrt(mi * kn);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (g.periodic[k]) continue;
      double delta = ri - X[k];
      if (delta > 0.0) Fc[k] += kn * delta - gw * U[k];
      delta = ri - ((double)g.n[k] - X[k]);
      if (delta > 0.0) Fc[k] -= kn * delta + gw * U[k];
    }
  }

  // --- particle update (Eq. 13) and force density (Eqs. 6-7) ---
  const double Ap = A.Ap[p], bu = A.buoy[p];
  double Un[3], Ub[3], gg[3];
  if (A.ph.implicit_drag) {
    const double inv = 1.0 / (mi + 2.0 * Ap * rho_l);
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
    double xn = X[k] + Un[k];
    if (g.periodic[k]) {
      const double N = (double)g.n[k];
      if (xn < 0.0) xn += N;
      else if (xn >= N) xn -= N;
      if (!(xn >= 0.0 && xn < N)) xn = xn - N * floor(xn / N);  // |U| > N: not physical
      if (!(xn >= 0.0 && xn < N)) xn = 0.0;
    } else if (xn < 0.0 || xn > (double)g.n[k]) {
      esc = true;
    }
    bad |= !isfinite(xn) || !isfinite(Un[k]);
    A.Xn[k * np + p] = xn;
    A.Un[k * np + p] = Un[k];
    A.gout[k * np + p] = gg[k];
    A.Fcout[k * np + p] = Fc[k];
  }
  if (bad) atomicOr(A.err, ERR_PARTICLE_NONFINITE);
  if (esc) atomicOr(A.err, ERR_ESCAPED);

  // --- spreading (Eq. 9): F += A_p g w at the interpolation taps ---
  if (A.spread) {
    FT* F = (FT*)A.F;
    const long long P = g.pitch;
#pragma unroll 1
    for (int iz = 0; iz < WZ; ++iz) {
      const double wz = (D == 3) ? tz.w[iz] : 1.0;
      const int z = (D == 3) ? tz.idx[iz] : 0;
      if (wz == 0.0) continue;
#pragma unroll 1
      for (int iy = 0; iy < W; ++iy) {
        const double wyz = ty.w[iy] * wz;
        if (wyz == 0.0) continue;
#pragma unroll 1
        for (int ix = 0; ix < W; ++ix) {
          const double wt = tx.w[ix] * wyz;
          if (wt == 0.0) continue;
          const long long c = tx.idx[ix] + (long long)g.n[0] * (ty.idx[iy] + (long long)g.n[1] * z);
#pragma unroll
          for (int k = 0; k < D; ++k) atomic_add_f(&F[k * P + c], Ap * gg[k] * wt);
        }
      }
    }
  }
}

// Deterministic spreading: every cell gathers, in a fixed order (bins by
// ascending z, y, x offset; particles by id inside a bin), the A_p g w of every
// particle whose stencil covers it. Writes every cell of F.
template <int D, int W, typename FT>
__global__ void __launch_bounds__(256) k_spread_gather(Geometry g, long long np,
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
  double acc[3] = {0.0, 0.0, 0.0};
  const int cell[3] = {x, y, z};
#pragma unroll 1
  for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz) {
    int cz = z + oz;
    if (D == 3 && (cz < 0 || cz >= g.n[2])) {
      if (!g.periodic[2]) continue;
      cz = ((cz % g.n[2]) + g.n[2]) % g.n[2];
    }
#pragma unroll 1
    for (int oy = -R; oy <= R; ++oy) {
      int cy = y + oy;
      if (cy < 0 || cy >= g.n[1]) {
        if (!g.periodic[1]) continue;
        cy = ((cy % g.n[1]) + g.n[1]) % g.n[1];
      }
#pragma unroll 1
      for (int ox = -R; ox <= R; ++ox) {
        int cx = x + ox;
        if (cx < 0 || cx >= g.n[0]) {
          if (!g.periodic[0]) continue;
          cx = ((cx % g.n[0]) + g.n[0]) % g.n[0];
        }
        const long long b = cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
        const unsigned lo = start[b], hi = start[b + 1];
        for (unsigned sl = lo; sl < hi; ++sl) {
          const unsigned p = perm[sl];
          double wt = 1.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            Taps<W> t;
            axis_taps<W>(X[k * np + p], g.n[k], g.periodic[k], t);
            double wk = 0.0;
#pragma unroll
            for (int i = 0; i < W; ++i)
              if (t.idx[i] == cell[k]) wk += t.w[i];
            wt *= wk;
          }
          if (wt == 0.0) continue;
          const double a = Ap[p];
#pragma unroll
          for (int k = 0; k < D; ++k) acc[k] += a * gin[k * np + p] * wt;
        }
      }
    }
  }
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
#pragma unroll
  for (int k = 0; k < D; ++k) F[k * g.pitch + c] = (FT)acc[k];
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
__global__ void k_particle_init(long long np, int d, double* __restrict__ rad,
                                double* __restrict__ mass, double* __restrict__ Ap,
                                double* __restrict__ buoy) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double dia = rad[p], rr = buoy[p];
  const double pi = 3.14159265358979323846;
  const double m = d == 2 ? rr * pi * dia * dia / 4.0 : rr * pi * dia * dia * dia / 6.0;
  rad[p] = 0.5 * dia;
  mass[p] = m;
  Ap[p] = pi * dia * dia / 4.0;
  buoy[p] = m * (1.0 - 1.0 / rr);
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
    k_bin_key<2><<<blocks_for(P.np, 256), 256, 0, st>>>(X, P.np, s.geo, P.key, P.rank, P.bin_cnt);
  else
    k_bin_key<3><<<blocks_for(P.np, 256), 256, 0, st>>>(X, P.np, s.geo, P.key, P.rank, P.bin_cnt);
  const long long n = P.nbin + 1;
  k_scan_reduce<<<P.scan_blocks, SCAN_THREADS, 0, st>>>(P.bin_cnt, n, P.block_sums);
  k_scan_top<<<1, SCAN_THREADS, 0, st>>>(P.block_sums, P.scan_blocks);
  k_scan_down<<<P.scan_blocks, SCAN_THREADS, 0, st>>>(P.bin_cnt, n, P.block_sums);
  k_bin_scatter<<<blocks_for(P.np, 256), 256, 0, st>>>(P.key, P.rank, P.bin_cnt, P.np, P.perm);
  k_bin_sort<<<blocks_for(P.np, 256), 256, 0, st>>>(P.key, P.rank, P.bin_cnt, P.np, P.perm);
  if (nk) *nk += 6;
  return cudaGetLastError();
}

namespace {
template <int Q, int W, class St, typename FT>
cudaError_t couple_t(const State& s, cudaStream_t st, int* nk) {
  const Particles& P = s.p;
  CoupleArgs A;
  A.g = s.geo;
  A.ph = s.phy;
  A.np = P.np;
  A.X = P.X[s.cur];
  A.U = P.U[s.cur];
  A.Xn = P.X[1 - s.cur];
  A.Un = P.U[1 - s.cur];
  A.rad = P.rad;
  A.mass = P.mass;
  A.Ap = P.Ap;
  A.buoy = P.buoy;
  A.gout = P.g;
  A.Fcout = P.Fc;
  A.perm = P.perm;
  A.start = P.bin_cnt;
  A.f = s.f[s.cur];
  A.F = s.F;
  A.err = s.err;
  A.spread = s.deterministic ? 0 : 1;
  k_couple<Q, W, St, FT><<<blocks_for(P.np, 128), 128, 0, st>>>(A);
  if (nk) *nk += 1;
  if (s.deterministic) {
    const Geometry& g = s.geo;
    int bx = g.n[0] <= 32 ? 32 : (g.n[0] <= 64 ? 64 : 128);
    dim3 blk(bx, 256 / bx, 1);
    dim3 grd((g.n[0] + blk.x - 1) / blk.x, (g.n[1] + blk.y - 1) / blk.y, g.n[2]);
    k_spread_gather<Lattice<Q>::D, W, FT><<<grd, blk, 0, st>>>(g, P.np, P.X[s.cur], P.Ap, P.g,
                                                               P.perm, P.bin_cnt, (FT*)s.F);
    if (nk) *nk += 1;
  }
  return cudaGetLastError();
}

template <int Q, class St, typename FT>
cudaError_t couple_w(const State& s, cudaStream_t st, int* nk) {
  return s.phy.width == 2 ? couple_t<Q, 2, St, FT>(s, st, nk) : couple_t<Q, 4, St, FT>(s, st, nk);
}
}  // namespace

cudaError_t launch_couple(const State& s, cudaStream_t st, int* nk) {
  if (s.p.np == 0) return cudaSuccess;
  const int q = s.geo.q;
  if (s.precision == PIBM_FP64) {
    if (q == 9) return couple_w<9, StoreF64, double>(s, st, nk);
    if (q == 15) return couple_w<15, StoreF64, double>(s, st, nk);
    if (q == 19) return couple_w<19, StoreF64, double>(s, st, nk);
  } else {
    if (q == 9) return couple_w<9, StoreF32, float>(s, st, nk);
    if (q == 15) return couple_w<15, StoreF32, float>(s, st, nk);
    if (q == 19) return couple_w<19, StoreF32, float>(s, st, nk);
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
  k_particle_init<<<blocks_for(s.p.np, 256), 256, 0, st>>>(s.p.np, s.geo.d, s.p.rad, s.p.mass,
                                                           s.p.Ap, s.p.buoy);
  return cudaGetLastError();
}

}  // namespace pibm
