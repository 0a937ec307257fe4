// Fluid kernels: the fused pull-stream + Guo-forced BGK collision (Eqs. 2, 3, 8
// of the paper, with the half-force velocity of section 2.2) and the kernels that
// move populations between the stored layout and plain FP64 arrays.
//
// Stored state: f[cur][a][c] holds the post-collision value f*_a of the last
// step at cell c, minus S w_a (S = 1 for shifted FP32 storage). The post-stream
// population of the current step is the pull f_a(x) = f*_a(x - e_a), or the
// bounced f*_opp(a)(x) when the link x - e_a crosses a wall (halfway
// bounce-back at resting walls). One thread owns one cell; its Q loads and Q
// stores walk Q structure-of-arrays planes with unit stride along x.
#include "pibm_internal.cuh"

namespace pibm {

namespace {

struct Cell {
  int x, y, z;
  long long c;
};

// Source index of population a arriving at (x, y, z); sets bb when the link
// crosses a wall (then the bounced population at the cell itself is used).
template <int Q>
__device__ __forceinline__ long long pull_src(const Geometry& g, int x, int y, int z, int a,
                                              bool& bb) {
  using L = Lattice<Q>;
  int s[3] = {x - L::e(a, 0), y - L::e(a, 1), z - L::e(a, 2)};
  bb = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (L::e(a, k) == 0) continue;
    if (s[k] < 0) {
      if (g.periodic[k]) s[k] += g.n[k];
      else bb = true;
    } else if (s[k] >= g.n[k]) {
      if (g.periodic[k]) s[k] -= g.n[k];
      else bb = true;
    }
  }
  return s[0] + (long long)g.n[0] * (s[1] + (long long)g.n[1] * s[2]);
}

__device__ __forceinline__ bool bad_density(double r) {
  unsigned long long b = (unsigned long long)__double_as_longlong(r);
  return (b >> 52) >= 0x7ffull || b == 0ull;  // NaN, inf, negative or zero
}
__device__ __forceinline__ bool bad_density(float r) {
  unsigned b = __float_as_uint(r);
  return (b >> 23) >= 0xffu || b == 0u;
}
__device__ __forceinline__ bool nonzero_bits(double v) { return __double_as_longlong(v) != 0; }
__device__ __forceinline__ bool nonzero_bits(float v) { return __float_as_uint(v) != 0u; }

// Pull-stream, collide, store. FT: type of the force field.
template <int Q, class St, typename FT>
__global__ void __launch_bounds__(256) k_collide_stream(const typename St::T* __restrict__ fin,
                                                        typename St::T* __restrict__ fout,
                                                        FT* __restrict__ F, Geometry g,
                                                        typename St::R om,
                                                        typename St::R cF,
                                                        unsigned* __restrict__ err) {
  using L = Lattice<Q>;
  using T = typename St::T;
  using R = typename St::R;
  constexpr int D = L::D;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.n[0] || y >= g.n[1]) return;
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  const long long P = g.pitch;

  R s[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    bool bb;
    long long src = pull_src<Q>(g, x, y, z, a, bb);
    s[a] = (R)(bb ? fin[opp(a) * P + c] : fin[a * P + src]);
  }

  // force of this step, consumed here and cleared for the next spread
  R Fv[3] = {R(0), R(0), R(0)};
  {
    FT v[3];
    load_force<D, FT>(F, c, v);
    bool any = false;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      any |= nonzero_bits(v[k]);
      Fv[k] = (R)v[k];
    }
    if (any) clear_force<D, FT>(F, c);
  }

  // moments: sum of stored values and first moment
  R sum = R(0), j[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 0; a < Q; ++a) sum += s[a];
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int a = 1; a < Q; a += 2) {
      if (L::e(a, k) > 0) j[k] += s[a] - s[a + 1];
      else if (L::e(a, k) < 0) j[k] -= s[a] - s[a + 1];
    }
  }
  const R rho = R(St::S) + sum;
  if (bad_density(rho)) atomicOr(err, ERR_FLUID_NONFINITE);
  const R inv = R(1) / rho;
  R u[3] = {R(0), R(0), R(0)};
  R uu = R(0), uF = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    u[k] = (j[k] + R(0.5) * Fv[k]) * inv;
    uu += u[k] * u[k];
    uF += u[k] * Fv[k];
  }
  const R om1 = R(1) - om;
  // Equilibrium minus the stored shift, Eq. (3):
  //   feq_a - S w_a = w_a sum + rho w_a (3 eu + 4.5 eu^2 - 1.5 uu)
  // Guo term, Eq. (8): cF w_a (3 (e_a - u).F + 9 (e_a.u)(e_a.F)).
  // For an opposite pair (a, a+1) eu and eF flip sign, so the relaxation target
  // splits into an even part Ev and an odd part Od:
  //   Ev = w (om (sum - 1.5 rho uu) - 3 cF uF) + w eu (4.5 om rho eu + 9 cF eF)
  //   Od = w (3 om rho eu + 3 cF eF)
  //   f*_a = (1 - om) s_a + Ev + Od,  f*_{a+1} = (1 - om) s_{a+1} + Ev - Od.
  const R G = om * (sum - R(1.5) * rho * uu) - R(3) * cF * uF;
  const R H = R(4.5) * om * rho;
  const R K = R(9) * cF;
  const R Dd = R(3) * om * rho;
  const R E3 = R(3) * cF;
  fout[c] = (T)(om1 * s[0] + R(L::w(0)) * G);
#pragma unroll
  for (int a = 1; a < Q; a += 2) {
    const R w = R(L::w(a));
    R eu = R(0), eF = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (L::e(a, k) > 0) {
        eu += u[k];
        eF += Fv[k];
      } else if (L::e(a, k) < 0) {
        eu -= u[k];
        eF -= Fv[k];
      }
    }
    const R Ev = w * (G + eu * (H * eu + K * eF));
    const R Od = w * (Dd * eu + E3 * eF);
    fout[a * P + c] = (T)(om1 * s[a] + (Ev + Od));
    fout[(a + 1) * P + c] = (T)(om1 * s[a + 1] + (Ev - Od));
  }
}

// Stored value of plane a from an already un-streamed FP64 plane (or the rest
// value w_a when src is NULL).
template <int Q, class St>
__global__ void k_store_plane(typename St::T* __restrict__ f, const double* __restrict__ src,
                              int a, long long ncell) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  double wa = 0.0;
#pragma unroll
  for (int b = 0; b < Q; ++b)
    if (b == a) wa = Lattice<Q>::w(b);
  double shift = St::S ? wa : 0.0;
  f[c] = (typename St::T)((src ? src[c] : wa) - shift);
}

// Post-stream population a of the current state, FP64.
template <int Q, class St>
__global__ void k_read_pop(const typename St::T* __restrict__ fin, double* __restrict__ dst,
                           Geometry g, int a) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int x = (int)(c % g.n[0]);
  int y = (int)((c / g.n[0]) % g.n[1]);
  int z = (int)(c / ((long long)g.n[0] * g.n[1]));
  double v = 0.0;
  // a is a runtime value here; unroll over the set to keep the table constant
#pragma unroll
  for (int b = 0; b < Q; ++b) {
    if (b != a) continue;
    bool bb;
    long long src = pull_src<Q>(g, x, y, z, b, bb);
    v = (double)(bb ? fin[opp(b) * g.pitch + c] : fin[b * g.pitch + src]);
    v += St::S ? Lattice<Q>::w(b) : 0.0;
  }
  dst[c] = v;
}

// rho (comp 0) or j_k (comp k+1) of the current state, FP64.
template <int Q, class St>
__global__ void k_read_moment(const typename St::T* __restrict__ fin, double* __restrict__ dst,
                              Geometry g, int comp) {
  using L = Lattice<Q>;
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int x = (int)(c % g.n[0]);
  int y = (int)((c / g.n[0]) % g.n[1]);
  int z = (int)(c / ((long long)g.n[0] * g.n[1]));
  double r = St::S ? 1.0 : 0.0, m = 0.0;
#pragma unroll
  for (int b = 0; b < Q; ++b) {
    bool bb;
    long long src = pull_src<Q>(g, x, y, z, b, bb);
    double v = (double)(bb ? fin[opp(b) * g.pitch + c] : fin[b * g.pitch + src]);
    r += v;
    if (comp > 0) m += L::e(b, comp - 1) * v;
  }
  dst[c] = comp == 0 ? r : m;
}


// Fixed-order reductions: RED_BLOCKS blocks stride over the cells in a fixed
// pattern, reduce in shared memory with a fixed tree, and one block sums the
// partials, so the result is identical run to run.
constexpr int RED_BLOCKS = 512;
constexpr int RED_THREADS = 256;

template <int NV>
__device__ void block_tree(double (&v)[NV], double* sm) {
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k * RED_THREADS + threadIdx.x] = v[k];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        sm[k * RED_THREADS + threadIdx.x] += sm[k * RED_THREADS + threadIdx.x + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sm[k * RED_THREADS];
}

template <int Q, class St>
__global__ void __launch_bounds__(RED_THREADS) k_fluid_sums(const typename St::T* __restrict__ fin,
                                                            Geometry g,
                                                            double* __restrict__ partial) {
  using L = Lattice<Q>;
  constexpr int D = L::D;
  __shared__ double sm[(D + 1) * RED_THREADS];
  double acc[D + 1];
#pragma unroll
  for (int k = 0; k <= D; ++k) acc[k] = 0.0;
  for (long long c = blockIdx.x * (long long)RED_THREADS + threadIdx.x; c < g.ncell;
       c += (long long)RED_BLOCKS * RED_THREADS) {
    int x = (int)(c % g.n[0]);
    int y = (int)((c / g.n[0]) % g.n[1]);
    int z = (int)(c / ((long long)g.n[0] * g.n[1]));
    double r = St::S ? 1.0 : 0.0, m[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      bool bb;
      long long src = pull_src<Q>(g, x, y, z, b, bb);
      double v = (double)(bb ? fin[opp(b) * g.pitch + c] : fin[b * g.pitch + src]);
      r += v;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (L::e(b, k)) m[k] += L::e(b, k) * v;
    }
    acc[0] += r;
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k + 1] += m[k];
  }
  block_tree<D + 1>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k <= D; ++k) partial[k * RED_BLOCKS + blockIdx.x] = acc[k];
  }
}

template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_sum_partials(const double* __restrict__ partial,
                                                              int nblocks,
                                                              double* __restrict__ out) {
  __shared__ double sm[NV * RED_THREADS];
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += RED_THREADS) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += partial[k * nblocks + b];
  }
  block_tree<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = acc[k];
  }
}

dim3 cell_block(const Geometry& g) {
  int bx = g.n[0] <= 32 ? 32 : (g.n[0] <= 64 ? 64 : 128);
  return dim3(bx, 256 / bx, 1);
}

template <int Q, class St, typename FT>
cudaError_t collide_stream_t(const State& s, cudaStream_t st) {
  const Geometry& g = s.geo;
  dim3 blk = cell_block(g);
  dim3 grd((g.n[0] + blk.x - 1) / blk.x, (g.n[1] + blk.y - 1) / blk.y, g.n[2]);
  using T = typename St::T;
  using R = typename St::R;
  k_collide_stream<Q, St, FT><<<grd, blk, 0, st>>>((const T*)s.f[s.cur], (T*)s.f[1 - s.cur],
                                                   (FT*)s.F, g, (R)s.phy.omega, (R)s.phy.cF,
                                                   s.err);
  return cudaGetLastError();
}

template <class Fn>
cudaError_t dispatch(const State& s, Fn fn) {
  // fn is a generic lambda taking (Lattice tag, Store tag, force type tag)
  if (s.precision == PIBM_FP64) {
    if (s.geo.q == 9) return fn(Lattice<9>{}, StoreF64{}, double{});
    if (s.geo.q == 15) return fn(Lattice<15>{}, StoreF64{}, double{});
    if (s.geo.q == 19) return fn(Lattice<19>{}, StoreF64{}, double{});
  } else if (s.precision == PIBM_FP32) {
    if (s.geo.q == 9) return fn(Lattice<9>{}, StoreF32{}, float{});
    if (s.geo.q == 15) return fn(Lattice<15>{}, StoreF32{}, float{});
    if (s.geo.q == 19) return fn(Lattice<19>{}, StoreF32{}, float{});
  }
  return cudaErrorInvalidValue;
}

template <class L>
struct QOf;
template <>
struct QOf<Lattice<9>> {
  static constexpr int Q = 9;
};
template <>
struct QOf<Lattice<15>> {
  static constexpr int Q = 15;
};
template <>
struct QOf<Lattice<19>> {
  static constexpr int Q = 19;
};

}  // namespace

cudaError_t launch_collide_stream(const State& s, cudaStream_t st) {
  return dispatch(s, [&](auto lat, auto store, auto ft) {
    constexpr int Q = QOf<decltype(lat)>::Q;
    return collide_stream_t<Q, decltype(store), decltype(ft)>(s, st);
  });
}

cudaError_t launch_store_plane(const State& s, int a, const double* src, cudaStream_t st) {
  return dispatch(s, [&](auto lat, auto store, auto) {
    constexpr int Q = QOf<decltype(lat)>::Q;
    using St = decltype(store);
    using T = typename St::T;
    long long n = s.geo.ncell;
    T* plane = (T*)s.f[s.cur] + a * s.geo.pitch;
    k_store_plane<Q, St><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(plane, src, a, n);
    return cudaGetLastError();
  });
}

cudaError_t launch_read_pop_plane(const State& s, int a, double* dst, cudaStream_t st) {
  return dispatch(s, [&](auto lat, auto store, auto) {
    constexpr int Q = QOf<decltype(lat)>::Q;
    using St = decltype(store);
    using T = typename St::T;
    long long n = s.geo.ncell;
    k_read_pop<Q, St><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const T*)s.f[s.cur], dst,
                                                                   s.geo, a);
    return cudaGetLastError();
  });
}

cudaError_t launch_read_moment(const State& s, int comp, double* dst, cudaStream_t st) {
  return dispatch(s, [&](auto lat, auto store, auto) {
    constexpr int Q = QOf<decltype(lat)>::Q;
    using St = decltype(store);
    using T = typename St::T;
    long long n = s.geo.ncell;
    k_read_moment<Q, St><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const T*)s.f[s.cur], dst,
                                                                      s.geo, comp);
    return cudaGetLastError();
  });
}

cudaError_t launch_invariants(const State& s, double* out_dev, cudaStream_t st) {
  // out_dev[0] = sum rho, out_dev[1..d] = sum j; s.red holds the partials
  return dispatch(s, [&](auto lat, auto store, auto) {
    constexpr int Q = QOf<decltype(lat)>::Q;
    constexpr int D = Lattice<Q>::D;
    using St = decltype(store);
    using T = typename St::T;
    k_fluid_sums<Q, St><<<RED_BLOCKS, RED_THREADS, 0, st>>>((const T*)s.f[s.cur], s.geo, s.red);
    k_sum_partials<D + 1><<<1, RED_THREADS, 0, st>>>(s.red, RED_BLOCKS, out_dev);
    return cudaGetLastError();
  });
}

}  // namespace pibm
