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
#include "lbm_device.cuh"

namespace pibm {

namespace {

// Pull-stream, collide, store; one thread per cell. FT: type of the force field.
template <int Q, class St, typename FT>
__global__ void __launch_bounds__(256, (Lattice<Q>::D == 3 && sizeof(typename St::T) == 4) ? 5 : 0)
    k_collide_stream(const typename St::T* __restrict__ fin,
                                                        typename St::T* __restrict__ fout,
                                                        FT* __restrict__ F, Geometry g,
                                                        typename St::R om,
                                                        typename St::R cF,
                                                        unsigned* __restrict__ err) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.n[0] || y >= g.n[1]) return;
  collide_stream_at<Q, St, FT>(fin, fout, F, g, om, cF, err, x, y, z);
}

// The same over the tiles of one list (the busy or the free tiles of the cell
// list, tn[which] of them), one thread per cell of a tile (TileDims), each CTA
// walking the list with a stride of the grid; the next tile's index is loaded
// before this tile's populations.
template <int Q, class St, typename FT, int HINT, bool NOF = false>
__global__ void __launch_bounds__(TileDims<Lattice<Q>::D>::TC,
                                  (Lattice<Q>::D == 2 && sizeof(typename St::T) == 4) ? 7 : 0)
    k_collide_tiles(const typename St::T* __restrict__ fin, typename St::T* __restrict__ fout,
                    FT* __restrict__ F, Geometry g, BinMap bm, const int* __restrict__ tiles,
                    const unsigned* __restrict__ tn, int which, typename St::R om,
                    typename St::R cF, unsigned* __restrict__ err) {
  using TD = TileDims<Lattice<Q>::D>;
  const int n = (int)tn[which];
  const int lx = threadIdx.x % TD::TX, ly = (threadIdx.x / TD::TX) % TD::TY,
            lz = threadIdx.x / (TD::TX * TD::TY);
  int i = blockIdx.x;
  int t = i < n ? tiles[i] : 0;
  for (; i < n; i += gridDim.x) {
    const int next = i + (int)gridDim.x < n ? tiles[i + gridDim.x] : 0;
    const int r = t / bm.nt[0];
    const int x = (t - r * bm.nt[0]) * TD::TX + lx;
    const int y = (r % bm.nt[1]) * TD::TY + ly;
    const int z = (r / bm.nt[1]) * TD::TZ + lz;
    if (x < g.n[0] && y < g.n[1] && z < g.n[2])
      collide_stream_at<Q, St, FT, HINT, NOF>(fin, fout, F, g, om, cF, err, x, y, z);
    t = next;
  }
}

// The same for 16-bit storage, two neighbouring cells (x0, x0 + 1) per thread
// and one warp per 64 cells of a row: every population row is read with aligned
// 32-bit pair loads; the value one cell to the left or right comes from the
// neighbouring lane (warp shuffle), and only the warp's edge lanes and the
// domain edges load a single extra element. Requires an even n[0]. IX: the
// index type of offsets inside one population plane (int when the plane pitch
// fits in 31 bits, which halves the registers of the per-population rows).
template <int Q, class St, typename FT, typename IX>
__global__ void __launch_bounds__(256) k_collide_stream_pair(const typename St::T* __restrict__ fin,
                                                             typename St::T* __restrict__ fout,
                                                             FT* __restrict__ F, Geometry g,
                                                             typename St::R om,
                                                             typename St::R cF,
                                                             unsigned* __restrict__ err) {
  using L = Lattice<Q>;
  using R = typename St::R;
  constexpr int D = L::D;
  static_assert(sizeof(typename St::T) == 2, "pair kernel is for 16-bit storage");
  const int lane = threadIdx.x;  // blockDim.x == 32
  const int x0 = 2 * (blockIdx.x * 32 + lane);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= g.n[1]) return;  // whole warp (one row per warp)
  const int n0 = g.n[0];
  const bool act = x0 < n0;
  const long long P = g.pitch;
  const IX c0 = x0 + (IX)n0 * (y + (IX)g.n[1] * z);
  const unsigned short* fb = reinterpret_cast<const unsigned short*>(fin);
  // element i of population plane a
  auto at = [&](int a, IX i) { return fb + (long long)a * P + i; };
  auto pair_at = [&](int a, IX i) -> unsigned {  // i even
    return *reinterpret_cast<const unsigned*>(at(a, i));
  };

  // source row of every population: wraps on periodic axes, bounces at walls
  // (then the whole row bounces); three passes keep every load in flight at once
  IX rowb[Q];
  bool rowbb[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    int ys = y - L::e(a, 1), zs = z - L::e(a, 2);
    bool bb = false;
    if (L::e(a, 1) != 0 && (ys < 0 || ys >= g.n[1])) {
      if (g.periodic[1]) ys = ys < 0 ? ys + g.n[1] : ys - g.n[1];
      else bb = true;
    }
    if (L::e(a, 2) != 0 && (zs < 0 || zs >= g.n[2])) {
      if (g.periodic[2]) zs = zs < 0 ? zs + g.n[2] : zs - g.n[2];
      else bb = true;
    }
    rowbb[a] = bb;
    rowb[a] = (IX)n0 * (ys + (IX)g.n[1] * zs);
  }
  // pass 1: one aligned pair per population
  unsigned mine[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    mine[a] = 0u;
    if (act) mine[a] = rowbb[a] ? pair_at(opp(a), c0) : pair_at(a, rowb[a] + x0);
  }
  // pass 2: the single elements the warp's edge lanes and the domain edges need
  unsigned short fix[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ex = L::e(a, 0);
    fix[a] = 0;
    if (ex == 0 || rowbb[a] || !act) continue;
    if (ex > 0 && (lane == 0 || x0 == 0)) {  // needs x0 - 1
      if (x0 == 0) fix[a] = g.periodic[0] ? *at(a, rowb[a] + (n0 - 1)) : *at(opp(a), c0);
      else fix[a] = *at(a, rowb[a] + x0 - 1);
    } else if (ex < 0 && (lane == 31 || x0 + 2 >= n0)) {  // needs x0 + 2
      if (x0 + 2 >= n0) fix[a] = g.periodic[0] ? *at(a, rowb[a]) : *at(opp(a), c0 + 1);
      else fix[a] = *at(a, rowb[a] + x0 + 2);
    }
  }
  // pass 3: neighbours through the warp, then the values of the two cells
  R s[2][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int ex = L::e(a, 0);
    unsigned short v0 = (unsigned short)(mine[a] & 0xffffu), v1 = (unsigned short)(mine[a] >> 16);
    if (ex > 0) {  // sources x0 - 1, x0 (rowbb is warp-uniform: one row per warp)
      const unsigned left = __shfl_up_sync(0xffffffffu, mine[a], 1);
      if (!rowbb[a]) {
        v1 = v0;
        v0 = (lane == 0 || x0 == 0) ? fix[a] : (unsigned short)(left >> 16);
      }
    } else if (ex < 0) {  // sources x0 + 1, x0 + 2
      const unsigned right = __shfl_down_sync(0xffffffffu, mine[a], 1);
      if (!rowbb[a]) {
        v0 = v1;
        v1 = (lane == 31 || x0 + 2 >= n0) ? fix[a] : (unsigned short)(right & 0xffffu);
      }
    }
    s[0][a] = St::load_bits(v0);
    s[1][a] = St::load_bits(v1);
  }
  if (!act) return;
  R Fv0[3], Fv1[3];
  take_force<D, FT, R>(F, c0, Fv0);
  take_force<D, FT, R>(F, c0 + 1, Fv1);
  R o0[Q], o1[Q];
  collide_cell<Q, St>(s[0], Fv0, om, cF, err, o0);
  collide_cell<Q, St>(s[1], Fv1, om, cF, err, o1);
  unsigned short* ob = reinterpret_cast<unsigned short*>(fout);
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const unsigned pr = (unsigned)St::store_bits(o0[a]) | ((unsigned)St::store_bits(o1[a]) << 16);
    *reinterpret_cast<unsigned*>(ob + (long long)a * P + c0) = pr;
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
  f[c] = St::store((typename St::R)((src ? src[c] : wa) - shift));
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
    v = (double)St::load(bb ? fin[opp(b) * g.pitch + c] : fin[b * g.pitch + src]);
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
    double v = (double)St::load(bb ? fin[opp(b) * g.pitch + c] : fin[b * g.pitch + src]);
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
      double v = (double)St::load(bb ? fin[opp(b) * g.pitch + c] : fin[b * g.pitch + src]);
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

// Block shape of the fused collide-stream: the tuned one when set, else the default.
dim3 collide_block(const State& s, bool pair) {
  if (s.cblk[0] > 0 && s.cblk[1] > 0) return dim3(s.cblk[0], s.cblk[1], 1);
  return pair ? dim3(32, 8, 1) : cell_block(s.geo);
}

template <int Q, class St, typename FT>
cudaError_t collide_stream_t(const State& s, cudaStream_t st) {
  const Geometry& g = s.geo;
  using T = typename St::T;
  using R = typename St::R;
  if constexpr (sizeof(T) == 2) {
    if ((g.n[0] & 1) == 0) {
      dim3 blk = collide_block(s, true);  // blk.x is 32: one warp per 64 cells of a row
      dim3 grd((g.n[0] + 63) / 64, (g.n[1] + blk.y - 1) / blk.y, g.n[2]);
      if (g.pitch < (1LL << 31))
        k_collide_stream_pair<Q, St, FT, int><<<grd, blk, 0, st>>>(
            (const T*)s.f[s.cur], (T*)s.f[1 - s.cur], (FT*)s.F, g, (R)s.phy.omega, (R)s.phy.cF,
            s.err);
      else
        k_collide_stream_pair<Q, St, FT, long long><<<grd, blk, 0, st>>>(
            (const T*)s.f[s.cur], (T*)s.f[1 - s.cur], (FT*)s.F, g, (R)s.phy.omega, (R)s.phy.cF,
            s.err);
      return cudaGetLastError();
    }
  }
  dim3 blk = collide_block(s, false);
  dim3 grd((g.n[0] + blk.x - 1) / blk.x, (g.n[1] + blk.y - 1) / blk.y, g.n[2]);
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
  } else if (s.precision == PIBM_FP16) {
    if (s.geo.q == 9) return fn(Lattice<9>{}, StoreF16{}, float{});
    if (s.geo.q == 15) return fn(Lattice<15>{}, StoreF16{}, float{});
    if (s.geo.q == 19) return fn(Lattice<19>{}, StoreF16{}, float{});
  } else if (s.precision == PIBM_BF16) {
    if (s.geo.q == 9) return fn(Lattice<9>{}, StoreBF16{}, float{});
    if (s.geo.q == 15) return fn(Lattice<15>{}, StoreBF16{}, float{});
    if (s.geo.q == 19) return fn(Lattice<19>{}, StoreBF16{}, float{});
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

// CTAs of a grid-stride kernel that fill the GPU once (grid <= 0), else grid.
template <class K>
cudaError_t full_grid(K kern, int threads, int& grid) {
  if (grid > 0) return cudaSuccess;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
  if (e != cudaSuccess) return e;
  grid = sms * (per > 0 ? per : 1);
  return cudaSuccess;
}

}  // namespace

bool collide_tiles_supported(const State& s) { return !collide_uses_pair_kernel(s); }

cudaError_t launch_collide_tiles(const State& s, cudaStream_t st, int which, int grid) {
  return dispatch(s, [&](auto lat, auto store, auto ft) {
    constexpr int Q = QOf<decltype(lat)>::Q;
    using St = decltype(store);
    using FT = decltype(ft);
    using T = typename St::T;
    using R = typename St::R;
    const Particles& P = s.p;
    constexpr int TC = TileDims<Lattice<Q>::D>::TC;
    // busy tiles: their output is read back by the next step's moment kernel
    constexpr int HB = sizeof(T) >= 4 ? 1 : 0, HF = sizeof(T) >= 4 ? 2 : 0;
    cudaError_t e;
    // the free tiles have no force: no particle stencil reaches them
    auto kern = which == 0 ? k_collide_tiles<Q, St, FT, HB> : k_collide_tiles<Q, St, FT, HF, true>;
    if ((e = full_grid(kern, TC, grid)) != cudaSuccess) return e;
    kern<<<grid, TC, 0, st>>>((const T*)s.f[s.cur], (T*)s.f[1 - s.cur], (FT*)s.F, s.geo, P.bm,
                              which == 0 ? P.tbusy : P.tfree, P.tn, which, (R)s.phy.omega,
                              (R)s.phy.cF, s.err);
    return cudaGetLastError();
  });
}

bool collide_uses_pair_kernel(const State& s) {
  return (s.precision == PIBM_FP16 || s.precision == PIBM_BF16) && (s.geo.n[0] & 1) == 0;
}

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
