// Internal declarations shared by the CUDA translation units of libpibm.
// Lattice tables, storage policies, the device state layout and the launchers
// each translation unit provides.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pibm.h"

namespace pibm {

// ---------------------------------------------------------------------------
// Velocity sets (Eq. 1 of the paper for D3Q15; D2Q9 and D3Q19 are the usual
// 2D and 3D sets). Order matches the C ABI: rest first, then opposite pairs.
// ---------------------------------------------------------------------------
template <int Q>
struct Lattice;

template <>
struct Lattice<9> {
  static constexpr int D = 2;
  __host__ __device__ static constexpr int e(int a, int k) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return t[a][k];
  }
  __host__ __device__ static constexpr double w(int a) {
    return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <>
struct Lattice<15> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int e(int a, int k) {
    constexpr int t[15][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},    {0, -1, 0},
                              {0, 0, 1},   {0, 0, -1},  {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                              {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},   {1, -1, -1}};
    return t[a][k];
  }
  __host__ __device__ static constexpr double w(int a) {
    return a == 0 ? 2.0 / 9.0 : (a < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
  }
};

template <>
struct Lattice<19> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int e(int a, int k) {
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
    return t[a][k];
  }
  __host__ __device__ static constexpr double w(int a) {
    return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

// ---------------------------------------------------------------------------
// Population storage. The stored value is s = f - S w_a (S = 1: shifted),
// held in type T (possibly scaled) and operated on in type R.
// ---------------------------------------------------------------------------
// load() turns a stored value into s (type R), store() the reverse. Every mode
// keeps the deviation from the rest state (S = 1): the populations are about w_a
// while the flow lives in f - w_a, so storing the deviation keeps the rounding of
// every step at the scale of the flow (in FP64 about 1e-4 of the rounding of f
// itself in a weakly driven flow).
struct StoreF64 {
  using T = double;
  using R = double;
  static constexpr int S = 1;
  __device__ static __forceinline__ R load(T v) { return v; }
  __device__ static __forceinline__ T store(R v) { return v; }
};
struct StoreF32 {
  using T = float;
  using R = float;
  static constexpr int S = 1;
  __device__ static __forceinline__ R load(T v) { return v; }
  __device__ static __forceinline__ T store(R v) { return v; }
};
// Half precision keeps f - w scaled by 2^12, so that deviations of 1e-7 .. 1e1
// stay in FP16's normal range (6.1e-5 .. 65504 after scaling).
struct StoreF16 {
  using T = __half;
  using R = float;
  static constexpr int S = 1;
  __device__ static __forceinline__ R load(T v) { return __half2float(v) * 2.44140625e-4f; }
  __device__ static __forceinline__ T store(R v) { return __float2half_rn(v * 4096.f); }
  __device__ static __forceinline__ R load_bits(unsigned short b) { return load(__ushort_as_half(b)); }
  __device__ static __forceinline__ unsigned short store_bits(R v) {
    return __half_as_ushort(store(v));
  }
};
// BF16 has FP32's exponent range, so f - w is stored unscaled.
struct StoreBF16 {
  using T = __nv_bfloat16;
  using R = float;
  static constexpr int S = 1;
  __device__ static __forceinline__ R load(T v) { return __bfloat162float(v); }
  __device__ static __forceinline__ T store(R v) { return __float2bfloat16_rn(v); }
  __device__ static __forceinline__ R load_bits(unsigned short b) {
    return load(__ushort_as_bfloat16(b));
  }
  __device__ static __forceinline__ unsigned short store_bits(R v) {
    return __bfloat16_as_ushort(store(v));
  }
};

// L2 eviction priorities for single accesses (PTX createpolicy and the
// .L2::cache_hint qualifier): a policy marks the lines an access touches to be
// evicted first or last.
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float ld_l2hint(const float* a, unsigned long long pol) {
  float v;
  asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_l2hint(const double* a, unsigned long long pol) {
  double v;
  asm("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_l2hint(float* a, float v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol));
}
__device__ __forceinline__ void st_l2hint(double* a, double v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol));
}

// Force and moment fields are cell-major: FSTRIDE force slots per cell (2 in 2D,
// 4 in 3D with the last slot unused) and 4 moment slots per cell (rho - S, jx,
// jy, jz), so that one vector access or one vector atomic moves a whole cell.
template <int D>
struct FieldStride {
  static constexpr int F = D == 2 ? 2 : 4;
};
constexpr int MOM_SLOTS = 4;

template <int D, typename FT>
__device__ __forceinline__ void load_force(const FT* __restrict__ F, long long c, FT (&v)[3]) {
  if constexpr (sizeof(FT) == 4 && D == 2) {
    const float2 a = reinterpret_cast<const float2*>(F)[c];
    v[0] = a.x; v[1] = a.y; v[2] = 0.f;
  } else if constexpr (sizeof(FT) == 4) {
    const float4 a = reinterpret_cast<const float4*>(F)[c];
    v[0] = a.x; v[1] = a.y; v[2] = a.z;
  } else if constexpr (D == 2) {
    const double2 a = reinterpret_cast<const double2*>(F)[c];
    v[0] = a.x; v[1] = a.y; v[2] = 0.0;
  } else {
    const double2 a = reinterpret_cast<const double2*>(F)[2 * c];
    const double2 b = reinterpret_cast<const double2*>(F)[2 * c + 1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x;
  }
}

template <int D, typename FT>
__device__ __forceinline__ void clear_force(FT* __restrict__ F, long long c) {
  if constexpr (sizeof(FT) == 4 && D == 2) {
    reinterpret_cast<float2*>(F)[c] = make_float2(0.f, 0.f);
  } else if constexpr (sizeof(FT) == 4) {
    reinterpret_cast<float4*>(F)[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  } else if constexpr (D == 2) {
    reinterpret_cast<double2*>(F)[c] = make_double2(0.0, 0.0);
  } else {
    reinterpret_cast<double2*>(F)[2 * c] = make_double2(0.0, 0.0);
    reinterpret_cast<double2*>(F)[2 * c + 1] = make_double2(0.0, 0.0);
  }
}

template <int D, typename FT>
__device__ __forceinline__ void store_force(FT* __restrict__ F, long long c, const FT (&v)[3]) {
  if constexpr (sizeof(FT) == 4 && D == 2) {
    reinterpret_cast<float2*>(F)[c] = make_float2(v[0], v[1]);
  } else if constexpr (sizeof(FT) == 4) {
    reinterpret_cast<float4*>(F)[c] = make_float4(v[0], v[1], v[2], 0.f);
  } else if constexpr (D == 2) {
    reinterpret_cast<double2*>(F)[c] = make_double2(v[0], v[1]);
  } else {
    reinterpret_cast<double2*>(F)[2 * c] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(F)[2 * c + 1] = make_double2(v[2], 0.0);
  }
}

// F(c) += v, atomically: one vector atomic per cell in FP32, one per component in FP64.
template <int D, typename FT>
__device__ __forceinline__ void add_force(FT* __restrict__ F, long long c, const FT (&v)[3]) {
  if constexpr (sizeof(FT) == 4 && D == 2) {
    atomicAdd(reinterpret_cast<float2*>(F) + c, make_float2(v[0], v[1]));
  } else if constexpr (sizeof(FT) == 4) {
    atomicAdd(reinterpret_cast<float4*>(F) + c, make_float4(v[0], v[1], v[2], 0.f));
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) atomicAdd(F + (long long)FieldStride<D>::F * c + k, v[k]);
  }
}

// In the single-simulation kernels the moment field is read only after the
// kernel that writes it has finished, so the loads take the read-only path
// (NC). A persistent kernel that writes the field in one phase and reads it in
// the next must use coherent loads (NC = false).
template <typename R, bool NC = true>
__device__ __forceinline__ void load_moments(const R* __restrict__ mom, long long c, R (&m)[4]) {
  if constexpr (sizeof(R) == 4) {
    const float4* p = reinterpret_cast<const float4*>(mom) + c;
    const float4 a = NC ? __ldg(p) : *p;
    m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
  } else {
    const double2* p = reinterpret_cast<const double2*>(mom) + 2 * c;
    const double2 a = NC ? __ldg(p) : p[0];
    const double2 b = NC ? __ldg(p + 1) : p[1];
    m[0] = a.x; m[1] = a.y; m[2] = b.x; m[3] = b.y;
  }
}

template <typename R>
__device__ __forceinline__ void store_moments(R* __restrict__ mom, long long c, R r, const R (&j)[3]) {
  if constexpr (sizeof(R) == 4) {
    reinterpret_cast<float4*>(mom)[c] = make_float4(r, j[0], j[1], j[2]);
  } else {
    reinterpret_cast<double2*>(mom)[2 * c] = make_double2(r, j[0]);
    reinterpret_cast<double2*>(mom)[2 * c + 1] = make_double2(j[1], j[2]);
  }
}

// Device health flags (bitwise OR into State::err).
enum : unsigned {
  ERR_FLUID_NONFINITE = 1u,
  ERR_PARTICLE_NONFINITE = 2u,
  ERR_ESCAPED = 4u,
  ERR_INDEX = 8u,  // an internal index check failed; the access was skipped
  ERR_SKIN = 16u,  // a particle moved farther than the cell list allows within a step
  ERR_MACH = 32u,  // a fluid velocity above the Mach guard (|u| > 0.3 lattice units)
};

// ---------------------------------------------------------------------------
// Device state. Every pointer below lives inside one workspace allocation.
// ---------------------------------------------------------------------------
struct Geometry {
  int q, d;
  int n[3];          // extents (n[2] = 1 in 2D)
  int periodic[3];   // per axis
  long long ncell;   // n0 * n1 * n2
  long long pitch;   // plane stride in elements (ncell rounded up to 64)
};

struct Physics {
  double tau, omega, cF;  // omega = 1/tau, cF = 1 - omega/2 (Guo prefactor)
  double gravity[3];
  float gravityf[3];       // the same in FP32 (FP32-storage particle increments)
  double kn, beta;        // contact stiffness; damping ratio from restitution
  int width;              // 2 or 4 (spreading, and interpolation unless lagrange)
  int implicit_drag;
  int lagrange;           // 1: interpolate with the 4-point Lagrange polynomials (Eq. 5)
  int hertz;              // 1: Hertz normal contact (Eq. 15)
  double Epp, Epw;        // Hertz: effective modulus particle-particle, particle-wall
  double hz_damp;         // Hertz: 2 sqrt(5/6) beta
  int substeps;           // DEM sub-steps per fluid step (>= 1)
  double skin;            // largest displacement allowed away from the cell of the last
                          // rebuild (or the step start when sub-cycling): (1 - d_max) / 2
  int rebin;              // cell-list rebuild period in steps (>= 1)
  double disp_skin;       // kept cell list: largest displacement per axis from the position at
                          // the rebuild, (1 - d_max) / 4; bounds the recorded candidates
  float skinf, disp_skinf;  // the same two in FP32 (tests on FP32 offsets)
  int p64;                // 32- and 16-bit storage: particle update in FP64
};

// Tile of lattice cells handled by one CTA of the particle kernel.
template <int D>
struct TileDims {
  static constexpr int TX = D == 2 ? 32 : 16, TY = 8, TZ = D == 2 ? 1 : 4;
  static constexpr int TC = TX * TY * TZ;
};

// Cell-list bins are lattice cells numbered tile-major (tiles of T[0] x T[1] x
// T[2] cells, nt tiles per axis, tc = cells per tile), so that the particles of
// one tile occupy one contiguous range of the sorted list.
struct BinMap {
  int T[3];
  int nt[3];
  int tc;
};

// Particle state is stored in cell-sorted order: the coupling kernel writes the
// state of step n + 1 (and each particle's constants and user id) at the particle's
// slot in the cell list of step n, so the next step's sort is nearly the identity
// and every per-particle access of binning, contacts and coupling is nearly
// coalesced. Every array with two buffers is indexed by storage position; pid maps
// a storage position to the user's particle index.
struct Particles {
  long long np;
  double* X[2];   // [d][np] SoA, ping-pong
  double* U[2];
  double* rad[2];   // radius
  double* mass[2];  // rho_r * (pi d^2 / 4) in 2D, rho_r * (pi d^3 / 6) in 3D
  double* Ap[2];    // cross-section pi d^2 / 4
  double* buoy[2];  // mass * (1 - 1 / rho_r)
  double* gw[2];    // wall damping coefficient 2 beta sqrt(mass kn)
  float4* cf[2];    // FP32 {mass, A_p, buoy, radius} (FP32 arithmetic, contact pre-filter)
  unsigned* pid[2];  // user index of the particle at each storage position
  float4* xr;     // [np] FP32 in-cell position and radius by storage position (binning)
  int4* cr;       // [np] cell (x, y, z) and storage position (binning)
  // sorted records by slot, double-buffered by state parity: written by the
  // cell-list scatter for the current state, or by the coupling kernel of the
  // previous step when the cell list is kept (cell of the last rebuild, offset
  // of the current position from it)
  float4* xs[2];  // FP32 position inside the cell and radius
  int4* cs[2];    // cell (x, y, z) and storage position
  double* g;      // [d][np] force density of the last step (Eq. 7), by slot of that step
  double* Fc;     // [d][np] contact force of the last step, by slot of that step
  float* Fcf;     // [d][np] the same in FP32 (32- and 16-bit storage: the FP32 update reads it)
  // DEM sub-cycling scratch, by slot (allocated when substeps > 1)
  double* rl;     // [np] interpolated rho_l of the step
  double* jl;     // [d][np] interpolated j_l of the step
  double* Fs;     // [d][np] contact force of the current sub-step
  // ordered spreading (deterministic mode): each particle's spreading taps, by slot
  int* ti;        // [np][3][4] cell index per axis and node
  double* tw;     // [np][3][4] weight per axis and node
  // kept cell list (rebin_every > 1): contact candidates recorded at the rebuild
  float4* xs0;    // [np] in-cell offsets at the last rebuild, by slot
  unsigned* nb;   // [nb_max][np] candidate slots
  int* nbn;       // [np] candidate count, -1 when more than nb_max
  int nb_max;
  // cell list (bins = lattice cells)
  unsigned* key;      // [np] bin of each particle
  unsigned* rank;     // [np] arrival rank inside the bin
  unsigned* bin_cnt;  // [nbin + 1] counts, then exclusive prefix (bin start)
  unsigned* perm;     // [np] storage position by sorted slot
  unsigned* block_sums;  // scan scratch
  BinMap bm;
  long long nbin;         // tiles * cells per tile (>= ncell)
  int scan_blocks;
  // tile lists, rebuilt with the cell list: the tiles that hold a particle or
  // touch one that does (busy: every stencil cell of the period lies in them)
  // and the others (free), each in tile order
  long long ntiles;
  int* tflag;       // [ntiles] busy flag (scratch of the list build)
  int* tbusy;       // [ntiles]
  int* tfree;       // [ntiles]
  unsigned* tblk;   // [tile_blocks] busy tiles per block of TILE_BLOCK tiles
  unsigned* tn;     // [2] number of busy and free tiles
};

// Tiles per CTA of the tile-list kernels.
constexpr int TILE_BLOCK = 256;

struct State {
  Geometry geo;
  Physics phy;
  int precision;
  int deterministic;
  void* f[2];     // population buffers (post-collision of the last step), [q][pitch]
  void* F;        // force field [pitch][FieldStride], double (FP64) or float (FP32)
  void* mom;      // moment field [pitch][4] of the current state (cells near particles)
  double* red;    // reduction scratch
  unsigned* err;  // device health word
  Particles p;
  int cur;        // index of the buffer holding the current f* / X / U
  int cblk[2];    // collide-stream block shape (x, y); 0 = built-in choice
  int nb_mode;    // this step's contact search: 1 traverse and record candidates, 2 reuse them
  int move_consts;  // 1: the coupling kernel moves the particles' constants to their slots
                    // (needed unless the order held for the last two steps)
};

// ---------------------------------------------------------------------------
// Cell-list and geometry helpers shared by the particle kernels and the adjoint
// ---------------------------------------------------------------------------
// Bin of lattice cell (x, y, z): cells numbered tile-major (TileDims).
template <int D>
__device__ __forceinline__ unsigned bin_index(const BinMap& b, int x, int y, int z) {
  using TD = TileDims<D>;
  const int tx = x / TD::TX, ty = y / TD::TY, tz = z / TD::TZ;
  const int lx = x - tx * TD::TX, ly = y - ty * TD::TY, lz = z - tz * TD::TZ;
  return (unsigned)(tx + b.nt[0] * (ty + b.nt[1] * tz)) * (unsigned)TD::TC +
         (unsigned)(lx + TD::TX * (ly + TD::TY * lz));
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

// Minimum-image separation along one axis (periodic axes).
__device__ __forceinline__ double min_image(double s, int n, int periodic) {
  if (periodic) {
    double N = (double)n;
    if (s > 0.5 * N) s -= N;
    if (s < -0.5 * N) s += N;
  }
  return s;
}

// ---------------------------------------------------------------------------
// Delta weights along one axis (Eqs. 10-11 and the 2-point hat), shared by the
// particle kernels and the collision that gathers the spread force, so that both
// apply bit-identical weights.
// ---------------------------------------------------------------------------
template <int W, typename WT>
struct Taps {
  int first;    // unwrapped index of the first node
  int idx[W];   // wrapped (periodic) or clamped (dropped wall node) index
  WT w[W];
};

__device__ __forceinline__ void sincospi_t(double a, double* s, double* c) { sincospi(a, s, c); }
__device__ __forceinline__ void sincospi_t(float a, float* s, float* c) { sincospif(a, s, c); }

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

// ---------------------------------------------------------------------------
// Launchers (defined in lbm.cu, particles.cu, reduce.cu)
// ---------------------------------------------------------------------------
// Fluid: one fused pull-stream + Guo-forced BGK collision, f[cur] -> f[1-cur];
// consumes F and leaves it zero.
cudaError_t launch_collide_stream(const State& s, cudaStream_t st);
// True when the collide-stream runs the two-cells-per-thread 16-bit kernel
// (its block is 32 wide); the autotuner picks only the block height then.
bool collide_uses_pair_kernel(const State& s);
// The same collision over the tiles of one list of the cell list (which = 0:
// busy, 1: free), `grid` CTAs walking the list; the two together cover every
// cell once. Available for 32- and 64-bit storage.
bool collide_tiles_supported(const State& s);
cudaError_t launch_collide_tiles(const State& s, cudaStream_t st, int which, int grid);

// Write plane a of the stored buffer f[cur] from FP64 values src (already
// un-streamed by the host), or from the rest value w_a when src is NULL.
cudaError_t launch_store_plane(const State& s, int a, const double* src, cudaStream_t st);
// Post-stream populations / moments of the current state into FP64 arrays.
cudaError_t launch_read_pop_plane(const State& s, int a, double* dst, cudaStream_t st);
cudaError_t launch_read_moment(const State& s, int comp, double* dst, cudaStream_t st);

// Particles: binning (counting sort into lattice-cell bins) and the coupled
// particle kernel (interpolate, contacts, update, spread).
cudaError_t launch_bin(const State& s, cudaStream_t st, int* nkernels);
cudaError_t launch_contacts(const State& s, cudaStream_t st, int* nkernels);
// When before_particles is given, the stream waits for it after the moment
// kernel and before the particle kernels (the contacts then run elsewhere).
cudaError_t launch_couple(const State& s, cudaStream_t st, int* nkernels,
                          cudaEvent_t before_particles = nullptr);
cudaError_t launch_particle_forces(const State& s, double* f_fpi, double* f_c, cudaStream_t st);
// X or U of the current state (SoA by storage position) into aos[user index][d].
cudaError_t launch_interleave(const State& s, const double* soa, double* aos, cudaStream_t st);
// aos [np][d] -> soa [d][np], both device memory.
cudaError_t launch_aos_to_soa(long long np, int d, const double* aos, double* soa,
                              cudaStream_t st);
// Derive radius, mass, A_p and buoyancy factor in buffer 0 and number the
// particles in user order; expects the diameter in p.rad[0] and the density ratio
// in p.buoy[0] on entry.
cudaError_t launch_particle_init(const State& s, cudaStream_t st);

// Internal view of a handle (api.cu): its state, workspace and stream.
struct HandleView {
  State* s;
  void* ws;
  size_t ws_bytes;
  cudaStream_t stream;
};
HandleView handle_view(pibm_t* h);

// Batched persistent step (ensemble.cu). The members must all be D2Q9 with
// FP32 or FP64 storage (the same for all), the same delta width, delta
// interpolation, linear contacts and no DEM sub-cycling.
constexpr int ENSEMBLE_PERSISTENT_MAX = 256;  // members
struct EnsembleDevice;
bool ensemble_persistent_supported(const State* const* s, int n);
int ensemble_device_create(const State* const* s, int n, int device, EnsembleDevice** out);
void ensemble_device_destroy(EnsembleDevice* e);
// CTAs per SM (0: as many as fit) and cells per collision item (0: unchanged;
// a multiple of 256).
int ensemble_device_configure(EnsembleDevice* e, int per_sm, int cpi, cudaStream_t st);
void ensemble_device_shape(const EnsembleDevice* e, int* per_sm, int* max_per_sm, int* cpi,
                           int* grid);
// Load each member's buffer parity and steps since its last rebuild into the
// device phase table, and clear the cell-list counts of members about to rebuild.
cudaError_t ensemble_device_set_phase(EnsembleDevice* e, const int* cur, const int* sr,
                                      cudaStream_t st);
cudaError_t ensemble_device_launch(EnsembleDevice* e, int nsteps, cudaStream_t st);
// Test hook: CTA `block` skips the first barrier of the next launch, every wait of
// that launch gives up after limit_s seconds.
int ensemble_device_inject(EnsembleDevice* e, int block, double limit_s);
bool ensemble_device_injected(const EnsembleDevice* e);
// 1 when a barrier wait gave up (where: its index in the launch), 0 if not, -1 on
// a CUDA error. Synchronises st.
int ensemble_device_timed_out(EnsembleDevice* e, cudaStream_t st, unsigned* where);

// Record a failed CUDA call for pibm_last_error (this thread).
void record_cuda_error(const char* what, cudaError_t e);

// Gradient of the mean settling velocity by the discrete adjoint (adjoint.cu).
int settling_gradient(const pibm_config* cfg, int64_t nsteps, int64_t K, void* stream,
                      double* loss, double* dtau, double* drho, double* dx0);

// Reductions in a fixed order (deterministic). The reduction scratch s.red holds
// RED_SCRATCH doubles: fluid partials first, particle partials after them.
constexpr long long RED_SCRATCH = 4 * 512 + 3 * 256;
cudaError_t launch_invariants(const State& s, double* out_dev, cudaStream_t st);
cudaError_t launch_particle_momentum(const State& s, double* out_dev, cudaStream_t st);

}  // namespace pibm
