// Internal declarations shared by the CUDA translation units of libpibm.
// Lattice tables, storage policies, the device state layout and the launchers
// each translation unit provides.
#pragma once

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
// held in type T and operated on in type R.
// ---------------------------------------------------------------------------
struct StoreF64 {
  using T = double;
  using R = double;
  static constexpr int S = 0;
};
struct StoreF32 {
  using T = float;
  using R = float;
  static constexpr int S = 1;
};

// Device health flags (bitwise OR into State::err).
enum : unsigned {
  ERR_FLUID_NONFINITE = 1u,
  ERR_PARTICLE_NONFINITE = 2u,
  ERR_ESCAPED = 4u,
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
  double kn, beta;        // contact stiffness; damping ratio from restitution
  int width;              // 2 or 4
  int implicit_drag;
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

struct Particles {
  long long np;
  double* X[2];   // [d][np] SoA, ping-pong
  double* U[2];
  double* rad;    // radius
  double* mass;   // rho_r * (pi d^2 / 4) in 2D, rho_r * (pi d^3 / 6) in 3D
  double* Ap;     // cross-section pi d^2 / 4
  double* buoy;   // mass * (1 - 1 / rho_r)
  double* gw;     // wall damping coefficient 2 beta sqrt(mass kn)
  float* radf;    // radius in FP32 (contact pre-filter)
  float* xf;      // [d][np] positions in FP32 (contact pre-filter), written by binning
  double* g;      // [d][np] force density of the last step (Eq. 7)
  double* Fc;     // [d][np] contact force of the last step
  // cell list (bins = lattice cells)
  unsigned* key;      // [np] bin of each particle
  unsigned* rank;     // [np] arrival rank inside the bin
  unsigned* bin_cnt;  // [nbin + 1] counts, then exclusive prefix (bin start)
  unsigned* perm;     // [np] particle id by sorted slot
  unsigned* block_sums;  // scan scratch
  BinMap bm;
  long long nbin;         // tiles * cells per tile (>= ncell)
  int scan_blocks;
};

struct State {
  Geometry geo;
  Physics phy;
  int precision;
  int deterministic;
  void* f[2];     // population buffers (post-collision of the last step), [q][pitch]
  void* F;        // force field [d][pitch], double (FP64) or float (FP32)
  double* red;    // reduction scratch
  unsigned* err;  // device health word
  Particles p;
  int cur;        // index of the buffer holding the current f* / X / U
};

// ---------------------------------------------------------------------------
// Launchers (defined in lbm.cu, particles.cu, reduce.cu)
// ---------------------------------------------------------------------------
// Fluid: one fused pull-stream + Guo-forced BGK collision, f[cur] -> f[1-cur];
// consumes F and leaves it zero.
cudaError_t launch_collide_stream(const State& s, cudaStream_t st);
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
cudaError_t launch_couple(const State& s, cudaStream_t st, int* nkernels);
cudaError_t launch_particle_forces(const State& s, double* f_fpi, double* f_c, cudaStream_t st);
cudaError_t launch_interleave(const State& s, const double* soa, double* aos, cudaStream_t st);
// Derive radius, mass, A_p and buoyancy factor; expects diameter in p.rad and
// the density ratio in p.buoy on entry.
cudaError_t launch_particle_init(const State& s, cudaStream_t st);

// Reductions in a fixed order (deterministic). The reduction scratch s.red holds
// RED_SCRATCH doubles: fluid partials first, particle partials after them.
constexpr long long RED_SCRATCH = 4 * 512 + 3 * 256;
cudaError_t launch_invariants(const State& s, double* out_dev, cudaStream_t st);
cudaError_t launch_particle_momentum(const State& s, double* out_dev, cudaStream_t st);

}  // namespace pibm
