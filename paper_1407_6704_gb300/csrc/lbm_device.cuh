// Device functions of the fluid step shared by the stream-collide kernels and
// the batched persistent kernel: the pull of one cell (halfway bounce-back at
// resting walls, wraps on periodic axes), the Guo-forced BGK collision of one
// cell (Eqs. 2, 3, 8 of the paper, with the half-force velocity of section
// 2.2) and the force consume-and-clear.
#pragma once

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
// |u|^2 above 0.3^2 (the Mach guard: the BGK equilibrium of Eq. 3 is a low-Mach
// expansion, c_s = 1/sqrt(3)), tested on the bit pattern of the non-negative
// value, so that the FP64 path spends no FP64 operation on it; NaN counts too.
__device__ __forceinline__ bool above_mach(double uu) {
  return (unsigned long long)__double_as_longlong(uu) > 0x3FB70A3D70A3D70Aull;  // 0.09
}
__device__ __forceinline__ bool above_mach(float uu) { return __float_as_uint(uu) > 0x3DB851ECu; }
__device__ __forceinline__ bool nonzero_bits(double v) { return __double_as_longlong(v) != 0; }
__device__ __forceinline__ bool nonzero_bits(float v) { return __float_as_uint(v) != 0u; }

// Guo-forced BGK collision of one cell (Eqs. 2, 3, 8), on stored values s
// (s = f - S w) and the force Fv of this step; writes the post-collision stored
// values to out.
template <int Q, class St>
__device__ __forceinline__ void collide_cell(const typename St::R (&s)[Q],
                                             const typename St::R (&Fv)[3], typename St::R om,
                                             typename St::R cF, unsigned* __restrict__ err,
                                             typename St::R (&out)[Q]) {
  using L = Lattice<Q>;
  using R = typename St::R;
  constexpr int D = L::D;
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
  if (above_mach(uu)) atomicOr(err, ERR_MACH);
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
  out[0] = om1 * s[0] + R(L::w(0)) * G;
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
    out[a] = om1 * s[a] + (Ev + Od);
    out[a + 1] = om1 * s[a + 1] + (Ev - Od);
  }
}

// Force of this step at cell c, consumed and cleared for the next spread.
template <int D, typename FT, typename R>
__device__ __forceinline__ void take_force(FT* __restrict__ F, long long c, R (&Fv)[3]) {
  FT v[3];
  load_force<D, FT>(F, c, v);
  bool any = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) Fv[k] = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    any |= nonzero_bits(v[k]);
    Fv[k] = (R)v[k];
  }
  if (any) clear_force<D, FT>(F, c);
}

// The post-stream populations of lattice cell (x, y, z) as stored values s (type
// R): f*_a(x - e_a), or f*_opp(a)(x) where the link crosses a wall. HINT != 0
// (32- and 64-bit storage): the loads are marked evict-first (the buffer read
// is dead after this step).
template <int Q, class St, int HINT = 0>
__device__ __forceinline__ void pull_cell(const typename St::T* __restrict__ fin,
                                          const Geometry& g, int x, int y, int z,
                                          typename St::R (&s)[Q]) {
  using L = Lattice<Q>;
  using T = typename St::T;
  constexpr int D = L::D;
  static_assert(HINT == 0 || sizeof(T) >= 4, "cache hints are for 32- and 64-bit storage");
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  const long long P = g.pitch;
  unsigned long long first = 0;
  if constexpr (HINT != 0) first = l2_policy_evict_first();
  auto ld = [&](const T* a) -> T {
    if constexpr (HINT != 0) return ld_l2hint(a, first);
    else return *a;
  };
  // a cell whose neighbours all lie inside the lattice (no wall, no wrap) pulls
  // from fixed offsets; only the cells on the lattice faces test every link
  const bool inner = x >= 1 && x <= g.n[0] - 2 && y >= 1 && y <= g.n[1] - 2 &&
                     (D == 2 || (z >= 1 && z <= g.n[2] - 2));
  if (inner) {
    const int n0 = g.n[0], n01 = g.n[0] * g.n[1];
    const T* fa = fin + c;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      s[a] = St::load(ld(fa - (L::e(a, 0) + n0 * L::e(a, 1) + n01 * L::e(a, 2))));
      fa += P;
    }
  } else {
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      bool bb;
      long long src = pull_src<Q>(g, x, y, z, a, bb);
      s[a] = St::load(ld(bb ? fin + (opp(a) * P + c) : fin + (a * P + src)));
    }
  }
}

// Collide the pulled values s of cell c with the force Fv of this step and store
// the post-collision values. HINT == 1: the stores are marked evict-last (the
// next step's moment kernel reads them back).
template <int Q, class St, int HINT = 0>
__device__ __forceinline__ void collide_store(typename St::T* __restrict__ fout,
                                              const Geometry& g, long long c,
                                              const typename St::R (&s)[Q],
                                              const typename St::R (&Fv)[3], typename St::R om,
                                              typename St::R cF, unsigned* __restrict__ err) {
  using R = typename St::R;
  using T = typename St::T;
  unsigned long long last = 0;
  if constexpr (HINT == 1) last = l2_policy_evict_last();
  R out[Q];
  collide_cell<Q, St>(s, Fv, om, cF, err, out);
  T* fo = fout + c;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    if constexpr (HINT == 1) st_l2hint(fo, St::store(out[a]), last);
    else *fo = St::store(out[a]);
    fo += g.pitch;
  }
}

// Pull-stream, collide and store the lattice cell (x, y, z). HINT (32- and
// 64-bit storage): 0 plain accesses; 1 loads marked evict-first (the buffer
// read is dead after this step) and stores evict-last (the next step's moment
// kernel reads them back); 2 loads evict-first only. NOF: the cell has no
// force (no particle stencil reaches it, and the force field is not kept).
template <int Q, class St, typename FT, int HINT = 0, bool NOF = false>
__device__ __forceinline__ void collide_stream_at(const typename St::T* __restrict__ fin,
                                                  typename St::T* __restrict__ fout,
                                                  FT* __restrict__ F, const Geometry& g,
                                                  typename St::R om, typename St::R cF,
                                                  unsigned* __restrict__ err, int x, int y,
                                                  int z) {
  using R = typename St::R;
  constexpr int D = Lattice<Q>::D;
  const long long c = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
  R s[Q];
  pull_cell<Q, St, HINT>(fin, g, x, y, z, s);
  R Fv[3] = {R(0), R(0), R(0)};
  if constexpr (!NOF) take_force<D, FT, R>(F, c, Fv);
  collide_store<Q, St, HINT == 1 ? 1 : 0>(fout, g, c, s, Fv, om, cF, err);
}

}  // namespace

}  // namespace pibm
