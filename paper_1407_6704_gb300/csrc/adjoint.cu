// Discrete adjoint of the coupled step, FP64: the exact gradient of the mean
// settling velocity (the particles' mean velocity along the last axis after the
// last step) with respect to tau, each particle's density ratio and each initial
// position.
//
// The forward run is the library's own step in deterministic mode, so a replayed
// stretch of steps reproduces the trajectory bit for bit. Every K steps the whole
// workspace is kept as a checkpoint; the reverse sweep replays each stretch from
// its checkpoint, keeping a tape of the workspace as it stands before each
// collision (stored populations of the step start, the spread force, the moment
// field, the particle state of both buffers and the cell list), then runs the
// adjoint of each step backwards:
//   1. collision (Eqs. 2, 3, 8) per cell: the adjoint of the post-stream
//      populations, of the force field, and the tau sensitivity;
//   2. spreading (Eq. 9) and the particle update (Eqs. 6-7, 13) per particle;
//   3. contacts (linear spring-dashpot) and interpolation (Eq. 4) per particle,
//      the latter spreading the adjoint of (rho_l, j_l) into a cell field;
//   4. streaming: the pull of the forward step becomes a pull in the opposite
//      direction (each stored population feeds exactly one post-stream one).
#include <math.h>

#include <vector>

#include "pibm_internal.cuh"

namespace pibm {

namespace {

// Delta-kernel taps with their derivatives d w / d X along one axis, FP64, the
// same nodes, weights and wall renormalisation as the forward interpolation.
template <int W>
struct TapsD {
  int idx[W];
  double w[W];
  double dw[W];
};

template <int W>
__device__ __forceinline__ void axis_taps_d(double X, int n, int periodic, TapsD<W>& t) {
  const int b = (int)floor(X - 0.5);
  const int first = (W == 2) ? b : b - 1;
  const double r0 = (double)first + 0.5 - X;  // d r0 / d X = -1
  if constexpr (W == 2) {
    t.w[0] = 1.0 + r0;
    t.dw[0] = -1.0;
    t.w[1] = -r0;
    t.dw[1] = 1.0;
  } else {
    // w = 1/4 (1 + cos th), 1/4 (1 - sin th), 1/4 (1 - cos th), 1/4 (1 + sin th),
    // th = pi r0 / 2, d th / d X = -pi / 2
    double sn, cs;
    sincospi(0.5 * r0, &sn, &cs);
    const double c = 0.125 * 3.14159265358979323846;
    t.w[0] = 0.25 * (1.0 + cs);
    t.dw[0] = c * sn;
    t.w[1] = 0.25 * (1.0 - sn);
    t.dw[1] = c * cs;
    t.w[2] = 0.25 * (1.0 - cs);
    t.dw[2] = -c * sn;
    t.w[3] = 0.25 * (1.0 + sn);
    t.dw[3] = -c * cs;
  }
  if (periodic) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      int k = (first + i) % n;
      t.idx[i] = k < 0 ? k + n : k;
    }
  } else {
    double s = 0.0, ds = 0.0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int k = first + i;
      const bool in = (k >= 0 && k < n);
      t.idx[i] = in ? k : (k < 0 ? 0 : n - 1);
      if (!in) {
        t.w[i] = 0.0;
        t.dw[i] = 0.0;
      }
      s += t.w[i];
      ds += t.dw[i];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      t.w[i] /= s;
      t.dw[i] = (t.dw[i] - t.w[i] * ds) / s;
    }
  }
}

// Source of population a arriving at (x, y, z) by the pull stream; bb when the
// link crosses a wall (the bounced population of the cell itself arrives).
template <int Q>
__device__ __forceinline__ long long adj_pull_src(const Geometry& g, int x, int y, int z, int a,
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

__device__ __forceinline__ void cell_xyz(const Geometry& g, long long c, int& x, int& y, int& z) {
  x = (int)(c % g.n[0]);
  const long long r = c / g.n[0];
  y = (int)(r % g.n[1]);
  z = (int)(r / g.n[1]);
}

constexpr int ADJ_THREADS = 256;

// 1. Collision adjoint per cell. Forward, with T_a = f*_a - (1 - om) f_a:
//   T_a = w_a [om rho (1 + 3 eu + 4.5 eu^2 - 1.5 uu) + cF (3 eF - 3 uF + 9 eu eF)],
//   u = (j + F/2) / rho, cF = 1 - om/2.
// Given gb = adjoint of f*, writes fb = adjoint of the post-stream populations
// (without the interpolation's moment terms), Fb = adjoint of the force, and
// adds this block's d L / d om to om_part[block].
template <int Q>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_collide(Geometry g, double om, double cF,
                                                             const double* __restrict__ fin,
                                                             const double* __restrict__ F,
                                                             const double* __restrict__ gbar,
                                                             double* __restrict__ fbar,
                                                             double* __restrict__ Fbar,
                                                             double* __restrict__ om_part) {
  using L = Lattice<Q>;
  constexpr int D = L::D;
  constexpr int FS = FieldStride<D>::F;
  __shared__ double red[ADJ_THREADS];
  const long long c = blockIdx.x * (long long)ADJ_THREADS + threadIdx.x;
  double omb = 0.0;
  if (c < g.ncell) {
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    const long long P = g.pitch;
    double f[Q], gb[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      bool bb;
      const long long src = adj_pull_src<Q>(g, x, y, z, a, bb);
      // the stored value is f - S w (StoreF64 keeps the deviation from rest)
      f[a] = (bb ? fin[opp(a) * P + c] : fin[a * P + src]) + StoreF64::S * L::w(a);
      gb[a] = gbar[a * P + c];
    }
    double Fv[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) Fv[k] = F[FS * c + k];
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      rho += f[a];
#pragma unroll
      for (int k = 0; k < D; ++k) j[k] += L::e(a, k) * f[a];
    }
    double u[3] = {0.0, 0.0, 0.0}, uu = 0.0, uF = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      u[k] = (j[k] + 0.5 * Fv[k]) / rho;
      uu += u[k] * u[k];
      uF += u[k] * Fv[k];
    }
    double rhob = 0.0, ub[3] = {0.0, 0.0, 0.0}, Fb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      double eu = 0.0, eF = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        eu += L::e(a, k) * u[k];
        eF += L::e(a, k) * Fv[k];
      }
      const double poly = 1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu;
      const double guo = 3.0 * eF - 3.0 * uF + 9.0 * eu * eF;
      const double wg = L::w(a) * gb[a];
      rhob += wg * om * poly;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double e = (double)L::e(a, k);
        ub[k] += wg * (om * rho * (3.0 * e + 9.0 * eu * e - 3.0 * u[k]) +
                       cF * (-3.0 * Fv[k] + 9.0 * e * eF));
        Fb[k] += wg * cF * (3.0 * e - 3.0 * u[k] + 9.0 * eu * e);
      }
      omb += gb[a] * (-f[a]) + wg * (rho * poly - 0.5 * guo);
    }
    double jb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < D; ++k) {
      jb[k] = ub[k] / rho;
      Fb[k] += 0.5 * ub[k] / rho;
      rhob -= ub[k] * u[k] / rho;
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      double v = (1.0 - om) * gb[a] + rhob;
#pragma unroll
      for (int k = 0; k < D; ++k) v += L::e(a, k) * jb[k];
      fbar[a * P + c] = v;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) Fbar[FS * c + k] = Fb[k];
  }
  red[threadIdx.x] = omb;
  __syncthreads();
  for (int s = ADJ_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) om_part[blockIdx.x] += red[0];
}

struct AdjArgs {
  Geometry g;
  Physics ph;
  BinMap bm;
  long long np;
  int cur;              // buffer of the step-start particle state in the tape
  // tape of the step (pointers into the tape copy of the workspace)
  const double* X;      // step-start state by storage position
  const double* U;
  const double* Un;     // U' by slot
  const double* gin;    // g by slot
  const double* mass;   // by storage position
  const double* Ap;
  const double* buoy;
  const double* rad;
  const double* gw;
  const unsigned* pid;
  const int4* cs;
  const unsigned* start;
  const double* mom;    // moment field of the post-stream state [pitch][4]
  // adjoint state
  const double* Fbar;   // [pitch][FS]
  const double* Xb_in;  // adjoint of X' by slot
  const double* Ub_in;
  double* Xb_tmp;       // by slot
  double* Ub_tmp;
  double* Fcb;          // adjoint of F_c by slot
  double* rlb;          // adjoint of rho_l by slot
  double* jlb;          // adjoint of j_l by slot
  double* mb_tmp;       // adjoint of the density ratio from the update, by slot
  double* rjbar;        // adjoint of the moment field [pitch][4] (accumulated)
  double* Xb_out;       // adjoint of X by storage position
  double* Ub_out;
  double* drho;         // user order, accumulated over steps
  unsigned* err;
};

// 2. Spreading and particle update adjoint, per slot (implicit drag):
//   U' = N / den, N = m U + 2 A_p j_l + b G + F_c, den = m + 2 A_p rho_l,
//   X' = X + U', g = 2 (rho_l U' - j_l), F += A_p g w(X).
template <int D, int W>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_update(AdjArgs A) {
  const long long sl = blockIdx.x * (long long)ADJ_THREADS + threadIdx.x;
  if (sl >= A.np) return;
  const long long np = A.np;
  const Geometry& g = A.g;
  constexpr int FS = FieldStride<D>::F;
  const unsigned p = (unsigned)A.cs[sl].w;
  if (p >= (unsigned)np) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
  double X[3] = {0.0, 0.0, 0.0}, U[3] = {0.0, 0.0, 0.0}, Un[3] = {0.0, 0.0, 0.0},
         gg[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    X[k] = A.X[k * np + p];
    U[k] = A.U[k * np + p];
    Un[k] = A.Un[k * np + sl];
    gg[k] = A.gin[k * np + sl];
  }
  const double m = A.mass[p], Ap = A.Ap[p], bu = A.buoy[p];
  TapsD<W> t[3];
#pragma unroll
  for (int k = 0; k < D; ++k) axis_taps_d<W>(X[k], g.n[k], g.periodic[k], t[k]);
  constexpr int WZ = D == 3 ? W : 1;
  double rho_l = 0.0, j_l[3] = {0.0, 0.0, 0.0}, gb[3] = {0.0, 0.0, 0.0}, xs[3] = {0.0, 0.0, 0.0};
  for (int iz = 0; iz < WZ; ++iz) {
    for (int iy = 0; iy < W; ++iy) {
      for (int ix = 0; ix < W; ++ix) {
        const double wz = D == 3 ? t[2].w[iz] : 1.0, dwz = D == 3 ? t[2].dw[iz] : 0.0;
        const double w = t[0].w[ix] * t[1].w[iy] * wz;
        const double dw[3] = {t[0].dw[ix] * t[1].w[iy] * wz, t[0].w[ix] * t[1].dw[iy] * wz,
                              t[0].w[ix] * t[1].w[iy] * dwz};
        const long long c = t[0].idx[ix] + (long long)g.n[0] *
                                               (t[1].idx[iy] + (long long)g.n[1] *
                                                                   (D == 3 ? t[2].idx[iz] : 0));
        const double* mc = A.mom + 4 * c;
        rho_l += w * mc[0];
        double Fg = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          j_l[k] += w * mc[1 + k];
          const double Fb = A.Fbar[FS * c + k];
          gb[k] += w * Fb;
          Fg += Fb * gg[k];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) xs[k] += dw[k] * Fg;
      }
    }
  }
  rho_l += StoreF64::S;  // the moment field holds rho - S, as in the forward step
  double Ubt[3], Nb[3], rlb = 0.0, jlb[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    gb[k] *= Ap;
    xs[k] *= Ap;
    Ubt[k] = A.Ub_in[k * np + sl] + A.Xb_in[k * np + sl] + 2.0 * rho_l * gb[k];
    rlb += 2.0 * gb[k] * Un[k];
    jlb[k] = -2.0 * gb[k];
  }
  const double den = m + 2.0 * Ap * rho_l;
  double denb = 0.0, mb = 0.0, bb = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    Nb[k] = Ubt[k] / den;
    denb -= Ubt[k] * Un[k] / den;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    A.Ub_tmp[k * np + sl] = m * Nb[k];
    jlb[k] += 2.0 * Ap * Nb[k];
    A.Fcb[k * np + sl] = Nb[k];
    mb += Nb[k] * U[k];
    bb += Nb[k] * A.ph.gravity[k];
    A.Xb_tmp[k * np + sl] = A.Xb_in[k * np + sl] + xs[k];
    A.jlb[k * np + sl] = jlb[k];
  }
  mb += denb;
  rlb += 2.0 * Ap * denb;
  A.rlb[sl] = rlb;
  // m = rho_r V, b = m (1 - 1/rho_r) = V (rho_r - 1), V = m - b
  A.mb_tmp[sl] = (m - bu) * (mb + bb);
}

// 3. Contact and interpolation adjoint, per slot. Pair force f_ij = (k_n delta -
// gamma v_n) n with n = s / |s|, s = X_i - X_j, delta = r_i + r_j - |s|,
// v_n = (U_i - U_j).n, gamma = 2 beta sqrt(m_eff k_n); it enters F_c,i with + and
// F_c,j with -, so particle i takes the transposed Jacobian of f_ij applied to
// (Fcb_i - Fcb_j). Walls: F_k += -(+/-) ... as in the forward kernel.
// Interpolation rho_l = sum w rho(c), j_l = sum w j(c): the adjoint moments are
// spread into rjbar with the same weights, and the weight derivatives add to X.
template <int D, int W>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_contact_interp(AdjArgs A) {
  const long long sl = blockIdx.x * (long long)ADJ_THREADS + threadIdx.x;
  if (sl >= A.np) return;
  const long long np = A.np;
  const Geometry& g = A.g;
  const BinMap& bm = A.bm;
  const int4 mc = A.cs[sl];
  const unsigned p = (unsigned)mc.w;
  if (p >= (unsigned)np) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
  double X[3] = {0.0, 0.0, 0.0}, U[3] = {0.0, 0.0, 0.0}, Xb[3] = {0.0, 0.0, 0.0},
         Ub[3] = {0.0, 0.0, 0.0}, ai[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    X[k] = A.X[k * np + p];
    U[k] = A.U[k * np + p];
    Xb[k] = A.Xb_tmp[k * np + sl];
    Ub[k] = A.Ub_tmp[k * np + sl];
    ai[k] = A.Fcb[k * np + sl];
  }
  const double m = A.mass[p], r = A.rad[p], kn = A.ph.kn, beta = A.ph.beta;
  double mb = 0.0;
  const int bc[3] = {mc.x, mc.y, mc.z};
  for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
    int cz = bc[2] + oz;
    if (D == 3 && !lattice_coord(cz, g.n[2], g.periodic[2])) continue;
    for (int oy = -1; oy <= 1; ++oy) {
      int cy = bc[1] + oy;
      if (!lattice_coord(cy, g.n[1], g.periodic[1])) continue;
      for (int ox = -1; ox <= 1; ++ox) {
        int cx = bc[0] + ox;
        if (!lattice_coord(cx, g.n[0], g.periodic[0])) continue;
        const unsigned b = bin_index<D>(bm, cx, cy, cz);
        const unsigned lo = A.start[b], hi = A.start[b + 1];
        if (hi > (unsigned)np || lo > hi) {
          atomicOr(A.err, ERR_INDEX);
          continue;
        }
        for (unsigned s2 = lo; s2 < hi; ++s2) {
          if (s2 == (unsigned)sl) continue;
          const unsigned q = (unsigned)A.cs[s2].w;
          if (q >= (unsigned)np) {
            atomicOr(A.err, ERR_INDEX);
            continue;
          }
          double s[3] = {0.0, 0.0, 0.0}, d2 = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            s[k] = min_image(X[k] - A.X[k * np + q], g.n[k], g.periodic[k]);
            d2 += s[k] * s[k];
          }
          const double dist = sqrt(d2);
          const double delta = r + A.rad[q] - dist;
          if (!(delta > 0.0) || !(dist > 0.0)) continue;
          const double mq = A.mass[q];
          const double meff = m * mq / (m + mq);
          const double gam = 2.0 * beta * sqrt(meff * kn);
          double n[3] = {0.0, 0.0, 0.0}, dU[3] = {0.0, 0.0, 0.0}, vn = 0.0, an = 0.0;
          double av[3] = {0.0, 0.0, 0.0};
#pragma unroll
          for (int k = 0; k < D; ++k) {
            n[k] = s[k] / dist;
            dU[k] = U[k] - A.U[k * np + q];
            vn += dU[k] * n[k];
            av[k] = ai[k] - A.Fcb[k * np + s2];
            an += av[k] * n[k];
          }
          const double mag = kn * delta - gam * vn;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const double dmag = -kn * n[k] - gam * (dU[k] - vn * n[k]) / dist;
            Xb[k] += an * dmag + mag * (av[k] - an * n[k]) / dist;
            Ub[k] -= an * gam * n[k];
          }
          const double mqs = mq / (m + mq);
          mb -= an * vn * gam / (2.0 * meff) * mqs * mqs;
        }
      }
    }
  }
  const double gw = A.gw[p];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (g.periodic[k]) continue;
    // wall at 0: F_k += k_n (r - X_k) - gw U_k; wall at n: F_k -= k_n (r - n + X_k) + gw U_k
    const bool lo = r - X[k] > 0.0, hi = r - ((double)g.n[k] - X[k]) > 0.0;
    const int cnt = (lo ? 1 : 0) + (hi ? 1 : 0);
    Xb[k] -= cnt * kn * ai[k];
    Ub[k] -= cnt * gw * ai[k];
    mb -= cnt * ai[k] * U[k] * gw / (2.0 * m);
  }
  // interpolation adjoint
  const double rlb = A.rlb[sl];
  double jlb[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < D; ++k) jlb[k] = A.jlb[k * np + sl];
  TapsD<W> t[3];
#pragma unroll
  for (int k = 0; k < D; ++k) axis_taps_d<W>(X[k], g.n[k], g.periodic[k], t[k]);
  constexpr int WZ = D == 3 ? W : 1;
  for (int iz = 0; iz < WZ; ++iz) {
    for (int iy = 0; iy < W; ++iy) {
      for (int ix = 0; ix < W; ++ix) {
        const double wz = D == 3 ? t[2].w[iz] : 1.0, dwz = D == 3 ? t[2].dw[iz] : 0.0;
        const double w = t[0].w[ix] * t[1].w[iy] * wz;
        const double dw[3] = {t[0].dw[ix] * t[1].w[iy] * wz, t[0].w[ix] * t[1].dw[iy] * wz,
                              t[0].w[ix] * t[1].w[iy] * dwz};
        const long long c = t[0].idx[ix] + (long long)g.n[0] *
                                               (t[1].idx[iy] + (long long)g.n[1] *
                                                                   (D == 3 ? t[2].idx[iz] : 0));
        const double* mcell = A.mom + 4 * c;
        double val = rlb * mcell[0];
#pragma unroll
        for (int k = 0; k < D; ++k) val += jlb[k] * mcell[1 + k];
#pragma unroll
        for (int k = 0; k < D; ++k) Xb[k] += dw[k] * val;
        if (w != 0.0) {
          atomicAdd(A.rjbar + 4 * c, rlb * w);
#pragma unroll
          for (int k = 0; k < D; ++k) atomicAdd(A.rjbar + 4 * c + 1 + k, jlb[k] * w);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    A.Xb_out[k * np + p] = Xb[k];
    A.Ub_out[k * np + p] = Ub[k];
  }
  const unsigned user = A.pid[p];
  if (user >= (unsigned)np) {
    atomicOr(A.err, ERR_INDEX);
    return;
  }
  A.drho[user] += (m - A.buoy[p]) * mb + A.mb_tmp[sl];
}

// 4. Stream adjoint per cell: the stored population (x, a) of the previous step
// reaches exactly one post-stream population: (x + e_a, a) when that cell is in
// the lattice (wrapped on periodic axes), else (x, opp a) by bounce-back. Adds
// the interpolation's moment adjoint rho_bar + e.j_bar of the receiving cell.
template <int Q>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_stream(Geometry g,
                                                            const double* __restrict__ fbar,
                                                            const double* __restrict__ rjbar,
                                                            double* __restrict__ gout) {
  using L = Lattice<Q>;
  constexpr int D = L::D;
  const long long c = blockIdx.x * (long long)ADJ_THREADS + threadIdx.x;
  if (c >= g.ncell) return;
  int x, y, z;
  cell_xyz(g, c, x, y, z);
  const long long P = g.pitch;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    int t[3] = {x + L::e(a, 0), y + L::e(a, 1), z + L::e(a, 2)};
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (L::e(a, k) == 0) continue;
      if (t[k] < 0 || t[k] >= g.n[k]) {
        if (g.periodic[k]) t[k] = t[k] < 0 ? t[k] + g.n[k] : t[k] - g.n[k];
        else in = false;
      }
    }
    long long y_c;
    int b;
    if (in) {
      y_c = t[0] + (long long)g.n[0] * (t[1] + (long long)g.n[1] * t[2]);
      b = a;
    } else {
      y_c = c;
      b = opp(a);
    }
    double v = fbar[b * P + y_c] + rjbar[4 * y_c];
#pragma unroll
    for (int k = 0; k < D; ++k) v += L::e(b, k) * rjbar[4 * y_c + 1 + k];
    gout[a * P + c] = v;
  }
}

__global__ void k_adj_seed(long long np, int d, double* __restrict__ Ub) {
  const long long i = blockIdx.x * (long long)ADJ_THREADS + threadIdx.x;
  if (i < np) Ub[(long long)(d - 1) * np + i] = 1.0 / (double)np;
}

__global__ void k_mean_last(long long np, int d, const double* __restrict__ U,
                            double* __restrict__ out) {
  __shared__ double red[ADJ_THREADS];
  double s = 0.0;
  for (long long i = threadIdx.x; i < np; i += ADJ_THREADS) s += U[(long long)(d - 1) * np + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = ADJ_THREADS / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / (double)np;
}

__global__ void k_sum_blocks(long long n, const double* __restrict__ in, double* __restrict__ out) {
  __shared__ double red[ADJ_THREADS];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += ADJ_THREADS) s += in[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = ADJ_THREADS / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

unsigned nblk(long long n) { return (unsigned)((n + ADJ_THREADS - 1) / ADJ_THREADS); }

template <typename T>
T* rebase(T* p, const char* from, char* to) {
  return p ? (T*)(to + ((const char*)p - from)) : nullptr;
}

// A copy of the state whose pointers address the tape copy of the workspace.
State rebase_state(const State& s, const void* ws, void* tape) {
  const char* a = (const char*)ws;
  char* b = (char*)tape;
  State t = s;
  for (int i = 0; i < 2; ++i) t.f[i] = rebase((char*)s.f[i], a, b);
  t.F = rebase((char*)s.F, a, b);
  t.mom = rebase((char*)s.mom, a, b);
  t.red = rebase(s.red, a, b);
  t.err = rebase(s.err, a, b);
  Particles& P = t.p;
  const Particles& Q = s.p;
  for (int i = 0; i < 2; ++i) {
    P.X[i] = rebase(Q.X[i], a, b);
    P.U[i] = rebase(Q.U[i], a, b);
    P.rad[i] = rebase(Q.rad[i], a, b);
    P.mass[i] = rebase(Q.mass[i], a, b);
    P.Ap[i] = rebase(Q.Ap[i], a, b);
    P.buoy[i] = rebase(Q.buoy[i], a, b);
    P.gw[i] = rebase(Q.gw[i], a, b);
    P.cf[i] = rebase(Q.cf[i], a, b);
    P.pid[i] = rebase(Q.pid[i], a, b);
  }
  P.xr = rebase(Q.xr, a, b);
  P.cr = rebase(Q.cr, a, b);
  for (int i = 0; i < 2; ++i) {
    P.xs[i] = rebase(Q.xs[i], a, b);
    P.cs[i] = rebase(Q.cs[i], a, b);
  }
  P.g = rebase(Q.g, a, b);
  P.Fc = rebase(Q.Fc, a, b);
  P.rl = rebase(Q.rl, a, b);
  P.jl = rebase(Q.jl, a, b);
  P.Fs = rebase(Q.Fs, a, b);
  P.key = rebase(Q.key, a, b);
  P.rank = rebase(Q.rank, a, b);
  P.bin_cnt = rebase(Q.bin_cnt, a, b);
  P.perm = rebase(Q.perm, a, b);
  P.block_sums = rebase(Q.block_sums, a, b);
  return t;
}

template <int Q, int W>
cudaError_t adjoint_step(const State& T, AdjArgs A, double* gbar, double* fbar, double* Fbar,
                         double* om_part, cudaStream_t st) {
  constexpr int D = Lattice<Q>::D;
  const Geometry& g = T.geo;
  const int cur = T.cur, nxt = 1 - T.cur;
  A.X = T.p.X[cur];
  A.U = T.p.U[cur];
  A.Un = T.p.U[nxt];
  A.gin = T.p.g;
  A.mass = T.p.mass[cur];
  A.Ap = T.p.Ap[cur];
  A.buoy = T.p.buoy[cur];
  A.rad = T.p.rad[cur];
  A.gw = T.p.gw[cur];
  A.pid = T.p.pid[cur];
  A.cs = T.p.cs[cur];
  A.start = T.p.bin_cnt;
  A.mom = (const double*)T.mom;
  cudaError_t e = cudaMemsetAsync(A.rjbar, 0, sizeof(double) * 4 * g.pitch, st);
  if (e != cudaSuccess) return e;
  k_adj_collide<Q><<<nblk(g.ncell), ADJ_THREADS, 0, st>>>(
      g, T.phy.omega, T.phy.cF, (const double*)T.f[cur], (const double*)T.F, gbar, fbar, Fbar,
      om_part);
  const unsigned pb = nblk(A.np);
  k_adj_update<D, W><<<pb, ADJ_THREADS, 0, st>>>(A);
  k_adj_contact_interp<D, W><<<pb, ADJ_THREADS, 0, st>>>(A);
  k_adj_stream<Q><<<nblk(g.ncell), ADJ_THREADS, 0, st>>>(g, fbar, A.rjbar, gbar);
  return cudaGetLastError();
}

template <int Q>
cudaError_t adjoint_step_w(const State& T, const AdjArgs& A, double* gbar, double* fbar,
                           double* Fbar, double* om_part, cudaStream_t st) {
  return T.phy.width == 2 ? adjoint_step<Q, 2>(T, A, gbar, fbar, Fbar, om_part, st)
                          : adjoint_step<Q, 4>(T, A, gbar, fbar, Fbar, om_part, st);
}

// Device allocations of the gradient run, released together.
struct Allocs {
  std::vector<void*> ptrs;
  ~Allocs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 256) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
};

struct HandleGuard {
  pibm_t* h = nullptr;
  ~HandleGuard() {
    if (h) pibm_destroy(h);
  }
};

}  // namespace

int settling_gradient(const pibm_config* cfg_in, int64_t nsteps, int64_t K, void* stream,
                      double* loss, double* dtau, double* drho, double* dx0) {
  if (!cfg_in || nsteps < 1 || K < 1 || !loss) return PIBM_EINVAL;
  if (cfg_in->n_particles < 1) return PIBM_EINVAL;
  if (cfg_in->precision != PIBM_FP64 || cfg_in->coupling != PIBM_IMPLICIT ||
      cfg_in->interp != PIBM_INTERP_DELTA || cfg_in->dem_model != PIBM_DEM_LINEAR ||
      cfg_in->dem_substeps > 1 || cfg_in->rebin_every > 1)
    return PIBM_ENOTSUP;
  pibm_config cfg = *cfg_in;
  cfg.deterministic = 1;  // replayed stretches reproduce the forward run bit for bit
  cudaStream_t st = (cudaStream_t)stream;
  HandleGuard hg;
  int rc = pibm_create(&cfg, nullptr, 0, stream, &hg.h);
  if (rc != PIBM_OK) return rc;
  HandleView v = handle_view(hg.h);
  State& s = *v.s;
  const long long np = s.p.np;
  const int d = s.geo.d, q = s.geo.q;
  const long long nseg = (nsteps + K - 1) / K;
  const size_t wsb = v.ws_bytes;
  const long long P = s.geo.pitch;
  const int FS = d == 2 ? 2 : 4;

  const bool grads = dtau || drho || dx0;
  Allocs al;
  char* ckpt = grads ? al.get<char>(wsb * (size_t)nseg) : nullptr;
  double* scal = al.get<double>(sizeof(double) * 4);
  if ((grads && !ckpt) || !scal) return PIBM_ENOMEM;

  auto fwd_step = [&](char* tape_slot) -> cudaError_t {
    cudaError_t e;
    if ((e = launch_bin(s, st, nullptr)) != cudaSuccess) return e;
    if ((e = launch_contacts(s, st, nullptr)) != cudaSuccess) return e;
    if ((e = launch_couple(s, st, nullptr)) != cudaSuccess) return e;
    if (tape_slot &&
        (e = cudaMemcpyAsync(tape_slot, v.ws, wsb, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
    if ((e = launch_collide_stream(s, st)) != cudaSuccess) return e;
    s.cur ^= 1;
    return cudaSuccess;
  };

  // forward sweep with checkpoints
  std::vector<int> par(nseg);
  for (long long sg = 0; sg < nseg; ++sg) {
    par[sg] = s.cur;
    if (grads &&
        cudaMemcpyAsync(ckpt + wsb * sg, v.ws, wsb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return PIBM_ECUDA;
    const long long n1 = sg == nseg - 1 ? nsteps : (sg + 1) * K;
    for (long long n = sg * K; n < n1; ++n)
      if (fwd_step(nullptr) != cudaSuccess) return PIBM_ECUDA;
  }
  k_mean_last<<<1, ADJ_THREADS, 0, st>>>(np, d, s.p.U[s.cur], scal);
  if (cudaMemcpyAsync(loss, scal, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PIBM_ECUDA;
  rc = pibm_status(hg.h);
  if (rc != PIBM_OK || !grads) return rc;

  char* tape = al.get<char>(wsb * (size_t)K);
  double* gbar = al.get<double>(sizeof(double) * q * P);
  double* fbar = al.get<double>(sizeof(double) * q * P);
  double* Fbar = al.get<double>(sizeof(double) * FS * P);
  double* rjbar = al.get<double>(sizeof(double) * 4 * P);
  double* om_part = al.get<double>(sizeof(double) * nblk(s.geo.ncell));
  double* pb[2][2] = {{al.get<double>(sizeof(double) * d * np), al.get<double>(sizeof(double) * d * np)},
                      {al.get<double>(sizeof(double) * d * np), al.get<double>(sizeof(double) * d * np)}};
  double* Xb_tmp = al.get<double>(sizeof(double) * d * np);
  double* Ub_tmp = al.get<double>(sizeof(double) * d * np);
  double* Fcb = al.get<double>(sizeof(double) * d * np);
  double* rlb = al.get<double>(sizeof(double) * np);
  double* jlb = al.get<double>(sizeof(double) * d * np);
  double* mb_tmp = al.get<double>(sizeof(double) * np);
  double* drho_d = al.get<double>(sizeof(double) * np);
  if (!tape || !gbar || !fbar || !Fbar || !rjbar || !om_part || !pb[0][0] || !pb[0][1] ||
      !pb[1][0] || !pb[1][1] || !Xb_tmp || !Ub_tmp || !Fcb || !rlb || !jlb || !mb_tmp || !drho_d)
    return PIBM_ENOMEM;
  // adjoint of the final state: d loss / d U_last = 1 / np
  int io = 0;  // pb[io] = adjoint of (X, U) of the state being reversed into
  if (cudaMemsetAsync(gbar, 0, sizeof(double) * q * P, st) != cudaSuccess ||
      cudaMemsetAsync(pb[io][0], 0, sizeof(double) * d * np, st) != cudaSuccess ||
      cudaMemsetAsync(pb[io][1], 0, sizeof(double) * d * np, st) != cudaSuccess ||
      cudaMemsetAsync(om_part, 0, sizeof(double) * nblk(s.geo.ncell), st) != cudaSuccess ||
      cudaMemsetAsync(drho_d, 0, sizeof(double) * np, st) != cudaSuccess)
    return PIBM_ECUDA;
  k_adj_seed<<<nblk(np), ADJ_THREADS, 0, st>>>(np, d, pb[io][1]);

  AdjArgs A{};
  A.g = s.geo;
  A.ph = s.phy;
  A.bm = s.p.bm;
  A.np = np;
  A.Fbar = Fbar;
  A.Xb_tmp = Xb_tmp;
  A.Ub_tmp = Ub_tmp;
  A.Fcb = Fcb;
  A.rlb = rlb;
  A.jlb = jlb;
  A.mb_tmp = mb_tmp;
  A.rjbar = rjbar;
  A.drho = drho_d;
  A.err = s.err;
  std::vector<int> step_par((size_t)K);
  for (long long sg = nseg - 1; sg >= 0; --sg) {
    // replay the stretch from its checkpoint, keeping the tape
    if (cudaMemcpyAsync(v.ws, ckpt + wsb * sg, wsb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return PIBM_ECUDA;
    s.cur = par[sg];
    const long long n0 = sg * K, n1 = sg == nseg - 1 ? nsteps : (sg + 1) * K;
    for (long long n = n0; n < n1; ++n) {
      step_par[n - n0] = s.cur;
      if (fwd_step(tape + wsb * (n - n0)) != cudaSuccess) return PIBM_ECUDA;
    }
    for (long long n = n1 - 1; n >= n0; --n) {
      State T = rebase_state(s, v.ws, tape + wsb * (n - n0));
      T.cur = step_par[n - n0];
      A.Xb_in = pb[io][0];
      A.Ub_in = pb[io][1];
      A.Xb_out = pb[1 - io][0];
      A.Ub_out = pb[1 - io][1];
      cudaError_t e = cudaErrorInvalidValue;
      if (q == 9) e = adjoint_step_w<9>(T, A, gbar, fbar, Fbar, om_part, st);
      else if (q == 15) e = adjoint_step_w<15>(T, A, gbar, fbar, Fbar, om_part, st);
      else if (q == 19) e = adjoint_step_w<19>(T, A, gbar, fbar, Fbar, om_part, st);
      if (e != cudaSuccess) return PIBM_ECUDA;
      io = 1 - io;
    }
  }
  k_sum_blocks<<<1, ADJ_THREADS, 0, st>>>(nblk(s.geo.ncell), om_part, scal + 1);
  double omb = 0.0;
  if (cudaMemcpyAsync(&omb, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIBM_ECUDA;
  // the initial storage order is the user order
  std::vector<double> xb((size_t)d * np);
  if (dx0 && cudaMemcpyAsync(xb.data(), pb[io][0], sizeof(double) * d * np,
                             cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIBM_ECUDA;
  if (drho && cudaMemcpyAsync(drho, drho_d, sizeof(double) * np, cudaMemcpyDeviceToHost, st) !=
                  cudaSuccess)
    return PIBM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIBM_ECUDA;
  if (dx0)
    for (long long i = 0; i < np; ++i)
      for (int k = 0; k < d; ++k) dx0[i * d + k] = xb[(size_t)k * np + i];
  // om = 1 / tau
  if (dtau) *dtau = -omb / (cfg.tau * cfg.tau);
  return pibm_status(hg.h);
}

}  // namespace pibm

extern "C" int pibm_settling_gradient(const pibm_config* cfg, int64_t nsteps,
                                      int64_t checkpoint_every, void* stream, double* loss,
                                      double* dtau, double* drho, double* dx0) {
  return pibm::settling_gradient(cfg, nsteps, checkpoint_every, stream, loss, dtau, drho, dx0);
}
