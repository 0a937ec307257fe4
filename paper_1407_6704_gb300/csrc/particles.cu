// Particle kernels: the cell list (counting sort of particles into lattice-cell
// bins) with its busy and free tile lists, the moment kernel over the busy
// tiles, the contact kernel, which sums the linear spring-dashpot (or Hertz)
// contact forces over the 3^d neighbouring bins (or the candidates recorded at
// the last rebuild) and the walls, and the coupled particle kernel, which for
// each particle
//   - interpolates the post-stream moments rho, j of the fluid with the per-axis
//     delta weights (Eq. 4 of the paper, the interpolant being the same kernel
//     as the spreading, Eqs. 10-11) or the Lagrange polynomials (Eq. 5),
//   - advances U and X (Eq. 13, with the drag implicit or explicit),
//   - forms the force density g = 2 (rho_l U - j_l) of the moving bounce-back
//     (Eqs. 6-7) and spreads A_p g back to the lattice (Eq. 9).
// Particle state is FP64 structure-of-arrays, double-buffered so that every
// contact reads the state of step n, and stored in cell-sorted order: the
// coupled kernel writes the new state at the particle's slot in the cell list.
#include "particles_device.cuh"

namespace pibm {

cudaError_t launch_bin(const State& s, cudaStream_t st, int* nk) {
  const Particles& P = s.p;
  if (P.np == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P.bin_cnt, 0, sizeof(unsigned) * (P.nbin + 1), st);
  if (e != cudaSuccess) return e;
  const double* X = P.X[s.cur];
  if (s.geo.d == 2)
    k_bin_key<2><<<blocks_for(P.np, 256), 256, 0, st>>>(X, P.np, s.geo, P.bm, P.cf[s.cur], P.key,
                                                        P.rank, P.bin_cnt, P.xr, P.cr);
  else
    k_bin_key<3><<<blocks_for(P.np, 256), 256, 0, st>>>(X, P.np, s.geo, P.bm, P.cf[s.cur], P.key,
                                                        P.rank, P.bin_cnt, P.xr, P.cr);
  const long long n = P.nbin + 1;
  k_scan_reduce<<<P.scan_blocks, SCAN_THREADS, 0, st>>>(P.bin_cnt, n, P.block_sums);
  k_scan_top<<<1, SCAN_THREADS, 0, st>>>(P.block_sums, P.scan_blocks);
  k_scan_down<<<P.scan_blocks, SCAN_THREADS, 0, st>>>(P.bin_cnt, n, P.block_sums);
  k_bin_scatter<<<blocks_for(P.np, 256), 256, 0, st>>>(P.key, P.rank, P.bin_cnt, P.np, P.xr,
                                                       P.cr, P.perm, P.xs[s.cur], P.cs[s.cur], P.xs0);
  if (nk) *nk += 5;
  if (s.deterministic) {
    // bins in storage order: every sum over a bin then runs in a fixed order
    k_bin_sort<<<blocks_for(P.np, 256), 256, 0, st>>>(P.key, P.rank, P.bin_cnt, P.np, P.xr,
                                                      P.cr, P.perm, P.xs[s.cur], P.cs[s.cur], P.xs0);
    if (nk) *nk += 1;
  }
  // the busy and free tile lists of this cell list
  const unsigned tb = (unsigned)((P.ntiles + TILE_BLOCK - 1) / TILE_BLOCK);
  if (s.geo.d == 2)
    k_tile_flags<2><<<tb, TILE_BLOCK, 0, st>>>(P.bin_cnt, P.bm, s.geo, P.ntiles, P.tflag, P.tblk);
  else
    k_tile_flags<3><<<tb, TILE_BLOCK, 0, st>>>(P.bin_cnt, P.bm, s.geo, P.ntiles, P.tflag, P.tblk);
  k_tile_lists<<<tb, TILE_BLOCK, 0, st>>>(P.tflag, P.tblk, P.ntiles, P.tbusy, P.tfree, P.tn);
  if (nk) *nk += 2;
  return cudaGetLastError();
}

namespace {

template <int Q, int W, class St, typename FT>
cudaError_t couple_t(const State& s, cudaStream_t st, int* nk, cudaEvent_t before_particles) {
  const Particles& P = s.p;
  constexpr int D = Lattice<Q>::D;
  using T = typename St::T;
  using R = typename St::R;
  CoupleArgs A = couple_args(s);
  const long long ntiles = P.nbin / P.bm.tc;
  constexpr int KT = MomentsShape<Q, St>::KT;
  const unsigned pb = blocks_for(P.np, 256);
  k_moments<Q, St><<<(unsigned)((ntiles + KT - 1) / KT), 256, 0, st>>>(
      s.geo, P.bm, P.tbusy, P.tn, (const T*)s.f[s.cur], (R*)s.mom);
  if (before_particles) {
    const cudaError_t e = cudaStreamWaitEvent(st, before_particles, 0);
    if (e != cudaSuccess) return e;
  }
  int n = 1;
  if (s.phy.substeps <= 1) {
    bool tiled = false;
    if constexpr (D == 3 && sizeof(R) == 4) {
      // 3D, FP32 arithmetic, delta interpolation, atomic spreading: by tiles
      if (!s.phy.lagrange && A.spread) {
        constexpr int TPC = CoupleWindow<D, W>::TPC;
        const long long groups = (P.ntiles + TPC - 1) / TPC;
        const unsigned grid = (unsigned)(groups * TILE_CHUNKS);
        if (s.phy.p64) k_couple_tiles<Q, W, St, FT, true><<<grid, 256, 0, st>>>(A);
        else k_couple_tiles<Q, W, St, FT, false><<<grid, 256, 0, st>>>(A);
        tiled = true;
      }
    }
    // 32- and 16-bit storage: the particle update in FP64 (P64) or FP32
    constexpr bool NARROW = sizeof(R) == 4;
    if (tiled) {
    } else if (s.phy.lagrange) {
      if (NARROW && s.phy.p64) k_couple<Q, W, St, FT, true, NARROW><<<pb, 256, 0, st>>>(A);
      else k_couple<Q, W, St, FT, true, false><<<pb, 256, 0, st>>>(A);
    } else {
      if (NARROW && s.phy.p64) k_couple<Q, W, St, FT, false, NARROW><<<pb, 256, 0, st>>>(A);
      else k_couple<Q, W, St, FT, false, false><<<pb, 256, 0, st>>>(A);
    }
    n += 1;
  } else {
    // DEM sub-cycling: interpolate once, S x (contacts, update), then spread
    if (s.phy.lagrange)
      k_sub_init<Q, 4, St, true><<<pb, 256, 0, st>>>(A);
    else
      k_sub_init<Q, W, St, false><<<pb, 256, 0, st>>>(A);
    const double h = 1.0 / (double)s.phy.substeps;
    // the first sub-step records the contact candidates, the others reuse them
    for (int k = 0; k < s.phy.substeps; ++k) {
      if (s.phy.hertz) {
        if (k == 0) k_contacts<D, true, true, 1><<<pb, 256, 0, st>>>(A);
        else k_contacts<D, true, true, 2><<<pb, 256, 0, st>>>(A);
      } else {
        if (k == 0) k_contacts<D, true, false, 1><<<pb, 256, 0, st>>>(A);
        else k_contacts<D, true, false, 2><<<pb, 256, 0, st>>>(A);
      }
      k_substep<D><<<pb, 256, 0, st>>>(A, h);
    }
    n += 1 + 2 * s.phy.substeps;
    if (A.spread) {
      k_sub_spread<Q, W, St, FT><<<pb, 256, 0, st>>>(A);
      n += 1;
    }
  }
  if (nk) *nk += n;
  if (s.deterministic) {
    const Geometry& g = s.geo;
    int bx = g.n[0] <= 32 ? 32 : (g.n[0] <= 64 ? 64 : 128);
    dim3 blk(bx, 256 / bx, 1);
    dim3 grd((g.n[0] + blk.x - 1) / blk.x, (g.n[1] + blk.y - 1) / blk.y, g.n[2]);
    constexpr int R0 = W == 2 ? 1 : 2;
    if (s.phy.rebin > 1)
      k_spread_gather<D, W, R0 + 1, FT><<<grd, blk, 0, st>>>(g, P.bm, P.np, P.ti, P.tw,
                                                             P.Ap[1 - s.cur], P.g, P.bin_cnt,
                                                             (FT*)s.F);
    else
      k_spread_gather<D, W, R0, FT><<<grd, blk, 0, st>>>(g, P.bm, P.np, P.ti, P.tw,
                                                         P.Ap[1 - s.cur], P.g, P.bin_cnt,
                                                         (FT*)s.F);
    if (nk) *nk += 1;
  }
  return cudaGetLastError();
}

template <int Q, class St, typename FT>
cudaError_t couple_w(const State& s, cudaStream_t st, int* nk, cudaEvent_t ev) {
  return s.phy.width == 2 ? couple_t<Q, 2, St, FT>(s, st, nk, ev)
                          : couple_t<Q, 4, St, FT>(s, st, nk, ev);
}
}  // namespace

namespace {
template <int D, bool HZ, bool HS>
void contacts_nb(const CoupleArgs& A, unsigned pb, cudaStream_t st) {
  if (A.nb_mode == 1) k_contacts<D, false, HZ, 1, HS><<<pb, 256, 0, st>>>(A);
  else if (A.nb_mode == 2) k_contacts<D, false, HZ, 2, HS><<<pb, 256, 0, st>>>(A);
  else k_contacts<D, false, HZ, 0, HS><<<pb, 256, 0, st>>>(A);
}
template <int D, bool HZ>
void contacts_hs(const CoupleArgs& A, bool hs, unsigned pb, cudaStream_t st) {
  if constexpr (D == 3) {
    if (hs) {
      contacts_nb<D, HZ, true>(A, pb, st);
      return;
    }
  }
  contacts_nb<D, HZ, false>(A, pb, st);
}
}  // namespace

cudaError_t launch_contacts(const State& s, cudaStream_t st, int* nk) {
  // with DEM sub-cycling the contacts run inside the particle phase, per sub-step
  if (s.p.np == 0 || s.phy.substeps > 1) return cudaSuccess;
  CoupleArgs A = couple_args(s);
  const unsigned pb = blocks_for(s.p.np, 256);
  const bool hs = contacts_half_shell(s);
  if (hs) {  // partner forces are added into the array: start from zero
    const cudaError_t e =
        cudaMemsetAsync(s.p.Fc, 0, sizeof(double) * s.geo.d * s.p.np, st);
    if (e != cudaSuccess) return e;
  }
  if (s.geo.d == 2) {
    if (s.phy.hertz) contacts_hs<2, true>(A, hs, pb, st);
    else contacts_hs<2, false>(A, hs, pb, st);
  } else {
    if (s.phy.hertz) contacts_hs<3, true>(A, hs, pb, st);
    else contacts_hs<3, false>(A, hs, pb, st);
  }
  if (nk) *nk += 1;
  return cudaGetLastError();
}

cudaError_t launch_couple(const State& s, cudaStream_t st, int* nk, cudaEvent_t ev) {
  if (s.p.np == 0) return cudaSuccess;
  const int q = s.geo.q;
  if (s.precision == PIBM_FP64) {
    if (q == 9) return couple_w<9, StoreF64, double>(s, st, nk, ev);
    if (q == 15) return couple_w<15, StoreF64, double>(s, st, nk, ev);
    if (q == 19) return couple_w<19, StoreF64, double>(s, st, nk, ev);
  } else if (s.precision == PIBM_FP32) {
    if (q == 9) return couple_w<9, StoreF32, float>(s, st, nk, ev);
    if (q == 15) return couple_w<15, StoreF32, float>(s, st, nk, ev);
    if (q == 19) return couple_w<19, StoreF32, float>(s, st, nk, ev);
  } else if (s.precision == PIBM_FP16) {
    if (q == 9) return couple_w<9, StoreF16, float>(s, st, nk, ev);
    if (q == 15) return couple_w<15, StoreF16, float>(s, st, nk, ev);
    if (q == 19) return couple_w<19, StoreF16, float>(s, st, nk, ev);
  } else if (s.precision == PIBM_BF16) {
    if (q == 9) return couple_w<9, StoreBF16, float>(s, st, nk, ev);
    if (q == 15) return couple_w<15, StoreBF16, float>(s, st, nk, ev);
    if (q == 19) return couple_w<19, StoreBF16, float>(s, st, nk, ev);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_particle_forces(const State& s, double* f_fpi, double* f_c, cudaStream_t st) {
  if (s.p.np == 0) return cudaSuccess;
  const Particles& P = s.p;
  k_forces<<<blocks_for(P.np, 256), 256, 0, st>>>(P.np, s.geo.d, P.Ap[s.cur], P.g, P.Fc,
                                                  P.pid[s.cur], f_fpi, f_c, s.err);
  return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(long long np, int d, const double* aos, double* soa,
                              cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  k_aos_to_soa<<<blocks_for(np, 256), 256, 0, st>>>(np, d, aos, soa);
  return cudaGetLastError();
}

cudaError_t launch_interleave(const State& s, const double* soa, double* aos, cudaStream_t st) {
  if (s.p.np == 0) return cudaSuccess;
  k_interleave<<<blocks_for(s.p.np, 256), 256, 0, st>>>(s.p.np, s.geo.d, soa, s.p.pid[s.cur],
                                                        aos, s.err);
  return cudaGetLastError();
}

cudaError_t launch_particle_momentum(const State& s, double* out_dev, cudaStream_t st) {
  // out_dev[0..d) = sum_p m_p U_p; s.red + 3 * PRED_BLOCKS... scratch after the fluid partials
  double* partial = s.red + 4 * 512;
  if (s.p.np == 0) {
    return cudaMemsetAsync(out_dev, 0, sizeof(double) * s.geo.d, st);
  }
  k_particle_momentum<<<PRED_BLOCKS, PRED_THREADS, 0, st>>>(s.p.np, s.geo.d, s.p.mass[s.cur],
                                                            s.p.U[s.cur], partial);
  k_particle_momentum_final<<<1, 32, 0, st>>>(s.geo.d, partial, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_particle_init(const State& s, cudaStream_t st) {
  if (s.p.np == 0) return cudaSuccess;
  const Particles& P = s.p;
  k_particle_init<<<blocks_for(P.np, 256), 256, 0, st>>>(P.np, s.geo.d, s.phy.kn, s.phy.beta,
                                                         P.rad[0], P.mass[0], P.Ap[0], P.buoy[0],
                                                         P.gw[0], P.cf[0], P.pid[0]);
  return cudaGetLastError();
}

}  // namespace pibm
