// Batched persistent step: many independent simulations (an ensemble of
// sedimentation runs with uneven lattices and particle counts) advanced by ONE
// cooperative kernel launch per group of steps, captured in a CUDA graph.
//
// The kernel runs every phase of the coupled step (cell list, contacts, moments,
// coupling, collision) for all members, phase after phase, with grid-wide
// barriers in between. Each phase is a list of work items: a group of 256
// particles, a chunk of the cell-list scan, a block of tiles, a group of busy
// tiles for the moment field, or a run of lattice cells. Items are numbered per
// member from an offset table (one per item kind), so one phase is a single
// range [0, total). Phases of even cost split it into contiguous shares per CTA;
// the contacts, the moment field and the coupling hand items out from a ticket
// counter. An item runs the same device function as the corresponding
// single-simulation kernel (particles_device.cuh, lbm_device.cuh), so a member
// advanced here follows exactly the arithmetic of the same simulation stepped on
// its own.
//
// Grid barriers wait with a limit (%globaltimer, plus a spin-count cap): a CTA
// that waits longer sets the barrier's abort word and returns, every other CTA
// returns at its next wait, and later launches return at once; the host reports
// PIBM_ETIMEOUT. The cooperative launch refuses a grid larger than what can be
// resident at once, so a barrier can only time out if a CTA fails to arrive.
#include <stdint.h>

#include <algorithm>
#include <array>
#include <new>
#include <vector>

#include "lbm_device.cuh"
#include "particles_device.cuh"

namespace pibm {

namespace {

constexpr int ENS_THREADS = 256;

// Item kinds of the persistent kernel's phases.
enum : int {
  IK_PART = 0,  // 256 particles (cell-list slots or storage positions)
  IK_SCAN,      // ENS_THREADS * SCAN_PER_THREAD counts of the cell-list scan
  IK_TBLK,      // TILE_BLOCK tiles (tile flags and lists)
  IK_CELL,      // cells_per_item consecutive lattice cells (collision)
  IK_GATH,      // 256 consecutive lattice cells (ordered spreading, deterministic members)
  IK_N
};

// What the persistent kernel needs of a member beyond the coupling arguments.
struct EnsExtra {
  void* fout[2];  // f[1 - cur] for cur = 0, 1
  unsigned* key;
  unsigned* rank;
  unsigned* bsum;
  float4* xr;
  int4* cr;
  int* tflag;
  int* tbusy;
  int* tfree;
  unsigned* tblk;
  unsigned* tn;
  long long ntiles;
  int rebin;
  int det;        // deterministic (ordered spreading)
  int ncitems;    // collision items of this member (the count clear is split over them)
  int pad;
};

struct EnsMember {
  CoupleArgs A[2];  // coupling arguments with the current buffer 0 and 1
  EnsExtra x;
};

struct GridBarrier {
  unsigned count;   // CTAs arrived at the current barrier
  unsigned gen;     // barriers completed
  unsigned abort;   // 1 once a wait gave up
  unsigned where;   // 1 + index (within its launch) of the barrier that gave up
  unsigned ticket;  // next work item of a dynamically scheduled phase (reset at every barrier)
  unsigned pad[3];
};

struct EnsParams {
  const EnsMember* mem;
  const int* off;    // [IK_N][nm + 1] item offsets, by position
  const int* ord;    // [IK_N][nm] member at each position
  int* cur;          // [nm] buffer of the current state at the launch's first step
  int* sr;           // [nm] steps since the last cell-list rebuild, same time
  GridBarrier* bar;
  unsigned long long limit_ns;
  int nm;
  int nsteps;
  int cpi;           // cells per collision item
  int skip_arrive;   // fault injection for tests: this CTA skips the first barrier (-1: none)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned BARRIER_SPIN_CAP = 1u << 26;  // with a 100 ns sleep: several seconds

// Grid-wide barrier with a bounded wait. Returns false when this CTA's wait gave
// up (limit reached: the abort word is set) or another CTA's did; the caller then
// returns. arrive = false (test hook only) waits without arriving.
__device__ bool grid_sync(GridBarrier* b, unsigned nblocks, unsigned long long limit_ns,
                          unsigned where, bool arrive = true) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    const unsigned g0 = ld_acquire_u32(&b->gen);
    __threadfence();
    bool last = false;
    if (arrive) {
      last = atomicAdd(&b->count, 1u) + 1u == nblocks;
      if (last) {
        atomicExch(&b->count, 0u);
        atomicExch(&b->ticket, 0u);  // every CTA has finished taking items
        __threadfence();
        atomicAdd(&b->gen, 1u);
      }
    }
    if (!last) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&b->gen) == g0) {
        if (ld_acquire_u32(&b->abort)) {
          good = 0;
          break;
        }
        ++spins;
        if (spins >= BARRIER_SPIN_CAP || ((spins & 15u) == 0 && global_ns() - t0 > limit_ns)) {
          if (atomicExch(&b->abort, 1u) == 0u) b->where = where;
          good = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Position of item i in the offset table o[0..nm]: the largest a with o[a] <= i.
__device__ __forceinline__ int item_pos(const int* o, int nm, long long i) {
  int a = 0, b = nm;
  while (b - a > 1) {
    const int mid = (a + b) >> 1;
    if (__ldg(o + mid) <= i) a = mid;
    else b = mid;
  }
  return a;
}

// Static schedule: the CTA's share [lo, hi) of the items of one kind, walked in
// order; fn(m, i) runs item i of member m. CTA-uniform. For phases whose items
// cost about the same.
template <class Fn>
__device__ __forceinline__ void for_items(const EnsParams& E, int kind, Fn&& fn) {
  const int* o = E.off + kind * (E.nm + 1);
  const int* ord = E.ord + kind * E.nm;
  const long long total = __ldg(o + E.nm);
  if (total == 0) return;
  const long long lo = (long long)blockIdx.x * total / gridDim.x;
  const long long hi = (long long)(blockIdx.x + 1) * total / gridDim.x;
  if (lo >= hi) return;
  int pos = item_pos(o, E.nm, lo);
  long long next = __ldg(o + pos + 1);
  for (long long i = lo; i < hi; ++i) {
    while (i >= next) next = __ldg(o + (++pos) + 1);
    fn(__ldg(ord + pos), (int)(i - __ldg(o + pos)));
  }
}

// Largest a in [0, n) with o[a] <= i, o in shared memory.
__device__ __forceinline__ int item_pos_shared(const int* o, int n, long long i) {
  int a = 0, b = n;
  while (b - a > 1) {
    const int mid = (a + b) >> 1;
    if (o[mid] <= i) a = mid;
    else b = mid;
  }
  return a;
}

// Exclusive sum of v over the NT threads of the CTA; sm: 33 words.
template <int NT>
__device__ __forceinline__ int block_exclusive_sum(int v, unsigned* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) sm[wid] = (unsigned)incl;
  __syncthreads();
  int base = 0;
  for (int w = 0; w < wid; ++w) base += (int)sm[w];
  __syncthreads();
  return base + incl - v;
}

// Dynamic schedule: each CTA takes the next ticket t < total from the barrier's
// counter (the following ticket is fetched while item t runs) and runs fn(t), so
// items of uneven cost spread over the CTAs. CTA-uniform. The counter is reset
// at every barrier, so one phase holds at most one such loop.
template <class Fn>
__device__ __forceinline__ void for_tickets(GridBarrier* bar, long long total, Fn&& fn) {
  __shared__ unsigned s_t[2];
  unsigned* ctr = &bar->ticket;
  __syncthreads();  // s_t may still be read from the previous phase
  if (threadIdx.x == 0) s_t[0] = atomicAdd(ctr, 1u);
  __syncthreads();
  int buf = 0;
  long long t = s_t[0];
  while (t < total) {
    if (threadIdx.x == 0) s_t[buf ^ 1] = atomicAdd(ctr, 1u);
    fn(t);
    __syncthreads();
    buf ^= 1;
    t = s_t[buf];
  }
}

template <int Q, class St>
struct EnsShape {
  // CTAs per SM the kernel is compiled for: 64 registers in FP32 (measured
  // faster than 80 on the 64-member workload, every phase), 128 in FP64 (the
  // FP64 coupling needs them)
  static constexpr int MINB = sizeof(typename St::R) == 4 ? 4 : 2;
};

// The persistent kernel: E.nsteps steps of every member.
template <int Q, int W, class St, typename FT>
__global__ void __launch_bounds__(ENS_THREADS, EnsShape<Q, St>::MINB) k_ensemble(EnsParams E) {
  using T = typename St::T;
  using R = typename St::R;
  using L = Lattice<Q>;
  constexpr int D = L::D;
  constexpr int R0 = W == 2 ? 1 : 2;  // ordered spreading reach (cells)
  // FP32 members update their particles in FP64 (the default particle_update)
  constexpr bool P64 = sizeof(R) == 4;
  __shared__ CoupleArgs sA;
  __shared__ EnsExtra sX;
  __shared__ int s_key;
  __shared__ unsigned s_scan[33];
  // [nm] parity, [nm] rebuild phase, [nm] period, [nm] np > 0, [nm + 1] moment items
  extern __shared__ int s_dyn[];
  int* s_cur = s_dyn;
  int* s_sr = s_dyn + E.nm;
  int* s_rb = s_dyn + 2 * E.nm;
  int* s_np = s_dyn + 3 * E.nm;
  int* s_moff = s_dyn + 4 * E.nm;
  GridBarrier* bar = E.bar;
  if (ld_acquire_u32(&bar->abort)) return;  // a barrier of an earlier launch gave up
  for (int m = threadIdx.x; m < E.nm; m += ENS_THREADS) {
    s_cur[m] = E.cur[m];
    s_sr[m] = E.sr[m];
    s_rb[m] = E.mem[m].x.rebin;
    s_np[m] = E.mem[m].A[0].np > 0;
  }
  if (threadIdx.x == 0) s_key = -1;
  __syncthreads();
  unsigned where = 0;
  bool table_done = false;
  // barrier between phases; after the first one every CTA has read the phase
  // table, so CTA 0 advances it to the state after this launch
  auto sync = [&]() -> bool {
    ++where;
    const bool arrive = !(E.skip_arrive >= 0 && (int)blockIdx.x == E.skip_arrive && where == 1);
    if (!grid_sync(bar, gridDim.x, E.limit_ns, where, arrive)) return false;
    if (!table_done) {
      table_done = true;
      if (blockIdx.x == 0)
        for (int m = threadIdx.x; m < E.nm; m += ENS_THREADS) {
          E.cur[m] = s_cur[m] ^ (E.nsteps & 1);
          E.sr[m] = (int)((s_sr[m] + (long long)E.nsteps) % s_rb[m]);
        }
    }
    return true;
  };
  auto phase_of = [&](int m, int k) { return (int)((s_sr[m] + (long long)k) % s_rb[m]); };
  // make sA / sX the arguments of member m at step k (CTA-uniform)
  auto use = [&](int m, int k) {
    const int key = k * 1024 + m;
    if (s_key == key) return;
    __syncthreads();
    const int cur = s_cur[m] ^ (k & 1);
    const unsigned* src = reinterpret_cast<const unsigned*>(&E.mem[m].A[cur]);
    unsigned* dst = reinterpret_cast<unsigned*>(&sA);
    for (int i = threadIdx.x; i < (int)(sizeof(CoupleArgs) / 4); i += ENS_THREADS)
      dst[i] = __ldg(src + i);
    const unsigned* srx = reinterpret_cast<const unsigned*>(&E.mem[m].x);
    unsigned* dsx = reinterpret_cast<unsigned*>(&sX);
    for (int i = threadIdx.x; i < (int)(sizeof(EnsExtra) / 4); i += ENS_THREADS)
      dsx[i] = __ldg(srx + i);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int ph = phase_of(m, k);
      if (sX.rebin > 1) {  // kept cell list: candidates recorded on a rebuild, reused after
        sA.nb_mode = ph == 0 ? 1 : 2;
        sA.move_consts = ph <= 1;
      }
      s_key = key;
    }
    __syncthreads();
  };
  const int tid = threadIdx.x;

  for (int k = 0; k < E.nsteps; ++k) {
    int any = 0;
    for (int m = tid; m < E.nm; m += ENS_THREADS) any |= s_np[m] && phase_of(m, k) == 0;
    any = __syncthreads_or(any);
    auto rebuilds = [&](int m) { return s_np[m] && phase_of(m, k) == 0; };

    if (any) {
      // cell list: bin of every particle and arrival rank (counts are zero on entry)
      for_items(E, IK_PART, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        bin_key_at<D>(sA.X, sA.np, sA.g, sA.bm, sA.cf, sX.key, sX.rank, (unsigned*)sA.start,
                      sX.xr, sX.cr, (long long)it * ENS_THREADS + tid);
      });
      if (!sync()) return;
      for_items(E, IK_SCAN, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        scan_reduce_chunk<ENS_THREADS>(sA.start, sA.nbin + 1, it, sX.bsum, s_scan);
      });
      if (!sync()) return;
      for_items(E, IK_SCAN, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        scan_down_chunk_self<ENS_THREADS>((unsigned*)sA.start, sA.nbin + 1, it, sX.bsum, s_scan);
      });
      if (!sync()) return;
      for_items(E, IK_PART, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        bin_scatter_at(sX.key, sX.rank, sA.start, sA.np, sX.xr, sX.cr, (unsigned*)sA.perm,
                       (float4*)sA.xs, (int4*)sA.cs, (float4*)sA.xs0,
                       (long long)it * ENS_THREADS + tid);
      });
      for_items(E, IK_TBLK, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        tile_flags_block<D>(sA.start, sA.bm, sA.g, sX.ntiles, sX.tflag, sX.tblk, it);
      });
      if (!sync()) return;
      for_items(E, IK_TBLK, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        tile_lists_block(sX.tflag, sX.tblk, sX.ntiles, sX.tbusy, sX.tfree, sX.tn, it);
      });
      for_items(E, IK_PART, [&](int m, int it) {
        if (!rebuilds(m)) return;
        use(m, k);
        if (!sX.det) return;
        bin_sort_at(sX.key, sX.rank, sA.start, sA.np, sX.xr, sX.cr, (unsigned*)sA.perm,
                    (float4*)sA.xs, (int4*)sA.cs, (float4*)sA.xs0,
                    (long long)it * ENS_THREADS + tid);
      });
      if (!sync()) return;
    }

    // contact forces and the moment field of the busy tiles, one dynamic schedule
    // (costs are uneven): first the particle items, the densest members first,
    // then the moment items, numbered over each member's busy tiles (KT per item;
    // every CTA forms the same prefix of the members' busy-tile counts)
    {
      constexpr int KT = MomentsShape<Q, St>::KT;
      int cnt = 0;
      if (tid < E.nm && s_np[tid]) cnt = (int)((*E.mem[tid].x.tn + KT - 1) / KT);
      const int excl = block_exclusive_sum<ENS_THREADS>(cnt, s_scan);
      if (tid < E.nm) s_moff[tid] = excl;
      if (tid == ENS_THREADS - 1) s_moff[E.nm] = excl + cnt;
      __syncthreads();
      const long long tp = __ldg(E.off + IK_PART * (E.nm + 1) + E.nm);
      for_tickets(E.bar, tp + s_moff[E.nm], [&](long long t) {
        if (t < tp) {
          const int* o = E.off + IK_PART * (E.nm + 1);
          const int pos = item_pos(o, E.nm, t);
          use(__ldg(E.ord + IK_PART * E.nm + pos), k);
          const long long sl = (t - __ldg(o + pos)) * ENS_THREADS + tid;
          if (sA.nb_mode == 1) contacts_at<D, false, false, 1>(sA, sl);
          else if (sA.nb_mode == 2) contacts_at<D, false, false, 2>(sA, sl);
          else contacts_at<D, false, false, 0>(sA, sl);
        } else {
          const long long i = t - tp;
          const int m = item_pos_shared(s_moff, E.nm, i);
          // the arguments by value: stores to the moment field could alias a
          // struct read in place, which would force reloads of every field
          const CoupleArgs& Am = E.mem[m].A[s_cur[m] ^ (k & 1)];
          const Geometry g = Am.g;
          const BinMap bm = Am.bm;
          const T* f = (const T*)Am.f;
          R* mom = (R*)Am.mom;
          const int* tbusy = E.mem[m].x.tbusy;
          const unsigned* tn = E.mem[m].x.tn;
          moments_block<Q, St>(g, bm, tbusy, tn, f, mom, (int)(i - s_moff[m]));
        }
      });
    }
    if (!sync()) return;
    // interpolation, particle update, spreading
    {
      const int* o = E.off + IK_PART * (E.nm + 1);
      for_tickets(E.bar, __ldg(o + E.nm), [&](long long t) {
        const int pos = item_pos(o, E.nm, t);
        use(__ldg(E.ord + IK_PART * E.nm + pos), k);
        couple_at<Q, W, St, FT, false, false, P64>(sA, (t - __ldg(o + pos)) * ENS_THREADS + tid);
      });
    }
    if (!sync()) return;
    // ordered spreading of the deterministic members
    if (__ldg(E.off + IK_GATH * (E.nm + 1) + E.nm) > 0) {
      for_items(E, IK_GATH, [&](int m, int it) {
        use(m, k);
        const long long c = (long long)it * ENS_THREADS + tid;
        if (c >= sA.g.ncell) return;
        const int x = (int)(c % sA.g.n[0]);
        const long long r = c / sA.g.n[0];
        const int y = (int)(r % sA.g.n[1]), z = (int)(r / sA.g.n[1]);
        if (sX.rebin > 1)
          spread_gather_at<D, W, R0 + 1, FT>(sA.g, sA.bm, sA.np, sA.ti, sA.tw, sA.Apn, sA.gout,
                                             sA.start, (FT*)sA.F, x, y, z);
        else
          spread_gather_at<D, W, R0, FT>(sA.g, sA.bm, sA.np, sA.ti, sA.tw, sA.Apn, sA.gout,
                                         sA.start, (FT*)sA.F, x, y, z);
      });
      if (!sync()) return;
    }
    // collision; clear the cell-list counts of members that rebuild next step
    for_items(E, IK_CELL, [&](int m, int it) {
      use(m, k);
      const int cur = s_cur[m] ^ (k & 1);
      const long long c0 = (long long)it * E.cpi;
      const long long ncell = sA.g.ncell;
      const long long c1 = c0 + E.cpi < ncell ? c0 + E.cpi : ncell;
      const unsigned n0 = (unsigned)sA.g.n[0], n1 = (unsigned)sA.g.n[1];
      const int* flag = s_np[m] ? sX.tflag : nullptr;
      using TD = TileDims<D>;
      // the thread's cells c0 + tid + 256 j; (x, y, z) of the first by division
      // (ncell < 2^31), then stepped along x with carries into y and z
      unsigned r0 = (unsigned)(c0 + tid) / n0;
      int x = (int)((unsigned)(c0 + tid) - r0 * n0), y = (int)(r0 % n1), z = (int)(r0 / n1);
      for (long long c = c0 + tid; c < c1; c += ENS_THREADS) {
        const unsigned cu = (unsigned)c;
        // no particle stencil reaches a cell of a free tile of the cell list, so
        // its force is zero and stays untouched (as in the single-simulation
        // step's free-tile collision)
        const bool busy =
            flag && flag[x / TD::TX + sA.bm.nt[0] * (y / TD::TY + sA.bm.nt[1] * (z / TD::TZ))];
        R sv[Q], Fv[3] = {R(0), R(0), R(0)};
        pull_cell<Q, St>((const T*)sA.f, sA.g, x, y, z, sv);
        if (busy) take_force<D, FT, R>((FT*)sA.F, (long long)cu, Fv);
        collide_store<Q, St>((T*)sX.fout[cur], sA.g, (long long)cu, sv, Fv, (R)sA.ph.omega,
                             (R)sA.ph.cF, sA.err);
        x += ENS_THREADS;
        while (x >= (int)n0) {
          x -= (int)n0;
          if (++y == (int)n1) {
            y = 0;
            ++z;
          }
        }
      }
      if (s_np[m] && phase_of(m, k + 1) == 0) {
        const long long n = sA.nbin + 1;
        const long long per = (n + sX.ncitems - 1) / sX.ncitems;
        unsigned* cnt = (unsigned*)sA.start;
        for (long long i = it * per + tid; i < (it + 1) * per && i < n; i += ENS_THREADS)
          cnt[i] = 0u;
      }
    });
    if (k + 1 < E.nsteps && !sync()) return;
  }
  // every step has at least two phase barriers, so the phase table was advanced
}

// Barrier self-test: nbar grid barriers; CTA skip (>= 0) does not arrive at the
// first one, so every CTA's wait runs out and the kernel returns.
__global__ void __launch_bounds__(ENS_THREADS) k_barrier_test(GridBarrier* b, int nbar, int skip,
                                                              unsigned long long limit_ns,
                                                              unsigned* passed) {
  for (int i = 0; i < nbar; ++i) {
    const bool arrive = !(i == 0 && (int)blockIdx.x == skip);
    if (!grid_sync(b, gridDim.x, limit_ns, (unsigned)i + 1, arrive)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *passed = (unsigned)nbar;
}

using KernelFn = void (*)(EnsParams);

KernelFn pick_kernel(int precision, int width) {
  if (precision == PIBM_FP32)
    return width == 2 ? k_ensemble<9, 2, StoreF32, float> : k_ensemble<9, 4, StoreF32, float>;
  if (precision == PIBM_FP64)
    return width == 2 ? k_ensemble<9, 2, StoreF64, double> : k_ensemble<9, 4, StoreF64, double>;
  return nullptr;
}

cudaError_t launch_coop(const void* fn, unsigned grid, size_t smem, cudaStream_t st, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(ENS_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct EnsembleDevice {
  int nm = 0;
  int precision = 0, width = 0;
  KernelFn fn = nullptr;
  int sms = 0, max_per_sm = 0;
  int per_sm = 0;  // CTAs per SM of the launch
  int cpi = 1024;  // cells per collision item
  size_t smem = 0;
  unsigned long long limit_ns = 1000000000ull;
  std::vector<const State*> st;
  char* dev = nullptr;  // one allocation: members, offsets, phase table, barrier
  EnsMember* mem = nullptr;
  int* off = nullptr;
  int* ord = nullptr;
  int* cur = nullptr;
  int* sr = nullptr;
  GridBarrier* bar = nullptr;
  int any_gather = 0;
  int skip = -1;  // test hook: CTA that skips the first barrier of the next launch
};

namespace {

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

void fill_member(const State& s, EnsMember& em, int cpi) {
  for (int c = 0; c < 2; ++c) {
    State t = s;
    t.cur = c;
    t.nb_mode = 0;
    t.move_consts = 1;
    em.A[c] = couple_args(t);
  }
  const Particles& P = s.p;
  EnsExtra& x = em.x;
  x.fout[0] = s.f[1];
  x.fout[1] = s.f[0];
  x.key = P.key;
  x.rank = P.rank;
  x.bsum = P.block_sums;
  x.xr = P.xr;
  x.cr = P.cr;
  x.tflag = P.tflag;
  x.tbusy = P.tbusy;
  x.tfree = P.tfree;
  x.tblk = P.tblk;
  x.tn = P.tn;
  x.ntiles = P.ntiles;
  x.rebin = s.phy.rebin > 0 ? s.phy.rebin : 1;
  x.det = s.deterministic ? 1 : 0;
  x.ncitems = (int)ceil_div(s.geo.ncell, cpi);
  x.pad = 0;
}

// Item counts of member s by kind.
void member_items(const State& s, int cpi, long long (&n)[IK_N]) {
  const Particles& P = s.p;
  const bool part = P.np > 0;
  n[IK_PART] = part ? ceil_div(P.np, ENS_THREADS) : 0;
  n[IK_SCAN] = part ? ceil_div(P.nbin + 1, ENS_THREADS * SCAN_PER_THREAD) : 0;
  n[IK_TBLK] = part ? ceil_div(P.ntiles, TILE_BLOCK) : 0;
  n[IK_CELL] = ceil_div(s.geo.ncell, cpi);
  n[IK_GATH] = (part && s.deterministic) ? ceil_div(s.geo.ncell, ENS_THREADS) : 0;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

bool ensemble_persistent_supported(const State* const* s, int n) {
  if (n <= 0 || n > ENSEMBLE_PERSISTENT_MAX) return false;
  for (int i = 0; i < n; ++i) {
    const State& a = *s[i];
    if (a.geo.q != 9 || (a.precision != PIBM_FP32 && a.precision != PIBM_FP64)) return false;
    if (a.phy.lagrange || a.phy.hertz || a.phy.substeps > 1) return false;
    if (a.precision != s[0]->precision || a.phy.width != s[0]->phy.width) return false;
    if (a.geo.ncell > INT_MAX || a.p.np > INT_MAX) return false;
    if (a.precision == PIBM_FP32 && !a.phy.p64) return false;  // built for the FP64 update
  }
  return pick_kernel(s[0]->precision, s[0]->phy.width) != nullptr;
}

static cudaError_t write_tables(EnsembleDevice* e, cudaStream_t st) {
  std::vector<EnsMember> mem(e->nm);
  std::vector<int> off((size_t)IK_N * (e->nm + 1), 0), ord((size_t)IK_N * e->nm);
  std::vector<std::array<long long, IK_N>> items(e->nm);
  for (int i = 0; i < e->nm; ++i) {
    fill_member(*e->st[i], mem[i], e->cpi);
    long long n[IK_N];
    member_items(*e->st[i], e->cpi, n);
    for (int k = 0; k < IK_N; ++k) items[i][k] = n[k];
  }
  // particle items in order of falling particle density (contact candidates per
  // particle grow with it), the other kinds in member order
  std::vector<int> dense(e->nm);
  for (int i = 0; i < e->nm; ++i) dense[i] = i;
  std::stable_sort(dense.begin(), dense.end(), [&](int a, int b) {
    const State& A = *e->st[a];
    const State& B = *e->st[b];
    return (double)A.p.np / (double)A.geo.ncell > (double)B.p.np / (double)B.geo.ncell;
  });
  long long tot[IK_N] = {};
  for (int k = 0; k < IK_N; ++k)
    for (int pos = 0; pos < e->nm; ++pos) {
      const int i = k == IK_PART ? dense[pos] : pos;
      ord[(size_t)k * e->nm + pos] = i;
      off[(size_t)k * (e->nm + 1) + pos] = (int)tot[k];
      tot[k] += items[i][k];
    }
  for (int k = 0; k < IK_N; ++k) {
    if (tot[k] > INT_MAX) return cudaErrorInvalidValue;
    off[(size_t)k * (e->nm + 1) + e->nm] = (int)tot[k];
  }
  e->any_gather = tot[IK_GATH] > 0;
  cudaError_t r = cudaMemcpyAsync(e->mem, mem.data(), sizeof(EnsMember) * e->nm,
                                  cudaMemcpyHostToDevice, st);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(e->off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, st);
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(e->ord, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice, st);
  // the vectors are pageable: the copies are staged before the calls return
  return r;
}

int ensemble_device_create(const State* const* s, int n, int device, EnsembleDevice** out) {
  *out = nullptr;
  if (!ensemble_persistent_supported(s, n)) return PIBM_ENOTSUP;
  EnsembleDevice* e = new (std::nothrow) EnsembleDevice();
  if (!e) return PIBM_ENOMEM;
  e->nm = n;
  e->st.assign(s, s + n);
  e->precision = s[0]->precision;
  e->width = s[0]->phy.width;
  e->fn = pick_kernel(e->precision, e->width);
  e->smem = sizeof(int) * (5 * (size_t)n + 1);
  cudaError_t r = cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, device);
  if (r == cudaSuccess)
    r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e->max_per_sm, (const void*)e->fn,
                                                      ENS_THREADS, e->smem);
  if (r != cudaSuccess || e->max_per_sm < 1) {
    record_cuda_error("ensemble occupancy", r);
    delete e;
    return PIBM_ECUDA;
  }
  e->per_sm = e->max_per_sm;
  const size_t b_mem = align256(sizeof(EnsMember) * n);
  const size_t b_off = align256(sizeof(int) * IK_N * (size_t)(n + 1)) +
                       align256(sizeof(int) * IK_N * (size_t)n);
  const size_t b_tab = align256(sizeof(int) * 2 * (size_t)n);
  const size_t b_bar = align256(sizeof(GridBarrier));
  if ((r = cudaMalloc(&e->dev, b_mem + b_off + b_tab + b_bar)) != cudaSuccess) {
    record_cuda_error("cudaMalloc (ensemble tables)", r);
    delete e;
    return PIBM_ENOMEM;
  }
  e->mem = reinterpret_cast<EnsMember*>(e->dev);
  e->off = reinterpret_cast<int*>(e->dev + b_mem);
  e->ord = reinterpret_cast<int*>(e->dev + b_mem + align256(sizeof(int) * IK_N * (size_t)(n + 1)));
  e->cur = reinterpret_cast<int*>(e->dev + b_mem + b_off);
  e->sr = e->cur + n;
  e->bar = reinterpret_cast<GridBarrier*>(e->dev + b_mem + b_off + b_tab);
  if ((r = cudaMemset(e->bar, 0, sizeof(GridBarrier))) != cudaSuccess ||
      (r = write_tables(e, 0)) != cudaSuccess || (r = cudaStreamSynchronize(0)) != cudaSuccess) {
    record_cuda_error("ensemble tables", r);
    ensemble_device_destroy(e);
    return PIBM_ECUDA;
  }
  *out = e;
  return PIBM_OK;
}

void ensemble_device_destroy(EnsembleDevice* e) {
  if (!e) return;
  if (e->dev) cudaFree(e->dev);
  delete e;
}

int ensemble_device_configure(EnsembleDevice* e, int per_sm, int cpi, cudaStream_t st) {
  if (per_sm < 0 || per_sm > e->max_per_sm || cpi < 0 || cpi % ENS_THREADS != 0)
    return PIBM_EINVAL;
  e->per_sm = per_sm > 0 ? per_sm : e->max_per_sm;
  if (cpi > 0 && cpi != e->cpi) {
    e->cpi = cpi;
    const cudaError_t r = write_tables(e, st);
    if (r != cudaSuccess) {
      record_cuda_error("ensemble tables", r);
      return PIBM_ECUDA;
    }
  }
  return PIBM_OK;
}

void ensemble_device_shape(const EnsembleDevice* e, int* per_sm, int* max_per_sm, int* cpi,
                           int* grid) {
  if (per_sm) *per_sm = e->per_sm;
  if (max_per_sm) *max_per_sm = e->max_per_sm;
  if (cpi) *cpi = e->cpi;
  if (grid) *grid = e->per_sm * e->sms;
}

cudaError_t ensemble_device_set_phase(EnsembleDevice* e, const int* cur, const int* sr,
                                      cudaStream_t st) {
  std::vector<int> t(2 * (size_t)e->nm);
  for (int i = 0; i < e->nm; ++i) {
    t[i] = cur[i];
    t[e->nm + i] = sr[i];
  }
  cudaError_t r = cudaMemcpyAsync(e->cur, t.data(), sizeof(int) * t.size(),
                                  cudaMemcpyHostToDevice, st);
  // the kernel expects zero counts for a member whose next step rebuilds
  for (int i = 0; i < e->nm && r == cudaSuccess; ++i) {
    const State& s = *e->st[i];
    if (s.p.np > 0 && sr[i] == 0)
      r = cudaMemsetAsync(s.p.bin_cnt, 0, sizeof(unsigned) * (s.p.nbin + 1), st);
  }
  return r;
}

cudaError_t ensemble_device_launch(EnsembleDevice* e, int nsteps, cudaStream_t st) {
  EnsParams p;
  p.mem = e->mem;
  p.off = e->off;
  p.ord = e->ord;
  p.cur = e->cur;
  p.sr = e->sr;
  p.bar = e->bar;
  p.limit_ns = e->limit_ns;
  p.nm = e->nm;
  p.nsteps = nsteps;
  p.cpi = e->cpi;
  p.skip_arrive = e->skip;
  e->skip = -1;
  void* args[] = {&p};
  return launch_coop((const void*)e->fn, (unsigned)(e->per_sm * e->sms), e->smem, st, args);
}

int ensemble_device_inject(EnsembleDevice* e, int block, double limit_s) {
  if (block < 0 || block >= e->per_sm * e->sms || !(limit_s > 0.0) || limit_s > 10.0)
    return PIBM_EINVAL;
  e->skip = block;
  e->limit_ns = (unsigned long long)(limit_s * 1e9);
  return PIBM_OK;
}

bool ensemble_device_injected(const EnsembleDevice* e) { return e->skip >= 0; }

int ensemble_device_timed_out(EnsembleDevice* e, cudaStream_t st, unsigned* where) {
  GridBarrier b;
  cudaError_t r = cudaMemcpyAsync(&b, e->bar, sizeof(b), cudaMemcpyDeviceToHost, st);
  if (r == cudaSuccess) r = cudaStreamSynchronize(st);
  if (r != cudaSuccess) {
    record_cuda_error("ensemble barrier state", r);
    return -1;
  }
  if (where) *where = b.where;
  return b.abort != 0;
}

}  // namespace pibm

extern "C" int pibm_grid_barrier_test(int nblocks, int skip_block, int nbarriers, double limit_s,
                                      int* passed) {
  using namespace pibm;
  if (nblocks < 1 || nbarriers < 1 || skip_block >= nblocks || !(limit_s > 0.0) ||
      limit_s > 10.0 || !passed)
    return PIBM_EINVAL;
  *passed = 0;
  int dev = 0, sms = 0, per = 0;
  cudaError_t r = cudaGetDevice(&dev);
  if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (r == cudaSuccess)
    r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_barrier_test, ENS_THREADS, 0);
  if (r != cudaSuccess) {
    record_cuda_error("barrier test setup", r);
    return PIBM_ECUDA;
  }
  if ((long long)nblocks > (long long)sms * per) return PIBM_EINVAL;  // not co-resident
  char* buf = nullptr;
  if ((r = cudaMalloc(&buf, 256 + sizeof(unsigned))) != cudaSuccess) {
    record_cuda_error("cudaMalloc (barrier test)", r);
    return PIBM_ENOMEM;
  }
  GridBarrier* b = reinterpret_cast<GridBarrier*>(buf);
  unsigned* pass = reinterpret_cast<unsigned*>(buf + 256);
  int rc = PIBM_OK;
  GridBarrier hb = {};
  unsigned hp = 0;
  unsigned long long lim = (unsigned long long)(limit_s * 1e9);
  int nbar = nbarriers;
  void* args[] = {&b, &nbar, &skip_block, &lim, &pass};
  if ((r = cudaMemset(buf, 0, 256 + sizeof(unsigned))) != cudaSuccess ||
      (r = launch_coop((const void*)k_barrier_test, (unsigned)nblocks, 0, 0, args)) !=
          cudaSuccess ||
      (r = cudaDeviceSynchronize()) != cudaSuccess ||
      (r = cudaMemcpy(&hb, b, sizeof(hb), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (r = cudaMemcpy(&hp, pass, sizeof(hp), cudaMemcpyDeviceToHost)) != cudaSuccess) {
    record_cuda_error("barrier test", r);
    rc = PIBM_ECUDA;
  }
  cudaFree(buf);
  if (rc != PIBM_OK) return rc;
  *passed = (int)hp;
  return hb.abort ? PIBM_ETIMEOUT : PIBM_OK;
}
