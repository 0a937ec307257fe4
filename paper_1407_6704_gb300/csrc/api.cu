// Host side of the C ABI declared in include/pibm.h: validation, workspace
// layout, upload of the initial state, the step loop (replayed from CUDA graphs
// of two steps) and the read-back calls.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "pibm_internal.cuh"

using namespace pibm;

struct pibm_t {
  State s;
  cudaStream_t stream;     // caller's stream
  cudaStream_t cap;        // private stream used for graph capture
  void* ws;                // workspace base
  size_t ws_bytes;
  int owns_ws;
  int device;
  cudaGraphExec_t graph[2];  // step graphs (graph_length steps), indexed by the parity of s.cur
  int graph_failed;
  double* out_dev;         // small device scratch for reductions
  int kernels_per_step;
  int debug_sync;          // synchronise after every phase (PIBM_DEBUG_SYNC=1)
  int since_rebin;         // steps since the cell list was last rebuilt (0: rebuild next)
  int64_t launches;        // kernels launched by pibm_step so far
  int64_t nstep;           // steps taken so far (any path)
  int64_t graph_kernels;   // kernels in one replay of the step graphs
  int graph_steps;         // steps in one replay of the step graphs
  // overlap: contacts and the free tiles' collision on a second stream
  int split;
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_contacts, ev_free;
  int side_grid;           // CTAs of the free tiles' collision (a share of the GPU)
};

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  size_t f, F, mom, red, err, out, X, U, rad, mass, Ap, buoy, gw, cf, pid, rl, jl, Fs, ti, tw, nb, nbn, xs0, xr, cr, xs, cs, g, Fc, Fcf, key, rank, perm, bin,
      bsum, tflag, tbusy, tfree, tblk, tn;
  size_t total;
};

int dims_of(int lattice) { return lattice == PIBM_D2Q9 ? 2 : 3; }

size_t pop_bytes(int precision) {
  return precision == PIBM_FP64 ? 8 : (precision == PIBM_FP32 ? 4 : 2);
}

// Tile shape of the particle kernel: 32 x 8 cells in 2D, 16 x 8 x 4 in 3D.
BinMap bin_map(const pibm_config* c) {
  BinMap b;
  const int d = dims_of(c->lattice);
  b.T[0] = d == 2 ? TileDims<2>::TX : TileDims<3>::TX;
  b.T[1] = d == 2 ? TileDims<2>::TY : TileDims<3>::TY;
  b.T[2] = d == 2 ? TileDims<2>::TZ : TileDims<3>::TZ;
  for (int k = 0; k < 3; ++k) b.nt[k] = (int)((c->n[k] + b.T[k] - 1) / b.T[k]);
  b.tc = b.T[0] * b.T[1] * b.T[2];
  return b;
}

long long bin_count(const pibm_config* c) {
  BinMap b = bin_map(c);
  return (long long)b.nt[0] * b.nt[1] * b.nt[2] * b.tc;
}

int validate(const pibm_config* c) {
  if (!c) return PIBM_EINVAL;
  if (c->lattice != PIBM_D2Q9 && c->lattice != PIBM_D3Q15 && c->lattice != PIBM_D3Q19)
    return PIBM_EINVAL;
  if (c->overlap < PIBM_OVERLAP_AUTO || c->overlap > PIBM_OVERLAP_OFF) return PIBM_EINVAL;
  const int d = dims_of(c->lattice);
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    if (c->n[k] < 1 || c->n[k] > (1 << 30)) return PIBM_EINVAL;
    if (k < d && c->boundary[k] != PIBM_WALL && c->boundary[k] != PIBM_PERIODIC)
      return PIBM_EINVAL;
    ncell *= c->n[k];
  }
  if (d == 2 && c->n[2] != 1) return PIBM_EINVAL;
  // bins are cells padded to whole tiles; the cell-list scan covers up to
  // 8192 * 8192 entries
  if (bin_count(c) + 1 > 8192LL * 8192LL) return PIBM_ENOTSUP;
  if (!(c->tau > 0.5) || !isfinite(c->tau)) return PIBM_EINVAL;
  if (c->delta_width != 2 && c->delta_width != 4) return PIBM_EINVAL;
  if (c->coupling != PIBM_IMPLICIT && c->coupling != PIBM_EXPLICIT) return PIBM_EINVAL;
  if (c->precision != PIBM_FP64 && c->precision != PIBM_FP32 && c->precision != PIBM_FP16 &&
      c->precision != PIBM_BF16)
    return PIBM_EINVAL;
  if (!(c->dem_kn >= 0.0) || !isfinite(c->dem_kn)) return PIBM_EINVAL;
  if (!(c->dem_restitution > 0.0 && c->dem_restitution <= 1.0)) return PIBM_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (!isfinite(c->gravity[k])) return PIBM_EINVAL;
  if (c->n_particles < 0 || c->n_particles > 0x7fffffffLL) return PIBM_EINVAL;
  if (c->interp != PIBM_INTERP_DELTA && c->interp != PIBM_INTERP_LAGRANGE4) return PIBM_EINVAL;
  if (c->interp == PIBM_INTERP_LAGRANGE4)
    for (int k = 0; k < d; ++k)
      if (c->boundary[k] == PIBM_WALL && c->n[k] < 4) return PIBM_EINVAL;
  if (c->dem_model != PIBM_DEM_LINEAR && c->dem_model != PIBM_DEM_HERTZ) return PIBM_EINVAL;
  if (c->dem_model == PIBM_DEM_HERTZ) {
    if (!(c->dem_young > 0.0) || !isfinite(c->dem_young)) return PIBM_EINVAL;
    if (!(c->dem_poisson >= 0.0 && c->dem_poisson < 0.5)) return PIBM_EINVAL;
    if (!(c->wall_young >= 0.0) || !isfinite(c->wall_young)) return PIBM_EINVAL;
    if (c->wall_young > 0.0 && !(c->wall_poisson >= 0.0 && c->wall_poisson < 0.5))
      return PIBM_EINVAL;
  }
  if (c->dem_substeps < 0 || c->dem_substeps > 4096) return PIBM_EINVAL;
  if (c->particle_update != PIBM_PARTICLE_FP64 && c->particle_update != PIBM_PARTICLE_FP32)
    return PIBM_EINVAL;
  if (c->rebin_every < 0 || c->rebin_every > 100000) return PIBM_EINVAL;
  if (c->rebin_every > 1 && c->dem_substeps > 1) return PIBM_ENOTSUP;
  if (c->n_particles > 0) {
    if (!c->x0 || !c->diameter || !c->density_ratio) return PIBM_EINVAL;
    // contact and spreading stencils must not alias on a periodic axis: the
    // contact search spans 3 cells, the ordered gather 2 R + 1
    const int reach = (c->delta_width == 2 ? 1 : 2) + (c->rebin_every > 1 ? 1 : 0);
    const int nmin = c->deterministic && 2 * reach + 1 > 5 ? 2 * reach + 1 : 5;
    for (int k = 0; k < d; ++k)
      if (c->boundary[k] == PIBM_PERIODIC && c->n[k] < nmin) return PIBM_EINVAL;
    for (long long p = 0; p < c->n_particles; ++p) {
      double dia = c->diameter[p], rr = c->density_ratio[p];
      if (!(dia > 0.0 && dia <= 1.0)) return PIBM_EINVAL;
      if (!(rr > 0.0) || !isfinite(rr)) return PIBM_EINVAL;
      for (int k = 0; k < d; ++k) {
        double x = c->x0[p * d + k];
        if (!isfinite(x)) return PIBM_EINVAL;
        if (c->boundary[k] == PIBM_PERIODIC) {
          if (x < 0.0 || x >= (double)c->n[k]) return PIBM_EINVAL;
        } else if (!(x > 0.0 && x < (double)c->n[k])) {
          return PIBM_EINVAL;
        }
        if (c->u0 && !isfinite(c->u0[p * d + k])) return PIBM_EINVAL;
      }
    }
  }
  return PIBM_OK;
}

Layout layout(const pibm_config* c) {
  Layout L;
  const int q = c->lattice, d = dims_of(q);
  const long long ncell = c->n[0] * c->n[1] * c->n[2];
  const long long pitch = (ncell + 63) / 64 * 64;
  const size_t ts = pop_bytes(c->precision);           // population element
  const size_t fs = c->precision == PIBM_FP64 ? 8 : 4;  // force and moment element
  const long long np = c->n_particles;
  const long long nbin = bin_count(c);
  const long long scan_blocks = (nbin + 1 + 8191) / 8192;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L.f = take(2 * align_up((size_t)q * pitch * ts));
  L.F = take((size_t)(d == 2 ? 2 : 4) * pitch * fs);
  L.mom = take(c->n_particles > 0 ? (size_t)MOM_SLOTS * pitch * fs : 0);
  L.red = take(sizeof(double) * RED_SCRATCH);
  L.err = take(sizeof(unsigned));
  L.out = take(sizeof(double) * 8);
  L.X = take(2 * align_up(sizeof(double) * d * np));
  L.U = take(2 * align_up(sizeof(double) * d * np));
  L.rad = take(2 * align_up(sizeof(double) * np));
  L.mass = take(2 * align_up(sizeof(double) * np));
  L.Ap = take(2 * align_up(sizeof(double) * np));
  L.buoy = take(2 * align_up(sizeof(double) * np));
  L.gw = take(2 * align_up(sizeof(double) * np));
  L.cf = take(2 * align_up(sizeof(float4) * np));
  L.pid = take(2 * align_up(sizeof(unsigned) * np));
  const bool sub = c->dem_substeps > 1;
  L.rl = take(sub ? sizeof(double) * np : 0);
  L.jl = take(sub ? sizeof(double) * d * np : 0);
  L.Fs = take(sub ? sizeof(double) * d * np : 0);
  L.ti = take(c->deterministic ? sizeof(int) * 12 * np : 0);
  L.tw = take(c->deterministic ? sizeof(double) * 12 * np : 0);
  const bool keep = c->rebin_every > 1;
  // contact candidates recorded at a rebuild (kept cell list) or at the first DEM
  // sub-step (sub-cycling)
  const bool record = keep || sub;
  L.nb = take(record ? sizeof(unsigned) * (d == 2 ? 24 : 64) * np : 0);
  L.nbn = take(record ? sizeof(int) * np : 0);
  L.xs0 = take(keep ? sizeof(float4) * np : 0);
  L.xr = take(sizeof(float4) * np);
  L.cr = take(sizeof(int4) * np);
  L.xs = take(2 * align_up(sizeof(float4) * np));
  L.cs = take(2 * align_up(sizeof(int4) * np));
  L.g = take(sizeof(double) * d * np);
  L.Fc = take(sizeof(double) * d * np);
  L.Fcf = take(sizeof(float) * d * np);
  L.key = take(sizeof(unsigned) * np);
  L.rank = take(sizeof(unsigned) * np);
  L.perm = take(sizeof(unsigned) * np);
  L.bin = take(sizeof(unsigned) * (nbin + 1));
  // chunk totals of the cell-list scan: chunks of 8192 counts in the step kernels,
  // of 2048 in the batched persistent kernel
  L.bsum = take(sizeof(unsigned) * std::max<long long>(scan_blocks, (nbin + 1 + 2047) / 2048));
  const long long ntiles = nbin / bin_map(c).tc;
  L.tflag = take(np > 0 ? sizeof(int) * ntiles : 0);
  L.tbusy = take(np > 0 ? sizeof(int) * ntiles : 0);
  L.tfree = take(np > 0 ? sizeof(int) * ntiles : 0);
  L.tblk = take(np > 0 ? sizeof(unsigned) * ((ntiles + TILE_BLOCK - 1) / TILE_BLOCK) : 0);
  L.tn = take(np > 0 ? sizeof(unsigned) * 2 : 0);
  L.total = off;
  return L;
}


// Description of the last failed CUDA call on this thread (pibm_last_error).
thread_local char g_last_error[256] = "";

void record_error(const char* what, cudaError_t e) { pibm::record_cuda_error(what, e); }

#define CK(expr)                          \
  do {                                    \
    cudaError_t e_ = (expr);              \
    if (e_ != cudaSuccess) {              \
      record_error(#expr, e_);            \
      return PIBM_ECUDA;                  \
    }                                     \
  } while (0)

// With PIBM_DEBUG_SYNC=1 in the environment at pibm_create, steps are launched
// without graphs and the stream is synchronised after every phase, so that an
// error is attributed to the phase that raised it.
#define PHASE(expr)                                        \
  do {                                                     \
    CK(expr);                                              \
    if (h->debug_sync) CK(cudaStreamSynchronize(st));      \
  } while (0)

// One step: the cell list (when due), contacts, coupling, collision. nk
// receives the number of kernels launched.
int enqueue_step(pibm_t* h, cudaStream_t st, int* nk_out, bool split_ok = true) {
  State& s = h->s;
  int nk = 0;
  const bool rebuild = h->since_rebin == 0;
  if (rebuild) PHASE(launch_bin(s, st, &nk));
  s.nb_mode = rebuild ? 1 : 2;
  // between rebuilds the storage order holds, so from the second step after a
  // rebuild the other buffer already holds the constants in that order
  s.move_consts = h->since_rebin <= 1;
  if (h->split && split_ok) {
    // side stream: contacts, then the collision of the free tiles (no particle
    // stencil reaches them, so their force is zero and stays untouched); main
    // stream: moments, the particle kernels after the contacts, then the busy
    // tiles' collision after the free ones
    CK(cudaEventRecord(h->ev_fork, st));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    PHASE(launch_contacts(s, h->side, &nk));
    CK(cudaEventRecord(h->ev_contacts, h->side));
    PHASE(launch_collide_tiles(s, h->side, 1, h->side_grid));
    CK(cudaEventRecord(h->ev_free, h->side));
    PHASE(launch_couple(s, st, &nk, h->ev_contacts));
    CK(cudaStreamWaitEvent(st, h->ev_free, 0));
    PHASE(launch_collide_tiles(s, st, 0, 0));
    nk += 2;
  } else {
    PHASE(launch_contacts(s, st, &nk));
    PHASE(launch_couple(s, st, &nk));
    PHASE(launch_collide_stream(s, st));
    nk += 1;
  }
  s.cur ^= 1;
  h->since_rebin = (h->since_rebin + 1) % s.phy.rebin;
  ++h->nstep;
  if (rebuild) h->kernels_per_step = nk;
  if (nk_out) *nk_out = nk;
  return PIBM_OK;
}

// Steps in one replay of the step graphs: a whole number of cell-list rebuild
// periods that is even, so that the buffers and the rebuild phase both return
// to where they started.
int graph_length(const pibm_t* h) {
  const int r = h->s.phy.rebin;
  return r % 2 == 0 ? r : 2 * r;
}

int build_graph(pibm_t* h, int parity) {
  // Capture graph_length() steps starting from buffer parity `parity` with a
  // cell-list rebuild due; afterwards the buffers and the rebuild phase are back
  // where they started, so the graph can be replayed.
  cudaGraph_t g = nullptr;
  const int saved = h->s.cur, saved_r = h->since_rebin, saved_k = h->kernels_per_step;
  const int64_t saved_n = h->nstep;
  h->s.cur = parity;
  h->since_rebin = 0;
  if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    h->s.cur = saved;
    h->since_rebin = saved_r;
    return PIBM_ECUDA;
  }
  int rc = PIBM_OK;
  int64_t total = 0;
  const int len = graph_length(h);
  for (int i = 0; i < len && rc == PIBM_OK; ++i) {
    int nk = 0;
    rc = enqueue_step(h, h->cap, &nk);
    total += nk;
  }
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  h->s.cur = saved;
  h->since_rebin = saved_r;
  h->nstep = saved_n;
  h->kernels_per_step = saved_k > 0 ? saved_k : h->kernels_per_step;
  h->graph_kernels = total;
  h->graph_steps = len;
  if (rc != PIBM_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  e = cudaGraphInstantiate(&h->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph[parity] = nullptr;
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  return PIBM_OK;
}

int health(pibm_t* h) {
  unsigned err = 0;
  CK(cudaMemcpyAsync(&err, h->s.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err & (ERR_FLUID_NONFINITE | ERR_PARTICLE_NONFINITE | ERR_SKIN | ERR_MACH))
    return PIBM_EUNSTABLE;
  if (err & ERR_ESCAPED) return PIBM_EESCAPED;
  if (err & ERR_INDEX) return PIBM_EINTERNAL;
  return PIBM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

namespace pibm {
HandleView handle_view(pibm_t* h) { return HandleView{&h->s, h->ws, h->ws_bytes, h->stream}; }

void record_cuda_error(const char* what, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e),
           cudaGetErrorString(e));
}
}  // namespace pibm

extern "C" {

const char* pibm_last_error(void) { return g_last_error; }

const char* pibm_strerror(int st) {
  switch (st) {
    case PIBM_OK: return "ok";
    case PIBM_EINVAL: return "invalid argument or configuration";
    case PIBM_ENOMEM: return "workspace too small or allocation failed";
    case PIBM_ECUDA: return "CUDA call failed";
    case PIBM_EUNSTABLE: return "non-finite fluid or particle state";
    case PIBM_EESCAPED: return "a particle crossed a wall";
    case PIBM_ENOTSUP: return "configuration not supported by this build";
    case PIBM_EINTERNAL: return "internal index check failed (access skipped)";
    case PIBM_ETOOBIG: return "size exceeds the fixed static scratch of the no-allocation call";
    case PIBM_ETIMEOUT: return "a grid barrier of the persistent ensemble kernel timed out";
    default: return "unknown status";
  }
}

int pibm_workspace_bytes(const pibm_config* cfg, size_t* bytes) {
  int rc = validate(cfg);
  if (rc != PIBM_OK) return rc;
  if (!bytes) return PIBM_EINVAL;
  *bytes = layout(cfg).total;
  return PIBM_OK;
}

int pibm_create(const pibm_config* cfg, void* workspace, size_t workspace_bytes, void* stream,
                pibm_t** out) {
  if (!out) return PIBM_EINVAL;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc != PIBM_OK) return rc;
  const Layout L = layout(cfg);
  if (workspace && (workspace_bytes < L.total || ((uintptr_t)workspace % ALIGN) != 0))
    return PIBM_ENOMEM;

  pibm_t* h = new (std::nothrow) pibm_t();
  if (!h) return PIBM_ENOMEM;
  memset(h, 0, sizeof(*h));
  cudaGetDevice(&h->device);
  h->stream = (cudaStream_t)stream;
  {
    const char* dbg = getenv("PIBM_DEBUG_SYNC");
    h->debug_sync = dbg && dbg[0] == '1';
    h->graph_failed = h->debug_sync;  // debug steps run eagerly
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return PIBM_ECUDA;
  }
  if (workspace) {
    h->ws = workspace;
    h->owns_ws = 0;
  } else {
    if (cudaMalloc(&h->ws, L.total) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamDestroy(h->cap);
      delete h;
      return PIBM_ENOMEM;
    }
    h->owns_ws = 1;
  }
  h->ws_bytes = L.total;
  char* base = (char*)h->ws;

  State& s = h->s;
  const int q = cfg->lattice, d = dims_of(q);
  s.geo.q = q;
  s.geo.d = d;
  for (int k = 0; k < 3; ++k) {
    s.geo.n[k] = (int)cfg->n[k];
    s.geo.periodic[k] = (k < d) ? (cfg->boundary[k] == PIBM_PERIODIC) : 1;
  }
  s.geo.ncell = cfg->n[0] * cfg->n[1] * cfg->n[2];
  s.geo.pitch = (s.geo.ncell + 63) / 64 * 64;
  s.phy.tau = cfg->tau;
  s.phy.omega = 1.0 / cfg->tau;
  s.phy.cF = 1.0 - 0.5 / cfg->tau;
  for (int k = 0; k < 3; ++k) {
    s.phy.gravity[k] = k < d ? cfg->gravity[k] : 0.0;
    s.phy.gravityf[k] = (float)s.phy.gravity[k];
  }
  s.phy.kn = cfg->dem_kn;
  {
    const double lne = log(cfg->dem_restitution);
    s.phy.beta = -lne / sqrt(M_PI * M_PI + lne * lne);
  }
  s.phy.width = cfg->delta_width;
  s.phy.implicit_drag = cfg->coupling == PIBM_IMPLICIT;
  s.phy.lagrange = cfg->interp == PIBM_INTERP_LAGRANGE4;
  s.phy.hertz = cfg->dem_model == PIBM_DEM_HERTZ;
  s.phy.Epp = s.phy.Epw = s.phy.hz_damp = 0.0;
  if (s.phy.hertz) {
    // 1/E* = (1 - nu_1^2)/E_1 + (1 - nu_2^2)/E_2 (Eq. 15)
    const double cp = (1.0 - cfg->dem_poisson * cfg->dem_poisson) / cfg->dem_young;
    const double cw = cfg->wall_young > 0.0
                          ? (1.0 - cfg->wall_poisson * cfg->wall_poisson) / cfg->wall_young
                          : cp;
    s.phy.Epp = 1.0 / (cp + cp);
    s.phy.Epw = 1.0 / (cp + cw);
    s.phy.hz_damp = 2.0 * sqrt(5.0 / 6.0) * s.phy.beta;
  }
  s.phy.substeps = cfg->dem_substeps > 1 ? cfg->dem_substeps : 1;
  s.phy.p64 = cfg->precision != PIBM_FP64 && cfg->particle_update == PIBM_PARTICLE_FP64;
  s.phy.rebin = cfg->rebin_every > 1 ? cfg->rebin_every : 1;
  {
    double dmax = 0.0;
    for (long long p = 0; p < cfg->n_particles; ++p) dmax = fmax(dmax, cfg->diameter[p]);
    s.phy.skin = 0.5 * (1.0 - dmax);
    s.phy.disp_skin = 0.25 * (1.0 - dmax);
    s.phy.skinf = (float)s.phy.skin;
    s.phy.disp_skinf = (float)s.phy.disp_skin;
  }
  s.precision = cfg->precision;
  s.deterministic = cfg->deterministic ? 1 : 0;
  const size_t ts = pop_bytes(cfg->precision);
  const size_t fs = cfg->precision == PIBM_FP64 ? 8 : 4;
  const size_t fbuf = align_up((size_t)q * s.geo.pitch * ts);
  s.f[0] = base + L.f;
  s.f[1] = base + L.f + fbuf;
  s.F = base + L.F;
  s.mom = base + L.mom;
  s.red = (double*)(base + L.red);
  s.err = (unsigned*)(base + L.err);
  h->out_dev = (double*)(base + L.out);
  const long long np = cfg->n_particles;
  Particles& P = s.p;
  P.np = np;
  const size_t xb = align_up(sizeof(double) * d * np);
  P.X[0] = (double*)(base + L.X);
  P.X[1] = (double*)(base + L.X + xb);
  P.U[0] = (double*)(base + L.U);
  P.U[1] = (double*)(base + L.U + xb);
  const size_t db = align_up(sizeof(double) * np), fb = align_up(sizeof(float) * np);
  for (int b = 0; b < 2; ++b) {
    P.rad[b] = (double*)(base + L.rad + b * db);
    P.mass[b] = (double*)(base + L.mass + b * db);
    P.Ap[b] = (double*)(base + L.Ap + b * db);
    P.buoy[b] = (double*)(base + L.buoy + b * db);
    P.gw[b] = (double*)(base + L.gw + b * db);
    P.cf[b] = (float4*)(base + L.cf + b * align_up(sizeof(float4) * np));
    P.pid[b] = (unsigned*)(base + L.pid + b * fb);
  }
  P.xr = (float4*)(base + L.xr);
  P.cr = (int4*)(base + L.cr);
  for (int b = 0; b < 2; ++b) {
    P.xs[b] = (float4*)(base + L.xs + b * align_up(sizeof(float4) * np));
    P.cs[b] = (int4*)(base + L.cs + b * align_up(sizeof(int4) * np));
  }
  P.g = (double*)(base + L.g);
  P.rl = (double*)(base + L.rl);
  P.jl = (double*)(base + L.jl);
  P.Fs = (double*)(base + L.Fs);
  P.ti = (int*)(base + L.ti);
  P.tw = (double*)(base + L.tw);
  P.nb = (unsigned*)(base + L.nb);
  P.nbn = (int*)(base + L.nbn);
  P.xs0 = cfg->rebin_every > 1 ? (float4*)(base + L.xs0) : nullptr;
  P.nb_max = d == 2 ? 24 : 64;
  P.Fc = (double*)(base + L.Fc);
  P.Fcf = (float*)(base + L.Fcf);
  P.key = (unsigned*)(base + L.key);
  P.rank = (unsigned*)(base + L.rank);
  P.perm = (unsigned*)(base + L.perm);
  P.bin_cnt = (unsigned*)(base + L.bin);
  P.block_sums = (unsigned*)(base + L.bsum);
  P.bm = bin_map(cfg);
  P.nbin = bin_count(cfg);
  P.scan_blocks = (int)((P.nbin + 1 + 8191) / 8192);
  P.ntiles = P.nbin / P.bm.tc;
  P.tflag = (int*)(base + L.tflag);
  P.tbusy = (int*)(base + L.tbusy);
  P.tfree = (int*)(base + L.tfree);
  P.tblk = (unsigned*)(base + L.tblk);
  P.tn = (unsigned*)(base + L.tn);
  s.cur = 0;

  cudaStream_t st = h->stream;
  auto fail = [&](int code) {
    pibm_destroy(h);
    return code;
  };
  // force field and health word start at zero
  if (cudaMemsetAsync(s.F, 0, (size_t)(d == 2 ? 2 : 4) * s.geo.pitch * fs, st) != cudaSuccess ||
      cudaMemsetAsync(s.err, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(PIBM_ECUDA);

  // populations: store f*_a(y) = f0_a(y + e_a), or f0_opp(a)(y) across a wall,
  // so that the first pull reproduces f0 (streaming is a permutation of slots)
  if (cfg->f0) {
    std::vector<double> plane((size_t)s.geo.ncell);
    double* stage = (double*)s.f[1];  // the partner buffer is free before the first step
    int e[19][3];
    for (int a = 0; a < q; ++a)
      for (int k = 0; k < 3; ++k)
        e[a][k] = q == 9 ? Lattice<9>::e(a, k) : (q == 15 ? Lattice<15>::e(a, k) : Lattice<19>::e(a, k));
    const int n0 = s.geo.n[0], n1 = s.geo.n[1], n2 = s.geo.n[2];
    for (int a = 0; a < q; ++a) {
      const int b = opp(a);
      for (int z = 0; z < n2; ++z)
        for (int y = 0; y < n1; ++y)
          for (int x = 0; x < n0; ++x) {
            int t[3] = {x + e[a][0], y + e[a][1], z + e[a][2]};
            bool wall = false;
            for (int k = 0; k < 3; ++k) {
              if (t[k] < 0 || t[k] >= s.geo.n[k]) {
                if (s.geo.periodic[k]) t[k] = (t[k] + s.geo.n[k]) % s.geo.n[k];
                else wall = true;
              }
            }
            const long long c = x + (long long)n0 * (y + (long long)n1 * z);
            const long long tc = t[0] + (long long)n0 * (t[1] + (long long)n1 * t[2]);
            plane[c] = wall ? cfg->f0[(size_t)b * s.geo.ncell + c]
                            : cfg->f0[(size_t)a * s.geo.ncell + tc];
          }
      if (cudaMemcpyAsync(stage, plane.data(), sizeof(double) * s.geo.ncell,
                          cudaMemcpyHostToDevice, st) != cudaSuccess ||
          launch_store_plane(s, a, stage, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail(PIBM_ECUDA);
    }
  } else {
    for (int a = 0; a < q; ++a)
      if (launch_store_plane(s, a, nullptr, st) != cudaSuccess) return fail(PIBM_ECUDA);
  }

  if (np > 0) {
    // The AoS arrays go up as they are, into the second particle buffers (free
    // before the first step), and are transposed to SoA on the device; one
    // synchronisation at the end covers every copy.
    const size_t vb = sizeof(double) * d * np;
    if (cudaMemcpyAsync(P.X[1], cfg->x0, vb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        launch_aos_to_soa(np, d, P.X[1], P.X[0], st) != cudaSuccess)
      return fail(PIBM_ECUDA);
    if (cfg->u0) {
      if (cudaMemcpyAsync(P.U[1], cfg->u0, vb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          launch_aos_to_soa(np, d, P.U[1], P.U[0], st) != cudaSuccess)
        return fail(PIBM_ECUDA);
    } else if (cudaMemsetAsync(P.U[0], 0, vb, st) != cudaSuccess) {
      return fail(PIBM_ECUDA);
    }
    if (cudaMemcpyAsync(P.rad[0], cfg->diameter, sizeof(double) * np, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(P.buoy[0], cfg->density_ratio, sizeof(double) * np,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(P.g, 0, vb, st) != cudaSuccess ||
        cudaMemsetAsync(P.Fc, 0, vb, st) != cudaSuccess ||
        cudaMemsetAsync(P.Fcf, 0, sizeof(float) * d * np, st) != cudaSuccess ||
        launch_particle_init(s, st) != cudaSuccess)
      return fail(PIBM_ECUDA);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(PIBM_ECUDA);
  // binning 5 (+1 ordered bins) and tile lists 2, contacts 1, moments + coupling
  // 2 (+1 ordered gather), collide 1 (2 with overlap); with S DEM sub-steps the
  // contacts and the coupling become 1 + 2 S (+1 spread unless gathered)
  {
    const int S = s.phy.substeps, det = s.deterministic;
    h->kernels_per_step = np == 0 ? 1 : (S <= 1 ? (det ? 13 : 11) : (det ? 12 : 11) + 2 * S);
  }
  // overlap: a second stream and its events. AUTO takes it for 2D lattices of
  // 2^20 cells or more; in 3D the tile-shaped collision (16-cell rows) is slower
  // than the plain kernel by more than the overlap gains.
  if (np > 0 && !s.deterministic && collide_tiles_supported(s) &&
      (cfg->overlap == PIBM_OVERLAP_ON ||
       (cfg->overlap == PIBM_OVERLAP_AUTO && d == 2 && s.geo.ncell >= (1LL << 20)))) {
    int lo = 0, hi = 0, sms = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_contacts, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_free, cudaEventDisableTiming) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
      return fail(PIBM_ECUDA);
    h->side_grid = 4 * sms;  // a share of the GPU beside the coupling kernels
    h->split = 1;
    h->kernels_per_step += 1;
  }
  *out = h;
  return PIBM_OK;
}

int pibm_step(pibm_t* h, int64_t nsteps) {
  if (!h || nsteps < 0) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  const int len = graph_length(h);
  while (nsteps > 0) {
    if (h->since_rebin == 0 && nsteps >= len && !h->graph_failed) {
      const int par = h->s.cur;
      if (!h->graph[par] && build_graph(h, par) != PIBM_OK) {
        h->graph_failed = 1;
        continue;
      }
      CK(cudaGraphLaunch(h->graph[par], h->stream));
      nsteps -= len;  // an even number of toggles leaves s.cur unchanged
      h->nstep += len;
      h->launches += h->graph_kernels;
    } else {
      int nk = 0;
      int rc = enqueue_step(h, h->stream, &nk);
      if (rc != PIBM_OK) return rc;
      h->launches += nk;
      nsteps -= 1;
    }
  }
  return PIBM_OK;
}

int pibm_forces(pibm_t* h, double* f_fpi, double* f_contact, int on_device) {
  if (!h) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  State& s = h->s;
  const long long np = s.p.np;
  const int d = s.geo.d;
  if (np > 0 && (f_fpi || f_contact)) {
    if (on_device) {
      CK(launch_particle_forces(s, f_fpi, f_contact, h->stream));
    } else {
      double* stage = (double*)s.f[1 - s.cur];  // free between steps
      double* a = stage;
      double* b = stage + (size_t)d * np;
      size_t need = sizeof(double) * 2 * d * np;
      size_t have = align_up((size_t)s.geo.q * s.geo.pitch * pop_bytes(s.precision));
      if (need > have) return PIBM_ENOMEM;
      CK(launch_particle_forces(s, f_fpi ? a : nullptr, f_contact ? b : nullptr, h->stream));
      if (f_fpi)
        CK(cudaMemcpyAsync(f_fpi, a, sizeof(double) * d * np, cudaMemcpyDeviceToHost, h->stream));
      if (f_contact)
        CK(cudaMemcpyAsync(f_contact, b, sizeof(double) * d * np, cudaMemcpyDeviceToHost,
                           h->stream));
    }
  }
  return health(h);
}

int pibm_read_fields(pibm_t* h, unsigned mask, void* const* dst, int on_device) {
  if (!h || (mask && !dst)) return PIBM_EINVAL;
  if (mask >> PIBM_NFIELDS) return PIBM_EINVAL;
  for (int k = 0; k < PIBM_NFIELDS; ++k)
    if ((mask >> k & 1u) && !dst[k]) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  State& s = h->s;
  const long long nc = s.geo.ncell, np = s.p.np;
  const int d = s.geo.d, q = s.geo.q;
  cudaStream_t st = h->stream;
  double* stage = (double*)s.f[1 - s.cur];  // partner buffer holds >= ncell doubles
  auto plane_out = [&](double* dstp, auto launch) -> int {
    if (on_device) {
      CK(launch(dstp));
    } else {
      CK(launch(stage));
      CK(cudaMemcpyAsync(dstp, stage, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    return PIBM_OK;
  };
  int rc;
  if (mask & PIBM_FIELD_RHO) {
    rc = plane_out((double*)dst[0], [&](double* o) { return launch_read_moment(s, 0, o, st); });
    if (rc) return rc;
  }
  if (mask & PIBM_FIELD_J) {
    for (int k = 0; k < d; ++k) {
      rc = plane_out((double*)dst[1] + (size_t)k * nc,
                     [&](double* o) { return launch_read_moment(s, k + 1, o, st); });
      if (rc) return rc;
    }
  }
  if (mask & PIBM_FIELD_POP) {
    for (int a = 0; a < q; ++a) {
      rc = plane_out((double*)dst[2] + (size_t)a * nc,
                     [&](double* o) { return launch_read_pop_plane(s, a, o, st); });
      if (rc) return rc;
    }
  }
  for (int f = 0; f < 2; ++f) {
    const unsigned bit = f == 0 ? PIBM_FIELD_X : PIBM_FIELD_U;
    if (!(mask & bit) || np == 0) continue;
    const double* src = f == 0 ? s.p.X[s.cur] : s.p.U[s.cur];
    double* o = (double*)dst[f == 0 ? 3 : 4];
    if (on_device) {
      CK(launch_interleave(s, src, o, st));
    } else if ((size_t)2 * d * np * sizeof(double) <=
               align_up((size_t)s.geo.q * s.geo.pitch * pop_bytes(s.precision))) {
      // storage order -> user order on the device, in the partner population
      // buffer (free between steps), then one copy into the caller's array
      double* aos = stage + (size_t)f * d * np;
      CK(launch_interleave(s, src, aos, st));
      CK(cudaMemcpyAsync(o, aos, sizeof(double) * d * np, cudaMemcpyDeviceToHost, st));
    } else {
      // a lattice too small to stage the particles: storage order -> user order
      // on the host
      std::vector<double> soa((size_t)d * np);
      std::vector<unsigned> pid((size_t)np);
      CK(cudaMemcpyAsync(soa.data(), src, sizeof(double) * d * np, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(pid.data(), s.p.pid[s.cur], sizeof(unsigned) * np,
                         cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (long long i = 0; i < np; ++i) {
        const unsigned p = pid[(size_t)i];
        if (p >= (unsigned long long)np) return PIBM_EINTERNAL;
        for (int k = 0; k < d; ++k) o[(size_t)p * d + k] = soa[(size_t)k * np + i];
      }
    }
  }
  return health(h);
}

int pibm_invariants(pibm_t* h, double* out) {
  if (!h || !out) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  State& s = h->s;
  const int d = s.geo.d;
  CK(launch_invariants(s, h->out_dev, h->stream));
  CK(launch_particle_momentum(s, h->out_dev + 1 + d, h->stream));
  CK(cudaMemcpyAsync(out, h->out_dev, sizeof(double) * (1 + 2 * d), cudaMemcpyDeviceToHost,
                     h->stream));
  return health(h);
}

int pibm_status(pibm_t* h) {
  if (!h) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  return health(h);
}

int pibm_kernels_per_step(pibm_t* h) { return h ? h->kernels_per_step : 0; }

int pibm_launch_count(pibm_t* h, int64_t* count) {
  if (!h || !count) return PIBM_EINVAL;
  *count = h->launches;
  return PIBM_OK;
}

int pibm_autotune(pibm_t* h, int* block_xy) {
  if (!h) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  State& s = h->s;
  cudaStream_t st = h->stream;
  // Candidate block shapes; the 16-bit pair kernel fixes x at one warp.
  static const int scal[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {32, 4}, {64, 2}, {128, 1}};
  static const int pair[][2] = {{32, 2}, {32, 4}, {32, 8}};  // kernels take <= 256 threads
  const bool pk = collide_uses_pair_kernel(s);
  const int ncand = pk ? 3 : 7;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PIBM_ECUDA;
  }
  int best = -1;
  float best_ms = 0.f;
  const int saved[2] = {s.cblk[0], s.cblk[1]};
  int rc = PIBM_OK;
  // Running the collide-stream without advancing the step only rewrites the
  // partner buffer and clears F, both of which hold nothing between steps.
  for (int i = 0; i < ncand && rc == PIBM_OK; ++i) {
    s.cblk[0] = pk ? pair[i][0] : scal[i][0];
    s.cblk[1] = pk ? pair[i][1] : scal[i][1];
    cudaError_t le = launch_collide_stream(s, st);
    if (le != cudaSuccess) {  // a shape this launch cannot take: skip it
      cudaGetLastError();
      continue;
    }
    if (cudaEventRecord(e0, st) != cudaSuccess) {
      record_error("cudaEventRecord", cudaGetLastError());
      rc = PIBM_ECUDA;
      break;
    }
    for (int r = 0; r < 3; ++r)
      if ((le = launch_collide_stream(s, st)) != cudaSuccess) {
        record_error("launch_collide_stream", le);
        rc = PIBM_ECUDA;
      }
    float ms = 0.f;
    cudaError_t te = cudaSuccess;
    if (rc == PIBM_OK && ((te = cudaEventRecord(e1, st)) != cudaSuccess ||
                          (te = cudaEventSynchronize(e1)) != cudaSuccess ||
                          (te = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)) {
      record_error("autotune timing", te);
      rc = PIBM_ECUDA;
    }
    if (rc != PIBM_OK) break;
    if (best < 0 || ms < best_ms) {
      best = i;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PIBM_OK || best < 0) {
    s.cblk[0] = saved[0];
    s.cblk[1] = saved[1];
    return rc != PIBM_OK ? rc : PIBM_ECUDA;
  }
  s.cblk[0] = pk ? pair[best][0] : scal[best][0];
  s.cblk[1] = pk ? pair[best][1] : scal[best][1];
  for (int k = 0; k < 2; ++k)  // graphs captured before hold the old launch shape
    if (h->graph[k]) {
      cudaGraphExecDestroy(h->graph[k]);
      h->graph[k] = nullptr;
    }
  if (block_xy) {
    block_xy[0] = s.cblk[0];
    block_xy[1] = s.cblk[1];
  }
  return health(h);
}

// ---------------------------------------------------------------------------
// Ensembles: independent simulations advanced together. Persistent mode (the
// default where every member qualifies, ensemble.cu): one cooperative kernel runs
// ENS_GRAPH_STEPS steps of all members per launch, replayed from a CUDA graph.
// Branch mode: a graph with one branch of ordinary step kernels per member.
// ---------------------------------------------------------------------------
constexpr int ENS_GRAPH_STEPS = 10;  // steps per persistent launch in the graph

struct pibm_ensemble_t {
  std::vector<pibm_t*> members;
  cudaStream_t stream;          // launch stream
  cudaStream_t origin;          // capture origin
  std::vector<cudaStream_t> lanes;
  std::vector<int> parity;      // member parities the branch graph was captured for
  cudaGraphExec_t graph;
  int device;
  // persistent mode
  int persistent;
  EnsembleDevice* pd;
  cudaGraphExec_t pgraph;       // one persistent launch of ENS_GRAPH_STEPS steps
  int pgraph_failed;
  std::vector<int64_t> seen;    // member step counts after the last ensemble step
  int64_t launches;             // kernels launched by pibm_ensemble_step
  int timed_out;
};

static int ensemble_capture(pibm_ensemble_t* e) {
  // Two steps of every member, each member on its own capture stream forked
  // from and joined back into the origin stream, so the graph's branches are
  // independent and run concurrently.
  cudaGraph_t g = nullptr;
  std::vector<cudaEvent_t> evs;
  auto ev = [&]() -> cudaEvent_t {
    cudaEvent_t x = nullptr;
    if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    evs.push_back(x);
    return x;
  };
  int rc = PIBM_OK;
  if (cudaStreamBeginCapture(e->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return PIBM_ECUDA;
  cudaEvent_t fork = ev();
  if (!fork || cudaEventRecord(fork, e->origin) != cudaSuccess) rc = PIBM_ECUDA;
  for (size_t i = 0; i < e->members.size() && rc == PIBM_OK; ++i) {
    pibm_t* m = e->members[i];
    cudaStream_t ln = e->lanes[i];
    if (cudaStreamWaitEvent(ln, fork, 0) != cudaSuccess) {
      rc = PIBM_ECUDA;
      break;
    }
    const int saved = m->s.cur;
    const int64_t saved_n = m->nstep;
    rc = enqueue_step(m, ln, nullptr, false);
    if (rc == PIBM_OK) rc = enqueue_step(m, ln, nullptr, false);
    m->s.cur = saved;
    m->nstep = saved_n;
    cudaEvent_t join = ev();
    if (rc == PIBM_OK && (!join || cudaEventRecord(join, ln) != cudaSuccess ||
                          cudaStreamWaitEvent(e->origin, join, 0) != cudaSuccess))
      rc = PIBM_ECUDA;
  }
  cudaError_t ee = cudaStreamEndCapture(e->origin, &g);
  for (auto x : evs)
    if (x) cudaEventDestroy(x);
  if (rc != PIBM_OK || ee != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  cudaError_t ie = cudaGraphInstantiate(&e->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    e->graph = nullptr;
    record_error("cudaGraphInstantiate", ie);
    return PIBM_ECUDA;
  }
  for (size_t i = 0; i < e->members.size(); ++i) e->parity[i] = e->members[i]->s.cur;
  return PIBM_OK;
}

// Persistent mode: the graph of one launch of ENS_GRAPH_STEPS steps. The kernel
// reads each member's buffer parity and rebuild phase from the device table and
// advances it, so the graph replays from any phase.
static int ensemble_capture_persistent(pibm_ensemble_t* e) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(e->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  const cudaError_t le = ensemble_device_launch(e->pd, ENS_GRAPH_STEPS, e->origin);
  const cudaError_t ee = cudaStreamEndCapture(e->origin, &g);
  if (le != cudaSuccess || ee != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&e->pgraph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    e->pgraph = nullptr;
    cudaGetLastError();
    return PIBM_ECUDA;
  }
  return PIBM_OK;
}

int pibm_ensemble_create(pibm_t* const* members, int count, void* stream, pibm_ensemble_t** out) {
  if (!members || count <= 0 || !out) return PIBM_EINVAL;
  *out = nullptr;
  int dev = -1;
  std::vector<const State*> st((size_t)count);
  for (int i = 0; i < count; ++i) {
    if (!members[i]) return PIBM_EINVAL;
    if (i == 0) dev = members[i]->device;
    if (members[i]->device != dev) return PIBM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return PIBM_EINVAL;
    st[i] = &members[i]->s;
  }
  DeviceGuard guard(dev);
  const bool persistent = ensemble_persistent_supported(st.data(), count);
  if (!persistent)
    for (int i = 0; i < count; ++i)
      if (members[i]->s.phy.rebin > 1) return PIBM_ENOTSUP;  // branch mode: rebuild every step
  pibm_ensemble_t* e = new (std::nothrow) pibm_ensemble_t();
  if (!e) return PIBM_ENOMEM;
  e->members.assign(members, members + count);
  e->stream = (cudaStream_t)stream;
  e->parity.assign(count, -1);
  e->graph = nullptr;
  e->device = dev;
  e->origin = nullptr;
  e->seen.assign(count, -1);
  if (cudaStreamCreateWithFlags(&e->origin, cudaStreamNonBlocking) != cudaSuccess) {
    delete e;
    return PIBM_ECUDA;
  }
  // members' own streams must be idle before the ensemble takes over
  for (int i = 0; i < count; ++i)
    if (cudaStreamSynchronize(members[i]->stream) != cudaSuccess) {
      pibm_ensemble_destroy(e);
      return PIBM_ECUDA;
    }
  if (persistent) {
    const int rc = ensemble_device_create(st.data(), count, dev, &e->pd);
    if (rc != PIBM_OK) {
      pibm_ensemble_destroy(e);
      return rc;
    }
    e->persistent = 1;
  } else {
    e->lanes.assign(count, nullptr);
    for (int i = 0; i < count; ++i)
      if (cudaStreamCreateWithFlags(&e->lanes[i], cudaStreamNonBlocking) != cudaSuccess) {
        pibm_ensemble_destroy(e);
        return PIBM_ECUDA;
      }
  }
  *out = e;
  return PIBM_OK;
}

static int ensemble_step_persistent(pibm_ensemble_t* e, int64_t nsteps) {
  const int n = (int)e->members.size();
  // a member stepped on its own since the last ensemble step: load the phase
  // table from the handles again (and clear the counts a rebuild expects)
  bool stale = false;
  for (int i = 0; i < n; ++i) stale |= e->seen[i] != e->members[i]->nstep;
  if (stale) {
    std::vector<int> cur(n), sr(n);
    for (int i = 0; i < n; ++i) {
      cur[i] = e->members[i]->s.cur;
      sr[i] = e->members[i]->since_rebin;
    }
    CK(ensemble_device_set_phase(e->pd, cur.data(), sr.data(), e->stream));
  }
  auto advance = [&](int k) {
    for (int i = 0; i < n; ++i) {
      pibm_t* m = e->members[i];
      m->s.cur ^= (k & 1);
      m->since_rebin = (int)((m->since_rebin + (int64_t)k) % m->s.phy.rebin);
      m->nstep += k;
      e->seen[i] = m->nstep;
    }
    e->launches += 1;
  };
  while (nsteps > 0) {
    if (nsteps >= ENS_GRAPH_STEPS && !e->pgraph_failed && !ensemble_device_injected(e->pd)) {
      if (!e->pgraph && ensemble_capture_persistent(e) != PIBM_OK) {
        e->pgraph_failed = 1;  // launch directly from now on
        continue;
      }
      CK(cudaGraphLaunch(e->pgraph, e->stream));
      advance(ENS_GRAPH_STEPS);
      nsteps -= ENS_GRAPH_STEPS;
    } else {
      const int k = (int)std::min<int64_t>(nsteps, ENS_GRAPH_STEPS);
      CK(ensemble_device_launch(e->pd, k, e->stream));
      advance(k);
      nsteps -= k;
    }
  }
  return PIBM_OK;
}

int pibm_ensemble_step(pibm_ensemble_t* e, int64_t nsteps) {
  if (!e || nsteps < 0) return PIBM_EINVAL;
  DeviceGuard guard(e->device);
  if (e->persistent) return ensemble_step_persistent(e, nsteps);
  while (nsteps > 0) {
    if (nsteps >= 2) {
      bool stale = !e->graph;
      for (size_t i = 0; i < e->members.size() && !stale; ++i)
        stale = e->parity[i] != e->members[i]->s.cur;
      if (stale) {
        if (e->graph) cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
        int rc = ensemble_capture(e);
        if (rc != PIBM_OK) return rc;
      }
      CK(cudaGraphLaunch(e->graph, e->stream));
      for (pibm_t* m : e->members) m->nstep += 2;
      nsteps -= 2;
    } else {
      for (pibm_t* m : e->members) {
        int rc = enqueue_step(m, e->stream, nullptr);
        if (rc != PIBM_OK) return rc;
      }
      nsteps -= 1;
    }
  }
  return PIBM_OK;
}

int pibm_ensemble_configure(pibm_ensemble_t* e, int ctas_per_sm, int cells_per_item) {
  if (!e) return PIBM_EINVAL;
  if (!e->pd) return PIBM_ENOTSUP;
  DeviceGuard guard(e->device);
  int before[4], after[4];
  ensemble_device_shape(e->pd, &before[0], &before[1], &before[2], &before[3]);
  const int rc = ensemble_device_configure(e->pd, ctas_per_sm, cells_per_item, e->stream);
  if (rc != PIBM_OK) return rc;
  ensemble_device_shape(e->pd, &after[0], &after[1], &after[2], &after[3]);
  if ((before[0] != after[0] || before[2] != after[2]) && e->pgraph) {
    CK(cudaStreamSynchronize(e->stream));  // the graph may still be running
    cudaGraphExecDestroy(e->pgraph);
    e->pgraph = nullptr;
  }
  return PIBM_OK;
}

int pibm_ensemble_autotune(pibm_ensemble_t* e, int steps_per_candidate, int* choice) {
  if (!e || steps_per_candidate < 1) return PIBM_EINVAL;
  if (!e->persistent) return PIBM_ENOTSUP;
  DeviceGuard guard(e->device);
  int per_sm = 0, max_per_sm = 0, cpi = 0;
  ensemble_device_shape(e->pd, &per_sm, &max_per_sm, &cpi, nullptr);
  static const int cpis[] = {256, 512, 1024, 2048, 4096};
  // timed steps per candidate: whole graph launches
  const int64_t timed = (steps_per_candidate + ENS_GRAPH_STEPS - 1) / ENS_GRAPH_STEPS *
                        (int64_t)ENS_GRAPH_STEPS;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PIBM_ECUDA;
  }
  int rc = PIBM_OK, best_p = per_sm, best_c = cpi, ncand = 0;
  float best_ms = 0.f;
  for (int p = 1; p <= max_per_sm && rc == PIBM_OK; ++p)
    for (int c : cpis) {
      if ((rc = pibm_ensemble_configure(e, p, c)) != PIBM_OK) break;
      // one untimed launch captures this shape's graph and warms up
      if ((rc = ensemble_step_persistent(e, ENS_GRAPH_STEPS)) != PIBM_OK) break;
      float ms = 0.f;
      cudaError_t te = cudaEventRecord(e0, e->stream);
      if (te == cudaSuccess) rc = ensemble_step_persistent(e, timed);
      if (rc != PIBM_OK) break;
      if (te != cudaSuccess || (te = cudaEventRecord(e1, e->stream)) != cudaSuccess ||
          (te = cudaEventSynchronize(e1)) != cudaSuccess ||
          (te = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        record_error("ensemble autotune timing", te);
        rc = PIBM_ECUDA;
        break;
      }
      ++ncand;
      if (ncand == 1 || ms < best_ms) {
        best_ms = ms;
        best_p = p;
        best_c = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PIBM_OK) return rc;
  if ((rc = pibm_ensemble_configure(e, best_p, best_c)) != PIBM_OK) return rc;
  if (choice) {
    choice[0] = best_p;
    choice[1] = best_c;
    choice[2] = ncand;
  }
  return pibm_ensemble_status(e);
}

int pibm_ensemble_set_mode(pibm_ensemble_t* e, int persistent) {
  if (!e || (persistent != 0 && persistent != 1)) return PIBM_EINVAL;
  DeviceGuard guard(e->device);
  if (persistent == e->persistent) return PIBM_OK;
  if (persistent) {
    if (!e->pd) return PIBM_ENOTSUP;
    e->seen.assign(e->members.size(), -1);  // reload the phase table at the next step
  } else {
    for (pibm_t* m : e->members)
      if (m->s.phy.rebin > 1) return PIBM_ENOTSUP;
    if (e->lanes.empty()) {
      e->lanes.assign(e->members.size(), nullptr);
      for (auto& ln : e->lanes) CK(cudaStreamCreateWithFlags(&ln, cudaStreamNonBlocking));
    }
  }
  e->persistent = persistent;
  return PIBM_OK;
}

int pibm_ensemble_inject_skip(pibm_ensemble_t* e, int block, double limit_s) {
  if (!e) return PIBM_EINVAL;
  if (!e->pd) return PIBM_ENOTSUP;
  return ensemble_device_inject(e->pd, block, limit_s);
}

int pibm_ensemble_info(pibm_ensemble_t* e, int* info) {
  if (!e || !info) return PIBM_EINVAL;
  for (int k = 0; k < 6; ++k) info[k] = 0;
  info[0] = e->persistent;
  if (e->pd) {
    ensemble_device_shape(e->pd, &info[1], &info[2], &info[3], &info[4]);
    info[5] = e->pgraph_failed ? 0 : 1;
  }
  return PIBM_OK;
}

int pibm_ensemble_launch_count(pibm_ensemble_t* e, int64_t* count) {
  if (!e || !count) return PIBM_EINVAL;
  *count = e->launches;
  return PIBM_OK;
}

int pibm_ensemble_status(pibm_ensemble_t* e) {
  if (!e) return PIBM_EINVAL;
  DeviceGuard guard(e->device);
  CK(cudaStreamSynchronize(e->stream));
  if (e->pd) {
    const int t = ensemble_device_timed_out(e->pd, e->stream, nullptr);
    if (t < 0) return PIBM_ECUDA;
    if (t > 0) return PIBM_ETIMEOUT;
  }
  int worst = PIBM_OK;
  for (pibm_t* m : e->members) {
    int rc = health(m);
    if (rc != PIBM_OK && worst == PIBM_OK) worst = rc;
  }
  return worst;
}

void pibm_ensemble_destroy(pibm_ensemble_t* e) {
  if (!e) return;
  DeviceGuard guard(e->device);
  if (e->stream) cudaStreamSynchronize(e->stream);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  if (e->pgraph) cudaGraphExecDestroy(e->pgraph);
  ensemble_device_destroy(e->pd);
  for (cudaStream_t s : e->lanes)
    if (s) cudaStreamDestroy(s);
  if (e->origin) cudaStreamDestroy(e->origin);
  delete e;
}

int pibm_profile_steps(pibm_t* h, int64_t nsteps, double* phase_ms) {
  if (!h || nsteps < 0 || !phase_ms) return PIBM_EINVAL;
  DeviceGuard guard(h->device);
  constexpr int NP = 4;  // bin, contacts, coupling, collide-stream
  for (int k = 0; k <= NP; ++k) phase_ms[k] = 0.0;
  if (nsteps == 0) return health(h);
  State& s = h->s;
  cudaStream_t st = h->stream;
  std::vector<cudaEvent_t> ev((size_t)NP * nsteps + 1, nullptr);
  int rc = PIBM_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = PIBM_ECUDA;
  if (rc == PIBM_OK) {
    int nk = 0;
    if (cudaEventRecord(ev[0], st) != cudaSuccess) rc = PIBM_ECUDA;
    for (int64_t i = 0; i < nsteps && rc == PIBM_OK; ++i) {
      cudaEvent_t* e = &ev[NP * i + 1];
      const bool rebuild = h->since_rebin == 0;
      s.move_consts = h->since_rebin <= 1;
      h->since_rebin = (h->since_rebin + 1) % s.phy.rebin;
      s.nb_mode = rebuild ? 1 : 2;
      if ((rebuild && launch_bin(s, st, &nk) != cudaSuccess) ||
          cudaEventRecord(e[0], st) != cudaSuccess ||
          launch_contacts(s, st, &nk) != cudaSuccess ||
          cudaEventRecord(e[1], st) != cudaSuccess ||
          launch_couple(s, st, &nk) != cudaSuccess || cudaEventRecord(e[2], st) != cudaSuccess ||
          launch_collide_stream(s, st) != cudaSuccess ||
          cudaEventRecord(e[3], st) != cudaSuccess) {
        rc = PIBM_ECUDA;
        break;
      }
      s.cur ^= 1;
      ++h->nstep;
    }
    if (rc == PIBM_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = PIBM_ECUDA;
    for (int64_t i = 0; i < nsteps && rc == PIBM_OK; ++i) {
      for (int k = 0; k < NP; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[NP * i + k], ev[NP * i + k + 1]) != cudaSuccess)
          rc = PIBM_ECUDA;
        phase_ms[k] += t;
      }
    }
    float tot = 0.f;
    if (rc == PIBM_OK && cudaEventElapsedTime(&tot, ev[0], ev[NP * nsteps]) != cudaSuccess)
      rc = PIBM_ECUDA;
    phase_ms[NP] = tot;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc != PIBM_OK) return rc;
  return health(h);
}

void pibm_destroy(pibm_t* h) {
  if (!h) return;
  DeviceGuard guard(h->device);
  cudaStreamSynchronize(h->stream);
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  for (cudaEvent_t e : {h->ev_fork, h->ev_contacts, h->ev_free})
    if (e) cudaEventDestroy(e);
  if (h->owns_ws && h->ws) cudaFree(h->ws);
  delete h;
}

}  // extern "C"
