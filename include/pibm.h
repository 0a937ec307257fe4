/*
 * pibm.h — C ABI of the GB300 library for the coupled LBM-PIBM-DEM time step of
 * Zhang et al., "PIBM: Particulate immersed boundary method for fluid-particle
 * interaction problems" (arXiv:1407.6704).
 *
 * One step of the method (section 2 of the paper):
 *   1. the fluid moments at every particle are interpolated from the lattice
 *      (Eq. 4; the interpolant is the same per-axis kernel as the spreading);
 *   2. the particle velocity is advanced under buoyancy-reduced gravity, the
 *      contact force and the fluid force (Eq. 13); the fluid force is the
 *      reaction -A_p g (Eq. 12) of the force density g that a moving bounce-back
 *      with the particle velocity exchanges with the fluid (Eqs. 6-7), which is
 *      g = 2 (rho_l U - j_l);
 *   3. A_p g is spread back to the lattice with the discrete delta (Eqs. 9-11);
 *   4. every cell collides with the BGK rule and the Guo body-force term
 *      (Eqs. 2, 3, 8; velocity u = (j + F/2) / rho) and streams.
 * Contacts are the linear spring-dashpot normal force (stiffness kn,
 * restitution e) between overlapping particles and against walls, found over a
 * cell list of lattice-sized bins. Units are lattice units (h = 1, dt = 1).
 *
 * Conventions shared by every call:
 *  - Status codes: PIBM_OK (0) on success, a negative PIBM_E* value otherwise;
 *    pibm_strerror() names it. A failed call leaves the handle usable unless it
 *    returns PIBM_ECUDA (the CUDA context may be lost).
 *  - Lattice node k of an axis sits at coordinate k + 1/2; a wall axis of extent
 *    N has resting walls at 0 and N (halfway bounce-back); a periodic axis wraps.
 *  - Cell index c = x + n[0] * (y + n[1] * z).
 *  - Velocity sets, in this order (opposites adjacent):
 *      D2Q9 : (0,0) (1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1) (1,-1) (-1,1)
 *      D3Q15: 0, +-x, +-y, +-z, (1,1,1) (-1,-1,-1) (1,1,-1) (-1,-1,1) (1,-1,1)
 *             (-1,1,-1) (-1,1,1) (1,-1,-1)
 *      D3Q19: 0, +-x, +-y, +-z, (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1)
 *             (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *  - Field arrays are structure-of-arrays FP64: populations [q][ncell],
 *    vectors [d][ncell]; particle arrays are AoS FP64 [n_particles][d].
 *  - The caller keeps ownership of every array it passes; the library copies
 *    what it needs during the call.
 *  - A handle is bound to the CUDA device that was current at pibm_create and
 *    to one stream; calls on one handle must not overlap (not thread-safe).
 */
#ifndef PIBM_H
#define PIBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PIBM_OK 0
#define PIBM_EINVAL (-1)    /* bad argument or configuration */
#define PIBM_ENOMEM (-2)    /* workspace too small or allocation failed */
#define PIBM_ECUDA (-3)     /* a CUDA call failed */
#define PIBM_EUNSTABLE (-4) /* non-finite fluid or particle state detected, a fluid speed
                               above 0.3 lattice units (Mach guard: the equilibrium of
                               Eq. 3 is a low-Mach expansion), or a particle moved farther
                               than the cell list allows (sub-cycling, rebin_every > 1) */
#define PIBM_EESCAPED (-5)  /* a particle crossed a wall */
#define PIBM_ENOTSUP (-6)   /* combination not built into this library */
#define PIBM_EINTERNAL (-7) /* a device-side index check failed; the access was skipped */
#define PIBM_ETOOBIG (-8)   /* larger than the fixed scratch of pibm_fluid_sums_noalloc */
#define PIBM_ETIMEOUT (-9)  /* a grid-wide barrier of the persistent ensemble kernel waited
                               longer than its limit; the kernel returned without finishing
                               (the members' states are then undefined) */

/* particle update precision in the 32- and 16-bit storage modes */
#define PIBM_PARTICLE_FP64 0
#define PIBM_PARTICLE_FP32 1

/* lattices (value = number of velocities q) */
#define PIBM_D2Q9 9
#define PIBM_D3Q15 15
#define PIBM_D3Q19 19

/* per-axis boundary */
#define PIBM_WALL 0
#define PIBM_PERIODIC 1

/* particle drag coupling */
#define PIBM_IMPLICIT 0 /* force density evaluated with U^{n+1} (solved in closed form) */
#define PIBM_EXPLICIT 1 /* force density evaluated with U^n */

/* interpolation of the fluid to the particles (Eq. 4) */
#define PIBM_INTERP_DELTA 0     /* the spreading kernel (delta_width), renormalised at walls */
#define PIBM_INTERP_LAGRANGE4 1 /* Eq. (5): 4-point Lagrange polynomials per axis over the
                                   nodes floor(X - 1/2) - 1 .. + 2, the block shifted inside
                                   the domain next to a wall; spreading keeps delta_width */

/* scheduling of a step (results are the same either way) */
#define PIBM_OVERLAP_AUTO 0 /* on for 2D lattices of at least 2^20 cells where supported */
#define PIBM_OVERLAP_ON 1   /* on wherever supported */
#define PIBM_OVERLAP_OFF 2  /* one stream, one collision kernel over the whole lattice */

/* normal contact law */
#define PIBM_DEM_LINEAR 0 /* k_n delta - gamma v_n, gamma = 2 beta sqrt(m_eff k_n) */
#define PIBM_DEM_HERTZ 1  /* Eq. (15): (4/3) E* sqrt(R*) delta^{3/2} - gamma v_n,
                             gamma = 2 sqrt(5/6) beta sqrt(2 E* sqrt(R* delta) m_eff);
                             1/E* = (1 - nu_1^2)/E_1 + (1 - nu_2^2)/E_2, 1/R* = 1/R_1 + 1/R_2
                             (R* = R against a wall); beta from dem_restitution as for
                             the linear law */

/* storage / arithmetic of the populations; particles, contacts and the
 * particle integration are FP64 in every mode */
#define PIBM_FP64 0 /* populations stored as f - w in FP64, FP64 collision and force */
#define PIBM_FP32 1 /* populations stored as f - w in FP32, FP32 collision and force field */
#define PIBM_FP16 2 /* populations stored as (f - w) * 2^12 in FP16, FP32 collision and force */
#define PIBM_BF16 3 /* populations stored as f - w in BF16, FP32 collision and force field */

/* fields for pibm_read_fields (bit k selects dst[k]) */
#define PIBM_FIELD_RHO (1u << 0) /* ncell: rho = sum_a f_a of the current state */
#define PIBM_FIELD_J (1u << 1)   /* d*ncell: j = sum_a e_a f_a (no half-force term) */
#define PIBM_FIELD_POP (1u << 2) /* q*ncell: post-stream populations f_a of the current state */
#define PIBM_FIELD_X (1u << 3)   /* n_particles*d: particle positions */
#define PIBM_FIELD_U (1u << 4)   /* n_particles*d: particle velocities */
#define PIBM_NFIELDS 5
/* The spread force field is consumed (and cleared) by the collision of the same
 * step; its content is fixed by the per-particle force density, which
 * pibm_forces returns as f_fpi = -A_p g. */

typedef struct pibm_config {
  int lattice;         /* PIBM_D2Q9, PIBM_D3Q15 or PIBM_D3Q19 */
  int64_t n[3];        /* lattice extents; n[2] = 1 for D2Q9 */
  int boundary[3];     /* PIBM_WALL or PIBM_PERIODIC per axis (ignored for z in 2D) */
  double tau;          /* BGK relaxation time, Eq. (2); must exceed 1/2 */
  double gravity[3];   /* acceleration on the particles; the fluid carries none */
  int delta_width;     /* 2 (linear hat) or 4 (cosine kernel, Eq. 11) */
  int coupling;        /* PIBM_IMPLICIT or PIBM_EXPLICIT */
  int precision;       /* PIBM_FP64, PIBM_FP32, PIBM_FP16 or PIBM_BF16 */
  int deterministic;   /* 0: spread with atomics; 1: ordered per-cell gather,
                          bitwise reproducible run to run. With particles, a periodic
                          axis then needs 2 R + 1 cells (and at least 5), R the gather's
                          reach: 1 for delta_width 2, 2 for 4, plus 1 when rebin_every
                          > 1; without ordered spreading it needs 5 cells. */
  double dem_kn;       /* contact stiffness */
  double dem_restitution; /* normal restitution coefficient, in (0, 1] */
  int64_t n_particles; /* may be 0 */
  const double* x0;    /* host, [n_particles][d]; every particle inside the
                          domain and at least its radius from every wall */
  const double* u0;    /* host, [n_particles][d], or NULL for particles at rest */
  const double* diameter;      /* host, [n_particles], each in (0, 1] */
  const double* density_ratio; /* host, [n_particles], rho_p / rho_f, > 0 */
  const double* f0;    /* host, [q][ncell] post-stream populations of step 0, or
                          NULL for the rest state f_a = w_a (rho = 1, u = 0) */
  /* Variants of the paper's method; a zero-initialised tail selects the
   * defaults (interpolation with the spreading kernel, linear contacts, no
   * sub-cycling). */
  int interp;          /* PIBM_INTERP_DELTA or PIBM_INTERP_LAGRANGE4 (every wall axis
                          then needs n >= 4) */
  int dem_model;       /* PIBM_DEM_LINEAR or PIBM_DEM_HERTZ (dem_kn is then unused) */
  double dem_young;    /* Hertz: Young's modulus of the particles, > 0 (lattice units) */
  double dem_poisson;  /* Hertz: Poisson ratio of the particles, in [0, 1/2) */
  double wall_young;   /* Hertz: Young's modulus of the walls; 0 = the particles' */
  double wall_poisson; /* Hertz: Poisson ratio of the walls (used when wall_young > 0) */
  int dem_substeps;    /* DEM sub-steps S per fluid step (0 or 1: none). With S > 1 the
                          interpolated rho_l, j_l stay fixed for the step, contacts and
                          the particle update run S times with h = 1/S, and the fluid
                          receives the sub-step average of the force density. Every
                          particle's displacement within one step must stay below
                          (1 - largest diameter) / 2 so that the cell list of the step
                          start still holds every pair that can touch; a larger one
                          raises PIBM_EUNSTABLE. */
  int rebin_every;     /* rebuild the cell list every R steps (0 or 1: every step). In
                          between, the contact search and the ordered spreading use the
                          bins of the last rebuild and the contact candidates it recorded;
                          this finds every touching pair as long as each particle stays
                          within (1 - largest diameter) / 2 of the cell it had at the last
                          rebuild and within (1 - largest diameter) / 4 of its position
                          then, on every axis, which is checked on the device every step
                          (PIBM_EUNSTABLE when violated). Results equal those of R = 1 up to
                          the summation order. Needs dem_substeps <= 1. */
  int overlap;         /* PIBM_OVERLAP_AUTO (0), PIBM_OVERLAP_ON or PIBM_OVERLAP_OFF.
                          With overlap a step runs the contact search, then the collision
                          of the free tiles (those no particle stencil reaches until the
                          next cell-list rebuild), on a second stream of the handle, beside
                          the moment and coupling kernels; the collision of the other tiles
                          follows both. Every cell's arithmetic is unchanged. Supported
                          with 32- or 64-bit storage and without ordered spreading
                          (deterministic); elsewhere the step runs on one stream. */
  int particle_update; /* 32- and 16-bit storage: PIBM_PARTICLE_FP64 (0, default) forms
                          U' - U and the force density g (Eqs. 6, 7, 13) in FP64 from the
                          FP64 mass, A_p, buoyancy and contact force, with the
                          interpolated rho_l, j_l widened from FP32; PIBM_PARTICLE_FP32
                          (1) forms them in FP32 and adds the increment to the FP64 state
                          (about 6 % faster per step on the 2048^2 workload). Positions
                          and velocities are FP64 state either way. FP64 storage always
                          updates in FP64. */
} pibm_config;

typedef struct pibm_t pibm_t; /* opaque handle owning the device state */

/* Device bytes that pibm_create needs for this configuration.
 * Returns PIBM_EINVAL for an invalid configuration. */
int pibm_workspace_bytes(const pibm_config* cfg, size_t* bytes);

/* Validate cfg, lay out the device state and upload the initial condition.
 * workspace: device memory of at least pibm_workspace_bytes() bytes, 256-byte
 *   aligned, owned by the caller and kept alive until pibm_destroy; or NULL, in
 *   which case the library allocates (and later frees) it with cudaMalloc.
 * stream: the cudaStream_t every later call is ordered on (NULL = legacy
 *   default stream). Returns with the upload complete.
 * Errors: PIBM_EINVAL (tau <= 1/2, bad lattice/width/precision, a particle
 *   outside the domain or closer than its radius to a wall, diameter outside
 *   (0, 1], NULL arrays with n_particles > 0), PIBM_ENOMEM, PIBM_ECUDA. */
int pibm_create(const pibm_config* cfg, void* workspace, size_t workspace_bytes, void* stream,
                pibm_t** out);

/* Advance nsteps coupled time steps, asynchronously on the handle's stream
 * (whole cell-list rebuild periods are replayed from CUDA graphs). With overlap
 * the work of each step forks onto a second stream of the handle and joins back
 * before the step ends, so the handle's stream orders everything after it.
 * Health flags raised on the device (non-finite state, a fluid speed above the
 * Mach guard, escaped particle, a particle beyond the skin of a kept cell list)
 * are reported by the next synchronising call; after such a flag the state is
 * not meaningful. */
int pibm_step(pibm_t* h, int64_t nsteps);

/* Per-particle forces of the last step, AoS [n_particles][d] FP64:
 * f_fpi = -A_p g (Eq. 12), f_contact = the contact force. Either pointer may be
 * NULL. on_device != 0: the pointers are device memory on the handle's device.
 * Synchronises the stream; returns the device health status. */
int pibm_forces(pibm_t* h, double* f_fpi, double* f_contact, int on_device);

/* Copy the fields selected by mask into dst[k] (bit k of mask), FP64, layouts
 * as documented at PIBM_FIELD_*. Entries of dst for unselected bits are ignored.
 * Synchronises the stream; returns the device health status. */
int pibm_read_fields(pibm_t* h, unsigned mask, void* const* dst, int on_device);

/* Global invariants of the current state, FP64, reduced in a fixed order:
 * out[0] = total mass sum rho, out[1..d] = fluid momentum sum j,
 * out[1+d..2d] = particle momentum sum m U. Synchronises the stream. */
int pibm_invariants(pibm_t* h, double* out);

/* Synchronise the stream and return the device health status. */
int pibm_status(pibm_t* h);

/* Number of kernels one pibm_step(h, 1) launches (for launch accounting); with
 * rebin_every > 1, the count of a step that rebuilds the cell list. With
 * overlap the collision counts as two kernels (free and busy tiles). */
int pibm_kernels_per_step(pibm_t* h);

/* Total number of kernels pibm_step has launched on this handle since it was
 * created (graph replays included), into *count. */
int pibm_launch_count(pibm_t* h, int64_t* count);

/* Advance nsteps steps like pibm_step, launched one phase at a time with CUDA
 * events between the phases, and return the summed device time of each phase
 * in milliseconds: phase_ms[0] cell-list binning, phase_ms[1] contact forces,
 * phase_ms[2] particle coupling (interpolation, update, spreading),
 * phase_ms[3] fused stream-collide, phase_ms[4] the whole steps (first event to
 * last). Synchronises the stream. Not part of the method; a timing aid. */
int pibm_profile_steps(pibm_t* h, int64_t nsteps, double* phase_ms);

/* Gradient of the mean settling velocity by the discrete adjoint of the
 * coupled step (FP64). Runs nsteps steps of cfg from its initial state and
 * returns in *loss the particles' mean velocity along the last axis after the
 * last step, L = (1/N) sum_p U_p[d-1], and the exact derivatives of the computed
 * L (the adjoint of every discrete operation of the step, Eqs. 2-13):
 *   dtau: dL/dtau (one double; may be NULL),
 *   drho: [n_particles] dL/d(density ratio of each particle) (may be NULL),
 *   dx0:  [n_particles][d] dL/d(initial position) (may be NULL);
 * all host pointers. The forward run is the library's deterministic step; the
 * state is checkpointed every checkpoint_every steps and each stretch is
 * replayed for the reverse sweep, which needs device memory for
 * (ceil(nsteps / checkpoint_every) + checkpoint_every) copies of the workspace of
 * pibm_workspace_bytes(cfg). The call allocates and frees that memory itself and
 * returns when done, on `stream` (a cudaStream_t, NULL = legacy default).
 * Supported: precision PIBM_FP64, PIBM_IMPLICIT, PIBM_INTERP_DELTA (width 2 or
 * 4), PIBM_DEM_LINEAR, no sub-cycling, rebin_every <= 1, n_particles >= 1; else PIBM_ENOTSUP or
 * PIBM_EINVAL. Contacts make L non-smooth where an overlap starts or ends; the
 * result is the derivative of the branch the run took. Errors as pibm_create,
 * PIBM_ENOMEM when the checkpoints do not fit, and the run's health status. */
int pibm_settling_gradient(const pibm_config* cfg, int64_t nsteps, int64_t checkpoint_every,
                           void* stream, double* loss, double* dtau, double* drho, double* dx0);

/* Pick the block shape of the fused stream-collide kernel for this handle by
 * timing a fixed list of candidates on its stream (not part of the method; a
 * tuning aid). The timing runs leave the simulation state unchanged. block_xy
 * (may be NULL) receives the chosen shape. Synchronises the stream. */
int pibm_autotune(pibm_t* h, int* block_xy);

/* Ensembles: independent simulations (each made by pibm_create, possibly with
 * different lattices, particle counts and parameters) that advance together.
 * Two modes, chosen by pibm_ensemble_create:
 *  - persistent, when every member is D2Q9 with FP32 or FP64 storage (the same
 *    for all), the same delta width, delta interpolation, linear contacts, no
 *    DEM sub-cycling, and there are at most 256 members: one cooperative kernel
 *    runs every phase of the coupled step (Eqs. 2-13: cell list, contacts,
 *    moment field, interpolation, update, spreading, stream-collide) for all
 *    members, with grid-wide barriers between the phases; a launch covers up to
 *    10 steps, and the 10-step launch is replayed from a CUDA graph. Work items
 *    (256 particles, a run of lattice cells, a block of tiles) are numbered per
 *    member from offset tables and split evenly over the CTAs. A member follows
 *    the same arithmetic as when stepped alone, with any rebin_every (each
 *    member keeps its own cell-list period);
 *  - branches, otherwise: pibm_ensemble_step captures two steps of every member
 *    into one CUDA graph, one independent branch per member, and replays it;
 *    members must then rebuild their cell list every step (rebin_every <= 1,
 *    else PIBM_ENOTSUP).
 * Members stay ordinary handles (read them with pibm_read_fields etc. after
 * pibm_ensemble_status); stepping a member on its own between ensemble steps is
 * allowed when the caller orders the two streams. All members must live on one
 * device; the ensemble does not own them and must be destroyed before them.
 * pibm_ensemble_create synchronises the members' streams. Errors: PIBM_EINVAL
 * (no members, NULL or repeated member, members on different devices),
 * PIBM_ENOTSUP, PIBM_ENOMEM (device tables of the persistent mode), PIBM_ECUDA. */
typedef struct pibm_ensemble_t pibm_ensemble_t;
int pibm_ensemble_create(pibm_t* const* members, int count, void* stream, pibm_ensemble_t** out);
int pibm_ensemble_step(pibm_ensemble_t* e, int64_t nsteps);
/* Synchronise the ensemble's stream; PIBM_ETIMEOUT if a barrier of the
 * persistent kernel gave up, else the first non-OK member health status. */
int pibm_ensemble_status(pibm_ensemble_t* e);
void pibm_ensemble_destroy(pibm_ensemble_t* e);
/* Persistent mode only (PIBM_ENOTSUP otherwise). Launch shape: ctas_per_sm CTAs
 * of 256 threads per SM (0: as many as fit; at most that many) and
 * cells_per_item lattice cells per collision work item (0: unchanged; a positive
 * multiple of 256; default 1024). Takes effect at the next launch; the graph
 * captured before is kept only when the shape is unchanged. Errors: PIBM_EINVAL. */
int pibm_ensemble_configure(pibm_ensemble_t* e, int ctas_per_sm, int cells_per_item);
/* Pick the persistent launch shape by timing: every candidate (CTAs per SM from
 * 1 to the largest that fits, x cells per item 256, 512, 1024, 2048, 4096)
 * advances the ensemble by 10 untimed steps (which capture its graph) and then
 * by steps_per_candidate steps rounded up to a multiple of 10, timed with
 * events on the ensemble's stream; the fastest is kept. These are real steps:
 * the ensemble moves on by candidates x (10 + that rounded count) steps.
 * choice (may be NULL) receives {ctas_per_sm, cells_per_item, candidates}.
 * Synchronises the stream. PIBM_ENOTSUP when the members do not qualify for
 * the persistent mode. */
int pibm_ensemble_autotune(pibm_ensemble_t* e, int steps_per_candidate, int* choice);
/* info[6]: {1 persistent / 0 branches, CTAs per SM, largest CTAs per SM that fit,
 * cells per collision item, CTAs of the grid, 1 when the launches replay from a
 * CUDA graph}; entries 1-5 are 0 when the members do not qualify for the
 * persistent mode. */
int pibm_ensemble_info(pibm_ensemble_t* e, int* info);
/* Switch between the persistent mode (1; PIBM_ENOTSUP when the members do not
 * qualify) and the branch mode (0; PIBM_ENOTSUP when a member keeps its cell
 * list, rebin_every > 1). Members keep their states; takes effect at the next
 * pibm_ensemble_step. */
int pibm_ensemble_set_mode(pibm_ensemble_t* e, int persistent);
/* Persistent kernel launches made by pibm_ensemble_step so far. */
int pibm_ensemble_launch_count(pibm_ensemble_t* e, int64_t* count);
/* Fault injection for tests (persistent mode): in the next launch, CTA `block`
 * does not arrive at the first grid barrier, and every barrier wait of the
 * ensemble gives up after limit_s seconds (0 < limit_s <= 10; the limit stays).
 * The launch then returns early, pibm_ensemble_status reports PIBM_ETIMEOUT and
 * every later launch of the ensemble returns at once. Nothing faults or hangs. */
int pibm_ensemble_inject_skip(pibm_ensemble_t* e, int block, double limit_s);

/* Grid-barrier self-test: one cooperative launch of nblocks CTAs that pass
 * nbarriers grid-wide barriers of the persistent kernel's kind; CTA skip_block
 * (-1: none) does not arrive at the first one. Each wait gives up after limit_s
 * seconds (0 < limit_s <= 10). Returns PIBM_OK when all barriers passed (*passed
 * = nbarriers), PIBM_ETIMEOUT when a wait gave up (*passed = 0), PIBM_EINVAL when
 * nblocks CTAs cannot all be resident at once or an argument is out of range,
 * PIBM_ENOMEM, PIBM_ECUDA. Synchronises the device. */
int pibm_grid_barrier_test(int nblocks, int skip_block, int nbarriers, double limit_s,
                           int* passed);

/* Free the handle (and the workspace when the library allocated it). NULL is a no-op. */
void pibm_destroy(pibm_t* h);

const char* pibm_strerror(int status);

/* Total mass and fluid momentum of a population field held by the caller, with
 * no device allocation of any kind (no cudaMalloc, cudaFree or allocating
 * library routine). The paper has no counterpart; this is a service for callers
 * that must not allocate device memory: code running inside a stream capture it
 * does not own (an allocation there would break the capture or synchronise the
 * device), real-time stepping loops held to a fixed memory budget, and
 * allocator hooks that must not re-enter the allocator.
 * f: device, [q][ncell] FP64 populations in the layout of PIBM_FIELD_POP, at
 *   least q * ncell doubles; lattice: PIBM_D2Q9 / PIBM_D3Q15 / PIBM_D3Q19;
 *   n: extents (n[2] = 1 for D2Q9); ncell = n[0] n[1] n[2].
 * out: device, 1 + d doubles, written with sum_a f_a (total mass) and
 *   sum_a e_a f_a (fluid momentum), summed in a fixed order (run to run
 *   identical for the same input and size).
 * stream: cudaStream_t to run on (NULL = legacy default stream); the call is
 *   asynchronous and reports launch errors only.
 * Limits and sharing: partial sums live in one file-scope static device array
 *   of 128 KiB that every GPU loading this library holds until the process
 *   exits; ncell may not exceed 16,777,216 (PIBM_ETOOBIG otherwise, nothing is
 *   launched). All calls on a device share that array and keep the last call's
 *   partials, so calls that overlap on the GPU (different streams without
 *   ordering) race and give wrong sums; order them on one stream.
 * The first call on each device looks up the array's device address with that
 *   device current (cudaGetSymbolAddress); make that first call before any
 *   stream capture that will contain later calls.
 * Errors: PIBM_EINVAL (NULL pointer, bad lattice or extents), PIBM_ETOOBIG (any
 *   extents whose product exceeds the limit, checked without overflow),
 *   PIBM_ECUDA (the failed call is named by pibm_last_error). On entry the call
 *   clears any CUDA error still pending on this thread from an earlier call, so
 *   that it is not reported as this call's own. */
int pibm_fluid_sums_noalloc(const double* f, int lattice, const int64_t n[3], double* out,
                            void* stream);

/* Text of the last failed CUDA call made by this library on the calling thread
 * (name of the call, CUDA error name and description), or "" if none failed.
 * The string stays valid until the next failing call on this thread. */
const char* pibm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PIBM_H */
