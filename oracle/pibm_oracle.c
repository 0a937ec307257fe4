/*
 * PIBM oracle: a plain, slow, double-precision CPU statement of one coupled
 * LBM-PIBM-DEM time step of Zhang et al., "PIBM: Particulate immersed boundary
 * method for fluid-particle interaction problems" (arXiv:1407.6704).
 *
 * TEST INFRASTRUCTURE. This file is the yardstick the CUDA library is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it. It shares no code, header, table generator or
 * helper with the CUDA path, and the CUDA path never calls it.
 *
 * Equation numbers are the paper's printed numbers:
 *   (1) velocity set, (2) BGK update, (3) equilibrium, (4) interpolation to a
 *   particle, (5) Lagrange interpolant, (6) moving bounce-back, (7) force
 *   density, (8) body-force term, (9) spreading, (10) discrete delta,
 *   (11) one-dimensional kernel, (12) reaction force, (13) translation ODE,
 *   (15) Hertz normal force-displacement law.
 *
 * Frame and readings used throughout (the paper is silent on them):
 *  - lattice units, h = 1, dt = 1, c = 1, c_s^2 = 1/3;
 *  - node k on an axis sits at coordinate k + 1/2; a wall axis of extent N has
 *    walls at 0 and N (halfway bounce-back); a periodic axis wraps;
 *  - f holds the post-stream (pre-collision) populations of step n, i.e. the
 *    f(r, t) of Eq. (2);
 *  - one step: interpolate the populations to every particle (Eq. 4), compute
 *    the DEM contact force on the old positions, update the particle velocity
 *    (implicit in the drag by default), form the force density with the
 *    moving bounce-back (Eqs. 6-7), move the particle, spread A_p g into F
 *    (Eq. 9), collide every cell with the Guo term (Eqs. 2, 3, 8), stream;
 *  - Eq. (7) is read as the momentum exchange sum_beta e_beta [f_beta(new) -
 *    f_beta(old)] at the particle, which equals 2 (rho_l U - j_l);
 *  - the interpolation weights are, by default, the same per-axis kernel as the
 *    spreading (2-point hat or the 4-point cosine of Eq. 11); taps that fall
 *    outside a wall axis are dropped and the remaining weights are renormalised
 *    per axis. The alternative (interp = 1) is the 4-point Lagrange polynomial
 *    of Eq. (5) over a 4-node block per axis, shifted to lie inside the domain
 *    next to a wall (one-sided, an extrapolation there as the paper describes);
 *  - contacts: linear spring-dashpot normal force (k_n, restitution e) by
 *    default, or (contact = 1) the Hertz law of Eq. (15) with the damping of the
 *    Hertz-Mindlin model of Tsuji et al. (1992) for the same restitution
 *    coefficient; brute force over all pairs, plus the walls; no tangential
 *    force, no rotation;
 *  - DEM sub-cycling (substeps S > 1): the interpolated rho_l, j_l stay fixed
 *    for the fluid step, the contact forces and the particle update run S
 *    times with h = 1/S, and the fluid receives the time average of the force
 *    density; S = 1 is the plain step.
 *
 * Stored populations: every array of populations holds g_a = f_a - w_a, the
 * deviation from the rest state (f_a = w_a, rho = 1, u = 0), with w_a the exact
 * weights of the velocity set. This is the same method with f = w + g
 * substituted: the rest state is a fixed point of Eqs. (2), (3) and (8) with
 * zero force, and of streaming (w_a is constant across the lattice and equal
 * for opposite directions), so g obeys the same update with
 * g^eq_a = f^eq_a - w_a = w_a [(rho - 1) + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)],
 * rho = 1 + sum_a g_a and j = sum_a e_a g_a. Only the rounding differs: in a weakly
 * driven flow f is about w while the flow lives in g, so every step rounds at the
 * scale of g rather than of w.
 *
 * Layouts: populations g[a * ncell + c], c = x + nx * (y + ny * z);
 * force F[k * ncell + c]; particle vectors are AoS with d components.
 *
 * Threads: built with -fopenmp, the loops over cells and the per-particle
 * updates (each reads the step-n state and writes only its own particle's
 * results) run in parallel; the spreading, whose sums into shared cells fix the
 * summation order, stays serial in particle index order. Every value is then
 * computed by the same operations as in the serial build, so the two builds give
 * bitwise identical results (a test checks this).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXQ 19
#define OR_PI 3.14159265358979323846

typedef struct {
  int q;              /* 9 (D2Q9), 15 (D3Q15) or 19 (D3Q19) */
  int n[3];           /* lattice extents; n[2] = 1 in 2D */
  int periodic[3];    /* 1 = periodic axis, 0 = walls at 0 and n */
  double tau;         /* relaxation time of Eq. (2) */
  int delta_width;    /* 2 (hat) or 4 (cosine, Eq. 11) */
  int implicit_drag;  /* 1: drag uses U^{n+1}; 0: drag uses U^n (explicit) */
  double gravity[3];  /* acceleration acting on particles */
  double kn;          /* contact spring stiffness */
  double restitution; /* normal restitution coefficient */
  int interp;         /* 0: same kernel as the spreading; 1: 4-point Lagrange, Eq. (5) */
  int contact;        /* 0: linear spring-dashpot; 1: Hertz, Eq. (15) */
  double young, poisson;           /* particle material (Hertz) */
  double wall_young, wall_poisson; /* wall material (Hertz) */
  int substeps;       /* DEM sub-steps per fluid step; <= 1 means 1 */
} or_params;

typedef struct {
  int d, q;
  int e[OR_MAXQ][3];
  double w[OR_MAXQ];
  int opp[OR_MAXQ];
} or_lattice_t;

/* Velocity sets, Eq. (1). Opposite directions are adjacent: a = 2k-1, 2k. */
static int or_lattice_get(int q, or_lattice_t* L) {
  static const int e9[9][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                               {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
  static const int e15[15][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                 {0, 0, 1},   {0, 0, -1},  {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                                 {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
  static const int e19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                 {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                 {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
  const int(*e)[3];
  if (q == 9) {
    e = e9;
    L->d = 2;
  } else if (q == 15) {
    e = e15;
    L->d = 3;
  } else if (q == 19) {
    e = e19;
    L->d = 3;
  } else {
    return -1;
  }
  L->q = q;
  for (int a = 0; a < q; ++a) {
    int s = 0;
    for (int k = 0; k < 3; ++k) {
      L->e[a][k] = e[a][k];
      s += e[a][k] * e[a][k];
    }
    /* weights by speed class */
    if (q == 9) L->w[a] = (s == 0) ? 4.0 / 9.0 : (s == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
    if (q == 15) L->w[a] = (s == 0) ? 2.0 / 9.0 : (s == 1) ? 1.0 / 9.0 : 1.0 / 72.0;
    if (q == 19) L->w[a] = (s == 0) ? 1.0 / 3.0 : (s == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
  }
  for (int a = 0; a < q; ++a) {
    L->opp[a] = -1;
    for (int b = 0; b < q; ++b)
      if (e[b][0] == -e[a][0] && e[b][1] == -e[a][1] && e[b][2] == -e[a][2]) L->opp[a] = b;
  }
  return 0;
}

int or_lattice(int q, int* d, int* e, double* w, int* opp) {
  or_lattice_t L;
  if (or_lattice_get(q, &L)) return -1;
  *d = L.d;
  for (int a = 0; a < q; ++a) {
    for (int k = 0; k < 3; ++k) e[3 * a + k] = L.e[a][k];
    w[a] = L.w[a];
    opp[a] = L.opp[a];
  }
  return 0;
}

static long or_ncell(const or_params* p) { return (long)p->n[0] * p->n[1] * p->n[2]; }

static long or_cell(const or_params* p, const int* x) {
  return x[0] + (long)p->n[0] * (x[1] + (long)p->n[1] * x[2]);
}

/* One-dimensional kernels. 2-point: the linear hat (the 2-point Lagrange
 * interpolant). 4-point: Eq. (11), 1/4 (1 + cos(pi a / 2)) for |a| <= 2. */
double or_phi(int width, double a) {
  double r = fabs(a);
  if (width == 2) return r < 1.0 ? 1.0 - r : 0.0;
  if (r > 2.0) return 0.0;
  return 0.25 * (1.0 + cos(OR_PI * a / 2.0));
}

/* Taps and weights along one axis for a particle at coordinate X.
 * b = floor(X - 1/2) is the node just below X; the 2-point stencil is {b, b+1},
 * the 4-point one {b-1, ..., b+2}. Weight of node k: phi(k + 1/2 - X).
 * Wall axis: taps outside [0, N-1] are dropped and the kept weights are
 * divided by their sum. Periodic axis: indices wrap. Returns the tap count. */
int or_taps(const or_params* p, int axis, double X, int* idx, double* w) {
  int N = p->n[axis];
  int b = (int)floor(X - 0.5);
  int first = (p->delta_width == 2) ? b : b - 1;
  int cnt = 0;
  double sum = 0.0;
  for (int t = 0; t < p->delta_width; ++t) {
    int k = first + t;
    double wk = or_phi(p->delta_width, (double)k + 0.5 - X);
    if (p->periodic[axis]) {
      int kk = ((k % N) + N) % N;
      idx[cnt] = kk;
      w[cnt] = wk;
      ++cnt;
    } else if (k >= 0 && k < N) {
      idx[cnt] = k;
      w[cnt] = wk;
      sum += wk;
      ++cnt;
    }
  }
  if (!p->periodic[axis]) {
    for (int t = 0; t < cnt; ++t) w[t] /= sum;
  }
  return cnt;
}

/* Eq. (5) along one axis: the 4-point Lagrange interpolant. The block is the
 * nodes first .. first + 3, first = floor(X - 1/2) - 1 (two nodes on each side
 * of X); on a wall axis it is shifted to lie inside [0, N - 1] (needs N >= 4),
 * on a periodic axis the indices wrap. Weight of node t, at x_t = first + t +
 * 1/2: the product over the other nodes l of (X - x_l) / (x_t - x_l). */
int or_lagrange_taps(const or_params* p, int axis, double X, int* idx, double* w) {
  int N = p->n[axis];
  int first = (int)floor(X - 0.5) - 1;
  if (!p->periodic[axis]) {
    if (first < 0) first = 0;
    if (first > N - 4) first = N - 4;
  }
  for (int t = 0; t < 4; ++t) {
    double xt = (double)(first + t) + 0.5;
    double L = 1.0;
    for (int l = 0; l < 4; ++l) {
      if (l == t) continue;
      double xl = (double)(first + l) + 0.5;
      L *= (X - xl) / (xt - xl);
    }
    int k = first + t;
    idx[t] = p->periodic[axis] ? ((k % N) + N) % N : k;
    w[t] = L;
  }
  return 4;
}

/* The interpolation taps of the configured interpolant (Eq. 4 with Eq. 5 or
 * with the spreading kernel). */
int or_interp_taps(const or_params* p, int axis, double X, int* idx, double* w) {
  if (p->interp == 1) return or_lagrange_taps(p, axis, X, idx, w);
  return or_taps(p, axis, X, idx, w);
}

/* Macroscopic moments of the stored populations g = f - w: rho = sum f =
 * 1 + sum g, j = sum e f = sum e g. */
void or_moments(const or_params* p, const double* f, double* rho, double* j) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  long nc = or_ncell(p);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < L.q; ++a) {
      double v = f[a * nc + c];
      r += v;
      for (int k = 0; k < L.d; ++k) m[k] += L.e[a][k] * v;
    }
    rho[c] = 1.0 + r;
    for (int k = 0; k < L.d; ++k) j[k * nc + c] = m[k];
  }
}

/* Eq. (4): every population interpolated to the particle position X with the
 * tensor-product weights of the per-axis interpolation taps, on the stored
 * deviations g = f - w (the weights sum to one, so f(X) = w + g(X)). */
void or_interp_pops(const or_params* p, const double* f, const double* X, double* fl) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  long nc = or_ncell(p);
  int idx[3][4], cnt[3] = {1, 1, 1};
  double w[3][4];
  idx[2][0] = 0;
  w[2][0] = 1.0;
  for (int k = 0; k < L.d; ++k) cnt[k] = or_interp_taps(p, k, X[k], idx[k], w[k]);
  for (int a = 0; a < L.q; ++a) fl[a] = 0.0;
  for (int tz = 0; tz < cnt[2]; ++tz)
    for (int ty = 0; ty < cnt[1]; ++ty)
      for (int tx = 0; tx < cnt[0]; ++tx) {
        int x[3] = {idx[0][tx], idx[1][ty], idx[2][tz]};
        double wt = w[0][tx] * w[1][ty] * w[2][tz];
        long c = or_cell(p, x);
        for (int a = 0; a < L.q; ++a) fl[a] += wt * f[a * nc + c];
      }
}

static double or_mass(int d, double dia, double rr) {
  if (d == 2) return rr * OR_PI * dia * dia / 4.0; /* per unit depth */
  return rr * OR_PI * dia * dia * dia / 6.0;
}

/* Minimum-image separation on periodic axes. */
static double or_sep(const or_params* p, int k, double a, double b) {
  double s = a - b;
  if (p->periodic[k]) {
    double N = (double)p->n[k];
    if (s > 0.5 * N) s -= N;
    if (s < -0.5 * N) s += N;
  }
  return s;
}

/* Magnitude of the normal contact force (positive = repulsive) for an overlap
 * delta > 0 and a normal relative velocity vn (positive = separating), with
 * reduced mass meff, effective radius Rs and effective modulus Es.
 * Linear: k_n delta - gamma vn, gamma = 2 beta sqrt(meff k_n).
 * Hertz, Eq. (15): (4/3) Es sqrt(Rs) delta^{3/2}, damped by gamma vn with
 * gamma = 2 sqrt(5/6) beta sqrt(S_n meff), S_n = 2 Es sqrt(Rs delta) the
 * contact stiffness (Tsuji et al. 1992). beta = -ln e / sqrt(pi^2 + ln^2 e). */
static double or_normal_force(const or_params* p, double beta, double delta, double vn,
                              double meff, double Rs, double Es) {
  if (p->contact == 1) {
    double Sn = 2.0 * Es * sqrt(Rs * delta);
    double gam = 2.0 * sqrt(5.0 / 6.0) * beta * sqrt(Sn * meff);
    return (4.0 / 3.0) * Es * sqrt(Rs) * pow(delta, 1.5) - gam * vn;
  }
  double gam = 2.0 * beta * sqrt(meff * p->kn);
  return p->kn * delta - gam * vn;
}

/* Contact force on particle i, summed over every other particle (brute force,
 * ascending index) and over the walls, along the normal. Effective radius
 * 1/R* = 1/R_1 + 1/R_2 (R* = R_i against a wall) and modulus
 * 1/E* = (1 - nu_1^2)/E_1 + (1 - nu_2^2)/E_2 (Eq. 15). */
void or_contact_force(const or_params* p, long np, const double* X, const double* U,
                      const double* dia, const double* rr, long i, double* Fc) {
  int d = (p->q == 9) ? 2 : 3;
  double lne = log(p->restitution);
  double beta = -lne / sqrt(OR_PI * OR_PI + lne * lne);
  double mi = or_mass(d, dia[i], rr[i]);
  double ri = 0.5 * dia[i];
  double cp = 0.0, Epp = 0.0, Epw = 0.0;
  if (p->contact == 1) {
    cp = (1.0 - p->poisson * p->poisson) / p->young;
    Epp = 1.0 / (cp + cp);
    Epw = 1.0 / (cp + (1.0 - p->wall_poisson * p->wall_poisson) / p->wall_young);
  }
  for (int k = 0; k < d; ++k) Fc[k] = 0.0;
  for (long jx = 0; jx < np; ++jx) {
    if (jx == i) continue;
    double s[3], dist2 = 0.0;
    for (int k = 0; k < d; ++k) {
      s[k] = or_sep(p, k, X[i * d + k], X[jx * d + k]);
      dist2 += s[k] * s[k];
    }
    double dist = sqrt(dist2);
    double rj = 0.5 * dia[jx];
    double delta = ri + rj - dist;
    if (delta <= 0.0 || dist <= 0.0) continue;
    double mj = or_mass(d, dia[jx], rr[jx]);
    double meff = mi * mj / (mi + mj);
    double vn = 0.0;
    for (int k = 0; k < d; ++k) vn += (U[i * d + k] - U[jx * d + k]) * (s[k] / dist);
    double mag = or_normal_force(p, beta, delta, vn, meff, ri * rj / (ri + rj), Epp);
    for (int k = 0; k < d; ++k) Fc[k] += mag * (s[k] / dist);
  }
  for (int k = 0; k < d; ++k) {
    if (p->periodic[k]) continue;
    /* wall at 0, normal +e_k */
    double delta = ri - X[i * d + k];
    if (delta > 0.0) Fc[k] += or_normal_force(p, beta, delta, U[i * d + k], mi, ri, Epw);
    /* wall at N, normal -e_k */
    delta = ri - ((double)p->n[k] - X[i * d + k]);
    if (delta > 0.0) Fc[k] -= or_normal_force(p, beta, delta, -U[i * d + k], mi, ri, Epw);
  }
}

/* Particle phase for particle i (§2.2-2.3) without sub-cycling (S = 1), from
 * the step-n state:
 * outputs X^{n+1}, U^{n+1}, the force density g (Eq. 7) and the contact force.
 * diag[0] receives |g_literal - 2 (rho_l U - j_l)| (max over components).
 * Returns 1 if the particle left the domain through a wall, else 0. */
int or_particle_update(const or_params* p, const double* f, long np, const double* X,
                       const double* U, const double* dia, const double* rr, long i,
                       double* Xn, double* Un, double* g, double* Fc, double* diag) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  int d = L.d;
  double fl[OR_MAXQ];
  or_interp_pops(p, f, X + i * d, fl); /* Eq. (4), fl = f(X_l) - w */
  double sum_l = 0.0, j_l[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < L.q; ++a) {
    sum_l += fl[a];
    for (int k = 0; k < d; ++k) j_l[k] += L.e[a][k] * fl[a];
  }
  double rho_l = 1.0 + sum_l;
  or_contact_force(p, np, X, U, dia, rr, i, Fc);
  double m = or_mass(d, dia[i], rr[i]);
  double Ap = OR_PI * dia[i] * dia[i] / 4.0;
  double buoy = m * (1.0 - 1.0 / rr[i]); /* Eq. (13): (1 - rho_f / rho_p) m g */
  double Ub[3];                           /* velocity seen by the bounce-back */
  for (int k = 0; k < d; ++k) {
    double Uo = U[i * d + k];
    if (p->implicit_drag) {
      /* m (U' - U) = buoy g + Fc - A_p * 2 (rho_l U' - j_l), solved for U' */
      Un[k] = (m * Uo + 2.0 * Ap * j_l[k] + buoy * p->gravity[k] + Fc[k]) /
              (m + 2.0 * Ap * rho_l);
      Ub[k] = Un[k];
    } else {
      Un[k] = Uo + (buoy * p->gravity[k] + Fc[k] - Ap * 2.0 * (rho_l * Uo - j_l[k])) / m;
      Ub[k] = Uo;
    }
  }
  /* Eq. (6): population bounced into beta = opposite(alpha) by the moving
   * particle; Eq. (7): momentum exchanged, sum_beta e_beta (new - old). Both
   * sides are taken minus w (w_alpha = w_beta), which leaves the differences
   * unchanged. */
  double fnew[OR_MAXQ];
  for (int a = 0; a < L.q; ++a) {
    double eu = 0.0;
    for (int k = 0; k < d; ++k) eu += L.e[a][k] * Ub[k];
    fnew[L.opp[a]] = fl[a] - 2.0 * L.w[a] * rho_l * eu * 3.0; /* 1 / c_s^2 = 3 */
  }
  double dev = 0.0;
  for (int k = 0; k < d; ++k) {
    double s = 0.0;
    for (int b = 0; b < L.q; ++b) s += L.e[b][k] * (fnew[b] - fl[b]);
    g[k] = s;
    double closed = 2.0 * (rho_l * Ub[k] - j_l[k]);
    double dd = fabs(s - closed);
    if (dd > dev) dev = dd;
  }
  if (diag) diag[0] = dev;
  int escaped = 0;
  for (int k = 0; k < d; ++k) {
    double x = X[i * d + k] + Un[k];
    if (p->periodic[k]) {
      double N = (double)p->n[k];
      if (x < 0.0) x += N;
      else if (x >= N) x -= N;
    } else if (x < 0.0 || x > (double)p->n[k]) {
      escaped = 1;
    }
    Xn[k] = x;
  }
  return escaped;
}

/* Eq. (9): add A_p g D(r - X) to the force field F for one particle, with the
 * same per-axis taps and weights as the interpolation (h = 1). */
void or_spread_one(const or_params* p, const double* X, double dia, const double* g, double* F) {
  int d = (p->q == 9) ? 2 : 3;
  long nc = or_ncell(p);
  double Ap = OR_PI * dia * dia / 4.0;
  int idx[3][4], cnt[3] = {1, 1, 1};
  double w[3][4];
  idx[2][0] = 0;
  w[2][0] = 1.0;
  for (int k = 0; k < d; ++k) cnt[k] = or_taps(p, k, X[k], idx[k], w[k]);
  for (int tz = 0; tz < cnt[2]; ++tz)
    for (int ty = 0; ty < cnt[1]; ++ty)
      for (int tx = 0; tx < cnt[0]; ++tx) {
        int x[3] = {idx[0][tx], idx[1][ty], idx[2][tz]};
        double wt = w[0][tx] * w[1][ty] * w[2][tz];
        long c = or_cell(p, x);
        for (int k = 0; k < d; ++k) F[k * nc + c] += Ap * g[k] * wt;
      }
}

/* Collision of one cell, Eqs. (2), (3), (8): u = (j + F/2) / rho, equilibrium,
 * Guo body-force term, relaxation. fc: the q stored populations g = f - w of the
 * cell (in), Fc: the d force components, out: post-collision g. */
static void or_collide_cell(const or_lattice_t* L, double tau, const double* fc, const double* Fc,
                            double* out) {
  int d = L->d;
  double sum = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < L->q; ++a) {
    sum += fc[a];
    for (int k = 0; k < d; ++k) j[k] += L->e[a][k] * fc[a];
  }
  double rho = 1.0 + sum;
  double uu = 0.0;
  for (int k = 0; k < d; ++k) {
    u[k] = (j[k] + 0.5 * Fc[k]) / rho;
    uu += u[k] * u[k];
  }
  for (int a = 0; a < L->q; ++a) {
    double eu = 0.0, eF = 0.0, emuF = 0.0;
    for (int k = 0; k < d; ++k) {
      eu += L->e[a][k] * u[k];
      eF += L->e[a][k] * Fc[k];
      emuF += (L->e[a][k] - u[k]) * Fc[k];
    }
    /* f^eq - w = w [(rho - 1) + rho (3 eu + 4.5 eu^2 - 1.5 uu)], rho - 1 = sum */
    double feq = L->w[a] * (sum + rho * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
    double Fb = (1.0 - 1.0 / (2.0 * tau)) * L->w[a] * (3.0 * emuF + 9.0 * eu * eF);
    out[a] = fc[a] - (fc[a] - feq) / tau + Fb;
  }
}

void or_collide(const or_params* p, const double* f, const double* F, double* fs) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  long nc = or_ncell(p);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    double fc[OR_MAXQ], out[OR_MAXQ], Fc[3];
    for (int a = 0; a < L.q; ++a) fc[a] = f[a * nc + c];
    for (int k = 0; k < L.d; ++k) Fc[k] = F ? F[k * nc + c] : 0.0;
    or_collide_cell(&L, p->tau, fc, Fc, out);
    for (int a = 0; a < L.q; ++a) fs[a * nc + c] = out[a];
  }
}

/* Source of population a arriving at cell x: x - e_a, wrapped on periodic
 * axes. Returns 0 and the source cell, or 1 when the link crosses a wall
 * (halfway bounce-back: the arriving value is fs[opp(a)] at x itself). */
static int or_source(const or_params* p, const or_lattice_t* L, const int* x, int a, int* src) {
  for (int k = 0; k < 3; ++k) {
    int s = x[k] - L->e[a][k];
    if (p->periodic[k]) {
      s = ((s % p->n[k]) + p->n[k]) % p->n[k];
    } else if (s < 0 || s >= p->n[k]) {
      return 1;
    }
    src[k] = s;
  }
  return 0;
}

/* Streaming, the left-hand side of Eq. (2), as a pull with halfway
 * bounce-back at resting walls. */
void or_stream(const or_params* p, const double* fs, double* f) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  long nc = or_ncell(p);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    int x[3] = {(int)(c % p->n[0]), (int)((c / p->n[0]) % p->n[1]),
                (int)(c / ((long)p->n[0] * p->n[1]))};
    int src[3];
    for (int a = 0; a < L.q; ++a) {
      if (or_source(p, &L, x, a, src))
        f[a * nc + c] = fs[L.opp[a] * nc + c];
      else
        f[a * nc + c] = fs[a * nc + or_cell(p, src)];
    }
  }
}

/* One full step in the order stated at the top of this file. f is advanced
 * in place (fs is scratch of the same size); X, U are replaced by the new
 * state. F receives the spread force of this step; g, Fc the per-particle
 * force density and contact force. diag[0]: max literal-vs-closed g deviation;
 * diag[1]: number of escaped particles. */
/* Particle phase of all particles with S = substeps DEM sub-steps of length
 * h = 1/S. rho_l, j_l are interpolated once at the step-n positions (Eq. 4);
 * each sub-step takes the contact forces of all particles at the sub-step
 * state and then advances every particle:
 *   implicit: m (U' - U) = h [buoy g + Fc - 2 A_p (rho_l U' - j_l)],
 *   explicit: m (U' - U) = h [buoy g + Fc - 2 A_p (rho_l U - j_l)],
 *   X' = X + h U'.
 * g (to the fluid) and Fc (reported) are the averages over the sub-steps of
 * 2 (rho_l U_b - j_l) and of the contact force. Returns the number of
 * sub-step moves that left the domain through a wall. */
static double or_particles_subcycled(const or_params* p, const double* f, long np,
                                     const double* X, const double* U, const double* dia,
                                     const double* rr, double* Xn, double* Un, double* g,
                                     double* Fc) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  int d = L.d;
  int S = p->substeps;
  double h = 1.0 / (double)S;
  double* rho = (double*)malloc(sizeof(double) * np);
  double* jl = (double*)malloc(sizeof(double) * np * d);
  double* Xs = (double*)malloc(sizeof(double) * np * d);
  double* Us = (double*)malloc(sizeof(double) * np * d);
  double* Fs = (double*)malloc(sizeof(double) * np * d);
  double esc = 0.0;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < np; ++i) {
    double fl[OR_MAXQ];
    or_interp_pops(p, f, X + i * d, fl);
    double sum_l = 0.0;
    for (int k = 0; k < d; ++k) jl[i * d + k] = 0.0;
    for (int a = 0; a < L.q; ++a) {
      sum_l += fl[a];
      for (int k = 0; k < d; ++k) jl[i * d + k] += L.e[a][k] * fl[a];
    }
    rho[i] = 1.0 + sum_l;
  }
  memcpy(Xs, X, sizeof(double) * np * d);
  memcpy(Us, U, sizeof(double) * np * d);
  memset(g, 0, sizeof(double) * np * d);
  memset(Fc, 0, sizeof(double) * np * d);
  for (int sub = 0; sub < S; ++sub) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < np; ++i) or_contact_force(p, np, Xs, Us, dia, rr, i, Fs + i * d);
#pragma omp parallel for schedule(static) reduction(+ : esc)
    for (long i = 0; i < np; ++i) {
      double m = or_mass(d, dia[i], rr[i]);
      double Ap = OR_PI * dia[i] * dia[i] / 4.0;
      double buoy = m * (1.0 - 1.0 / rr[i]);
      for (int k = 0; k < d; ++k) {
        double Uo = Us[i * d + k], Ub;
        double fc = Fs[i * d + k];
        if (p->implicit_drag) {
          Un[i * d + k] = (m * Uo + h * (2.0 * Ap * jl[i * d + k] + buoy * p->gravity[k] + fc)) /
                          (m + 2.0 * Ap * rho[i] * h);
          Ub = Un[i * d + k];
        } else {
          Un[i * d + k] =
              Uo + h * (buoy * p->gravity[k] + fc - Ap * 2.0 * (rho[i] * Uo - jl[i * d + k])) / m;
          Ub = Uo;
        }
        g[i * d + k] += h * 2.0 * (rho[i] * Ub - jl[i * d + k]);
        Fc[i * d + k] += h * fc;
        double x = Xs[i * d + k] + h * Un[i * d + k];
        if (p->periodic[k]) {
          double N = (double)p->n[k];
          if (x < 0.0) x += N;
          else if (x >= N) x -= N;
        } else if (x < 0.0 || x > (double)p->n[k]) {
          esc += 1.0;
        }
        Xn[i * d + k] = x;
      }
    }
    memcpy(Xs, Xn, sizeof(double) * np * d);
    memcpy(Us, Un, sizeof(double) * np * d);
  }
  free(rho);
  free(jl);
  free(Xs);
  free(Us);
  free(Fs);
  return esc;
}

void or_step(const or_params* p, double* f, double* fs, double* F, long np, double* X, double* U,
             const double* dia, const double* rr, double* Xn, double* Un, double* g, double* Fc,
             double* diag) {
  int d = (p->q == 9) ? 2 : 3;
  long nc = or_ncell(p);
  double dev_max = 0.0, esc = 0.0;
  if (p->substeps > 1) {
    esc = or_particles_subcycled(p, f, np, X, U, dia, rr, Xn, Un, g, Fc);
  } else {
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : esc) reduction(max : dev_max)
    for (long i = 0; i < np; ++i) {
      double dv = 0.0;
      esc += or_particle_update(p, f, np, X, U, dia, rr, i, Xn + i * d, Un + i * d, g + i * d,
                                Fc + i * d, &dv);
      if (dv > dev_max) dev_max = dv;
    }
  }
  memset(F, 0, sizeof(double) * d * nc);
  for (long i = 0; i < np; ++i) or_spread_one(p, X + i * d, dia[i], g + i * d, F);
  or_collide(p, f, F, fs);
  or_stream(p, fs, f);
  memcpy(X, Xn, sizeof(double) * np * d);
  memcpy(U, Un, sizeof(double) * np * d);
  if (diag) {
    if (dev_max > diag[0]) diag[0] = dev_max;
    diag[1] += esc;
  }
}

void or_run(const or_params* p, long nsteps, double* f, double* fs, double* F, long np, double* X,
            double* U, const double* dia, const double* rr, double* Xn, double* Un, double* g,
            double* Fc, double* diag) {
  for (long s = 0; s < nsteps; ++s) or_step(p, f, fs, F, np, X, U, dia, rr, Xn, Un, g, Fc, diag);
}

/* Sampled evaluation for large lattices. */

/* F at one cell after the particle phase: the sum over every particle whose
 * stencil covers the cell, in ascending particle index, of A_p g w. */
void or_force_at_cell(const or_params* p, const double* f, long np, const double* X,
                      const double* U, const double* dia, const double* rr, long cell,
                      double* Fout) {
  int d = (p->q == 9) ? 2 : 3;
  int x[3] = {(int)(cell % p->n[0]), (int)((cell / p->n[0]) % p->n[1]),
              (int)(cell / ((long)p->n[0] * p->n[1]))};
  for (int k = 0; k < d; ++k) Fout[k] = 0.0;
  for (long i = 0; i < np; ++i) {
    int idx[3][4], cnt[3] = {1, 1, 1};
    double w[3][4];
    idx[2][0] = 0;
    w[2][0] = 1.0;
    for (int k = 0; k < d; ++k) cnt[k] = or_taps(p, k, X[i * d + k], idx[k], w[k]);
    double wt = 0.0;
    int hit = 0;
    for (int tz = 0; tz < cnt[2]; ++tz)
      for (int ty = 0; ty < cnt[1]; ++ty)
        for (int tx = 0; tx < cnt[0]; ++tx)
          if (idx[0][tx] == x[0] && idx[1][ty] == x[1] && idx[2][tz] == x[2]) {
            wt += w[0][tx] * w[1][ty] * w[2][tz];
            hit = 1;
          }
    if (!hit) continue;
    double Xn[3], Un[3], gg[3], Fc[3];
    or_particle_update(p, f, np, X, U, dia, rr, i, Xn, Un, gg, Fc, NULL);
    double Ap = OR_PI * dia[i] * dia[i] / 4.0;
    for (int k = 0; k < d; ++k) Fout[k] += Ap * gg[k] * wt;
  }
}

/* Post-step populations at one cell: each arriving population is the
 * post-collision value at its source (or the bounced one at the cell itself);
 * the collision at a source needs F there, evaluated with or_force_at_cell. */
void or_cell_after_step(const or_params* p, const double* f, long np, const double* X,
                        const double* U, const double* dia, const double* rr, long cell,
                        double* out) {
  or_lattice_t L;
  or_lattice_get(p->q, &L);
  long nc = or_ncell(p);
  int x[3] = {(int)(cell % p->n[0]), (int)((cell / p->n[0]) % p->n[1]),
              (int)(cell / ((long)p->n[0] * p->n[1]))};
  int src[3];
  double fc[OR_MAXQ], post[OR_MAXQ], Fc[3];
  for (int a = 0; a < L.q; ++a) {
    long sc;
    int b;
    if (or_source(p, &L, x, a, src)) {
      sc = cell;
      b = L.opp[a];
    } else {
      sc = or_cell(p, src);
      b = a;
    }
    for (int k = 0; k < L.q; ++k) fc[k] = f[k * nc + sc];
    or_force_at_cell(p, f, np, X, U, dia, rr, sc, Fc);
    or_collide_cell(&L, p->tau, fc, Fc, post);
    out[a] = post[b];
  }
}
