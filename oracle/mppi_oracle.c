/*
 * CPU FP64 oracle for one iteration of DBaS-Log-MPPI (arXiv 2504.06437).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The product
 * path (the CUDA library) shares no code, header, table or constant with it.
 *
 * Everything here is written plainly, in the order of the paper's
 * Algorithm 1, in double precision, with no blocking or fusion.  Where the
 * paper is silent or ambiguous the reading used is stated at the function.
 *
 * Paper map:
 *   Eq. 1   x_{k+1} = f(x_k, u_k)                     -> orc_dynamics
 *   Eq. 5   beta = B(h(x)), B(h) = 1/h                -> orc_bsum
 *   Eq. 7   beta_{k+1} = B(h(f)) - gamma (B(h(x_d)) - beta_k)
 *   Eq. 8   rollout with v = u + du                   -> rollout_sample
 *   Eq. 9   cost-to-go with barrier cost C_B          -> rollout_sample
 *   Eq. 4   min-shifted exponentiated weights, update -> orc_weights, orc_step
 *   Eq. 10  S_e = mu log(e + C_B(X*))                  -> orc_step
 *   Eq. 11  NLN product of a normal and a log-normal  -> orc_noise
 *   Eq. 12  planar quadrotor (6-state two-thrust form of Sec. V-A constants)
 *   Eq. 13/15 h = |p_i - c_j|^2 - r_j^2 over shape points and obstacles
 *   Sec. V-C  the grid map's h at a shape point          -> orc_grid_h
 *   Alg. 1  the outer-loop body: sample, roll out, weight, update, actuate,
 *           nominal rollout for C_B, S_e, shift.
 *   Alg. 1  SGF: Savitzky-Golay smoothing of the weighted perturbation
 *           (Sec. III-A, last paragraph)                -> orc_sgf, orc_step
 *
 * Test-only outputs, not part of the method: per sample, the barrier cost's
 * sensitivity to position error (bsum_grad, summed with Eq. 7's weights in
 * rollout_sample) and the rollout's reach from x0, with which the tests
 * bound the cost error an FP32 rollout may make near an obstacle.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), counter (k, t, iter_lo,
 * iter_hi), key (seed_lo, seed_hi).  The paper does not name a generator.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_UNICYCLE 0
#define ORC_QUAD2D 1
#define ORC_ACKERMANN 2
#define ORC_QUAD5 3
#define ORC_MAXN 6
#ifndef M_E
#define M_E 2.7182818284590452354
#endif

/* Parameter block.  Field meanings follow the paper's problem statement
 * (Eq. 2, Eq. 7, Eq. 9, Eq. 10, Eq. 11, Algorithm 1 "Require"). */
typedef struct {
  int32_t model; /* ORC_UNICYCLE: x=(x,y,theta), u=(v,omega);
                    ORC_QUAD2D:   x=(y,z,phi,ydot,zdot,phidot), u=(u1,u2) thrust
                                  deviations, F_i = m g / 2 + u_i;
                    ORC_ACKERMANN: x=(x,y,theta,v), u=(steering phi, accel a)
                                  (Eq. 14);
                    ORC_QUAD5:    x=(x,z,theta,vx,vz), u=(pitch rate omega,
                                  thrust deviation u_t) (Eq. 12) */
  int32_t K, T;
  double dt, lambda;      /* lambda: temperature of Eq. 4 (divides the cost) */
  double sigma[4];        /* Sigma_u, 2x2 row-major, symmetric PSD */
  double ln_mu, ln_sigma; /* log-normal factor parameters of Eq. 11 */
  double mu_coarse;       /* mu of Eq. 10; <= 0 keeps S_e = 1 */
  double gamma_ctrl;      /* gamma of Eq. 9 (control-cost weight) */
  double gamma_bas;       /* gamma of Eq. 7, in (0,1) */
  double R_B;             /* barrier-state cost weight of Eq. 9 */
  double C_coll;          /* indicator cost per collided step */
  double h_eps;           /* floor on h inside B(h) = 1/h */
  double Q[6], Qf[6];     /* diagonal stage / terminal weights */
  double u_min[2], u_max[2];
  double x_goal[6];       /* x_d of Eq. 7 */
  int32_t n_shape;
  double shape[16];       /* body-frame shape points (sx, sy) */
  uint64_t seed;
  double mass, inertia, arm, gravity; /* quadrotor constants */
  double wheelbase;                   /* L of Eq. 14 */
  int32_t sgf_window, sgf_order;      /* Savitzky-Golay smoothing of the
                                         update (Algorithm 1); window 0 = off */
  const float* grid;                  /* grid map (orc_grid_h), or NULL */
  int32_t grid_nx, grid_ny;
  double grid_ox, grid_oy, grid_res;
} orc_params;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11 paper, Sec. 3.3 / Table 2 constants).          */
/* ------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (round < 9) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 32-bit word -> uniform in (0,1): the top 23 bits as an odd multiple of
 * 2^-24, i.e. ((r >> 8) | 1) * 2^-24.  Exact in float and double. */
double orc_uniform(uint32_t r) {
  return (double)((r >> 8) | 1u) * (1.0 / 16777216.0);
}

static int state_dim(int model) {
  switch (model) {
    case ORC_QUAD2D: return 6;
    case ORC_ACKERMANN: return 4;
    case ORC_QUAD5: return 5;
    default: return 3;
  }
}

/* Lower Cholesky factor of a symmetric PSD 2x2 matrix A (row-major):
 * L = [[l00, 0], [l10, l11]], A = L L^T. */
static void chol2(const double A[4], double L[3]) {
  double l00 = sqrt(A[0] > 0.0 ? A[0] : 0.0);
  double l10 = l00 > 0.0 ? A[2] / l00 : 0.0;
  double r = A[3] - l10 * l10;
  L[0] = l00;
  L[1] = l10;
  L[2] = sqrt(r > 0.0 ? r : 0.0);
}

/* Eq. 11 / Algorithm 1 "Sample du ~ NLN(0, S_e Sigma)":
 * du = (chol(S_e Sigma) z_n) .* exp(ln_mu + ln_sigma z_ln), element-wise,
 * with z_n, z_ln standard normals from two Box-Muller pairs over the four
 * Philox words of counter (k, t, iter).  z (optional) returns
 * (z_n0, z_n1, z_ln0, z_ln1). */
void orc_noise(const orc_params* p, double S_e, int32_t k, int32_t t,
               uint64_t iter, double du[2], double z[4]) {
  uint32_t ctr[4] = {(uint32_t)k, (uint32_t)t, (uint32_t)(iter & 0xffffffffu),
                     (uint32_t)(iter >> 32)};
  uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu),
                     (uint32_t)(p->seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  double U0 = orc_uniform(r[0]), U1 = orc_uniform(r[1]);
  double U2 = orc_uniform(r[2]), U3 = orc_uniform(r[3]);
  const double two_pi = 6.283185307179586476925286766559;
  double ra = sqrt(-2.0 * log(U0));
  double zn0 = ra * cos(two_pi * U1);
  double zn1 = ra * sin(two_pi * U1);
  double rb = sqrt(-2.0 * log(U2));
  double zl0 = rb * cos(two_pi * U3);
  double zl1 = rb * sin(two_pi * U3);
  double A[4];
  for (int i = 0; i < 4; ++i) A[i] = S_e * p->sigma[i];
  double L[3];
  chol2(A, L);
  double n0 = L[0] * zn0;
  double n1 = L[1] * zn0 + L[2] * zn1;
  du[0] = n0 * exp(p->ln_mu + p->ln_sigma * zl0);
  du[1] = n1 * exp(p->ln_mu + p->ln_sigma * zl1);
  if (z) {
    z[0] = zn0; z[1] = zn1; z[2] = zl0; z[3] = zl1;
  }
}

/* Eq. 1 with explicit Euler, right-hand side evaluated at step k
 * (as Eq. 12 and Eq. 14 are written). */
void orc_dynamics(const orc_params* p, const double* x, const double* v,
                  double* xn) {
  const double dt = p->dt;
  if (p->model == ORC_UNICYCLE) {
    xn[0] = x[0] + v[0] * cos(x[2]) * dt;
    xn[1] = x[1] + v[0] * sin(x[2]) * dt;
    xn[2] = x[2] + v[1] * dt;
  } else if (p->model == ORC_ACKERMANN) {
    /* Eq. 14: position along the heading at speed v_k, heading rate
     * v_k tan(phi) / L, speed rate a */
    xn[0] = x[0] + x[3] * cos(x[2]) * dt;
    xn[1] = x[1] + x[3] * sin(x[2]) * dt;
    xn[2] = x[2] + x[3] * tan(v[0]) / p->wheelbase * dt;
    xn[3] = x[3] + v[1] * dt;
  } else if (p->model == ORC_QUAD5) {
    /* Eq. 12, read with z in the second and fifth rows (the printed rows
     * say y and v_y): pitch rate omega, thrust m g + u_t */
    const double acc = (p->mass * p->gravity + v[1]) / p->mass;
    xn[0] = x[0] + x[3] * dt;
    xn[1] = x[1] + x[4] * dt;
    xn[2] = x[2] + v[0] * dt;
    xn[3] = x[3] - acc * sin(x[2]) * dt;
    xn[4] = x[4] + (acc * cos(x[2]) - p->gravity) * dt;
  } else {
    double F1 = 0.5 * p->mass * p->gravity + v[0];
    double F2 = 0.5 * p->mass * p->gravity + v[1];
    xn[0] = x[0] + x[3] * dt;
    xn[1] = x[1] + x[4] * dt;
    xn[2] = x[2] + x[5] * dt;
    xn[3] = x[3] - (F1 + F2) / p->mass * sin(x[2]) * dt;
    xn[4] = x[4] + ((F1 + F2) / p->mass * cos(x[2]) - p->gravity) * dt;
    xn[5] = x[5] + (F2 - F1) * p->arm / p->inertia * dt;
  }
}

/* Fused barrier over all (shape point, obstacle) pairs (Eq. 5, Eq. 13/15,
 * Algorithm 1 "sum B o h^(i)"): bsum = sum 1 / max(h_ij, h_eps),
 * collided = any h_ij <= 0, minh = min h_ij.  The pose is (x[0], x[1]) with
 * heading x[2] for both models; shape point s is placed at
 * position + R(heading) s.  obst is J x 3 (cx, cy, r). */
/* Grid map (Sec. V-C: the local point cloud is turned into a 2D grid map
 * for the optimisation; the paper does not say how h is read from it).
 * Reading: the grid holds signed distances (m) to the nearest obstacle,
 * negative inside one; sample (i, j) sits at (ox + i res, oy + j res),
 * stored at grid[j nx + i].  h at a point is the bilinear interpolation of
 * the four samples around it, the point's grid coordinates first clamped to
 * [0, nx - 1] x [0, ny - 1] (beyond the map the edge values continue).
 * Needs nx, ny >= 2. */
double orc_grid_h(const orc_params* p, double px, double py) {
  const int nx = p->grid_nx, ny = p->grid_ny;
  double u = (px - p->grid_ox) / p->grid_res;
  double v = (py - p->grid_oy) / p->grid_res;
  if (u < 0.0) u = 0.0;
  if (u > nx - 1) u = nx - 1;
  if (v < 0.0) v = 0.0;
  if (v > ny - 1) v = ny - 1;
  int i = (int)floor(u), j = (int)floor(v);
  if (i > nx - 2) i = nx - 2;
  if (j > ny - 2) j = ny - 2;
  const double fx = u - i, fy = v - j;
  const float* g = p->grid;
  const double g00 = g[(size_t)j * nx + i], g10 = g[(size_t)j * nx + i + 1];
  const double g01 = g[(size_t)(j + 1) * nx + i], g11 = g[(size_t)(j + 1) * nx + i + 1];
  return (1.0 - fy) * ((1.0 - fx) * g00 + fx * g10) + fy * ((1.0 - fx) * g01 + fx * g11);
}

/* The fused barrier of Eq. 13 at state x: over the shape points, the sum of
 * B(h) = 1 / max(h, h_eps) over the circle obstacles and, when a grid map is
 * set, one more term per point with the grid's h; collided when any h <= 0. */
void orc_bsum(const orc_params* p, const double* obst, int32_t J,
              const double* x, double* bsum, int32_t* collided, double* minh) {
  double c = cos(x[2]), s = sin(x[2]);
  double B = 0.0, mh = INFINITY;
  int coll = 0;
  for (int i = 0; i < p->n_shape; ++i) {
    double sx = p->shape[2 * i], sy = p->shape[2 * i + 1];
    double px = x[0] + c * sx - s * sy;
    double py = x[1] + s * sx + c * sy;
    for (int j = 0; j < J; ++j) {
      double dx = px - obst[3 * j];
      double dy = py - obst[3 * j + 1];
      double r = obst[3 * j + 2];
      double h = dx * dx + dy * dy - r * r;
      if (h <= 0.0) coll = 1;
      if (h < mh) mh = h;
      B += 1.0 / (h > p->h_eps ? h : p->h_eps);
    }
    if (p->grid) {
      const double h = orc_grid_h(p, px, py);
      if (h <= 0.0) coll = 1;
      if (h < mh) mh = h;
      B += 1.0 / (h > p->h_eps ? h : p->h_eps);
    }
  }
  *bsum = B;
  if (collided) *collided = coll;
  if (minh) *minh = mh;
}

/* Sensitivity of the fused barrier at state x to the positions of its shape
 * points: the sum over points and obstacles of |dB/dp| = 2 |p - c| / h^2
 * where h > h_eps (a floored term does not move), and 1 / h^2 for the grid
 * map's term (a signed-distance map: |grad h| taken as 1).  It is the
 * first-order change of the barrier sum when every point moves by one unit
 * of length; the tests scale it by the position error an FP32 rollout may
 * make, to bound the per-sample cost error of samples that pass close to
 * an obstacle (test infrastructure, not part of the method). */
static double bsum_grad(const orc_params* p, const double* obst, int32_t J, const double* x) {
  double c = cos(x[2]), s = sin(x[2]);
  double G = 0.0;
  for (int i = 0; i < p->n_shape; ++i) {
    double sx = p->shape[2 * i], sy = p->shape[2 * i + 1];
    double px = x[0] + c * sx - s * sy;
    double py = x[1] + s * sx + c * sy;
    for (int j = 0; j < J; ++j) {
      double dx = px - obst[3 * j];
      double dy = py - obst[3 * j + 1];
      double r = obst[3 * j + 2];
      double h = dx * dx + dy * dy - r * r;
      if (h > p->h_eps) G += 2.0 * sqrt(dx * dx + dy * dy) / (h * h);
    }
    if (p->grid) {
      const double h = orc_grid_h(p, px, py);
      if (h > p->h_eps) G += 1.0 / (h * h);
    }
  }
  return G;
}

/* Roll the plant forward under a given control sequence V (T x 2), no
 * noise, no clamping: X is (T+1) x n. */
void orc_simulate(const orc_params* p, const double* x0, const double* V,
                  double* X) {
  int n = state_dim(p->model);
  memcpy(X, x0, sizeof(double) * n);
  for (int t = 0; t < p->T; ++t) orc_dynamics(p, X + t * n, V + 2 * t, X + (t + 1) * n);
}

static double clampd(double a, double lo, double hi) {
  return a < lo ? lo : (a > hi ? hi : a);
}

/* Neumaier compensated summation, fixed order. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}
static double nsum_get(const nsum* a) { return a->s + a->c; }

/* One sampled rollout of Algorithm 1 (inner t loop) with the DBaS cost of
 * Eq. 9, for sample k.  Readings:
 *  - v_t = clamp(u_t + du_t, u_min, u_max) (the box G(u) <= 0 of Eq. 2);
 *    the perturbation kept for the update is the applied one, v_t - u_t.
 *  - stage terms are taken at x_{t+1}, t = 0..T-1, and phi at x_T
 *    (Algorithm 1 accumulates after each step).
 *  - control cost gamma u_t^T (S_e Sigma)^-1 v_t (Algorithm 1 form).
 *  - collided step adds C_coll; collision means min h <= 0.
 * Minv = (S_e Sigma)^-1 (row-major), ignored when gamma_ctrl == 0.
 * Optional test outputs: *sens_out = sum_t (dS/dB_t) bsum_grad(x_{t+1}),
 * where the Eq. 7 recursion gives dS/dB_t = R_B sum_{t' >= t} gamma^(t'-t),
 * and *reach_out = max_t |(x, y)_{t+1} - (x, y)_0|. */
static void rollout_sample(const orc_params* p, const double* obst, int32_t J,
                           const double* x0, const double* xref,
                           const double* U, double S_e, double beta0,
                           double beta_d, uint64_t iter, int32_t k,
                           const double Minv[4], double* S_out,
                           uint8_t* coll_out, double* minh_out,
                           double* du_eff, double* sens_out, double* reach_out) {
  const int n = state_dim(p->model);
  double x[ORC_MAXN], xn[ORC_MAXN];
  memcpy(x, x0, sizeof(double) * n);
  double w = beta0;
  nsum S = {0.0, 0.0};
  int coll = 0;
  double minh = INFINITY, sens = 0.0, reach = 0.0;
  for (int t = 0; t < p->T; ++t) {
    double du[2], v[2];
    orc_noise(p, S_e, k, t, iter, du, NULL);
    for (int d = 0; d < 2; ++d) {
      v[d] = clampd(U[2 * t + d] + du[d], p->u_min[d], p->u_max[d]);
      if (du_eff) du_eff[2 * t + d] = v[d] - U[2 * t + d];
    }
    orc_dynamics(p, x, v, xn);
    memcpy(x, xn, sizeof(double) * n);
    double B, mh;
    int32_t c;
    orc_bsum(p, obst, J, x, &B, &c, &mh);
    w = B - p->gamma_bas * (beta_d - w); /* Eq. 7 */
    double q = 0.0;
    for (int d = 0; d < n; ++d) {
      double e = x[d] - xref[(t + 1) * n + d];
      q += p->Q[d] * e * e;
    }
    double ctrl = 0.0;
    if (p->gamma_ctrl != 0.0) {
      double Mv0 = Minv[0] * v[0] + Minv[1] * v[1];
      double Mv1 = Minv[2] * v[0] + Minv[3] * v[1];
      ctrl = p->gamma_ctrl * (U[2 * t] * Mv0 + U[2 * t + 1] * Mv1);
    }
    nsum_add(&S, q);
    nsum_add(&S, ctrl);
    nsum_add(&S, p->R_B * w);
    if (c) nsum_add(&S, p->C_coll);
    coll |= c;
    if (mh < minh) minh = mh;
    if (sens_out) {
      const double g = p->gamma_bas, m = (double)(p->T - t);
      const double dS_dB = p->R_B * (fabs(1.0 - g) > 1e-12 ? (1.0 - pow(g, m)) / (1.0 - g) : m);
      sens += dS_dB * bsum_grad(p, obst, J, x);
    }
    if (reach_out) {
      const double dist = hypot(x[0] - x0[0], x[1] - x0[1]);
      if (dist > reach) reach = dist;
    }
  }
  double phi = 0.0;
  for (int d = 0; d < n; ++d) {
    double e = x[d] - xref[p->T * n + d];
    phi += p->Qf[d] * e * e;
  }
  nsum_add(&S, phi);
  *S_out = nsum_get(&S);
  *coll_out = (uint8_t)coll;
  *minh_out = minh;
  if (sens_out) *sens_out = sens;
  if (reach_out) *reach_out = reach;
}

/* Eq. 4 weights: rho = min_k S_k, e_k = exp(-(S_k - rho) / lambda),
 * w_k = e_k / sum e.  Returns rho; *Z_out gets the normaliser. */
double orc_weights(const double* S, int32_t K, double lambda, double* w,
                   double* Z_out) {
  double rho = INFINITY;
  for (int k = 0; k < K; ++k)
    if (S[k] < rho) rho = S[k];
  nsum Z = {0.0, 0.0};
  for (int k = 0; k < K; ++k) {
    w[k] = exp(-(S[k] - rho) / lambda);
    nsum_add(&Z, w[k]);
  }
  double z = nsum_get(&Z);
  for (int k = 0; k < K; ++k) w[k] /= z;
  if (Z_out) *Z_out = z;
  return rho;
}

/* Savitzky-Golay smoothing (Algorithm 1: U* = U + SGF(weighted
 * perturbation); Sec. III-A names the filter but gives no window or order).
 * Reading: y holds T samples (element t at y[t * stride]); out[t] is the
 * value at t of the degree-`order` polynomial fitted by least squares to the
 * W samples of the window centred on t, or, within W/2 of an end, to the
 * first or last W samples (the fit is evaluated off centre there).  Needs W
 * odd, order < W <= T.
 * Written as the definition: per t, the normal equations of the fit on the
 * window's abscissae scaled to [-1, 1], solved by Gaussian elimination with
 * partial pivoting, then the polynomial evaluated at t.  The polynomial is
 * written in the Legendre basis P_0..P_order (Bonnet's recurrence), which
 * spans the same polynomials as the monomials and keeps the normal matrix
 * close to diagonal on [-1, 1]. */
static void legendre_row(double z, int m, double* P) {
  P[0] = 1.0;
  if (m > 1) P[1] = z;
  for (int k = 1; k + 1 < m; ++k) P[k + 1] = ((2 * k + 1) * z * P[k] - k * P[k - 1]) / (k + 1);
}

#define ORC_SGF_MAXORDER 6
void orc_sgf(const double* y, int32_t stride, int32_t T, int32_t W,
             int32_t order, double* out, int32_t out_stride) {
  const int m = order + 1, h = W / 2;
  const double c = 0.5 * (W - 1);
  for (int t = 0; t < T; ++t) {
    int s = t - h;
    if (s < 0) s = 0;
    if (s > T - W) s = T - W;
    double A[ORC_SGF_MAXORDER + 1][ORC_SGF_MAXORDER + 2];
    for (int r = 0; r < m; ++r)
      for (int q = 0; q <= m; ++q) A[r][q] = 0.0;
    for (int i = 0; i < W; ++i) {
      const double yi = y[(size_t)(s + i) * stride];
      double P[ORC_SGF_MAXORDER + 1];
      legendre_row((i - c) / c, m, P);
      for (int r = 0; r < m; ++r) {
        for (int q = 0; q < m; ++q) A[r][q] += P[r] * P[q];
        A[r][m] += P[r] * yi;
      }
    }
    for (int col = 0; col < m; ++col) {
      int piv = col;
      for (int r = col + 1; r < m; ++r)
        if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
      if (piv != col)
        for (int q = 0; q <= m; ++q) {
          double tmp = A[col][q];
          A[col][q] = A[piv][q];
          A[piv][q] = tmp;
        }
      for (int r = col + 1; r < m; ++r) {
        const double f = A[r][col] / A[col][col];
        for (int q = col; q <= m; ++q) A[r][q] -= f * A[col][q];
      }
    }
    double a[ORC_SGF_MAXORDER + 1];
    for (int r = m - 1; r >= 0; --r) {
      double v = A[r][m];
      for (int q = r + 1; q < m; ++q) v -= A[r][q] * a[q];
      a[r] = v / A[r][r];
    }
    double P[ORC_SGF_MAXORDER + 1];
    legendre_row(((t - s) - c) / c, m, P);
    double v = 0.0;
    for (int k = 0; k < m; ++k) v += a[k] * P[k];
    out[(size_t)t * out_stride] = v;
  }
}

/* Per-controller state carried between iterations. */
typedef struct {
  double* U;      /* T x 2 nominal control sequence (in/out) */
  double S_e;     /* exploration rate of Eq. 10 */
  double beta;    /* barrier state of the real system */
  int32_t first;  /* 1 until the first step has run */
  uint64_t iter;  /* Philox counter word pair (iteration index) */
} orc_state;

/* Outputs of one iteration (any pointer may be NULL). */
typedef struct {
  double* costs;    /* K */
  uint8_t* coll;    /* K */
  double* minh;     /* K */
  double* weights;  /* K */
  double* du_eff;   /* K x T x 2 */
  double* Ustar;    /* T x 2, before the shift */
  double* u0;       /* 2 */
  double CB_star;   /* barrier cost of the nominal rollout of U* */
  double beta_used; /* barrier state the rollouts started from */
  double beta_d;    /* B summed at the goal pose */
  double rho, Z;
  double* sens;     /* K: barrier sensitivity to position (rollout_sample), or NULL */
  double* reach;    /* K: farthest distance of the rollout from x0, or NULL */
} orc_out;

static int g_threads = 0;
void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

/* One Algorithm 1 outer-loop body.  xref is (T+1) x n.
 * Returns 0, -1 on allocation failure, -2 for smoothing parameters that
 * orc_sgf does not accept. */
int orc_step(const orc_params* p, const double* obst, int32_t J,
             const double* x0, const double* xref, orc_state* st,
             orc_out* out) {
  const int K = p->K, T = p->T, n = state_dim(p->model);
  if (p->sgf_window != 0 &&
      (p->sgf_window % 2 != 1 || p->sgf_window > T || p->sgf_order < 0 ||
       p->sgf_order >= p->sgf_window || p->sgf_order > ORC_SGF_MAXORDER))
    return -2;
  double* S = (double*)malloc(sizeof(double) * K);
  uint8_t* coll = (uint8_t*)malloc(K);
  double* minh = (double*)malloc(sizeof(double) * K);
  double* w = (double*)malloc(sizeof(double) * K);
  double* du = (double*)malloc(sizeof(double) * (size_t)K * T * 2);
  double* Us = (double*)malloc(sizeof(double) * T * 2);
  if (!S || !coll || !minh || !w || !du || !Us) {
    free(S); free(coll); free(minh); free(w); free(du); free(Us);
    return -1;
  }

  /* beta_d = fused barrier at the desired equilibrium x_d (Eq. 7). */
  double beta_d;
  orc_bsum(p, obst, J, p->x_goal, &beta_d, NULL, NULL);

  /* Barrier state of the measured state: Eq. 7 applied to the plant. */
  double B0;
  orc_bsum(p, obst, J, x0, &B0, NULL, NULL);
  double beta = st->first ? B0 : B0 - p->gamma_bas * (beta_d - st->beta);

  /* (S_e Sigma)^-1 for the control cost. */
  double Minv[4] = {0, 0, 0, 0};
  if (p->gamma_ctrl != 0.0) {
    double a = st->S_e * p->sigma[0], b = st->S_e * p->sigma[1];
    double c = st->S_e * p->sigma[2], d = st->S_e * p->sigma[3];
    double det = a * d - b * c;
    Minv[0] = d / det; Minv[1] = -b / det;
    Minv[2] = -c / det; Minv[3] = a / det;
  }

  /* Sampled rollouts (Algorithm 1: one rollout per sample k). */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(orc_get_threads())
#endif
  for (int k = 0; k < K; ++k)
    rollout_sample(p, obst, J, x0, xref, st->U, st->S_e, beta, beta_d,
                   st->iter, k, Minv, &S[k], &coll[k], &minh[k],
                   du + (size_t)k * T * 2, out && out->sens ? out->sens + k : NULL,
                   out && out->reach ? out->reach + k : NULL);

  /* Eq. 4: weights and the weighted perturbation dU (held in Us), then
   * Algorithm 1's U* = U + SGF(dU), clamped to the box of Eq. 2. */
  double Z;
  double rho = orc_weights(S, K, p->lambda, w, &Z);
  for (int t = 0; t < T; ++t)
    for (int d = 0; d < 2; ++d) {
      nsum acc = {0.0, 0.0};
      for (int k = 0; k < K; ++k) nsum_add(&acc, w[k] * du[(size_t)k * T * 2 + 2 * t + d]);
      Us[2 * t + d] = nsum_get(&acc);
    }
  if (p->sgf_window > 0) {
    double* raw = (double*)malloc(sizeof(double) * T * 2);
    if (!raw) {
      free(S); free(coll); free(minh); free(w); free(du); free(Us);
      return -1;
    }
    memcpy(raw, Us, sizeof(double) * T * 2);
    for (int d = 0; d < 2; ++d) orc_sgf(raw + d, 2, T, p->sgf_window, p->sgf_order, Us + d, 2);
    free(raw);
  }
  for (int t = 0; t < T; ++t)
    for (int d = 0; d < 2; ++d)
      Us[2 * t + d] = clampd(st->U[2 * t + d] + Us[2 * t + d], p->u_min[d], p->u_max[d]);

  /* Nominal rollout of U* over the horizon (Algorithm 1) for C_B(X*). */
  double x[ORC_MAXN], xn[ORC_MAXN];
  memcpy(x, x0, sizeof(double) * n);
  double wn = beta;
  nsum CB = {0.0, 0.0};
  for (int t = 0; t < T; ++t) {
    orc_dynamics(p, x, Us + 2 * t, xn);
    memcpy(x, xn, sizeof(double) * n);
    double B;
    orc_bsum(p, obst, J, x, &B, NULL, NULL);
    wn = B - p->gamma_bas * (beta_d - wn);
    nsum_add(&CB, p->R_B * wn);
  }
  double CB_star = nsum_get(&CB);

  /* Eq. 10.  The paper treats the barrier state as positive; when the
   * DBaS recursion leaves C_B(X*) below zero (start barrier below the goal
   * barrier) the argument of the logarithm is floored at e, so S_e >= mu. */
  double S_e_next =
      p->mu_coarse > 0.0 ? p->mu_coarse * log(M_E + (CB_star > 0.0 ? CB_star : 0.0)) : 1.0;

  if (out) {
    if (out->costs) memcpy(out->costs, S, sizeof(double) * K);
    if (out->coll) memcpy(out->coll, coll, K);
    if (out->minh) memcpy(out->minh, minh, sizeof(double) * K);
    if (out->weights) memcpy(out->weights, w, sizeof(double) * K);
    if (out->du_eff) memcpy(out->du_eff, du, sizeof(double) * (size_t)K * T * 2);
    if (out->Ustar) memcpy(out->Ustar, Us, sizeof(double) * T * 2);
    if (out->u0) { out->u0[0] = Us[0]; out->u0[1] = Us[1]; }
    out->CB_star = CB_star;
    out->beta_used = beta;
    out->beta_d = beta_d;
    out->rho = rho;
    out->Z = Z;
  }

  /* Receding-horizon shift (Algorithm 1): u_{t-1} <- u*_t, last element kept. */
  for (int t = 0; t + 1 < T; ++t) {
    st->U[2 * t] = Us[2 * (t + 1)];
    st->U[2 * t + 1] = Us[2 * (t + 1) + 1];
  }
  st->U[2 * (T - 1)] = Us[2 * (T - 1)];
  st->U[2 * (T - 1) + 1] = Us[2 * (T - 1) + 1];
  st->S_e = S_e_next;
  st->beta = beta;
  st->first = 0;
  st->iter += 1;

  free(S); free(coll); free(minh); free(w); free(du); free(Us);
  return 0;
}

/* K x T draws of orc_noise for one iteration (moment tests).
 * du is K x T x 2; z (optional) is K x T x 4. */
void orc_noise_batch(const orc_params* p, double S_e, int32_t K, int32_t T,
                     uint64_t iter, double* du, double* z) {
  for (int k = 0; k < K; ++k)
    for (int t = 0; t < T; ++t)
      orc_noise(p, S_e, k, t, iter, du + ((size_t)k * T + t) * 2,
                z ? z + ((size_t)k * T + t) * 4 : NULL);
}

/* Cost-to-go (Eq. 9) of selected samples only, for comparisons at sizes where
 * the full step is too slow: the state (U, S_e, beta, first, iter) is the one
 * the step would start from.  ks[i] are sample indices; outputs per index. */
int orc_sample_costs(const orc_params* p, const double* obst, int32_t J,
                     const double* x0, const double* xref, const orc_state* st,
                     const int32_t* ks, int32_t nk, double* S, uint8_t* coll,
                     double* minh, double* sens, double* reach) {
  double beta_d, B0;
  orc_bsum(p, obst, J, p->x_goal, &beta_d, NULL, NULL);
  orc_bsum(p, obst, J, x0, &B0, NULL, NULL);
  double beta = st->first ? B0 : B0 - p->gamma_bas * (beta_d - st->beta);
  double Minv[4] = {0, 0, 0, 0};
  if (p->gamma_ctrl != 0.0) {
    double a = st->S_e * p->sigma[0], b = st->S_e * p->sigma[1];
    double c = st->S_e * p->sigma[2], d = st->S_e * p->sigma[3];
    double det = a * d - b * c;
    Minv[0] = d / det; Minv[1] = -b / det;
    Minv[2] = -c / det; Minv[3] = a / det;
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_get_threads())
#endif
  for (int i = 0; i < nk; ++i)
    rollout_sample(p, obst, J, x0, xref, st->U, st->S_e, beta, beta_d, st->iter,
                   ks[i], Minv, &S[i], &coll[i], &minh[i], NULL, sens ? sens + i : NULL,
                   reach ? reach + i : NULL);
  return 0;
}
