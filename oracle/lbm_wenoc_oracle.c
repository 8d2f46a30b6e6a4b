/*
 * FP64 CPU oracle of the coupled lattice-Boltzmann + WENO5 time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what one step of the method computes.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, table or header with the CUDA library and must never be called by it.
 *
 * Every routine follows the paper's statement of the method, step by step,
 * in double precision, with plain loops over nodes (OpenMP only splits those
 * loops; reductions are serial and in index order):
 *
 *   a1  moments   rho = sum f_i,  rho u = sum f_i c_i + F/2        (Sec. 2.3.1, Eqs. dens, mom_dens, LBE_Guo)
 *   a2  BGK collision with the Guo (2002) source term              (Sec. 2.3.1, Eqs. LBE, LBE_Guo, tau)
 *   a3  streaming with halfway bounce-back at floor and lid        (Sec. 2.3.1, no-slip walls of Sec. 2.2.1)
 *   a4  global Lax-Friedrichs split  h+- = (w +- alpha) c / 2     (Supplement Eqs. S8, S17-S20 "upwind splitting")
 *   a5  WENO5 (Jiang & Shu 1996) face reconstruction              (Supplement Eqs. S9-S16, order raised to 5)
 *   a6  central diffusion flux  kappa (c_{i+1} - c_i)              (Supplement Eq. S4; Eq. ADS)
 *   a7  conservative divergence of the face fluxes                 (Supplement Eq. S9; Eq. ADS)
 *   a8  SSP-RK3 (Shu-Osher) with the velocity frozen at step n     (Supplement Eqs. S21-S23)
 *   a9  deposit: settling flux through the floor, RK3 b-weights    (Sec. 4, deposited mass m_b)
 *
 * With ORC_SUGAR, a second scalar S (sugar, normalised by its lower-layer value S0):
 *   s1  force F_v = -g [R c + S* S (1 - phi0 c)]                   (Eq. forceterm; rho/rho0 - 1 = S* S)
 *   s2  settling velocity Vs (1 - kS S) in every face velocity     (Eq. stokes_vel with rho(S))
 * Variants of a4/a5: ORC_WENO3, the paper's third-order WENO with two two-point stencils
 * (Supplement Eqs. S10, S11, S14-S16 for the left-biased side, S17-S20 as its mirror
 * image), linear weights (2/3, 1/3) of Eq. S16; ORC_SIGN_SPLIT, the whole flux w c
 * reconstructed from the upwind side chosen by the sign of the face velocity
 * (w_i + w_{i+1})/2 (ties: left-biased), the paper's "upwind splitting of the flux".
 * Polydisperse (n_classes >= 2, Eqs. forceterm_poly, poly): classes c_k, each transported by
 * a4-a9 with its own settling velocity and deposit; the force (and the sugar term's
 * (1 - phi) factor) reads phi_tot = sum_k c_k.
 *   s3  S advanced by first-order upwind in advective form, one    (Eq. AD; Supplement Eqs. S5, S6)
 *       explicit step per axis sign, plus central diffusion D_s,
 *       with the velocity of a1 and Neumann walls (Eq. neum2)
 *
 * Readings of points the paper leaves open (garbled LBE right-hand side,
 * WENO order, split, epsilon, wall fluxes, coupling order, initial state) are
 * the ones listed in the design notes: fluid nodes sit at v = 0..N-1 on the
 * vertical axis, walls at v = -1/2 and v = N-1/2; stencils that cross a wall
 * read ghosts with c even-reflected (Neumann, Eq. neum1) and the fluid
 * velocity odd-reflected (no-slip); the lid face carries no flux and the floor
 * face carries the settling outflow -Vs c_0, which is tallied as deposit.
 *
 * Lattice units throughout (dx = dt = 1, c_s^2 = 1/3).  Vertical axis = y in
 * 2D, z in 3D.  Node index = (z*ny + y)*nx + x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PERIODIC_VERTICAL 1u /* vertical axis periodic too: no walls, no deposit */
#define ORC_FROZEN_VELOCITY 2u   /* fluid not advanced; transport uses the velocity given at init */
#define ORC_SUGAR 4u             /* second scalar S (sugar) in the force, Vs and its own transport */
#define ORC_WENO3 8u             /* the paper's third-order WENO (Supplement Eqs. S10-S20) instead of WENO5 */
#define ORC_SIGN_SPLIT 16u       /* split by the sign of the face velocity instead of Lax-Friedrichs */

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EUNSTABLE -4

typedef struct {
  int32_t dim; /* 2 or 3 */
  int32_t nx, ny, nz;
  double tau;
  double gravity;
  double density_contrast;
  double settling_velocity;
  double diffusivity;
  double lf_alpha; /* 0 selects the (largest class) settling velocity + u_cap */
  double u_cap;    /* 0 selects 0.1 */
  double body_force[3];
  uint32_t flags;
  double sugar_contrast;    /* S*: rho/rho0 - 1 at S = 1 */
  double sugar_diffusivity; /* D_s */
  double phi0;              /* particle volume fraction at c = 1, in the (1 - phi) factor */
  double vs_sugar;          /* kS: Vs(S) = Vs (1 - kS S) */
  int32_t n_classes;        /* >= 2: polydisperse, class k settles at class_vs[k] */
  double class_vs[8];
} orc_params;

typedef struct {
  orc_params p;
  int Q;
  int ci[19][3];
  double wi[19];
  int opp[19];
  int n[3];     /* extents along x, y, z (z = 1 in 2D) */
  size_t nn;    /* number of nodes */
  int vaxis;    /* index of the vertical axis */
  double alpha; /* Lax-Friedrichs split speed */
  double eps;   /* WENO epsilon = 1e-6 alpha^2 */
  double *f;    /* populations, natural layout f[i*nn + node] */
  double *fpost;
  double *c;
  double *u; /* dim*nn: velocity that transports c during the current step */
  double *rho;
  double *c1, *c2, *L, *flux;
  double *S, *Snew; /* sugar (ORC_SUGAR) */
  int ncls;         /* particle classes (1, or n_classes) */
  double *cls;      /* classes 1..ncls-1 (class 0 is c) */
  double *ctot;     /* sum of the classes: the phi_tot of the force */
  double cls_dep[8];
  double vs_cur;    /* settling velocity of the class being transported */
  double deposit;
  int64_t steps;
  int status;
} orc_sim;

/* ---- velocity sets (Kruger et al. 2017, the LBM text the paper cites) ---- */

static void set_d2q9(orc_sim *s) {
  /* rest, 4 axis neighbours (w = 1/9), 4 diagonals (w = 1/36) */
  static const int c[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                              {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
  s->Q = 9;
  for (int i = 0; i < 9; ++i) {
    s->ci[i][0] = c[i][0];
    s->ci[i][1] = c[i][1];
    s->ci[i][2] = 0;
    int len2 = c[i][0] * c[i][0] + c[i][1] * c[i][1];
    s->wi[i] = len2 == 0 ? 4.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
}

static void set_d3q19(orc_sim *s) {
  /* rest (1/3), 6 face neighbours (1/18), 12 edge neighbours (1/36) */
  int q = 0;
  for (int cz = -1; cz <= 1; ++cz)
    for (int cy = -1; cy <= 1; ++cy)
      for (int cx = -1; cx <= 1; ++cx) {
        int len2 = cx * cx + cy * cy + cz * cz;
        if (len2 == 3) continue; /* corners are not in D3Q19 */
        s->ci[q][0] = cx;
        s->ci[q][1] = cy;
        s->ci[q][2] = cz;
        s->wi[q] = len2 == 0 ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        ++q;
      }
  s->Q = q; /* 19 */
}

static void set_opposites(orc_sim *s) {
  for (int i = 0; i < s->Q; ++i)
    for (int j = 0; j < s->Q; ++j)
      if (s->ci[j][0] == -s->ci[i][0] && s->ci[j][1] == -s->ci[i][1] &&
          s->ci[j][2] == -s->ci[i][2])
        s->opp[i] = j;
}

/* ---- small helpers ---- */

static size_t node_index(const orc_sim *s, int x, int y, int z) {
  return ((size_t)z * s->n[1] + y) * s->n[0] + x;
}

static void node_coords(const orc_sim *s, size_t k, int xyz[3]) {
  xyz[0] = (int)(k % s->n[0]);
  xyz[1] = (int)((k / s->n[0]) % s->n[1]);
  xyz[2] = (int)(k / ((size_t)s->n[0] * s->n[1]));
}

static int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

static int vertical_walls(const orc_sim *s) { return !(s->p.flags & ORC_PERIODIC_VERTICAL); }

static int sugar_on(const orc_sim *s) { return (s->p.flags & ORC_SUGAR) != 0; }

/* Buoyancy + external body force at a node: F = body - A c e_v, A = g (rho_p - rho_0)/rho_0
 * (Eq. forceterm with phi read as c); with sugar also - g S* S (1 - phi0 c) e_v (its
 * second term, rho/rho0 - 1 = S* S). */
static void node_force_s(const orc_sim *s, double cval, double sval, double F[3]) {
  for (int d = 0; d < 3; ++d) F[d] = s->p.body_force[d];
  F[s->vaxis] -= s->p.gravity * s->p.density_contrast * cval;
  if (sugar_on(s)) F[s->vaxis] -= s->p.gravity * s->p.sugar_contrast * sval * (1.0 - s->p.phi0 * cval);
}

static void node_force(const orc_sim *s, size_t k, double F[3]) {
  node_force_s(s, s->ncls > 1 ? s->ctot[k] : s->c[k], sugar_on(s) ? s->S[k] : 0.0, F);
}

/* Settling velocity at node k of the class being transported: Vs, or Vs (1 - kS S_k) with
 * sugar. */
static double settling_at(const orc_sim *s, size_t k) {
  return sugar_on(s) ? s->vs_cur * (1.0 - s->p.vs_sugar * s->S[k]) : s->vs_cur;
}

/* Class k's concentration array. */
static double *class_c(const orc_sim *s, int k) { return k == 0 ? s->c : s->cls + (size_t)(k - 1) * s->nn; }

/* phi_tot / phi0 = sum of the classes, serial in class order. */
static void sum_classes(orc_sim *s) {
  if (s->ncls < 2) return;
  for (size_t j = 0; j < s->nn; ++j) {
    double acc = 0.0;
    for (int k = 0; k < s->ncls; ++k) acc += class_c(s, k)[j];
    s->ctot[j] = acc;
  }
}

/* ---- a1 + a2: moments and BGK-Guo collision at every node ---- */

static void collide_all(orc_sim *s) {
  const int Q = s->Q, dim = s->p.dim;
  const size_t nn = s->nn;
  const double tau = s->p.tau, cs2 = 1.0 / 3.0;
#pragma omp parallel for schedule(static)
  for (long long kk = 0; kk < (long long)nn; ++kk) {
    size_t k = (size_t)kk;
    double F[3];
    node_force(s, k, F);
    double rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      double fi = s->f[(size_t)i * nn + k];
      rho += fi;
      for (int d = 0; d < 3; ++d) mom[d] += fi * s->ci[i][d];
    }
    double u[3];
    for (int d = 0; d < 3; ++d) u[d] = (mom[d] + 0.5 * F[d]) / rho; /* Guo: b = 1/2 */
    s->rho[k] = rho;
    for (int d = 0; d < dim; ++d) s->u[(size_t)d * nn + k] = u[d];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
      double cu = s->ci[i][0] * u[0] + s->ci[i][1] * u[1] + s->ci[i][2] * u[2];
      double feq = s->wi[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
      /* Guo source: (1 - 1/(2 tau)) w_i [ (c_i - u)/cs2 + (c_i.u) c_i / cs2^2 ] . F */
      double src = 0.0;
      for (int d = 0; d < 3; ++d)
        src += ((s->ci[i][d] - u[d]) / cs2 + cu * s->ci[i][d] / (cs2 * cs2)) * F[d];
      src *= (1.0 - 1.0 / (2.0 * tau)) * s->wi[i];
      double fi = s->f[(size_t)i * nn + k];
      s->fpost[(size_t)i * nn + k] = fi - (fi - feq) / tau + src;
    }
  }
}

/* ---- a3: streaming with halfway bounce-back ---- */

static void stream_all(orc_sim *s) {
  const int Q = s->Q;
  const size_t nn = s->nn;
  const int walls = vertical_walls(s), va = s->vaxis;
#pragma omp parallel for schedule(static)
  for (long long kk = 0; kk < (long long)nn; ++kk) {
    size_t k = (size_t)kk;
    int xyz[3];
    node_coords(s, k, xyz);
    for (int i = 0; i < Q; ++i) {
      int to[3];
      int hits_wall = 0;
      for (int d = 0; d < 3; ++d) {
        to[d] = xyz[d] + s->ci[i][d];
        if (d == va && walls && (to[d] < 0 || to[d] >= s->n[d]))
          hits_wall = 1;
        else
          to[d] = wrap(to[d], s->n[d]);
      }
      double v = s->fpost[(size_t)i * nn + k];
      if (hits_wall) /* reflected back to the node it left, reversed */
        s->f[(size_t)s->opp[i] * nn + k] = v;
      else
        s->f[(size_t)i * nn + node_index(s, to[0], to[1], to[2])] = v;
    }
  }
}

/* ---- a5: one WENO5-JS reconstruction, upwind side on the left ----
 * v[0..4] are the split-flux values at i-2 .. i+2; the result approximates the
 * flux at the face i+1/2.  Candidate third-order fluxes on the three sub-stencils,
 * Jiang-Shu smoothness indicators, linear weights (1/10, 6/10, 3/10), and
 * nonlinear weights d_k/(eps + beta_k)^2 normalised to sum to one (S15-S16). */
double orc_weno5_left(const double v[5], double eps) {
  const double a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
  double q[3], beta[3];
  q[0] = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  q[1] = (-b + 5.0 * c + 2.0 * d) / 6.0;
  q[2] = (2.0 * c + 5.0 * d - e) / 6.0;
  beta[0] = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c) +
            0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
  beta[1] = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d) + 0.25 * (b - d) * (b - d);
  beta[2] = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e) +
            0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
  const double lin[3] = {0.1, 0.6, 0.3};
  double wt[3], sum = 0.0;
  for (int k = 0; k < 3; ++k) {
    wt[k] = lin[k] / ((eps + beta[k]) * (eps + beta[k]));
    sum += wt[k];
  }
  double h = 0.0;
  for (int k = 0; k < 3; ++k) h += wt[k] / sum * q[k];
  return h;
}

/* ---- a5 variant: one third-order WENO reconstruction, upwind side on the left ----
 * v[0..2] are the flux values at i-1, i, i+1; the result approximates the flux at the
 * face i+1/2: candidates h1 = (h_i + h_{i+1})/2 (S10) and h2 = -(h_{i-1} - 3 h_i)/2 (S11),
 * smoothness indicators beta1 = (h_{i+1} - h_i)^2, beta2 = (h_i - h_{i-1})^2 and weights
 * alpha_j/(eps + beta_j)^2 with alpha = (2/3, 1/3), normalised (S14-S16).  For the other
 * side the caller passes the mirror image (S17-S20). */
double orc_weno3_left(const double v[3], double eps) {
  const double hm1 = v[0], h0 = v[1], hp1 = v[2];
  const double q[2] = {0.5 * (h0 + hp1), -0.5 * (hm1 - 3.0 * h0)};
  const double beta[2] = {(hp1 - h0) * (hp1 - h0), (h0 - hm1) * (h0 - hm1)};
  const double lin[2] = {2.0 / 3.0, 1.0 / 3.0};
  double wt[2], sum = 0.0;
  for (int k = 0; k < 2; ++k) {
    wt[k] = lin[k] / ((eps + beta[k]) * (eps + beta[k]));
    sum += wt[k];
  }
  return wt[0] / sum * q[0] + wt[1] / sum * q[1];
}

/* Vertical ghost handling: index reflected into the fluid and whether it was a ghost. */
static int reflect_vertical(int v, int n, int *ghost) {
  *ghost = 0;
  if (v < 0) {
    *ghost = 1;
    return -1 - v;
  }
  if (v >= n) {
    *ghost = 1;
    return 2 * n - 1 - v;
  }
  return v;
}

/* ---- a4-a6: total flux through the face between node k and its +1 neighbour along axis d.
 * The caller never asks for the wall faces. */
static double face_flux(const orc_sim *s, const double *c, int xyz[3], int d) {
  const size_t nn = s->nn;
  const int va = s->vaxis;
  const int walls = vertical_walls(s) && d == va;
  double hp[6], hm[6], cv[6], wv[6];
  for (int m = -2; m <= 3; ++m) {
    int p[3] = {xyz[0], xyz[1], xyz[2]};
    int ghost = 0;
    if (walls)
      p[d] = reflect_vertical(xyz[d] + m, s->n[d], &ghost);
    else
      p[d] = wrap(xyz[d] + m, s->n[d]);
    size_t k = node_index(s, p[0], p[1], p[2]);
    double cval = c[k];
    double ud = s->u[(size_t)d * nn + k];
    if (ghost) ud = -ud; /* no-slip wall: velocity odd about the wall */
    double w = ud - (d == va ? settling_at(s, k) : 0.0);
    cv[m + 2] = cval;
    wv[m + 2] = w;
    hp[m + 2] = 0.5 * (w + s->alpha) * cval;
    hm[m + 2] = 0.5 * (w - s->alpha) * cval;
  }
  /* a6: central diffusion, flux = -kappa dc/dx at the face */
  const double fdiff = -s->p.diffusivity * (cv[3] - cv[2]);
  const int weno3 = (s->p.flags & ORC_WENO3) != 0;
  if (s->p.flags & ORC_SIGN_SPLIT) {
    /* whole flux h = w c, from the side the face velocity (w_i + w_{i+1})/2 comes from */
    double h[6];
    for (int m = 0; m < 6; ++m) h[m] = wv[m] * cv[m];
    const int from_left = 0.5 * (wv[2] + wv[3]) >= 0.0;
    if (weno3) {
      const double left[3] = {h[1], h[2], h[3]}, right[3] = {h[4], h[3], h[2]};
      return orc_weno3_left(from_left ? left : right, s->eps) + fdiff;
    }
    const double left[5] = {h[0], h[1], h[2], h[3], h[4]}, right[5] = {h[5], h[4], h[3], h[2], h[1]};
    return orc_weno5_left(from_left ? left : right, s->eps) + fdiff;
  }
  if (weno3) {
    /* h+ : points i-1..i+1; h- : mirror image, points i+2..i */
    const double left[3] = {hp[1], hp[2], hp[3]}, right[3] = {hm[4], hm[3], hm[2]};
    return orc_weno3_left(left, s->eps) + orc_weno3_left(right, s->eps) + fdiff;
  }
  /* h+ : upwind from the left, points i-2..i+2 */
  double fplus = orc_weno5_left(hp, s->eps);
  /* h- : mirror image, points i+3..i-1 read right to left */
  const double mirror[5] = {hm[5], hm[4], hm[3], hm[2], hm[1]};
  double fminus = orc_weno5_left(mirror, s->eps);
  return fplus + fminus + fdiff;
}

/* ---- a7: L(c) = -div(flux), conservative form ---- */

static void transport_rate(orc_sim *s, const double *c, double *L) {
  const size_t nn = s->nn;
  const int dim = s->p.dim, va = s->vaxis, walls = vertical_walls(s);
  for (size_t k = 0; k < nn; ++k) L[k] = 0.0;
  for (int d = 0; d < dim; ++d) {
    /* flux[k] = flux through the face on the + side of node k along d */
#pragma omp parallel for schedule(static)
    for (long long kk = 0; kk < (long long)nn; ++kk) {
      size_t k = (size_t)kk;
      int xyz[3];
      node_coords(s, k, xyz);
      if (d == va && walls && xyz[d] == s->n[d] - 1)
        s->flux[k] = 0.0; /* lid: no flux */
      else
        s->flux[k] = face_flux(s, c, xyz, d);
    }
#pragma omp parallel for schedule(static)
    for (long long kk = 0; kk < (long long)nn; ++kk) {
      size_t k = (size_t)kk;
      int xyz[3];
      node_coords(s, k, xyz);
      double fminus;
      if (d == va && walls && xyz[d] == 0) {
        fminus = -settling_at(s, k) * c[k]; /* floor: settling outflow */
      } else {
        int p[3] = {xyz[0], xyz[1], xyz[2]};
        p[d] = wrap(xyz[d] - 1, s->n[d]);
        fminus = s->flux[node_index(s, p[0], p[1], p[2])];
      }
      L[k] -= s->flux[k] - fminus;
    }
  }
}

/* Sum of c over the floor row/plane (v = 0), serial and in index order. */
static double floor_sum(const orc_sim *s, const double *c) {
  double acc = 0.0;
  if (s->p.dim == 2) {
    for (int x = 0; x < s->n[0]; ++x) acc += c[node_index(s, x, 0, 0)];
  } else {
    for (int y = 0; y < s->n[1]; ++y)
      for (int x = 0; x < s->n[0]; ++x) acc += c[node_index(s, x, y, 0)];
  }
  return acc;
}

/* With sugar: settling outflow through the floor, the sum of Vs(S) c over the floor
 * row/plane, serial and in index order. */
static double floor_outflow(const orc_sim *s, const double *c) {
  double acc = 0.0;
  if (s->p.dim == 2) {
    for (int x = 0; x < s->n[0]; ++x) {
      const size_t k = node_index(s, x, 0, 0);
      acc += settling_at(s, k) * c[k];
    }
  } else {
    for (int y = 0; y < s->n[1]; ++y)
      for (int x = 0; x < s->n[0]; ++x) {
        const size_t k = node_index(s, x, y, 0);
        acc += settling_at(s, k) * c[k];
      }
  }
  return acc;
}

/* ---- a8 + a9: SSP-RK3 (S21-S23) with dt = 1, velocity frozen, deposit by b-weights ---- */

static double rk3_transport(orc_sim *s, double *c) {
  const size_t nn = s->nn;
  double *c1 = s->c1, *c2 = s->c2, *L = s->L;
  transport_rate(s, c, L);
  for (size_t k = 0; k < nn; ++k) c1[k] = c[k] + L[k];
  transport_rate(s, c1, L);
  for (size_t k = 0; k < nn; ++k) c2[k] = 0.75 * c[k] + 0.25 * c1[k] + 0.25 * L[k];
  double dep = 0.0;
  if (vertical_walls(s)) {
    if (sugar_on(s))
      dep = floor_outflow(s, c) / 6.0 + floor_outflow(s, c1) / 6.0 + 2.0 * floor_outflow(s, c2) / 3.0;
    else
      dep = s->vs_cur * (floor_sum(s, c) / 6.0 + floor_sum(s, c1) / 6.0 + 2.0 * floor_sum(s, c2) / 3.0);
  }
  transport_rate(s, c2, L);
  for (size_t k = 0; k < nn; ++k) c[k] = c[k] / 3.0 + 2.0 * c2[k] / 3.0 + 2.0 * L[k] / 3.0;
  return dep;
}

/* a4-a9 for every particle class, each with its own settling velocity and deposit. */
static void transport_classes(orc_sim *s) {
  for (int k = 0; k < s->ncls; ++k) {
    s->vs_cur = s->ncls > 1 ? s->p.class_vs[k] : s->p.settling_velocity;
    const double dep = rk3_transport(s, class_c(s, k));
    s->cls_dep[k] += dep;
    s->deposit += dep;
  }
  s->vs_cur = s->ncls > 1 ? s->p.class_vs[0] : s->p.settling_velocity;
  sum_classes(s);
}

/* ---- s3: sugar, first-order upwind (S5 for u > 0, S6 for u < 0) per axis, explicit, in
 * the advective form the paper prints, plus central diffusion; Neumann walls read the
 * mirror node (S_{-1} = S_0). ---- */
static void sugar_transport(orc_sim *s) {
  const size_t nn = s->nn;
  const int dim = s->p.dim, va = s->vaxis, walls = vertical_walls(s);
  const double Ds = s->p.sugar_diffusivity;
#pragma omp parallel for schedule(static)
  for (long long kk = 0; kk < (long long)nn; ++kk) {
    const size_t k = (size_t)kk;
    int xyz[3];
    node_coords(s, k, xyz);
    const double a = s->S[k];
    double next = a;
    for (int d = 0; d < dim; ++d) {
      int pm[3] = {xyz[0], xyz[1], xyz[2]}, pp[3] = {xyz[0], xyz[1], xyz[2]};
      if (d == va && walls) {
        int g;
        pm[d] = reflect_vertical(xyz[d] - 1, s->n[d], &g);
        pp[d] = reflect_vertical(xyz[d] + 1, s->n[d], &g);
      } else {
        pm[d] = wrap(xyz[d] - 1, s->n[d]);
        pp[d] = wrap(xyz[d] + 1, s->n[d]);
      }
      const double am = s->S[node_index(s, pm[0], pm[1], pm[2])];
      const double ap = s->S[node_index(s, pp[0], pp[1], pp[2])];
      const double u = s->u[(size_t)d * nn + k];
      if (u > 0.0)
        next -= u * (a - am); /* S5, dt = dx = 1 */
      else
        next -= u * (ap - a); /* S6 */
      next += Ds * (ap - 2.0 * a + am);
    }
    s->Snew[k] = next;
  }
  double *t = s->S;
  s->S = s->Snew;
  s->Snew = t;
}

static void check_state(orc_sim *s) {
  const size_t nn = s->nn;
  for (size_t k = 0; k < nn; ++k) {
    for (int m = 0; m < s->ncls; ++m)
      if (!isfinite(class_c(s, m)[k])) s->status = ORC_EUNSTABLE;
    for (int d = 0; d < s->p.dim; ++d) {
      double ud = s->u[(size_t)d * nn + k];
      if (!isfinite(ud) || fabs(ud) > s->p.u_cap) s->status = ORC_EUNSTABLE;
    }
  }
}

/* ---- public entry points (ctypes) ---- */

orc_sim *orc_create(const orc_params *p) {
  if (!p || (p->dim != 2 && p->dim != 3) || p->nx < 4 || p->ny < 4 || p->tau <= 0.5) return NULL;
  if (p->dim == 3 && p->nz < 4) return NULL;
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  if (!s) return NULL;
  s->p = *p;
  if (s->p.dim == 2) s->p.nz = 1;
  if (s->p.u_cap <= 0.0) s->p.u_cap = 0.1;
  s->n[0] = s->p.nx;
  s->n[1] = s->p.ny;
  s->n[2] = s->p.nz;
  s->vaxis = s->p.dim - 1;
  s->nn = (size_t)s->n[0] * s->n[1] * s->n[2];
  if (s->p.n_classes > 8) {
    free(s);
    return NULL;
  }
  s->ncls = s->p.n_classes >= 2 ? s->p.n_classes : 1;
  s->vs_cur = s->ncls > 1 ? s->p.class_vs[0] : s->p.settling_velocity;
  double vs_max = s->p.settling_velocity;
  for (int k = 0; k < s->ncls && s->ncls > 1; ++k) vs_max = k == 0 || s->p.class_vs[k] > vs_max ? s->p.class_vs[k] : vs_max;
  s->alpha = s->p.lf_alpha > 0.0 ? s->p.lf_alpha : vs_max + s->p.u_cap;
  s->eps = 1e-6 * s->alpha * s->alpha;
  if (s->p.dim == 2)
    set_d2q9(s);
  else
    set_d3q19(s);
  set_opposites(s);
  const size_t nn = s->nn;
  s->f = (double *)calloc((size_t)s->Q * nn, sizeof(double));
  s->fpost = (double *)calloc((size_t)s->Q * nn, sizeof(double));
  s->c = (double *)calloc(nn, sizeof(double));
  s->c1 = (double *)calloc(nn, sizeof(double));
  s->c2 = (double *)calloc(nn, sizeof(double));
  s->L = (double *)calloc(nn, sizeof(double));
  s->flux = (double *)calloc(nn, sizeof(double));
  s->rho = (double *)calloc(nn, sizeof(double));
  s->u = (double *)calloc((size_t)s->p.dim * nn, sizeof(double));
  s->S = (double *)calloc(nn, sizeof(double));
  s->Snew = (double *)calloc(nn, sizeof(double));
  s->cls = (double *)calloc((size_t)s->ncls * nn, sizeof(double)); /* classes 1.. (one spare) */
  s->ctot = (double *)calloc(nn, sizeof(double));
  if (!s->f || !s->fpost || !s->c || !s->c1 || !s->c2 || !s->L || !s->flux || !s->rho || !s->u || !s->S ||
      !s->Snew || !s->cls || !s->ctot) {
    free(s->f); free(s->fpost); free(s->c); free(s->c1); free(s->c2);
    free(s->L); free(s->flux); free(s->rho); free(s->u); free(s->S); free(s->Snew);
    free(s->cls); free(s->ctot); free(s);
    return NULL;
  }
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->f); free(s->fpost); free(s->c); free(s->c1); free(s->c2);
  free(s->L); free(s->flux); free(s->rho); free(s->u); free(s->S); free(s->Snew);
  free(s->cls); free(s->ctot);
  free(s);
}

/* c0[nn] required.  u0[dim*nn] optional: populations start at equilibrium
 * f_i = f_i^eq(rho = 1, u0) (or f_i = w_i when u0 is NULL). */
int orc_init(orc_sim *s, const double *c0, const double *u0) {
  if (!s || !c0) return ORC_EINVAL;
  const size_t nn = s->nn;
  const double cs2 = 1.0 / 3.0;
  memcpy(s->c, c0, nn * sizeof(double));
  for (size_t k = 0; k < nn; ++k) {
    double u[3] = {0.0, 0.0, 0.0};
    if (u0)
      for (int d = 0; d < s->p.dim; ++d) u[d] = u0[(size_t)d * nn + k];
    for (int d = 0; d < s->p.dim; ++d) s->u[(size_t)d * nn + k] = u[d];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < s->Q; ++i) {
      double cu = s->ci[i][0] * u[0] + s->ci[i][1] * u[1] + s->ci[i][2] * u[2];
      s->f[(size_t)i * nn + k] =
          s->wi[i] * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    }
    s->rho[k] = 1.0;
  }
  memset(s->S, 0, nn * sizeof(double));
  memset(s->cls, 0, (size_t)s->ncls * nn * sizeof(double));
  memset(s->cls_dep, 0, sizeof(s->cls_dep));
  sum_classes(s);
  s->deposit = 0.0;
  s->steps = 0;
  s->status = ORC_OK;
  return ORC_OK;
}

/* Sugar field (ORC_SUGAR), set after orc_init and read back. */
int orc_set_sugar(orc_sim *s, const double *S0) {
  if (!s || !S0 || !sugar_on(s)) return ORC_EINVAL;
  memcpy(s->S, S0, s->nn * sizeof(double));
  return ORC_OK;
}

void orc_sugar(const orc_sim *s, double *S) { memcpy(S, s->S, s->nn * sizeof(double)); }

/* Particle class k (polydisperse): set after orc_init (which puts c0 in class 0 and zeros
 * the others), read, and its deposit. */
int orc_set_class(orc_sim *s, int k, const double *ck) {
  if (!s || !ck || k < 0 || k >= s->ncls) return ORC_EINVAL;
  memcpy(class_c(s, k), ck, s->nn * sizeof(double));
  sum_classes(s);
  return ORC_OK;
}

int orc_class(const orc_sim *s, int k, double *out) {
  if (!s || !out || k < 0 || k >= s->ncls) return ORC_EINVAL;
  memcpy(out, class_c(s, k), s->nn * sizeof(double));
  return ORC_OK;
}

double orc_class_deposit(const orc_sim *s, int k) { return (k >= 0 && k < s->ncls) ? s->cls_dep[k] : 0.0; }

/* One coupled step = a1..a3 on the populations (unless the velocity is frozen),
 * then a4..a9 on c with the velocity of a1 (O7: u at time n, frozen over the stages). */
int orc_step(orc_sim *s, int64_t nsteps) {
  if (!s) return ORC_EINVAL;
  for (int64_t t = 0; t < nsteps; ++t) {
    if (!(s->p.flags & ORC_FROZEN_VELOCITY)) {
      collide_all(s);
      stream_all(s);
    }
    transport_classes(s);
    if (sugar_on(s)) sugar_transport(s);
    check_state(s);
    s->steps++;
  }
  return s->status;
}

/* Macroscopic fields of the current state: rho, the half-force-corrected
 * velocity u = (sum f c + F/2)/rho computed with the current c, and c.
 * With a frozen velocity, rho = 1 and u is the frozen field.  Any pointer may be NULL. */
void orc_fields(const orc_sim *s, double *rho, double *u, double *c) {
  const size_t nn = s->nn;
  for (size_t k = 0; k < nn; ++k) {
    if (s->p.flags & ORC_FROZEN_VELOCITY) {
      if (rho) rho[k] = 1.0;
      if (u)
        for (int d = 0; d < s->p.dim; ++d) u[(size_t)d * nn + k] = s->u[(size_t)d * nn + k];
    } else {
      double F[3];
      node_force(s, k, F);
      double r = 0.0, mom[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < s->Q; ++i) {
        double fi = s->f[(size_t)i * nn + k];
        r += fi;
        for (int d = 0; d < 3; ++d) mom[d] += fi * s->ci[i][d];
      }
      if (rho) rho[k] = r;
      if (u)
        for (int d = 0; d < s->p.dim; ++d) u[(size_t)d * nn + k] = (mom[d] + 0.5 * F[d]) / r;
    }
    if (c) c[k] = s->ncls > 1 ? s->ctot[k] : s->c[k];
  }
}

/* Raw population sums over the domain: out[0] = sum f, out[1..3] = sum f c_i (serial). */
void orc_population_moments(const orc_sim *s, double out[4]) {
  const size_t nn = s->nn;
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (size_t k = 0; k < nn; ++k)
    for (int i = 0; i < s->Q; ++i) {
      double fi = s->f[(size_t)i * nn + k];
      out[0] += fi;
      for (int d = 0; d < 3; ++d) out[1 + d] += fi * s->ci[i][d];
    }
}

double orc_deposit(const orc_sim *s) { return s->deposit; }
int64_t orc_steps(const orc_sim *s) { return s->steps; }
double orc_alpha(const orc_sim *s) { return s->alpha; }

/* Total c over the domain, serial and in index order. */
double orc_total_mass(const orc_sim *s) {
  double acc = 0.0;
  for (size_t k = 0; k < s->nn; ++k) acc += s->ncls > 1 ? s->ctot[k] : s->c[k];
  return acc;
}

/* Particle mass below the horizontal plane under vertical level `level` (Sec. 4.2.3,
 * Eq. flux: the mass in the volume below the plane, m_i = c_i in lattice units), plus
 * the deposited mass, which lies below every plane: the cells with vertical index
 * v < level, summed serially in index order.  Returns NaN for a level outside 0..N. */
double orc_mass_below(const orc_sim *s, int level) {
  const int vax = s->p.dim - 1;
  const int nv = s->n[vax];
  if (level < 0 || level > nv) return NAN;
  double acc = 0.0;
  for (size_t k = 0; k < s->nn; ++k) {
    const int v = (int)(k / ((size_t)s->nn / (size_t)nv));  /* vertical index: the slowest axis */
    if (v < level) acc += s->ncls > 1 ? s->ctot[k] : s->c[k];
  }
  return acc + s->deposit;
}

/* L(c) for a given c and transport velocity u (dim*nn), using the walls and
 * parameters of the simulation; used to pin the spatial operator alone. */
void orc_transport_rate(orc_sim *s, const double *c, const double *u, double *L) {
  memcpy(s->u, u, (size_t)s->p.dim * s->nn * sizeof(double));
  transport_rate(s, c, L);
}

int orc_lattice(const orc_sim *s, int *ci, double *wi) {
  for (int i = 0; i < s->Q; ++i) {
    for (int d = 0; d < 3; ++d) ci[3 * i + d] = s->ci[i][d];
    wi[i] = s->wi[i];
  }
  return s->Q;
}

/* =====================================================================================
 * Reverse sweep: gradient of the deposited mass (Sec. 4, m_b) after nsteps steps with
 * respect to the initial concentration c0 and the settling velocity Vs (2D, walls, the
 * Lax-Friedrichs alpha held fixed).
 *
 * The forward run keeps every step's state (populations and c before the step, the
 * step's u, c1 and c2).  The reverse run then applies, step by step from the last, the
 * transpose of each forward operation to the adjoint fields.  The local Jacobians are
 * not derived by hand: each is the complex-step derivative  dF/dx = Im F(x + i h) / h
 * (h = 1e-30, exact to rounding for the rational functions used here) of a complex twin
 * of the forward routine above -- the WENO5 reconstruction, the face flux and the
 * per-node BGK-Guo collision -- which restates it operation for operation in complex
 * arithmetic.  Streaming, the Shu-Osher combinations and the deposit are linear and are
 * transposed directly.
 * ===================================================================================== */
#include <complex.h>

typedef double complex cplx;
static const double kCstep = 1e-30;

static cplx weno5_left_cx(const cplx v[5], double eps) {
  const cplx a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
  cplx q[3], beta[3];
  q[0] = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  q[1] = (-b + 5.0 * c + 2.0 * d) / 6.0;
  q[2] = (2.0 * c + 5.0 * d - e) / 6.0;
  beta[0] = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c) +
            0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
  beta[1] = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d) + 0.25 * (b - d) * (b - d);
  beta[2] = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e) +
            0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
  const double lin[3] = {0.1, 0.6, 0.3};
  cplx wt[3], sum = 0.0;
  for (int k = 0; k < 3; ++k) {
    wt[k] = lin[k] / ((eps + beta[k]) * (eps + beta[k]));
    sum += wt[k];
  }
  cplx h = 0.0;
  for (int k = 0; k < 3; ++k) h += wt[k] / sum * q[k];
  return h;
}

/* Face flux from its six stencil values c[0..5] and face-normal velocities w[0..5]
 * (positions i-2 .. i+3; ghosts already mirrored by the caller), as in face_flux. */
static cplx face_flux_cx(const orc_sim *s, const cplx cv[6], const cplx w[6]) {
  cplx hp[6], hm[6];
  for (int m = 0; m < 6; ++m) {
    hp[m] = 0.5 * (w[m] + s->alpha) * cv[m];
    hm[m] = 0.5 * (w[m] - s->alpha) * cv[m];
  }
  const cplx fplus = weno5_left_cx(hp, s->eps);
  const cplx mirror[5] = {hm[5], hm[4], hm[3], hm[2], hm[1]};
  const cplx fminus = weno5_left_cx(mirror, s->eps);
  const cplx fdiff = -s->p.diffusivity * (cv[3] - cv[2]);
  return fplus + fminus + fdiff;
}

/* Stencil of the face on the + side of node xyz along d, as face_flux reads it: node
 * indices, ghost flags, c and w = u_d (odd at a wall) - Vs (vertical). */
static void face_stencil(const orc_sim *s, const double *c, const int xyz[3], int d, size_t idx[6], int ghost[6],
                         double cv[6], double w[6]) {
  const int va = s->vaxis;
  const int walls = vertical_walls(s) && d == va;
  for (int m = -2; m <= 3; ++m) {
    int p[3] = {xyz[0], xyz[1], xyz[2]};
    int g = 0;
    if (walls)
      p[d] = reflect_vertical(xyz[d] + m, s->n[d], &g);
    else
      p[d] = wrap(xyz[d] + m, s->n[d]);
    const size_t k = node_index(s, p[0], p[1], p[2]);
    double ud = s->u[(size_t)d * s->nn + k];
    if (g) ud = -ud;
    idx[m + 2] = k;
    ghost[m + 2] = g;
    cv[m + 2] = c[k];
    w[m + 2] = ud - (d == va ? s->p.settling_velocity : 0.0);
  }
}

/* Transpose of L(c; u) applied to lamL: lam_c += (dL/dc)^T lamL, lam_u += (dL/du)^T lamL,
 * *lam_vs += (dL/dVs)^T lamL.  L_k = sum_d (F_{k-1/2} - F_{k+1/2}), so the face on the +
 * side of k carries lamF = lamL[next] - lamL[k]; the floor face F = -Vs c_0 enters L_0. */
static void rate_adjoint(orc_sim *s, const double *c, const double *lamL, double *lam_c, double *lam_u,
                         double *lam_vs, double *dfc, double *dfw) {
  const size_t nn = s->nn;
  const int dim = s->p.dim, va = s->vaxis, walls = vertical_walls(s);
  for (int d = 0; d < dim; ++d) {
    /* derivatives of every face flux (parallel), then the scatter (serial, index order) */
#pragma omp parallel for schedule(static)
    for (long long kk = 0; kk < (long long)nn; ++kk) {
      const size_t k = (size_t)kk;
      int xyz[3];
      node_coords(s, k, xyz);
      if (d == va && walls && xyz[d] == s->n[d] - 1) continue; /* lid: no face */
      size_t idx[6];
      int ghost[6];
      double cv[6], w[6];
      face_stencil(s, c, xyz, d, idx, ghost, cv, w);
      for (int j = 0; j < 6; ++j) {
        cplx cc[6], ww[6];
        for (int m = 0; m < 6; ++m) {
          cc[m] = cv[m];
          ww[m] = w[m];
        }
        cc[j] += I * kCstep;
        dfc[6 * k + j] = cimag(face_flux_cx(s, cc, ww)) / kCstep;
        cc[j] = cv[j];
        ww[j] += I * kCstep;
        dfw[6 * k + j] = cimag(face_flux_cx(s, cc, ww)) / kCstep;
      }
    }
    for (size_t k = 0; k < nn; ++k) {
      int xyz[3];
      node_coords(s, k, xyz);
      if (d == va && walls && xyz[d] == s->n[d] - 1) continue;
      int q[3] = {xyz[0], xyz[1], xyz[2]};
      q[d] = wrap(xyz[d] + 1, s->n[d]);
      const double lamF = lamL[node_index(s, q[0], q[1], q[2])] - lamL[k];
      size_t idx[6];
      int ghost[6];
      double cv[6], w[6];
      face_stencil(s, c, xyz, d, idx, ghost, cv, w);
      for (int j = 0; j < 6; ++j) {
        lam_c[idx[j]] += lamF * dfc[6 * k + j];
        lam_u[(size_t)d * nn + idx[j]] += lamF * (ghost[j] ? -dfw[6 * k + j] : dfw[6 * k + j]);
        if (d == va) *lam_vs -= lamF * dfw[6 * k + j]; /* w = +-u - Vs */
      }
    }
  }
  if (walls) {
    for (size_t k = 0; k < nn; ++k) {
      int xyz[3];
      node_coords(s, k, xyz);
      if (xyz[va] != 0) continue;
      lam_c[k] -= s->p.settling_velocity * lamL[k];
      *lam_vs -= c[k] * lamL[k];
    }
  }
}

/* Complex twin of one node of collide_all: populations f and concentration c in,
 * post-collision populations and the velocity out. */
static void collide_node_cx(const orc_sim *s, const cplx *f, cplx cval, cplx *fpost, cplx u[3]) {
  const int Q = s->Q;
  const double tau = s->p.tau, cs2 = 1.0 / 3.0;
  cplx F[3];
  for (int d = 0; d < 3; ++d) F[d] = s->p.body_force[d];
  F[s->vaxis] -= s->p.gravity * s->p.density_contrast * cval;
  cplx rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    for (int d = 0; d < 3; ++d) mom[d] += f[i] * s->ci[i][d];
  }
  for (int d = 0; d < 3; ++d) u[d] = (mom[d] + 0.5 * F[d]) / rho;
  const cplx uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    const cplx cu = s->ci[i][0] * u[0] + s->ci[i][1] * u[1] + s->ci[i][2] * u[2];
    const cplx feq = s->wi[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    cplx src = 0.0;
    for (int d = 0; d < 3; ++d) src += ((s->ci[i][d] - u[d]) / cs2 + cu * s->ci[i][d] / (cs2 * cs2)) * F[d];
    src *= (1.0 - 1.0 / (2.0 * tau)) * s->wi[i];
    fpost[i] = f[i] - (f[i] - feq) / tau + src;
  }
}

/* Reverse of collide + stream at every node: lam_next = lambda of the populations after
 * streaming, lam_u = lambda of the step's velocity; out: lambda of the populations
 * before the step (lam_f) and the buoyancy's share of lambda(c) (added to lam_c). */
static void fluid_adjoint(orc_sim *s, const double *f, const double *c, const double *lam_next,
                          const double *lam_u, double *lam_f, double *lam_c) {
  const int Q = s->Q, dim = s->p.dim, va = s->vaxis, walls = vertical_walls(s);
  const size_t nn = s->nn;
#pragma omp parallel for schedule(static)
  for (long long kk = 0; kk < (long long)nn; ++kk) {
    const size_t k = (size_t)kk;
    int xyz[3];
    node_coords(s, k, xyz);
    /* adjoint of the post-collision populations: where streaming sent each one */
    double lpost[19];
    for (int i = 0; i < Q; ++i) {
      int to[3];
      int hits_wall = 0;
      for (int d = 0; d < 3; ++d) {
        to[d] = xyz[d] + s->ci[i][d];
        if (d == va && walls && (to[d] < 0 || to[d] >= s->n[d]))
          hits_wall = 1;
        else
          to[d] = wrap(to[d], s->n[d]);
      }
      lpost[i] = hits_wall ? lam_next[(size_t)s->opp[i] * nn + k]
                           : lam_next[(size_t)i * nn + node_index(s, to[0], to[1], to[2])];
    }
    /* Jacobian columns of (fpost, u) with respect to each f_j and c, by complex step */
    cplx fin[19], fpost[19], u[3];
    for (int j = 0; j <= Q; ++j) {
      for (int i = 0; i < Q; ++i) fin[i] = f[(size_t)i * nn + k];
      cplx cval = c[k];
      if (j < Q)
        fin[j] += I * kCstep;
      else
        cval += I * kCstep;
      collide_node_cx(s, fin, cval, fpost, u);
      double acc = 0.0;
      for (int i = 0; i < Q; ++i) acc += lpost[i] * cimag(fpost[i]) / kCstep;
      for (int d = 0; d < dim; ++d) acc += lam_u[(size_t)d * nn + k] * cimag(u[d]) / kCstep;
      if (j < Q)
        lam_f[(size_t)j * nn + k] = acc;
      else
        lam_c[k] += acc;
    }
  }
}

/* J = deposited mass after nsteps steps from c0 (fluid at rest); grad_c0 = dJ/dc0,
 * *dJ_dVs = dJ/dVs at fixed alpha.  2D with walls, lf_alpha > 0, velocity not frozen. */
int orc_deposit_gradient(const orc_params *p, const double *c0, int64_t nsteps, double *grad_c0, double *dJ_dVs,
                         double *J) {
  if (!p || !c0 || !grad_c0 || !dJ_dVs || !J || nsteps < 1) return ORC_EINVAL;
  if (p->dim != 2 ||
      (p->flags & (ORC_PERIODIC_VERTICAL | ORC_FROZEN_VELOCITY | ORC_SUGAR | ORC_WENO3 | ORC_SIGN_SPLIT)) ||
      p->n_classes >= 2 ||
      !(p->lf_alpha > 0.0))
    return ORC_EINVAL;
  orc_sim *s = orc_create(p);
  if (!s) return ORC_EINVAL;
  const int Q = s->Q, dim = s->p.dim;
  const size_t nn = s->nn, per = (size_t)(Q + 3 + dim) * nn; /* f, c, c1, c2, u */
  double *hist = (double *)malloc(per * (size_t)nsteps * sizeof(double));
  double *work = (double *)calloc((size_t)(2 * Q + 5 + dim + 12) * nn, sizeof(double));
  if (!hist || !work) {
    free(hist);
    free(work);
    orc_destroy(s);
    return ORC_ENOMEM;
  }
  orc_init(s, c0, NULL);
  for (int64_t t = 0; t < nsteps; ++t) {
    double *h = hist + per * (size_t)t;
    memcpy(h, s->f, (size_t)Q * nn * sizeof(double));
    memcpy(h + (size_t)Q * nn, s->c, nn * sizeof(double));
    orc_step(s, 1);
    memcpy(h + (size_t)(Q + 1) * nn, s->c1, nn * sizeof(double));
    memcpy(h + (size_t)(Q + 2) * nn, s->c2, nn * sizeof(double));
    memcpy(h + (size_t)(Q + 3) * nn, s->u, (size_t)dim * nn * sizeof(double));
  }
  *J = s->deposit;
  double *lam_next = work, *lam_f = work + (size_t)Q * nn;
  double *mu = work + (size_t)2 * Q * nn, *lc2 = mu + nn, *lc1 = lc2 + nn, *lc = lc1 + nn, *lamL = lc + nn;
  double *lam_u = lamL + nn, *dfc = lam_u + (size_t)dim * nn, *dfw = dfc + 6 * nn;
  double lam_vs = 0.0;
  const double vs = s->p.settling_velocity;
  /* lambda(c^N) = 0 and lambda(f^N) = 0: J does not depend on the final state */
  for (int64_t t = nsteps - 1; t >= 0; --t) {
    const double *h = hist + per * (size_t)t;
    const double *f = h, *c = h + (size_t)Q * nn, *c1 = h + (size_t)(Q + 1) * nn, *c2 = h + (size_t)(Q + 2) * nn;
    memcpy(s->u, h + (size_t)(Q + 3) * nn, (size_t)dim * nn * sizeof(double));
    for (size_t k = 0; k < (size_t)dim * nn; ++k) lam_u[k] = 0.0;
    /* deposit += Vs (sum_floor c/6 + c1/6 + 2 c2/3) */
    for (int x = 0; x < s->n[0]; ++x) {
      const size_t k = node_index(s, x, 0, 0);
      lam_vs += c[k] / 6.0 + c1[k] / 6.0 + 2.0 * c2[k] / 3.0;
    }
    /* stage 3: c' = c/3 + 2 c2/3 + 2 L(c2)/3 */
    for (size_t k = 0; k < nn; ++k) {
      lamL[k] = 2.0 * mu[k] / 3.0;
      lc2[k] = 2.0 * mu[k] / 3.0;
    }
    for (int x = 0; x < s->n[0]; ++x) lc2[node_index(s, x, 0, 0)] += 2.0 * vs / 3.0;
    rate_adjoint(s, c2, lamL, lc2, lam_u, &lam_vs, dfc, dfw);
    /* stage 2: c2 = 3c/4 + c1/4 + L(c1)/4 */
    for (size_t k = 0; k < nn; ++k) {
      lamL[k] = 0.25 * lc2[k];
      lc1[k] = 0.25 * lc2[k];
    }
    for (int x = 0; x < s->n[0]; ++x) lc1[node_index(s, x, 0, 0)] += vs / 6.0;
    rate_adjoint(s, c1, lamL, lc1, lam_u, &lam_vs, dfc, dfw);
    /* stage 1: c1 = c + L(c) */
    for (size_t k = 0; k < nn; ++k) {
      lamL[k] = lc1[k];
      lc[k] = mu[k] / 3.0 + 0.75 * lc2[k] + lc1[k];
    }
    for (int x = 0; x < s->n[0]; ++x) lc[node_index(s, x, 0, 0)] += vs / 6.0;
    rate_adjoint(s, c, lamL, lc, lam_u, &lam_vs, dfc, dfw);
    /* fluid step */
    fluid_adjoint(s, f, c, lam_next, lam_u, lam_f, lc);
    memcpy(lam_next, lam_f, (size_t)Q * nn * sizeof(double));
    memcpy(mu, lc, nn * sizeof(double));
  }
  memcpy(grad_c0, mu, nn * sizeof(double));
  *dJ_dVs = lam_vs;
  free(hist);
  free(work);
  orc_destroy(s);
  return ORC_OK;
}
