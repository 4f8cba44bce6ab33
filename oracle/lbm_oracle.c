/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle for the LB-IMB-DEM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library: only
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Method (Xiong et al., "Large-Scale DNS of Gas-Solid Flow on Mole-8.5"):
 *   - LBGK on D2Q9 / D3Q19 (section "Numerical scheme").
 *   - Noble-Torczynski immersed moving boundary, Eq. (1) with beta of Eq. (2)
 *     and the solid collision term Omega^S printed after Eq. (2).
 *   - solid fraction eps per lattice cell = covered area/volume (text after
 *     the Omega^S equation); computed here exactly from its definition.
 *   - hydrodynamic force and torque, Eq. (3).
 *   - frictionless spring-dashpot DEM, Eqs. (4)-(5).
 *
 * Readings where the paper is silent or garbled (identical in the CUDA path):
 *   R1 state between steps = post-collision populations f*; a step is
 *      rasterise eps -> stream (pull) -> moments -> collide -> force -> DEM.
 *   R2 several particles on one node: eps = min(1, sum_p e_p),
 *      V_S = sum_p e_p V_p / sum_p e_p, node force split by e_p / sum_p e_p.
 *   R3 V_S includes rotation: V_p = v_p + omega_p x (x_n - x_p), minimum image.
 *   R4 body force F_i = 3 w_i rho (c_i . g_f), at every node.
 *   R5 force on the particle = -sum_n beta_n sum_i Omega_i^S c_i (momentum given
 *      to the fluid is taken from the particle), torque likewise with
 *      (x_n - x_p) x.  Sum over all lattice directions, h^d/dt = 1.
 *   R6 halfway bounce-back walls at y = -1/2 and y = ny - 1/2 when wall_y.
 *   R7 DEM (Eqs. 4-5 garbled): overlap xi = R_i + R_j - |r_i - r_j|, force on i
 *      = k xi n_ij - eta v_n,ij with n_ij = (r_i - r_j)/|r_i - r_j|, damping
 *      eta = -2 ln(e) sqrt(m* k / (pi^2 + ln^2 e)), m* = m_i m_j/(m_i + m_j);
 *      walls use m* = m_i.  Symplectic Euler: v += (F_f + F_c + m g_s)/m dt,
 *      x += v dt, omega += T_f/I dt, `substeps` sub-steps of dt = 1/substeps.
 *   R8 masses: 2D m = rho_s pi R^2 (per unit depth), I = m R^2 / 2;
 *      3D m = rho_s 4/3 pi R^3, I = 2/5 m R^2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_MAX_OWNERS 8

/* ------------------------------------------------------------------ */
/* Lattices (McNamara & Zanetti D2Q9 / D3Q19, standard weights).       */
/* Direction order is the library's documented interface order.        */
/* ------------------------------------------------------------------ */
static const int D2Q9_C[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const double D2Q9_W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                 1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int D3Q19_C[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
static const double D3Q19_W[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
  int Q;
  int c[19][3];
  double w[19];
  int opp[19];
} lattice_t;

static void lattice_init(lattice_t* L, int dim) {
  L->Q = dim == 2 ? 9 : 19;
  for (int i = 0; i < L->Q; i++) {
    for (int d = 0; d < 3; d++) L->c[i][d] = dim == 2 ? D2Q9_C[i][d] : D3Q19_C[i][d];
    L->w[i] = dim == 2 ? D2Q9_W[i] : D3Q19_W[i];
  }
  /* opposite direction found by search: c_opp = -c */
  for (int i = 0; i < L->Q; i++)
    for (int j = 0; j < L->Q; j++)
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
          L->c[j][2] == -L->c[i][2])
        L->opp[i] = j;
}

/* ------------------------------------------------------------------ */
/* Exact covered area / volume (definition of eps).                    */
/* ------------------------------------------------------------------ */

/* integral_0^t sqrt(R^2 - s^2) ds for t in [-R, R], written with atan2 and
 * (R-t)(R+t) so that it stays well conditioned near t = +-R */
static double chord_prim(double t, double R) {
  if (t <= -R) return -0.25 * M_PI * R * R;
  if (t >= R) return 0.25 * M_PI * R * R;
  double s = sqrt((R - t) * (R + t));
  return 0.5 * (t * s + R * R * atan2(t, s));
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Area of disk(centre (cx,cy), radius R) intersected with [x0,x1]x[y0,y1]:
 * the integral over x of the length of [y0,y1] n [cy - s(x), cy + s(x)],
 * s(x) = sqrt(R^2 - (x-cx)^2), split where an end of the chord crosses y0 or
 * y1 so that each piece integrates in closed form.  Coordinates are taken
 * relative to the centre first, so the ends of the disk sit exactly at +-R. */
double oracle_area_disk_rect(double cx, double cy, double R, double x0,
                             double x1, double y0, double y1) {
  if (R <= 0.0) return 0.0;
  double X0 = x0 - cx, X1 = x1 - cx, Y0 = y0 - cy, Y1 = y1 - cy;
  double a = fmax(X0, -R), b = fmin(X1, R);
  if (!(a < b) || !(Y0 < Y1)) return 0.0;
  /* every corner inside the disk: the whole rectangle is covered */
  double fx = fmax(fabs(X0), fabs(X1)), fy = fmax(fabs(Y0), fabs(Y1));
  if (fx * fx + fy * fy <= R * R) return (x1 - x0) * (y1 - y0);
  double bp[8];
  int nb = 0;
  bp[nb++] = a;
  bp[nb++] = b;
  double ys[2] = {Y0, Y1};
  for (int k = 0; k < 2; k++) {
    double d = fabs(ys[k]);
    if (d < R) {
      double h = sqrt((R - d) * (R + d));
      if (-h > a && -h < b) bp[nb++] = -h;
      if (h > a && h < b) bp[nb++] = h;
    }
  }
  qsort(bp, nb, sizeof(double), cmp_double);
  double total = 0.0;
  for (int k = 0; k + 1 < nb; k++) {
    double p = bp[k], q = bp[k + 1];
    if (!(q > p)) continue;
    double xm = 0.5 * (p + q);
    double sm = sqrt((R - fabs(xm)) * (R + fabs(xm)));
    int top_circle = sm <= Y1; /* <=: tangent chord at the midpoint */
    int bot_circle = -sm >= Y0;
    double top_m = top_circle ? sm : Y1;
    double bot_m = bot_circle ? -sm : Y0;
    if (!(top_m > bot_m)) continue; /* chord misses the strip on this piece */
    double Is = chord_prim(q, R) - chord_prim(p, R); /* int s dx */
    double top_int = top_circle ? Is : Y1 * (q - p);
    double bot_int = bot_circle ? -Is : Y0 * (q - p);
    total += top_int - bot_int;
  }
  return total;
}

/* Gauss-Legendre nodes/weights on [0,1] (Newton on P_n). */
#define GL_N 24
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;
static void gl_init(void) {
  if (gl_ready) return;
  const int n = GL_N;
  for (int i = 0; i < n; i++) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; k++) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; k++) {
      double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    double dp = n * (x * p1 - p0) / (x * x - 1.0);
    gl_x[i] = 0.5 * (x + 1.0);
    gl_w[i] = 1.0 / ((1.0 - x * x) * dp * dp); /* = 2/((1-x^2)P'^2) scaled by 1/2 */
  }
  gl_ready = 1;
}

/* Volume of ball(centre, R) intersected with the box: the integral over z of
 * the exact slice area (disk of radius sqrt(R^2 - (z-cz)^2) against the
 * rectangle).  The slice area is analytic in z between the heights where the
 * slice circle becomes tangent to an edge line of the rectangle or passes
 * through a corner; each such piece is integrated by Gauss-Legendre after the
 * substitution z = za + (zb-za)(3t^2 - 2t^3), which removes the (z-zb)^{3/2}
 * tangency behaviour at the piece ends. */
double oracle_volume_ball_box(double cx, double cy, double cz, double R,
                              double x0, double x1, double y0, double y1,
                              double z0, double z1) {
  if (R <= 0.0) return 0.0;
  double za = fmax(z0, cz - R), zb = fmin(z1, cz + R);
  if (!(za < zb)) return 0.0;
  /* nearest point of the box to the centre beyond R: empty */
  double nx = fmax(fmax(x0 - cx, 0.0), cx - x1);
  double ny = fmax(fmax(y0 - cy, 0.0), cy - y1);
  double nz = fmax(fmax(z0 - cz, 0.0), cz - z1);
  if (nx * nx + ny * ny + nz * nz >= R * R) return 0.0;
  /* farthest corner inside R: the whole box is covered */
  double fx = fmax(fabs(x0 - cx), fabs(x1 - cx));
  double fy = fmax(fabs(y0 - cy), fabs(y1 - cy));
  double fz = fmax(fabs(z0 - cz), fabs(z1 - cz));
  if (fx * fx + fy * fy + fz * fz <= R * R)
    return (x1 - x0) * (y1 - y0) * (z1 - z0);
  gl_init();
  double radii[8];
  int nr = 0;
  double dx[2] = {x0 - cx, x1 - cx}, dy[2] = {y0 - cy, y1 - cy};
  for (int k = 0; k < 2; k++) radii[nr++] = fabs(dx[k]);
  for (int k = 0; k < 2; k++) radii[nr++] = fabs(dy[k]);
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) radii[nr++] = sqrt(dx[i] * dx[i] + dy[j] * dy[j]);
  double bp[20];
  int nb = 0;
  bp[nb++] = za;
  bp[nb++] = zb;
  for (int k = 0; k < nr; k++) {
    if (radii[k] < R) {
      double h = sqrt((R - radii[k]) * (R + radii[k]));
      if (cz - h > za && cz - h < zb) bp[nb++] = cz - h;
      if (cz + h > za && cz + h < zb) bp[nb++] = cz + h;
    }
  }
  qsort(bp, nb, sizeof(double), cmp_double);
  double total = 0.0;
  for (int k = 0; k + 1 < nb; k++) {
    double p = bp[k], q = bp[k + 1];
    if (!(q > p)) continue;
    double piece = 0.0;
    for (int g = 0; g < GL_N; g++) {
      double t = gl_x[g];
      double z = p + (q - p) * t * t * (3.0 - 2.0 * t);
      double jac = (q - p) * 6.0 * t * (1.0 - t);
      double dz = fabs(z - cz);
      double r = dz < R ? sqrt((R - dz) * (R + dz)) : 0.0;
      piece += gl_w[g] * jac * oracle_area_disk_rect(cx, cy, r, x0, x1, y0, y1);
    }
    total += piece;
  }
  return total;
}

/* covered fraction of the unit lattice cell centred on node (i,j,k) */
double oracle_cell_fraction(int dim, double cx, double cy, double cz, double R,
                            double i, double j, double k) {
  if (dim == 2)
    return oracle_area_disk_rect(cx, cy, R, i - 0.5, i + 0.5, j - 0.5, j + 0.5);
  return oracle_volume_ball_box(cx, cy, cz, R, i - 0.5, i + 0.5, j - 0.5,
                                j + 0.5, k - 0.5, k + 0.5);
}

/* ------------------------------------------------------------------ */
/* LBGK + IMB node update                                              */
/* ------------------------------------------------------------------ */

/* f_i^eq(rho, v) = w_i rho (1 + 3 c.v + 4.5 (c.v)^2 - 1.5 v.v) */
static double feq(const lattice_t* L, int i, double rho, const double v[3]) {
  double cu = L->c[i][0] * v[0] + L->c[i][1] * v[1] + L->c[i][2] * v[2];
  double uu = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  return L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* One node: post-stream populations ft -> post-collision fout (Eq. 1).
 * nown owners with covered fractions e[] and solid velocities vs[3*k] at the
 * node.  m_out = beta * sum_i Omega_i^S c_i (momentum given to the fluid).
 * Returns beta. */
static double collide_node(const lattice_t* L, double tau, const double g[3],
                           const double* ft, int nown, const double* e,
                           const double* vs, double* fout, double* m_out,
                           double* rho_out, double* u_out) {
  const int Q = L->Q;
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; i++) {
    rho += ft[i];
    for (int d = 0; d < 3; d++) j[d] += ft[i] * L->c[i][d];
  }
  double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double esum = 0.0, VS[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < nown; k++) esum += e[k];
  double beta = 0.0;
  if (nown > 0 && esum > 0.0) {
    for (int k = 0; k < nown; k++)
      for (int d = 0; d < 3; d++) VS[d] += e[k] * vs[3 * k + d];
    for (int d = 0; d < 3; d++) VS[d] /= esum;
    double eps = esum < 1.0 ? esum : 1.0;
    beta = eps * (tau - 0.5) / ((1.0 - eps) + (tau - 0.5)); /* Eq. (2) */
  }
  double m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; i++) {
    int o = L->opp[i];
    double Fi = 3.0 * L->w[i] * rho *
                (L->c[i][0] * g[0] + L->c[i][1] * g[1] + L->c[i][2] * g[2]);
    double OmS = 0.0;
    if (beta != 0.0)
      OmS = ft[o] - ft[i] + feq(L, i, rho, VS) - feq(L, o, rho, u);
    fout[i] = ft[i] - (1.0 - beta) / tau * (ft[i] - feq(L, i, rho, u)) +
              beta * OmS + Fi;
    for (int d = 0; d < 3; d++) m[d] += OmS * L->c[i][d];
  }
  for (int d = 0; d < 3; d++) m_out[d] = beta * m[d];
  if (rho_out) *rho_out = rho;
  if (u_out)
    for (int d = 0; d < 3; d++) u_out[d] = u[d];
  return beta;
}

/* exported per-node entry for invariant tests */
double oracle_collide_node(int dim, double tau, const double* g,
                           const double* ft, int nown, const double* e,
                           const double* vs, double* fout, double* m_out) {
  lattice_t L;
  lattice_init(&L, dim);
  return collide_node(&L, tau, g, ft, nown, e, vs, fout, m_out, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* DEM (Eqs. 4-5, reading R7)                                          */
/* ------------------------------------------------------------------ */

static double wrap_delta(double d, double Lx) {
  if (d > 0.5 * Lx) d -= Lx;
  else if (d < -0.5 * Lx) d += Lx;
  return d;
}

/* Contact forces at the current state; fc[3*np]. */
static void dem_contacts(int dim, const int Ld[3], int wall_y, int np,
                         const double* pos, const double* vel,
                         const double* rad, const double* mass, double kn,
                         double e, double* fc) {
  double le = log(e);
  double den = M_PI * M_PI + le * le;
  memset(fc, 0, sizeof(double) * 3 * np);
  for (int i = 0; i < np; i++) {
    for (int j = 0; j < np; j++) {
      if (j == i) continue;
      double r[3], d2 = 0.0;
      for (int d = 0; d < 3; d++) {
        r[d] = pos[3 * i + d] - pos[3 * j + d];
        if (d < dim && !(d == 1 && wall_y)) r[d] = wrap_delta(r[d], Ld[d]);
        if (d >= dim) r[d] = 0.0;
        d2 += r[d] * r[d];
      }
      double dist = sqrt(d2);
      double xi = rad[i] + rad[j] - dist;
      if (!(xi > 0.0) || dist == 0.0) continue;
      double n[3] = {r[0] / dist, r[1] / dist, r[2] / dist};
      double vr = 0.0;
      for (int d = 0; d < 3; d++) vr += (vel[3 * i + d] - vel[3 * j + d]) * n[d];
      double ms = mass[i] * mass[j] / (mass[i] + mass[j]);
      double eta = -2.0 * le * sqrt(ms * kn / den);
      for (int d = 0; d < 3; d++) fc[3 * i + d] += kn * xi * n[d] - eta * vr * n[d];
    }
    if (wall_y) {
      /* bottom wall plane y = -1/2 (normal +y), top y = ny - 1/2 (normal -y) */
      double eta = -2.0 * le * sqrt(mass[i] * kn / den);
      double xb = rad[i] - (pos[3 * i + 1] + 0.5);
      if (xb > 0.0) {
        double vr = vel[3 * i + 1];
        fc[3 * i + 1] += kn * xb - eta * vr;
      }
      double xt = rad[i] - ((Ld[1] - 0.5) - pos[3 * i + 1]);
      if (xt > 0.0) {
        double vr = -vel[3 * i + 1];
        fc[3 * i + 1] += -(kn * xt - eta * vr);
      }
    }
  }
}

/* exported for tests: contact forces of the current state */
void oracle_dem_contacts(int dim, const int* Ld, int wall_y, int np,
                         const double* pos, const double* vel, const double* rad,
                         const double* mass, double kn, double e, double* fc) {
  dem_contacts(dim, Ld, wall_y, np, pos, vel, rad, mass, kn, e, fc);
}

/* Advance particles by one lattice time step given hydrodynamic force ff and
 * torque tf (reading R7).  fc_out receives the contact force of the last
 * sub-step. */
void oracle_dem_advance(int dim, const int* Ld, int wall_y, int np,
                        double* pos, double* vel, double* omg,
                        const double* rad, const double* mass,
                        const double* inertia, const double* ff,
                        const double* tf, const double* gs, double kn,
                        double e, int substeps, double* fc_out) {
  double* fc = (double*)malloc(sizeof(double) * 3 * (np > 0 ? np : 1));
  double dt = 1.0 / substeps;
  for (int s = 0; s < substeps; s++) {
    dem_contacts(dim, Ld, wall_y, np, pos, vel, rad, mass, kn, e, fc);
    for (int i = 0; i < np; i++) {
      for (int d = 0; d < dim; d++) {
        double a = (ff[3 * i + d] + fc[3 * i + d] + mass[i] * gs[d]) / mass[i];
        vel[3 * i + d] += a * dt;
        pos[3 * i + d] += vel[3 * i + d] * dt;
        if (!(d == 1 && wall_y)) {
          if (pos[3 * i + d] >= Ld[d]) pos[3 * i + d] -= Ld[d];
          else if (pos[3 * i + d] < 0.0) pos[3 * i + d] += Ld[d];
        }
      }
      for (int d = 0; d < 3; d++) omg[3 * i + d] += tf[3 * i + d] / inertia[i] * dt;
    }
  }
  if (fc_out) memcpy(fc_out, fc, sizeof(double) * 3 * np);
  free(fc);
}

/* ------------------------------------------------------------------ */
/* Simulation state                                                    */
/* ------------------------------------------------------------------ */
typedef struct oracle_sim {
  lattice_t L;
  int dim, n[3], wall_y, substeps, np;
  long N;
  double tau, gf[3], gs[3], kn, e;
  double *pos, *vel, *omg, *rad, *mass, *inertia;
  double *ff, *tf, *fc;
  double *f, *ft, *fn; /* stored post-collision, post-stream scratch, next */
  int* own_n;          /* owners per node */
  int* own_p;          /* [N*OR_MAX_OWNERS] particle ids, ascending */
  double* own_e;       /* [N*OR_MAX_OWNERS] covered fraction per owner */
  long step;
  int eps_method;      /* 0 exact covered fractions, 1 the table of Eq. (6) */
  float* tab;          /* Eq. (6) table */
  float tab_lo_r, tab_h_r, tab_h_s, tab_h_t;
} oracle_sim;

static long node_index(const oracle_sim* s, int x, int y, int z) {
  return ((long)z * s->n[1] + y) * s->n[0] + x;
}

int oracle_rasterize(oracle_sim* s);

/* ------------------------------------------------------------------ */
/* Eq. (6): covered fraction looked up in a table over the cell's      */
/* position relative to the particle centre (one radius R).            */
/* With the sorted offsets a >= b (>= c) >= 0 of the cell centre:       */
/*   2D: r = |(a,b)| on [R - sqrt(2)/2, R + sqrt(2)/2], 256 points;     */
/*       t = b/a on [0, 1], 128 points;                                 */
/*   3D: r = |(a,b,c)| on [R - sqrt(3)/2, R + sqrt(3)/2], 96 points;    */
/*       s = |(b,c)|/a on [0, sqrt(2)], 64 points; t = c/b on [0,1], 48. */
/* Entries: the exact fraction at the grid point, stored in FP32;       */
/* lookup: (bi/tri)linear interpolation in FP32, each operation rounded */
/* on its own.  Cells entirely inside take 1, outside 0 (as R10).        */
/* ------------------------------------------------------------------ */
#define OT_R2 256
#define OT_T2 128
#define OT_R3 96
#define OT_S3 64
#define OT_T3 48

static float ot_lerp(float x, float y, float w) {
  float a = (1.0f - w) * x;
  float b = w * y;
  return a + b;
}

static float ot_coord(float x, float lo, float h, int n, int* i) {
  float f = (x - lo) / h;
  if (f < 0.0f) f = 0.0f;
  if (f > (float)(n - 1)) f = (float)(n - 1);
  int k = (int)f;
  if (k > n - 2) k = n - 2;
  *i = k;
  return f - (float)k;
}

static float ot_lookup(const oracle_sim* s, const double off[3]) {
  float a = fabsf((float)off[0]), b = fabsf((float)off[1]), c = s->dim == 3 ? fabsf((float)off[2]) : 0.0f;
  float t0;
  if (a < b) { t0 = a; a = b; b = t0; }
  if (s->dim == 3) {
    if (b < c) { t0 = b; b = c; c = t0; }
    if (a < b) { t0 = a; a = b; b = t0; }
  }
  if (s->dim == 2) {
    float r = sqrtf(a * a + b * b);
    float t = a > 0.0f ? b / a : 0.0f;
    int i, j;
    float wr = ot_coord(r, s->tab_lo_r, s->tab_h_r, OT_R2, &i);
    float wt = ot_coord(t, 0.0f, s->tab_h_t, OT_T2, &j);
    const float* T = s->tab;
    float lo_r = ot_lerp(T[i * OT_T2 + j], T[i * OT_T2 + j + 1], wt);
    float hi_r = ot_lerp(T[(i + 1) * OT_T2 + j], T[(i + 1) * OT_T2 + j + 1], wt);
    return ot_lerp(lo_r, hi_r, wr);
  }
  float aa = a * a, bb = b * b, cc = c * c;
  float r = sqrtf((aa + bb) + cc);
  float sv = a > 0.0f ? sqrtf(bb + cc) / a : 0.0f;
  float t = b > 0.0f ? c / b : 0.0f;
  int i, j, k;
  float wr = ot_coord(r, s->tab_lo_r, s->tab_h_r, OT_R3, &i);
  float ws = ot_coord(sv, 0.0f, s->tab_h_s, OT_S3, &j);
  float wt = ot_coord(t, 0.0f, s->tab_h_t, OT_T3, &k);
  float v[2];
  for (int di = 0; di < 2; di++) {
    const float* T = s->tab + ((i + di) * OT_S3 + j) * OT_T3 + k;
    float lo_s = ot_lerp(T[0], T[1], wt);
    float hi_s = ot_lerp(T[OT_T3], T[OT_T3 + 1], wt);
    v[di] = ot_lerp(lo_s, hi_s, ws);
  }
  return ot_lerp(v[0], v[1], wr);
}

/* switch a simulation to the table (all radii equal and > 1); rebuilds the
 * owners.  Returns 0, or -1 if the radii differ. */
int oracle_set_eps_table(oracle_sim* s) {
  if (s->np == 0) return 0;
  double R = s->rad[0];
  for (int p = 1; p < s->np; p++)
    if (s->rad[p] != R) return -1;
  if (!(R > 1.0)) return -1;
  free(s->tab);
  if (s->dim == 2) {
    s->tab = (float*)malloc(sizeof(float) * OT_R2 * OT_T2);
    for (int i = 0; i < OT_R2; i++)
      for (int j = 0; j < OT_T2; j++) {
        double r = (R - sqrt(2.0) / 2.0) + i * (sqrt(2.0) / (OT_R2 - 1));
        double t = j * (1.0 / (OT_T2 - 1));
        double a = r / sqrt(1.0 + t * t);
        s->tab[i * OT_T2 + j] = (float)oracle_cell_fraction(2, 0.0, 0.0, 0.0, R, a, a * t, 0.0);
      }
    s->tab_lo_r = (float)(R - sqrt(2.0) / 2.0);
    s->tab_h_r = (float)(sqrt(2.0) / (OT_R2 - 1));
    s->tab_h_s = 0.0f;
    s->tab_h_t = (float)(1.0 / (OT_T2 - 1));
  } else {
    s->tab = (float*)malloc(sizeof(float) * OT_R3 * OT_S3 * OT_T3);
    for (int i = 0; i < OT_R3; i++)
      for (int j = 0; j < OT_S3; j++)
        for (int k = 0; k < OT_T3; k++) {
          double r = (R - sqrt(3.0) / 2.0) + i * (sqrt(3.0) / (OT_R3 - 1));
          double sv = j * (sqrt(2.0) / (OT_S3 - 1));
          double t = k * (1.0 / (OT_T3 - 1));
          double a = r / sqrt(1.0 + sv * sv);
          double b = a * sv / sqrt(1.0 + t * t);
          s->tab[(i * OT_S3 + j) * OT_T3 + k] = (float)oracle_cell_fraction(3, 0.0, 0.0, 0.0, R, a, b, b * t);
        }
    s->tab_lo_r = (float)(R - sqrt(3.0) / 2.0);
    s->tab_h_r = (float)(sqrt(3.0) / (OT_R3 - 1));
    s->tab_h_s = (float)(sqrt(2.0) / (OT_S3 - 1));
    s->tab_h_t = (float)(1.0 / (OT_T3 - 1));
  }
  s->eps_method = 1;
  return oracle_rasterize(s);
}

/* the table value at an arbitrary offset of the cell centre (test hook) */
double oracle_eps_table_value(const oracle_sim* s, double ox, double oy, double oz) {
  double off[3] = {ox, oy, oz};
  return (double)ot_lookup(s, off);
}

/* Eq. (6) fraction of cell (i,j,k) for the ball (c, R): 1 inside, 0 outside,
 * the table in between (clamped to [0, 1]) */
static double table_cell_fraction(const oracle_sim* s, const double c[3], double R, int i, int j, int k) {
  int idx[3] = {i, j, k};
  double near2 = 0.0, far2 = 0.0, off[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < s->dim; d++) {
    double bl = ((double)idx[d] - 0.5) - c[d], bh = ((double)idx[d] + 0.5) - c[d];
    double nd = bl > 0.0 ? bl : (bh < 0.0 ? -bh : 0.0);
    double fd = fabs(bl) > fabs(bh) ? fabs(bl) : fabs(bh);
    near2 += nd * nd;
    far2 += fd * fd;
    off[d] = (double)idx[d] - c[d];
  }
  if (near2 >= R * R) return 0.0;
  if (far2 <= R * R) return 1.0;
  float e = ot_lookup(s, off);
  if (e < 0.0f) e = 0.0f;
  if (e > 1.0f) e = 1.0f;
  return (double)e;
}

/* eps rasterisation: for each particle (ascending id) every node whose cell
 * meets the disk/ball receives (p, e_p) when e_p > 0.  Returns -1 when a node
 * would get more than OR_MAX_OWNERS owners. */
/* The OpenMP pragmas below matter only to the timing build of this file
 * (compiled with -fopenmp to time the oracle on all host cores); the parity
 * build ignores them and runs every loop in the order written.  In the timing
 * build particles rasterise concurrently (owner slots are appended under a
 * critical section, so their order on a shared node may differ) and the
 * force and torque sums are atomic (another summation order). */
int oracle_rasterize(oracle_sim* s) {
  memset(s->own_n, 0, sizeof(int) * s->N);
  int status = 0;
#pragma omp parallel for schedule(dynamic, 4)
  for (int p = 0; p < s->np; p++) {
    double c[3] = {s->pos[3 * p], s->pos[3 * p + 1], s->pos[3 * p + 2]};
    double R = s->rad[p];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < s->dim; d++) {
      lo[d] = (int)ceil(c[d] - R - 0.5);
      hi[d] = (int)floor(c[d] + R + 0.5);
    }
    for (int k = lo[2]; k <= hi[2]; k++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          int idx[3] = {i, j, k};
          int skip = 0;
          for (int d = 0; d < s->dim; d++) {
            if (d == 1 && s->wall_y) {
              if (idx[1] < 0 || idx[1] >= s->n[1]) skip = 1;
            } else {
              idx[d] = ((idx[d] % s->n[d]) + s->n[d]) % s->n[d];
            }
          }
          if (skip) continue;
          double ev = s->eps_method == 1 ? table_cell_fraction(s, c, R, i, j, k)
                                         : oracle_cell_fraction(s->dim, c[0], c[1], c[2], R, i, j, k);
          if (!(ev > 0.0)) continue;
          long n = node_index(s, idx[0], idx[1], idx[2]);
#pragma omp critical(oracle_owner_slots)
          {
            int m = s->own_n[n];
            if (m >= OR_MAX_OWNERS) {
              status = -1;
            } else {
              s->own_p[n * OR_MAX_OWNERS + m] = p;
              s->own_e[n * OR_MAX_OWNERS + m] = ev;
              s->own_n[n] = m + 1;
            }
          }
        }
  }
  return status;
}

oracle_sim* oracle_create(int dim, int nx, int ny, int nz, int wall_y,
                          double tau, const double* gf, const double* gs,
                          double rho0, double kn, double e, int substeps,
                          int np, const double* pos, const double* vel,
                          const double* omg, const double* rad,
                          const double* rho_s) {
  oracle_sim* s = (oracle_sim*)calloc(1, sizeof(oracle_sim));
  lattice_init(&s->L, dim);
  s->dim = dim;
  s->n[0] = nx;
  s->n[1] = ny;
  s->n[2] = dim == 2 ? 1 : nz;
  s->N = (long)s->n[0] * s->n[1] * s->n[2];
  s->wall_y = wall_y;
  s->tau = tau;
  for (int d = 0; d < 3; d++) {
    s->gf[d] = gf[d];
    s->gs[d] = gs[d];
  }
  s->kn = kn;
  s->e = e;
  s->substeps = substeps > 0 ? substeps : 1;
  s->np = np;
  int npa = np > 0 ? np : 1;
  s->pos = (double*)calloc(3 * npa, sizeof(double));
  s->vel = (double*)calloc(3 * npa, sizeof(double));
  s->omg = (double*)calloc(3 * npa, sizeof(double));
  s->ff = (double*)calloc(3 * npa, sizeof(double));
  s->tf = (double*)calloc(3 * npa, sizeof(double));
  s->fc = (double*)calloc(3 * npa, sizeof(double));
  s->rad = (double*)calloc(npa, sizeof(double));
  s->mass = (double*)calloc(npa, sizeof(double));
  s->inertia = (double*)calloc(npa, sizeof(double));
  for (int p = 0; p < np; p++) {
    for (int d = 0; d < 3; d++) {
      s->pos[3 * p + d] = pos[3 * p + d];
      s->vel[3 * p + d] = vel[3 * p + d];
      s->omg[3 * p + d] = omg[3 * p + d];
    }
    if (dim == 2) {
      s->pos[3 * p + 2] = 0.0;
      s->vel[3 * p + 2] = 0.0;
      s->omg[3 * p + 0] = 0.0;
      s->omg[3 * p + 1] = 0.0;
    }
    double R = rad[p];
    s->rad[p] = R;
    if (dim == 2) {
      s->mass[p] = rho_s[p] * M_PI * R * R;
      s->inertia[p] = 0.5 * s->mass[p] * R * R;
    } else {
      s->mass[p] = rho_s[p] * (4.0 / 3.0) * M_PI * R * R * R;
      s->inertia[p] = 0.4 * s->mass[p] * R * R;
    }
  }
  const int Q = s->L.Q;
  s->f = (double*)malloc(sizeof(double) * Q * s->N);
  s->ft = (double*)malloc(sizeof(double) * Q * s->N);
  s->fn = (double*)malloc(sizeof(double) * Q * s->N);
  for (int i = 0; i < Q; i++)
    for (long n = 0; n < s->N; n++) s->f[i * s->N + n] = s->L.w[i] * rho0;
  s->own_n = (int*)calloc(s->N, sizeof(int));
  s->own_p = (int*)malloc(sizeof(int) * s->N * OR_MAX_OWNERS);
  s->own_e = (double*)malloc(sizeof(double) * s->N * OR_MAX_OWNERS);
  oracle_rasterize(s);
  return s;
}

void oracle_destroy(oracle_sim* s) {
  if (!s) return;
  free(s->pos); free(s->vel); free(s->omg); free(s->ff); free(s->tf);
  free(s->fc); free(s->rad); free(s->mass); free(s->inertia); free(s->tab);
  free(s->f); free(s->ft); free(s->fn);
  free(s->own_n); free(s->own_p); free(s->own_e);
  free(s);
}

/* pull streaming of the stored post-collision populations into dst */
static void stream_pull(const oracle_sim* s, const double* src, double* dst) {
  const int Q = s->L.Q;
#pragma omp parallel for collapse(2)
  for (int z = 0; z < s->n[2]; z++)
    for (int y = 0; y < s->n[1]; y++)
      for (int x = 0; x < s->n[0]; x++) {
        long n = node_index(s, x, y, z);
        for (int i = 0; i < Q; i++) {
          int sx = x - s->L.c[i][0], sy = y - s->L.c[i][1], sz = z - s->L.c[i][2];
          if (s->wall_y && (sy < 0 || sy >= s->n[1])) {
            dst[i * s->N + n] = src[s->L.opp[i] * s->N + n]; /* bounce-back */
            continue;
          }
          sx = (sx + s->n[0]) % s->n[0];
          sy = (sy + s->n[1]) % s->n[1];
          sz = (sz + s->n[2]) % s->n[2];
          dst[i * s->N + n] = src[i * s->N + node_index(s, sx, sy, sz)];
        }
      }
}

/* node position minus particle centre, minimum image on periodic axes */
static void node_offset(const oracle_sim* s, int x, int y, int z, int p,
                        double r[3]) {
  double xn[3] = {x, y, z};
  for (int d = 0; d < 3; d++) {
    if (d >= s->dim) {
      r[d] = 0.0;
      continue;
    }
    r[d] = xn[d] - s->pos[3 * p + d];
    if (!(d == 1 && s->wall_y)) r[d] = wrap_delta(r[d], s->n[d]);
  }
}

int oracle_step(oracle_sim* s, int nsteps) {
  const int Q = s->L.Q;
  int status = 0;
  for (int t = 0; t < nsteps; t++) {
    /* 1. solid fraction from the current particle positions */
    if (oracle_rasterize(s) != 0) status = -1;
    /* 2. streaming */
    stream_pull(s, s->f, s->ft);
    /* 3-5. collision with IMB, force and torque */
    memset(s->ff, 0, sizeof(double) * 3 * s->np);
    memset(s->tf, 0, sizeof(double) * 3 * s->np);
#pragma omp parallel for collapse(2)
    for (int z = 0; z < s->n[2]; z++)
      for (int y = 0; y < s->n[1]; y++)
        for (int x = 0; x < s->n[0]; x++) {
          double ftn[19], fo[19];
          long n = node_index(s, x, y, z);
          for (int i = 0; i < Q; i++) ftn[i] = s->ft[i * s->N + n];
          int no = s->own_n[n];
          double e[OR_MAX_OWNERS], vs[3 * OR_MAX_OWNERS], r[OR_MAX_OWNERS][3];
          for (int k = 0; k < no; k++) {
            int p = s->own_p[n * OR_MAX_OWNERS + k];
            e[k] = s->own_e[n * OR_MAX_OWNERS + k];
            node_offset(s, x, y, z, p, r[k]);
            const double* w = &s->omg[3 * p];
            const double* v = &s->vel[3 * p];
            vs[3 * k + 0] = v[0] + (w[1] * r[k][2] - w[2] * r[k][1]);
            vs[3 * k + 1] = v[1] + (w[2] * r[k][0] - w[0] * r[k][2]);
            vs[3 * k + 2] = v[2] + (w[0] * r[k][1] - w[1] * r[k][0]);
          }
          double m[3];
          collide_node(&s->L, s->tau, s->gf, ftn, no, e, vs, fo, m, NULL, NULL);
          for (int i = 0; i < Q; i++) s->fn[i * s->N + n] = fo[i];
          if (no > 0) {
            double esum = 0.0;
            for (int k = 0; k < no; k++) esum += e[k];
            if (esum > 0.0) {
              for (int k = 0; k < no; k++) {
                int p = s->own_p[n * OR_MAX_OWNERS + k];
                double a = e[k] / esum;
                double mp[3] = {a * m[0], a * m[1], a * m[2]};
                double tq[3] = {r[k][1] * mp[2] - r[k][2] * mp[1], r[k][2] * mp[0] - r[k][0] * mp[2],
                                r[k][0] * mp[1] - r[k][1] * mp[0]};
                for (int d = 0; d < 3; d++) {
#pragma omp atomic
                  s->ff[3 * p + d] -= mp[d];
#pragma omp atomic
                  s->tf[3 * p + d] -= tq[d];
                }
              }
            }
          }
        }
    double* tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
    /* 6. DEM */
    oracle_dem_advance(s->dim, s->n, s->wall_y, s->np, s->pos, s->vel, s->omg,
                       s->rad, s->mass, s->inertia, s->ff, s->tf, s->gs, s->kn,
                       s->e, s->substeps, s->fc);
    s->step++;
  }
  /* leave eps/owners describing the current positions */
  if (oracle_rasterize(s) != 0) status = -1;
  return status;
}

/* ------------------------------------------------------------------ */
/* Accessors                                                           */
/* ------------------------------------------------------------------ */
long oracle_num_nodes(const oracle_sim* s) { return s->N; }
int oracle_num_dirs(const oracle_sim* s) { return s->L.Q; }

void oracle_get_populations(const oracle_sim* s, double* f) {
  memcpy(f, s->f, sizeof(double) * s->L.Q * s->N);
}
void oracle_set_populations(oracle_sim* s, const double* f) {
  memcpy(s->f, f, sizeof(double) * s->L.Q * s->N);
}
void oracle_get_particles(const oracle_sim* s, double* pos, double* vel,
                          double* omg, double* ff, double* tf, double* fc) {
  size_t b = sizeof(double) * 3 * s->np;
  if (pos) memcpy(pos, s->pos, b);
  if (vel) memcpy(vel, s->vel, b);
  if (omg) memcpy(omg, s->omg, b);
  if (ff) memcpy(ff, s->ff, b);
  if (tf) memcpy(tf, s->tf, b);
  if (fc) memcpy(fc, s->fc, b);
}
void oracle_get_mass(const oracle_sim* s, double* mass, double* inertia) {
  if (mass) memcpy(mass, s->mass, sizeof(double) * s->np);
  if (inertia) memcpy(inertia, s->inertia, sizeof(double) * s->np);
}

/* rho and the fluid velocity of the populations the next collision sees (the
 * stored state streamed): u = sum_i ft_i c_i / rho + g_f / 2, the average of
 * the momentum before and after the body force of Eq. (1) (this is the
 * velocity that solves the body-force driven channel flow exactly); eps =
 * min(1, sum of owner fractions) at the current particle positions. */
void oracle_fields(oracle_sim* s, double* rho, double* u, double* eps) {
  const int Q = s->L.Q;
  stream_pull(s, s->f, s->ft);
  for (long n = 0; n < s->N; n++) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) {
      double v = s->ft[i * s->N + n];
      r += v;
      for (int d = 0; d < 3; d++) j[d] += v * s->L.c[i][d];
    }
    if (rho) rho[n] = r;
    if (u)
      for (int d = 0; d < s->dim; d++) u[d * s->N + n] = j[d] / r + 0.5 * s->gf[d];
    if (eps) {
      double es = 0.0;
      for (int k = 0; k < s->own_n[n]; k++) es += s->own_e[n * OR_MAX_OWNERS + k];
      eps[n] = es < 1.0 ? es : 1.0;
    }
  }
}

/* owner lists (ascending particle id) for tests: cnt[N], ids/eps [N*maxo] */
void oracle_get_owners(const oracle_sim* s, int* cnt, int* ids, double* e,
                       int maxo) {
  for (long n = 0; n < s->N; n++) {
    cnt[n] = s->own_n[n];
    for (int k = 0; k < maxo; k++) {
      int ok = k < s->own_n[n];
      ids[n * maxo + k] = ok ? s->own_p[n * OR_MAX_OWNERS + k] : -1;
      e[n * maxo + k] = ok ? s->own_e[n * OR_MAX_OWNERS + k] : 0.0;
    }
  }
}
