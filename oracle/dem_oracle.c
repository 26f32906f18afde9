/*
 * dem_oracle.c -- plain FP64 CPU oracle of one soft-sphere DEM time step.
 *
 * TEST INFRASTRUCTURE ONLY: the reference against which the CUDA path is checked.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.  It is written from Golshan et al., "Lethe-DEM"
 * (arXiv 2106.09576) and shares no code with the CUDA library.  It is deliberately
 * simple: serial loops, FP64 throughout, compiled with -ffp-contract=off.
 *
 * One step n -> n+1 follows the paper's order:
 *   1. velocity Verlet half kick and drift (Sec. 2.2, Eq. halfstep);
 *   2. contact-search decision, constant or dynamic (Sec. 3.1), and if due the broad
 *      search over cells and the fine search with threshold r_c (Sec. 3.2);
 *   3. particle-particle and particle-wall contact forces (Sec. 2.1, Eqs. deltan to
 *      coulomb_overlap3, Table equation_parameters, Table rolling_torque);
 *   4. second half kick (Eq. newvv) with the accelerations of Eqs. main1 and main2.
 * With the explicit Euler integrator (Eq. integ_EE) a step is instead v^{n+1} = v^n + a^n dt
 * and x^{n+1} = x^n + v^n dt with the forces at (x^n, v^n), then the search when due and
 * the forces at (x^{n+1}, v^{n+1}).
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - the torque of Eq. torque_t uses the tangential force after the Coulomb limit;
 *   - the tangential overlap is incremented first, then used (Eq. delta_t);
 *     no re-projection onto the tangent plane (Sec. 2.1, the LIGGGHTS-like update);
 *   - a pair in the list that is not in contact has zero tangential overlap;
 *   - the Coulomb test is |F_t| >= mu |F_n| with the full normal force, skipped when F_t = 0;
 *   - rolling torque is zero when the relative angular velocity is zero;
 *   - a wall acts as a partner of infinite mass and radius (m_e = m_i, R_e = R_i),
 *     with e, mu and mu_r of the wall material, surface velocity Omega x (p*-c) + V at
 *     the nearest wall point p*, and spin Omega;
 *   - forces at step n+1 use x^{n+1} and the half-step velocities;
 *   - moment of inertia of a solid sphere, I = 2/5 m R^2;
 *   - the forces before the first step use the stored tangential overlap without the
 *     v_rt dt increment;
 *   - particles whose centre drops below z_sink leave the simulation;
 *   - linear model: the same k and eta in the normal and tangential directions (the
 *     paper says both directions use Eqs. linearkn and linearetan);
 *   - viscous rolling: V_omega = (R_i w_i + R_j w_j) x n for a particle pair and
 *     R_i (w_i - Omega) x n against a wall spinning with Omega;
 *   - explicit Euler: every force evaluation after the first of a run adds v_rt dt to
 *     the tangential overlap first (as in the velocity Verlet steps).
 */
#include "dem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_WALLS 8
#define ORC_PI 3.14159265358979323846

struct orc_sim {
  orc_config cfg;
  int64_t n;
  double *x, *v, *w;       /* [n][3] */
  double *F, *M;           /* [n][3] contact force / torque sums of the last evaluation */
  double *Fabs, *Mabs;     /* [n] sums of |contact force| and |contact torque| (error scales) */
  double *R, *m, *I;       /* radius, mass, moment of inertia */
  uint8_t* active;
  double* xref;            /* positions at the last contact search */
  /* fine-search list: pairs (pi[k], pj[k]) with pi < pj, lexicographic, and the
     tangential overlap H[k] of the (pi, pj) orientation */
  int64_t np, cap;
  int32_t *pi, *pj;
  double* H;
  int have_list;
  int64_t since_search;
  orc_wall walls[ORC_MAX_WALLS];
  double wall_Omega[ORC_MAX_WALLS][3];
  int nwalls;
  double* Hw;              /* [n][ORC_MAX_WALLS][3] particle-wall tangential overlap */
  int64_t step, searches;
  int forces_valid;
  double rc, dmax;
  int64_t n_touch, n_wall_touch;
};

/* ---------------------------------------------------------------- vectors */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* ---------------------------------------------- effective material constants
 * Table "equation_parameters": 1/Y_e = (1-nu_i^2)/Y_i + (1-nu_j^2)/Y_j,
 * 1/G_e = 2(2-nu_i)(1+nu_i)/Y_i + 2(2-nu_j)(1+nu_j)/Y_j,
 * beta = ln(e) / sqrt(ln(e)^2 + pi^2). */
static double eff_young(const orc_material* a, const orc_material* b) {
  return 1.0 / ((1.0 - a->poisson * a->poisson) / a->young + (1.0 - b->poisson * b->poisson) / b->young);
}
static double eff_shear(const orc_material* a, const orc_material* b) {
  return 1.0 / (2.0 * (2.0 - a->poisson) * (1.0 + a->poisson) / a->young +
                2.0 * (2.0 - b->poisson) * (1.0 + b->poisson) / b->young);
}
static double damping_beta(double e) {
  double le = log(e);
  return le / sqrt(le * le + ORC_PI * ORC_PI);
}
/* 1 + (pi / ln e)^2, the denominator of Eq. linearetan (infinite for e = 1: no damping) */
static double linear_damping_den(double e) {
  double q = ORC_PI / log(e);
  return 1.0 + q * q;
}

/* ------------------------------------------------------------ contact law
 * One contact of particle i with a partner (particle j or a wall), Sec. 2.1.
 *   nrm   : unit normal from i towards the partner (Eq. vecn)
 *   dn    : normal overlap > 0 (Eq. deltan)
 *   vij   : relative contact velocity v_i - v_j + (R_i w_i + R_j w_j) x n
 *   dw    : relative angular velocity w_i - w_j (rolling, Table rolling_torque)
 *   Re,me : effective radius and mass; Ye, Ge, beta: Table equation_parameters
 *   dt_t  : in: tangential overlap before the step; out: after (Eq. delta_t and the
 *           Coulomb limit, Eqs. coulomb_overlap..coulomb_overlap3)
 *   incr  : 1 = add v_rt dt (a time step), 0 = evaluate with the stored overlap
 * Outputs: F_n and F_t on i, n x F_t (the caller multiplies by the lever R_i or R_j
 * of Eq. torque_t), the rolling torque on i, and |F_n|. */
typedef struct {
  double Fn[3], Ft[3], nxFt[3], Mr[3], absFn;
} contact_out;

typedef struct {
  int model;         /* 0 non-linear, 1 linear */
  double V;          /* characteristic impact velocity of Eq. linearkn */
  double lin_den;    /* 1 + (pi / ln e)^2 of Eq. linearetan */
} law_opts;

static void contact_law(const double* nrm, double dn, const double* vij, const double* dw,
                        const double* vomega, double Re, double me, double Ye, double Ge, double beta,
                        double mu, double mu_r, int rolling, const law_opts* lo, double dt, double* dt_t,
                        int incr, contact_out* o) {
  /* v_rn = (v_ij . n) n ; v_rt = v_ij - v_rn */
  double vn = dot3(vij, nrm);
  double vrn[3], vrt[3];
  for (int d = 0; d < 3; d++) {
    vrn[d] = vn * nrm[d];
    vrt[d] = vij[d] - vrn[d];
  }
  /* Eq. delta_t: delta_t^new = delta_t^old + v_rt dt */
  if (incr)
    for (int d = 0; d < 3; d++) dt_t[d] = dt_t[d] + vrt[d] * dt;
  double kn, kt, eta_n, eta_t;
  if (lo->model == 0) {
    /* Eqs. nonlinearkn..nonlinearetat with S_n, S_t of Table equation_parameters */
    double sq = sqrt(Re * dn);
    kn = 4.0 / 3.0 * Ye * sq;
    double Sn = 2.0 * Ye * sq;
    kt = 8.0 * Ge * sq;
    double St = 8.0 * Ge * sq;
    eta_n = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(Sn * me);
    eta_t = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(St * me);
  } else {
    /* Eqs. linearkn, linearetan; the tangential constants are the same */
    double sR = sqrt(Re);
    double arg = 15.0 * me * lo->V * lo->V / (16.0 * sR * Ye);
    kn = 16.0 / 15.0 * sR * Ye * pow(arg, 0.2);
    eta_n = sqrt(4.0 * me * kn / lo->lin_den);
    kt = kn;
    eta_t = eta_n;
  }
  /* Eq. normal_force and Eq. tangential_force */
  for (int d = 0; d < 3; d++) {
    o->Fn[d] = -(kn * dn) * nrm[d] - eta_n * vrn[d];
    o->Ft[d] = -(kt * dt_t[d]) - eta_t * vrt[d];
  }
  double aFn = norm3(o->Fn);
  double aFt = norm3(o->Ft);
  /* Coulomb limit: if |F_t| >= mu |F_n|, F_t <- mu |F_n| F_t / |F_t| (Eq.
     coulomb_overlap3) and delta_t <- (F_t + eta_t v_rt) / (-k_t) (Eqs. elastic and
     coulomb_overlap) */
  if (aFt > 0.0 && aFt >= mu * aFn) {
    for (int d = 0; d < 3; d++) {
      o->Ft[d] = mu * aFn * o->Ft[d] / aFt;
      dt_t[d] = (o->Ft[d] + eta_t * vrt[d]) / (-kt);
    }
  }
  /* Eq. torque_t: M_t = R_i n x F_t (lever applied by the caller) */
  cross3(nrm, o->Ft, o->nxFt);
  /* Table rolling_torque: constant model M_r = -mu_r R_e |F_n| w_hat; viscous model
     M_r = -mu_r R_e |F_n| |V_omega| w_hat */
  o->Mr[0] = o->Mr[1] = o->Mr[2] = 0.0;
  double adw = norm3(dw);
  if (rolling == 1 && adw > 0.0)
    for (int d = 0; d < 3; d++) o->Mr[d] = -mu_r * Re * aFn * dw[d] / adw;
  if (rolling == 2 && adw > 0.0) {
    double avw = norm3(vomega);
    for (int d = 0; d < 3; d++) o->Mr[d] = -mu_r * Re * aFn * avw * dw[d] / adw;
  }
  o->absFn = aFn;
}

/* ------------------------------------------------------------ walls
 * Nearest point p* of wall k to the sphere centre x and the normal overlap.
 * Returns 0 if there is no contact (overlap <= 0), else fills nrm (unit vector from
 * the particle towards p*), dn and p*. */
static int wall_contact(const orc_wall* W, const double* x, double R, double* nrm, double* dn,
                        double* pstar) {
  if (W->kind == 0) { /* half-space: signed distance along the inward normal */
    double rel[3] = {x[0] - W->point[0], x[1] - W->point[1], x[2] - W->point[2]};
    double dist = dot3(rel, W->normal);
    double ov = R - dist;
    if (!(ov > 0.0)) return 0;
    for (int d = 0; d < 3; d++) {
      nrm[d] = -W->normal[d];
      pstar[d] = x[d] - dist * W->normal[d];
    }
    *dn = ov;
    return 1;
  }
  if (W->kind == 1) { /* inside of a cylinder: distance to the mantle */
    double rel[3] = {x[0] - W->point[0], x[1] - W->point[1], x[2] - W->point[2]};
    double ax = dot3(rel, W->normal);
    double rad[3] = {rel[0] - ax * W->normal[0], rel[1] - ax * W->normal[1], rel[2] - ax * W->normal[2]};
    double rho = norm3(rad);
    if (!(rho > 0.0)) return 0;
    double ov = R - (W->radius - rho);
    if (!(ov > 0.0)) return 0;
    for (int d = 0; d < 3; d++) {
      nrm[d] = rad[d] / rho;
      pstar[d] = W->point[d] + ax * W->normal[d] + W->radius * nrm[d];
    }
    *dn = ov;
    return 1;
  }
  if (W->kind == 2) { /* annulus: nearest point of a flat ring (face, or the rim of the hole) */
    double rel[3] = {x[0] - W->point[0], x[1] - W->point[1], x[2] - W->point[2]};
    double h = dot3(rel, W->normal);
    double q[3] = {rel[0] - h * W->normal[0], rel[1] - h * W->normal[1], rel[2] - h * W->normal[2]};
    double rho = norm3(q);
    double loc[3]; /* p* relative to the centre */
    if (rho < W->inner_radius || rho > W->radius) {
      double target = rho < W->inner_radius ? W->inner_radius : W->radius;
      double u[3];
      if (rho > 0.0) {
        for (int d = 0; d < 3; d++) u[d] = q[d] / rho;
      } else { /* centre on the axis: any rim point is nearest; take one fixed in-plane direction */
        double e[3] = {1.0, 0.0, 0.0};
        if (fabs(W->normal[0]) > 0.9) { e[0] = 0.0; e[1] = 1.0; }
        double c = dot3(e, W->normal);
        for (int d = 0; d < 3; d++) u[d] = e[d] - c * W->normal[d];
        double nu = norm3(u);
        for (int d = 0; d < 3; d++) u[d] /= nu;
      }
      for (int d = 0; d < 3; d++) loc[d] = target * u[d];
    } else {
      for (int d = 0; d < 3; d++) loc[d] = q[d];
    }
    double D[3];
    for (int d = 0; d < 3; d++) {
      pstar[d] = W->point[d] + loc[d];
      D[d] = pstar[d] - x[d];
    }
    double dist = norm3(D);
    double ov = R - dist;
    if (!(ov > 0.0) || !(dist > 0.0)) return 0;
    for (int d = 0; d < 3; d++) nrm[d] = D[d] / dist;
    *dn = ov;
    return 1;
  }
  return 0;
}

/* ------------------------------------------------------------ contact search
 * Broad search over a uniform cell grid (cell edge >= r_c, neighbour cells sharing a
 * vertex) followed by the fine search |x_j - x_i|^2 < r_c^2 (Sec. 3.2).  The squared
 * distance is formed as dx*dx + dy*dy + dz*dz, left to right, without contraction. */
static double sqdist(const double* a, const double* b) {
  double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  double s = dx * dx;
  s = s + dy * dy;
  s = s + dz * dz;
  return s;
}

typedef struct {
  int32_t i, j;
  int64_t src;
} ij_pair;
static int cmp_pair(const void* a, const void* b) {
  const ij_pair* p = (const ij_pair*)a;
  const ij_pair* q = (const ij_pair*)b;
  if (p->i != q->i) return p->i < q->i ? -1 : 1;
  if (p->j != q->j) return p->j < q->j ? -1 : 1;
  return 0;
}

static int64_t cell_search(const orc_sim* s, ij_pair** out) {
  const orc_config* c = &s->cfg;
  int64_t n = s->n;
  int nc[3];
  double h[3];
  for (int d = 0; d < 3; d++) {
    double L = c->domain_hi[d] - c->domain_lo[d];
    int k = (int)floor(L / s->rc);
    if (k < 1) k = 1;
    if (k > 1024) k = 1024;
    nc[d] = k;
    h[d] = L / k;
  }
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * ncell);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int* cidx = (int*)malloc(sizeof(int) * 3 * (n > 0 ? n : 1));
  for (int64_t k = 0; k < ncell; k++) head[k] = -1;
  /* insert in descending order so each cell's chain is in ascending id order */
  for (int64_t i = n - 1; i >= 0; i--) {
    if (!s->active[i]) continue;
    int ci[3];
    for (int d = 0; d < 3; d++) {
      double f = floor((s->x[3 * i + d] - c->domain_lo[d]) / h[d]);
      int k = f < 0 ? 0 : (f >= nc[d] ? nc[d] - 1 : (int)f);
      ci[d] = k;
      cidx[3 * i + d] = k;
    }
    int64_t cell = ((int64_t)ci[2] * nc[1] + ci[1]) * nc[0] + ci[0];
    next[i] = head[cell];
    head[cell] = i;
  }
  double rc2 = s->rc * s->rc;
  int64_t cap = 1024, np = 0;
  ij_pair* P = (ij_pair*)malloc(sizeof(ij_pair) * cap);
  for (int64_t i = 0; i < n; i++) {
    if (!s->active[i]) continue;
    for (int dz = -1; dz <= 1; dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          int a = cidx[3 * i] + dx, b = cidx[3 * i + 1] + dy, g = cidx[3 * i + 2] + dz;
          if (a < 0 || b < 0 || g < 0 || a >= nc[0] || b >= nc[1] || g >= nc[2]) continue;
          int64_t cell = ((int64_t)g * nc[1] + b) * nc[0] + a;
          for (int64_t j = head[cell]; j >= 0; j = next[j]) {
            if (j <= i) continue;
            if (sqdist(&s->x[3 * i], &s->x[3 * j]) < rc2) {
              if (np == cap) {
                cap *= 2;
                P = (ij_pair*)realloc(P, sizeof(ij_pair) * cap);
              }
              P[np].i = (int32_t)i;
              P[np].j = (int32_t)j;
              np++;
            }
          }
        }
  }
  free(head);
  free(next);
  free(cidx);
  qsort(P, (size_t)np, sizeof(ij_pair), cmp_pair);
  *out = P;
  return np;
}

/* New list; the tangential overlap of pairs present in both lists is carried over,
 * that of pairs no longer in the list is dropped. */
static void contact_search(orc_sim* s) {
  ij_pair* P;
  int64_t np = cell_search(s, &P);
  int32_t* pi = (int32_t*)malloc(sizeof(int32_t) * (np > 0 ? np : 1));
  int32_t* pj = (int32_t*)malloc(sizeof(int32_t) * (np > 0 ? np : 1));
  double* H = (double*)calloc((size_t)(np > 0 ? np : 1) * 3, sizeof(double));
  int64_t a = 0;
  for (int64_t k = 0; k < np; k++) {
    pi[k] = P[k].i;
    pj[k] = P[k].j;
    while (a < s->np && (s->pi[a] < P[k].i || (s->pi[a] == P[k].i && s->pj[a] < P[k].j))) a++;
    if (a < s->np && s->pi[a] == P[k].i && s->pj[a] == P[k].j)
      for (int d = 0; d < 3; d++) H[3 * k + d] = s->H[3 * a + d];
  }
  free(P);
  free(s->pi);
  free(s->pj);
  free(s->H);
  s->pi = pi;
  s->pj = pj;
  s->H = H;
  s->np = np;
  s->cap = np;
  memcpy(s->xref, s->x, sizeof(double) * 3 * s->n);
  s->have_list = 1;
  s->since_search = 0;
  s->searches++;
}

static int search_due(const orc_sim* s) {
  if (!s->have_list) return 1;
  if (s->cfg.rebuild_every > 0) return s->since_search >= s->cfg.rebuild_every;
  double half = 0.5 * s->cfg.skin;
  double lim = half * half;
  for (int64_t i = 0; i < s->n; i++)
    if (s->active[i] && sqdist(&s->xref[3 * i], &s->x[3 * i]) > lim) return 1;
  return 0;
}

/* ------------------------------------------------------------ forces */
static void evaluate_forces(orc_sim* s, int incr) {
  const orc_config* c = &s->cfg;
  int64_t n = s->n;
  memset(s->F, 0, sizeof(double) * 3 * n);
  memset(s->M, 0, sizeof(double) * 3 * n);
  memset(s->Fabs, 0, sizeof(double) * n);
  memset(s->Mabs, 0, sizeof(double) * n);
  double Ye = eff_young(&c->particle, &c->particle);
  double Ge = eff_shear(&c->particle, &c->particle);
  double beta = damping_beta(c->particle.restitution);
  law_opts lo_pp = {c->contact_model, c->linear_velocity, linear_damping_den(c->particle.restitution)};
  law_opts lo_pw = {c->contact_model, c->linear_velocity, linear_damping_den(c->wall.restitution)};
  double t = (double)s->step * c->dt;
  int64_t touch = 0, wtouch = 0;
  /* particle-particle contacts, list order */
  for (int64_t k = 0; k < s->np; k++) {
    int64_t i = s->pi[k], j = s->pj[k];
    double* H = &s->H[3 * k];
    if (!s->active[i] || !s->active[j]) {
      H[0] = H[1] = H[2] = 0.0;
      continue;
    }
    const double* xi = &s->x[3 * i];
    const double* xj = &s->x[3 * j];
    double dx[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
    double r = sqrt(sqdist(xi, xj));
    double dn = (s->R[i] + s->R[j]) - r; /* Eq. deltan */
    if (!(dn > 0.0)) {
      H[0] = H[1] = H[2] = 0.0; /* a new contact starts with zero tangential overlap */
      continue;
    }
    touch++;
    double nrm[3] = {dx[0] / r, dx[1] / r, dx[2] / r}; /* Eq. vecn */
    double rw[3], rwxn[3], vij[3], dw[3];
    for (int d = 0; d < 3; d++) rw[d] = s->R[i] * s->w[3 * i + d] + s->R[j] * s->w[3 * j + d];
    cross3(rw, nrm, rwxn);
    for (int d = 0; d < 3; d++) {
      vij[d] = (s->v[3 * i + d] - s->v[3 * j + d]) + rwxn[d];
      dw[d] = s->w[3 * i + d] - s->w[3 * j + d];
    }
    double Re = 1.0 / (1.0 / s->R[i] + 1.0 / s->R[j]);
    double me = 1.0 / (1.0 / s->m[i] + 1.0 / s->m[j]);
    contact_out o;
    /* V_omega of the viscous rolling model: (R_i w_i + R_j w_j) x n */
    contact_law(nrm, dn, vij, dw, rwxn, Re, me, Ye, Ge, beta, c->particle.mu_slide, c->particle.mu_roll,
                c->rolling_model, &lo_pp, c->dt, H, incr, &o);
    for (int d = 0; d < 3; d++) {
      double f = o.Fn[d] + o.Ft[d];
      s->F[3 * i + d] += f;
      s->F[3 * j + d] -= f;
      s->M[3 * i + d] += s->R[i] * o.nxFt[d] + o.Mr[d];
      s->M[3 * j + d] += s->R[j] * o.nxFt[d] - o.Mr[d];
    }
    {
      double f[3] = {o.Fn[0] + o.Ft[0], o.Fn[1] + o.Ft[1], o.Fn[2] + o.Ft[2]};
      double af = norm3(f), at = norm3(o.nxFt), ar = norm3(o.Mr);
      s->Fabs[i] += af;
      s->Fabs[j] += af;
      s->Mabs[i] += s->R[i] * at + ar;
      s->Mabs[j] += s->R[j] * at + ar;
    }
  }
  /* particle-wall contacts */
  double Yw = eff_young(&c->particle, &c->wall);
  double Gw = eff_shear(&c->particle, &c->wall);
  double bw = damping_beta(c->wall.restitution);
  for (int64_t i = 0; i < n; i++) {
    for (int k = 0; k < s->nwalls; k++) {
      double* H = &s->Hw[(i * ORC_MAX_WALLS + k) * 3];
      /* a translating wall is where its motion has carried it by time t */
      orc_wall Wt = s->walls[k];
      if (Wt.translates)
        for (int d = 0; d < 3; d++) {
          Wt.point[d] = Wt.point[d] + Wt.velocity[d] * t;
          Wt.rot_origin[d] = Wt.rot_origin[d] + Wt.velocity[d] * t;
        }
      const orc_wall* W = &Wt;
      int on = s->active[i] && t >= W->t_on && t < W->t_off;
      double nrm[3], dn, ps[3];
      if (!on || !wall_contact(W, &s->x[3 * i], s->R[i], nrm, &dn, ps)) {
        H[0] = H[1] = H[2] = 0.0;
        continue;
      }
      wtouch++;
      /* wall surface velocity at p*: Omega x (p* - c) + V; wall spin Omega */
      const double* Om = s->wall_Omega[k];
      double arm[3] = {ps[0] - W->rot_origin[0], ps[1] - W->rot_origin[1], ps[2] - W->rot_origin[2]};
      double Vw[3], rw[3], rwxn[3], vij[3], dw[3];
      cross3(Om, arm, Vw);
      for (int d = 0; d < 3; d++) {
        Vw[d] += W->velocity[d];
        rw[d] = s->R[i] * s->w[3 * i + d];
      }
      cross3(rw, nrm, rwxn);
      double rdw[3], vom[3];
      for (int d = 0; d < 3; d++) {
        vij[d] = (s->v[3 * i + d] - Vw[d]) + rwxn[d];
        dw[d] = s->w[3 * i + d] - Om[d];
        rdw[d] = s->R[i] * dw[d];
      }
      cross3(rdw, nrm, vom); /* V_omega against the wall: R_i (w_i - Omega) x n */
      contact_out o;
      contact_law(nrm, dn, vij, dw, vom, s->R[i], s->m[i], Yw, Gw, bw, c->wall.mu_slide, c->wall.mu_roll,
                  c->rolling_model, &lo_pw, c->dt, H, incr, &o);
      for (int d = 0; d < 3; d++) {
        s->F[3 * i + d] += o.Fn[d] + o.Ft[d];
        s->M[3 * i + d] += s->R[i] * o.nxFt[d] + o.Mr[d];
      }
      {
        double f[3] = {o.Fn[0] + o.Ft[0], o.Fn[1] + o.Ft[1], o.Fn[2] + o.Ft[2]};
        s->Fabs[i] += norm3(f);
        s->Mabs[i] += s->R[i] * norm3(o.nxFt) + norm3(o.Mr);
      }
    }
  }
  s->n_touch = touch;
  s->n_wall_touch = wtouch;
  s->forces_valid = 1;
}

/* Before the first step (or after a state change): search, then forces at the
 * current state with the stored tangential overlaps. */
static void ensure_forces(orc_sim* s) {
  if (s->forces_valid) return;
  contact_search(s);
  evaluate_forces(s, 0);
}

/* ------------------------------------------------------------ time step */
static void half_kick(orc_sim* s) {
  const orc_config* c = &s->cfg;
  double h = 0.5 * c->dt;
  for (int64_t i = 0; i < s->n; i++) {
    if (!s->active[i]) continue;
    for (int d = 0; d < 3; d++) {
      double a = s->F[3 * i + d] / s->m[i] + c->gravity[d]; /* Eq. main1 */
      double al = s->M[3 * i + d] / s->I[i];                /* Eq. main2 */
      s->v[3 * i + d] = s->v[3 * i + d] + a * h;
      s->w[3 * i + d] = s->w[3 * i + d] + al * h;
    }
  }
}

/* Explicit Euler (Eq. integ_EE): v^{n+1} = v^n + a^n dt and x^{n+1} = x^n + v^n dt
   (likewise for w) with the forces evaluated at (x^n, v^n) at the end of the previous
   step, then the contact search when due and the forces at (x^{n+1}, v^{n+1}). */
static void one_step_euler(orc_sim* s) {
  const orc_config* c = &s->cfg;
  for (int64_t i = 0; i < s->n; i++) {
    if (!s->active[i]) continue;
    for (int d = 0; d < 3; d++) {
      double a = s->F[3 * i + d] / s->m[i] + c->gravity[d]; /* Eq. main1 */
      double al = s->M[3 * i + d] / s->I[i];                /* Eq. main2 */
      s->x[3 * i + d] = s->x[3 * i + d] + s->v[3 * i + d] * c->dt;
      s->v[3 * i + d] = s->v[3 * i + d] + a * c->dt;
      s->w[3 * i + d] = s->w[3 * i + d] + al * c->dt;
    }
    if (s->x[3 * i + 2] < c->z_sink) s->active[i] = 0;
  }
  s->step++;
  s->since_search++;
  if (search_due(s)) contact_search(s);
  evaluate_forces(s, 1);
}

static void one_step(orc_sim* s) {
  const orc_config* c = &s->cfg;
  if (c->integrator == 1) {
    one_step_euler(s);
    return;
  }
  /* 1. v^{n+1/2} = v^n + a^n dt/2 ; x^{n+1} = x^n + v^{n+1/2} dt (Eq. halfstep) */
  half_kick(s);
  for (int64_t i = 0; i < s->n; i++) {
    if (!s->active[i]) continue;
    for (int d = 0; d < 3; d++) s->x[3 * i + d] = s->x[3 * i + d] + s->v[3 * i + d] * c->dt;
    if (s->x[3 * i + 2] < c->z_sink) s->active[i] = 0;
  }
  s->step++;
  s->since_search++;
  /* 2. contact search when due */
  if (search_due(s)) contact_search(s);
  /* 3. forces at x^{n+1} with the half-step velocities */
  evaluate_forces(s, 1);
  /* 4. v^{n+1} = v^{n+1/2} + a^{n+1} dt/2 (Eq. newvv) */
  half_kick(s);
}

/* ------------------------------------------------------------ public API */
orc_sim* orc_create(const orc_config* cfg, const double* x, const double* v, const double* w,
                    const float* radius) {
  if (!cfg || cfg->n < 0 || !(cfg->dt > 0.0) || !(cfg->density > 0.0)) return NULL;
  if (!(cfg->particle.restitution > 0.0 && cfg->particle.restitution <= 1.0)) return NULL;
  if (!(cfg->wall.restitution > 0.0 && cfg->wall.restitution <= 1.0)) return NULL;
  if (cfg->rolling_model < 0 || cfg->rolling_model > 2 || cfg->integrator < 0 || cfg->integrator > 1) return NULL;
  if (cfg->contact_model < 0 || cfg->contact_model > 1) return NULL;
  if (cfg->contact_model == 1 && !(cfg->linear_velocity > 0.0)) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->cfg = *cfg;
  int64_t n = cfg->n, n1 = n > 0 ? n : 1;
  s->n = n;
  s->x = (double*)malloc(sizeof(double) * 3 * n1);
  s->v = (double*)malloc(sizeof(double) * 3 * n1);
  s->w = (double*)malloc(sizeof(double) * 3 * n1);
  s->F = (double*)calloc((size_t)(3 * n1), sizeof(double));
  s->M = (double*)calloc((size_t)(3 * n1), sizeof(double));
  s->Fabs = (double*)calloc((size_t)n1, sizeof(double));
  s->Mabs = (double*)calloc((size_t)n1, sizeof(double));
  s->xref = (double*)malloc(sizeof(double) * 3 * n1);
  s->R = (double*)malloc(sizeof(double) * n1);
  s->m = (double*)malloc(sizeof(double) * n1);
  s->I = (double*)malloc(sizeof(double) * n1);
  s->active = (uint8_t*)malloc(n1);
  s->Hw = (double*)calloc((size_t)(n1 * ORC_MAX_WALLS * 3), sizeof(double));
  memcpy(s->x, x, sizeof(double) * 3 * n);
  memcpy(s->v, v, sizeof(double) * 3 * n);
  memcpy(s->w, w, sizeof(double) * 3 * n);
  double dmax = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double R = (double)radius[i];
    s->R[i] = R;
    s->m[i] = cfg->density * (4.0 / 3.0) * ORC_PI * R * R * R;
    s->I[i] = 0.4 * s->m[i] * R * R; /* solid sphere */
    s->active[i] = 1;
    if (2.0 * R > dmax) dmax = 2.0 * R;
  }
  s->dmax = dmax;
  /* threshold: r_c = factor * d_max, or d_max + skin when a skin is given */
  if (cfg->skin > 0.0) {
    s->rc = dmax + cfg->skin;
  } else {
    s->rc = cfg->neighbor_factor * dmax;
    s->cfg.skin = s->rc - dmax;
  }
  if (!(s->rc > 0.0)) s->rc = 1e-300;
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->x); free(s->v); free(s->w); free(s->F); free(s->M); free(s->xref);
  free(s->Fabs); free(s->Mabs);
  free(s->R); free(s->m); free(s->I); free(s->active); free(s->Hw);
  free(s->pi); free(s->pj); free(s->H);
  free(s);
}

int orc_set_walls(orc_sim* s, const orc_wall* walls, int32_t n_walls) {
  if (!s || n_walls < 0 || n_walls > ORC_MAX_WALLS) return 1;
  for (int k = 0; k < n_walls; k++) {
    orc_wall W = walls[k];
    double nn = norm3(W.normal);
    if (!(nn > 0.0)) return 1;
    for (int d = 0; d < 3; d++) W.normal[d] /= nn;
    double na = norm3(W.rot_axis);
    for (int d = 0; d < 3; d++) s->wall_Omega[k][d] = na > 0.0 ? W.omega * W.rot_axis[d] / na : 0.0;
    s->walls[k] = W;
  }
  s->nwalls = n_walls;
  memset(s->Hw, 0, sizeof(double) * 3 * ORC_MAX_WALLS * (s->n > 0 ? s->n : 1));
  s->forces_valid = 0;
  return 0;
}

int orc_step(orc_sim* s, int64_t n_steps) {
  if (!s || n_steps < 0) return 1;
  ensure_forces(s);
  for (int64_t k = 0; k < n_steps; k++) one_step(s);
  return 0;
}

int orc_get_state(const orc_sim* s, double* x, double* v, double* w, uint8_t* active) {
  if (!s) return 1;
  if (x) memcpy(x, s->x, sizeof(double) * 3 * s->n);
  if (v) memcpy(v, s->v, sizeof(double) * 3 * s->n);
  if (w) memcpy(w, s->w, sizeof(double) * 3 * s->n);
  if (active) memcpy(active, s->active, (size_t)s->n);
  return 0;
}

int orc_set_state(orc_sim* s, const double* x, const double* v, const double* w,
                  const uint8_t* active) {
  if (!s) return 1;
  if (x) memcpy(s->x, x, sizeof(double) * 3 * s->n);
  if (v) memcpy(s->v, v, sizeof(double) * 3 * s->n);
  if (w) memcpy(s->w, w, sizeof(double) * 3 * s->n);
  if (active) memcpy(s->active, active, (size_t)s->n);
  s->forces_valid = 0;
  return 0;
}

int orc_get_forces(orc_sim* s, double* F, double* M) {
  if (!s) return 1;
  ensure_forces(s);
  if (F) memcpy(F, s->F, sizeof(double) * 3 * s->n);
  if (M) memcpy(M, s->M, sizeof(double) * 3 * s->n);
  return 0;
}

int orc_get_force_scales(orc_sim* s, double* Fabs, double* Mabs) {
  if (!s) return 1;
  ensure_forces(s);
  if (Fabs) memcpy(Fabs, s->Fabs, sizeof(double) * s->n);
  if (Mabs) memcpy(Mabs, s->Mabs, sizeof(double) * s->n);
  return 0;
}

int64_t orc_get_pairs(orc_sim* s, int32_t* pairs, int64_t cap) {
  if (!s) return -1;
  ensure_forces(s);
  for (int64_t k = 0; k < s->np && k < cap; k++) {
    pairs[2 * k] = s->pi[k];
    pairs[2 * k + 1] = s->pj[k];
  }
  return s->np;
}

int64_t orc_get_history(orc_sim* s, int32_t* pairs, double* dt_pair, int64_t cap, double* dt_wall) {
  if (!s) return -1;
  ensure_forces(s);
  int64_t c = 0;
  for (int64_t k = 0; k < s->np; k++) {
    const double* H = &s->H[3 * k];
    if (H[0] == 0.0 && H[1] == 0.0 && H[2] == 0.0) continue;
    if (c < cap) {
      pairs[2 * c] = s->pi[k];
      pairs[2 * c + 1] = s->pj[k];
      for (int d = 0; d < 3; d++) dt_pair[3 * c + d] = H[d];
    }
    c++;
  }
  if (dt_wall)
    for (int64_t i = 0; i < s->n; i++)
      for (int k = 0; k < s->nwalls; k++)
        for (int d = 0; d < 3; d++)
          dt_wall[(i * s->nwalls + k) * 3 + d] = s->Hw[(i * ORC_MAX_WALLS + k) * 3 + d];
  return c;
}

int orc_set_history(orc_sim* s, int64_t n_pairs, const int32_t* pairs, const double* dt_pair,
                    const double* dt_wall) {
  if (!s || n_pairs < 0) return 1;
  /* The given pairs become the previous list; the next search carries them over. */
  ij_pair* P = (ij_pair*)malloc(sizeof(ij_pair) * (n_pairs > 0 ? n_pairs : 1));
  for (int64_t k = 0; k < n_pairs; k++) {
    int32_t a = pairs[2 * k], b = pairs[2 * k + 1];
    if (a < 0 || b < 0 || a >= s->n || b >= s->n || a == b) {
      free(P);
      return 1;
    }
    P[k].i = a < b ? a : b;
    P[k].j = a < b ? b : a;
  }
  free(s->pi); free(s->pj); free(s->H);
  s->pi = (int32_t*)malloc(sizeof(int32_t) * (n_pairs > 0 ? n_pairs : 1));
  s->pj = (int32_t*)malloc(sizeof(int32_t) * (n_pairs > 0 ? n_pairs : 1));
  s->H = (double*)calloc((size_t)(n_pairs > 0 ? n_pairs : 1) * 3, sizeof(double));
  /* sort by (i, j) keeping the value of each pair; the sign flips when given as (j, i) */
  for (int64_t k = 0; k < n_pairs; k++) {
    P[k].src = k;
  }
  qsort(P, (size_t)n_pairs, sizeof(ij_pair), cmp_pair);
  for (int64_t k = 0; k < n_pairs; k++) {
    int64_t src = P[k].src;
    s->pi[k] = P[k].i;
    s->pj[k] = P[k].j;
    double sg = pairs[2 * src] < pairs[2 * src + 1] ? 1.0 : -1.0;
    for (int d = 0; d < 3; d++) s->H[3 * k + d] = sg * dt_pair[3 * src + d];
  }
  s->np = n_pairs;
  free(P);
  if (dt_wall)
    for (int64_t i = 0; i < s->n; i++)
      for (int k = 0; k < s->nwalls; k++)
        for (int d = 0; d < 3; d++)
          s->Hw[(i * ORC_MAX_WALLS + k) * 3 + d] = dt_wall[(i * s->nwalls + k) * 3 + d];
  s->have_list = 0;
  s->forces_valid = 0;
  return 0;
}

int orc_get_stats(const orc_sim* s, orc_stats* out) {
  if (!s || !out) return 1;
  out->steps = s->step;
  out->rebuilds = s->searches;
  out->n_pairs = s->np;
  out->n_touch = s->n_touch;
  out->n_wall_touch = s->n_wall_touch;
  int64_t a = 0;
  for (int64_t i = 0; i < s->n; i++) a += s->active[i];
  out->n_active = a;
  out->time = (double)s->step * s->cfg.dt;
  return 0;
}

int64_t orc_brute_pairs(int64_t n, const double* x, const uint8_t* active, double rc,
                        int32_t* pairs, int64_t cap) {
  double rc2 = rc * rc;
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    if (active && !active[i]) continue;
    for (int64_t j = i + 1; j < n; j++) {
      if (active && !active[j]) continue;
      if (sqdist(&x[3 * i], &x[3 * j]) < rc2) {
        if (c < cap) {
          pairs[2 * c] = (int32_t)i;
          pairs[2 * c + 1] = (int32_t)j;
        }
        c++;
      }
    }
  }
  return c;
}

