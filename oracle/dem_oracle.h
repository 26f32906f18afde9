/*
 * dem_oracle.h -- interface of the CPU oracle for the soft-sphere DEM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This header belongs to the plain, slow FP64 CPU
 * restatement of the method of Golshan et al., "Lethe-DEM: an open-source parallel
 * discrete element solver with load balancing" (arXiv 2106.09576).  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Units are SI.  Arrays of vectors are row-major [n][3] FP64; particle order is the
 * caller's (the "id" of a particle is its row).  Radii are FP32 inputs, widened to
 * FP64 exactly.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Material of one body type (particle or wall): Young's modulus Y, Poisson ratio nu,
 * coefficient of restitution e, sliding friction mu, rolling friction mu_r
 * (Sec. 2.1, Table "equation_parameters" and Table "rolling_torque"). */
typedef struct {
  double young, poisson, restitution, mu_slide, mu_roll;
} orc_material;

typedef struct {
  int64_t n;                 /* number of particles */
  double density;            /* particle density, kg/m^3 */
  orc_material particle, wall;
  double gravity[3];         /* m/s^2 */
  double dt;                 /* time step, s */
  double neighbor_factor;    /* fine-search threshold r_c = factor * d_max (Sec. 3.2; 1.3 typical) */
  double skin;               /* dynamic search: rebuild when a displacement exceeds skin/2 (Sec. 3.1) */
  int32_t rebuild_every;     /* > 0: constant search mode, rebuild every n steps (Sec. 3.1) */
  int32_t rolling_model;     /* 0: none, 1: constant, 2: viscous rolling resistance (Table
                                "rolling_torque") */
  int32_t contact_model;     /* 0: non-linear (Eqs. nonlinearkn..nonlinearetat), 1: linear
                                (Eqs. linearkn, linearetan, same constants tangentially) */
  int32_t integrator;        /* 0: velocity Verlet (Sec. 2.2), 1: explicit Euler (Eq. integ_EE) */
  double linear_velocity;    /* characteristic impact velocity V of Eq. linearkn, m/s */
  double domain_lo[3], domain_hi[3]; /* extent of the search grid (outside points are clamped) */
  double z_sink;             /* particles whose centre falls below z_sink are removed */
} orc_config;

/* Analytic wall.  kind 0: half-space {(x-point).normal >= 0}; 1: inside of an infinite
 * cylinder (point on axis, normal = axis, radius); 2: annulus = flat plate with a
 * circular hole (point = centre, normal, radius = outer, inner_radius = hole).
 * A wall moves with surface velocity Omega x (p - rot_origin) + velocity, Omega =
 * omega * unit(rot_axis) (Sec. 3.6, boundary motion); with `translates` set its geometry
 * moves too: point and rot_origin at time t are point + velocity t and rot_origin +
 * velocity t (translational boundary motion).  It exists for t_on <= t < t_off
 * (floating wall, Sec. 3.6). */
typedef struct {
  int32_t kind;
  int32_t translates;
  double point[3], normal[3];
  double radius, inner_radius;
  double omega, rot_origin[3], rot_axis[3], velocity[3];
  double t_on, t_off;
} orc_wall;

typedef struct {
  int64_t steps, rebuilds, n_pairs, n_touch, n_wall_touch, n_active;
  double time;
} orc_stats;

typedef struct orc_sim orc_sim;

/* Copies the initial state in.  Returns NULL on invalid arguments. */
orc_sim* orc_create(const orc_config* cfg, const double* x, const double* v, const double* w,
                    const float* radius);
void orc_destroy(orc_sim* s);
int orc_set_walls(orc_sim* s, const orc_wall* walls, int32_t n_walls);   /* <= 8 walls */
int orc_step(orc_sim* s, int64_t n_steps);
/* State at the current step (v, w are the full-step velocities v^n, w^n). */
int orc_get_state(const orc_sim* s, double* x, double* v, double* w, uint8_t* active);
int orc_set_state(orc_sim* s, const double* x, const double* v, const double* w,
                  const uint8_t* active);
/* Contact force and torque sums (gravity excluded) of the last force evaluation. */
int orc_get_forces(orc_sim* s, double* F, double* M);
/* Per particle: sum over its contacts of |F_n + F_t| and of |R n x F_t| + |M_r| in the
 * last force evaluation (scales for relative error measures). */
int orc_get_force_scales(orc_sim* s, double* Fabs, double* Mabs);
/* Current fine-search list as (i, j) pairs with i < j, lexicographic order. */
int64_t orc_get_pairs(orc_sim* s, int32_t* pairs, int64_t cap);
/* Pairs with non-zero tangential overlap (i < j, delta_t of the (i,j) orientation),
 * and the particle-wall overlaps [n][n_walls][3]. */
int64_t orc_get_history(orc_sim* s, int32_t* pairs, double* dt_pair, int64_t cap, double* dt_wall);
int orc_set_history(orc_sim* s, int64_t n_pairs, const int32_t* pairs, const double* dt_pair,
                    const double* dt_wall);
int orc_get_stats(const orc_sim* s, orc_stats* out);
/* O(n^2) reference contact search: all i < j with |x_j - x_i|^2 < rc^2. */
int64_t orc_brute_pairs(int64_t n, const double* x, const uint8_t* active, double rc,
                        int32_t* pairs, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
