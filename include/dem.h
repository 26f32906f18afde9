/*
 * dem.h -- C ABI of the GB300 soft-sphere DEM hot path (libdem_gb300.so).
 *
 * The library advances a system of spheres by explicit time steps of the method of
 * Golshan et al., "Lethe-DEM: an open-source parallel discrete element solver with
 * load balancing" (arXiv 2106.09576):
 *   - contact search: particles sorted by cell key at each rebuild, broad search over
 *     the cells sharing a vertex, fine search |x_j - x_i| < r_c (Sec. 3.2); rebuild
 *     every n steps ("constant") or when a displacement exceeds skin/2 ("dynamic",
 *     Sec. 3.1);
 *   - nonlinear viscoelastic (Hertz-Mindlin) particle-particle and particle-wall forces
 *     with tangential-overlap history, Coulomb limit and constant rolling resistance
 *     (Sec. 2.1: Eqs. deltan..coulomb_overlap3, Tables equation_parameters and
 *     rolling_torque);
 *   - velocity Verlet integration (Sec. 2.2, Eqs. halfstep and newvv) of Eqs. main1
 *     and main2.
 *
 * Conventions for every call:
 *   - Units are SI.  Vectors of particles are row-major [n][3] FP64 in the caller's
 *     order; radii are FP32 [n]; "active" flags are uint8 [n].
 *   - Array arguments may be host or device pointers (unified addressing decides);
 *     they are read or written on the context's stream and the call returns only when
 *     host memory is no longer touched.  Device arrays must not be freed before the
 *     call returns.
 *   - The library never allocates device memory.  All device storage lives in the
 *     caller's workspace (size from dem_workspace_bytes), which must stay valid until
 *     dem_destroy.  CUDA graphs created by the library are released by dem_destroy.
 *   - Errors are returned as dem_status and never thrown.  Errors found on the device
 *     (capacity, non-finite state, excessive overlap) are sticky: they are reported by
 *     the next call that synchronises (dem_get_state, dem_get_stats, dem_sync, and
 *     dem_step when it finds the flag already set) and clear only through dem_set_state.
 *     A capacity error is reported before the others: once a list or table has been
 *     truncated the state that follows is not defined (it may turn non-finite).
 *   - A context is used by one host thread at a time.
 */
#ifndef DEM_GB300_H
#define DEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dem_status;
#define DEM_OK 0
#define DEM_ERR_ARG 1        /* invalid argument or configuration */
#define DEM_ERR_CUDA 2       /* a CUDA runtime call failed */
#define DEM_ERR_CAPACITY 3   /* workspace, neighbour slots, contacts or hash table too small */
#define DEM_ERR_NONFINITE 4  /* a position or velocity became NaN or infinite */
#define DEM_ERR_OVERLAP 5    /* a normal overlap exceeded max_overlap_ratio * radius */
#define DEM_ERR_TIMEOUT 6    /* a bounded device wait gave up */
#define DEM_ERR_STATE 7      /* call out of order, or the context holds a sticky error */

#define DEM_PRECISION_FP64 0   /* every operation in FP64 */
#define DEM_PRECISION_MIXED 1  /* contact-force arithmetic in FP32; positions, velocities,
                                  integration and tangential-overlap accumulation in FP64 */

#define DEM_PAIR_EVAL_ONCE 0   /* dem_config.pair_eval */
#define DEM_PAIR_EVAL_BOTH 1

#define DEM_MAX_WALLS 8
#define DEM_MAX_NEIGHBORS 56   /* fine-search entries kept per particle */
#define DEM_MAX_CONTACTS 32    /* simultaneous contacts (particles + walls) per particle */

/* One material: Young's modulus Y, Poisson ratio nu, restitution e, sliding friction mu,
 * rolling friction mu_r (Table equation_parameters; Table rolling_torque). */
typedef struct {
  double young, poisson, restitution, mu_slide, mu_roll;
} dem_material;

typedef struct {
  int64_t n;                 /* particles, 0 < n < 2^31 */
  double density;            /* kg/m^3; m = density * 4/3 pi R^3, I = 2/5 m R^2 */
  double radius_max;         /* largest particle radius; d_max = 2 radius_max sets the search
                                threshold and the cell grid (dem_create checks every radius
                                is <= radius_max) */
  dem_material particle;     /* particle-particle contacts use this material */
  dem_material wall;         /* particle-wall contacts: Y_e, G_e mix both; e, mu, mu_r of the wall */
  double gravity[3];         /* m/s^2 */
  double dt;                 /* s */
  double neighbor_factor;    /* fine-search threshold r_c = factor * d_max when skin <= 0
                                (Sec. 3.2 uses 1.3); then skin = r_c - d_max */
  double skin;               /* > 0: r_c = d_max + skin */
  int32_t rebuild_every;     /* > 0: constant search every n steps; 0: dynamic, rebuild when
                                some |x - x_ref| > skin/2 (Sec. 3.1) */
  int32_t precision;         /* DEM_PRECISION_FP64 or DEM_PRECISION_MIXED */
  int32_t rolling_model;     /* 0 none, 1 constant, 2 viscous torque model (Table rolling_torque) */
  int32_t n_instances;       /* 0 or 1: one system.  > 1: a batch of independent systems in
                                one context (dem_set_instances); no counterpart in the paper */
  double domain_lo[3];       /* box of the cell grid; particles outside are clamped to */
  double domain_hi[3];       /* the border cells (correct, but slower if many) */
  double z_sink;             /* a particle whose centre drops below z_sink leaves the system */
  double max_overlap_ratio;  /* > 0: DEM_ERR_OVERLAP when delta_n > ratio * R_min; 0 = off */
  int32_t step_block;        /* threads per block of the step kernel: 32, 64 or 128; 0 = chosen
                                from n and the SM count (a launch parameter, not physics) */
  int32_t contact_model;     /* 0 non-linear (Eqs. nonlinearkn..nonlinearetat), 1 linear
                                (Eqs. linearkn, linearetan; same constants tangentially) */
  int32_t integrator;        /* 0 velocity Verlet (Eqs. halfstep, newvv), 1 explicit Euler
                                (Eq. integ_EE) */
  int32_t pair_eval;         /* mixed precision: DEM_PAIR_EVAL_ONCE (0, default) evaluates each
                                touching pair once, by its partner of smaller id, and hands the
                                reaction to the other (Sec. 2.1: the pair force and its
                                reaction, Eq. torque_t); DEM_PAIR_EVAL_BOTH evaluates it from
                                both sides.  Same pairs and law, sums in another order: a
                                launch choice, not physics.  FP64 contexts always use BOTH */
  double linear_velocity;    /* characteristic impact velocity V of Eq. linearkn (m/s, > 0 for
                                the linear model) */
} dem_config;

/* Analytic wall (the paper meshes the boundary; see Sec. 2.1 last paragraph and
 * Sec. 3.6 for moving and floating walls).
 *   kind 0, plane:    half-space {(x - point) . normal >= 0}; contact on the side the
 *                     normal points to, signed distance (a centre behind the plane is
 *                     still pushed out).
 *   kind 1, cylinder: particles inside an infinite circular cylinder of `radius` whose
 *                     axis passes through `point` along `normal`.
 *   kind 2, annulus:  flat plate through `point` with unit `normal`, the ring
 *                     inner_radius <= rho <= radius around `point` (a silo bottom with an
 *                     orifice); nearest-point contact, including the rim of the hole.
 * Motion: the surface moves with velocity Omega x (p - rot_origin) + velocity at the
 * contact point p, Omega = omega * rot_axis / |rot_axis|.  With translates = 0 the
 * geometry itself does not move (rotation about the wall's own symmetry axis, or sliding
 * within its plane); with translates = 1 the wall is carried by `velocity`: at time t its
 * point and rot_origin are point + velocity t and rot_origin + velocity t (translational
 * boundary motion, Sec. 3.6).
 * Existence: the wall acts for t_on <= t < t_off (floating wall). */
typedef struct {
  int32_t kind;
  int32_t translates;
  double point[3], normal[3];
  double radius, inner_radius;
  double omega, rot_origin[3], rot_axis[3], velocity[3];
  double t_on, t_off;
} dem_wall;

#define DEM_MAX_INSTANCE_WALLS 4

/* One member of a batch (dem_config.n_instances > 1).  The paper simulates one system at
 * a time; a batch runs many independent systems -- each with its own particles, materials
 * and walls -- through the same kernels, one step of all of them per launch.  Instance k
 * owns the particles first[k] <= i < first[k+1] (caller order; first[n_instances] = n).
 * Particles of different instances never interact, even where their regions overlap;
 * placing instances in disjoint regions of the domain keeps the cells sparse.  The
 * top-level dem_config materials and dem_set_walls are not used by a batch. */
typedef struct {
  int64_t first;              /* first particle of the instance, caller order, increasing */
  dem_material particle;      /* particle-particle contacts */
  dem_material wall;          /* particle-wall contacts (mixing as for a single system) */
  int32_t n_walls;            /* <= DEM_MAX_INSTANCE_WALLS */
  int32_t reserved0;
  dem_wall walls[DEM_MAX_INSTANCE_WALLS];
} dem_instance;

typedef struct {
  int64_t steps;              /* time steps taken since the state was set */
  int64_t rebuilds;           /* contact searches (including the first) */
  int64_t n_pairs;            /* entries of the last fine-search list (each pair once) */
  int64_t n_touch;            /* particle-particle contacts (each pair once) at the last step */
  int64_t n_wall_touch;       /* particle-wall contacts at the last step */
  int64_t n_active;           /* particles still in the system */
  double time;                /* simulated time, s */
  double max_overlap_ratio;   /* max delta_n / R over contacts of the last step */
  uint32_t status_bits;       /* sticky device flags: 1 capacity, 2 non-finite, 4 overlap, 8 timeout */
  int32_t max_neighbors_seen; /* largest fine-search list of one particle at the last rebuild */
  size_t required_workspace;  /* bytes dem_workspace_bytes reports for this configuration */
  int64_t inner_builds;       /* mixed contexts: refreshes of the inner list, the pairs of the
                                 fine-search list within R_i + R_j + delta (delta = min(0.1 d_max,
                                 skin / 4)) that the force kernel walks; refreshed when a particle
                                 has moved delta / 2, and at each contact search */
} dem_stats;

typedef struct dem_ctx dem_ctx;

/* Bytes of device workspace that dem_create needs for `cfg` (>= 256-byte aligned start). */
dem_status dem_workspace_bytes(const dem_config* cfg, size_t* bytes);

/* Creates a context: validates cfg, lays out the workspace, copies the initial state
 * (x, v, w [n][3] FP64; radius [n] FP32 > 0) in.  `stream` is a cudaStream_t (NULL =
 * legacy default stream) on which every later call runs.  Forces are first evaluated
 * (without advancing the tangential overlap) at the start of the first dem_step. */
dem_status dem_create(const dem_config* cfg, const double* x, const double* v, const double* w,
                      const float* radius, void* workspace, size_t workspace_bytes, void* stream,
                      dem_ctx** out);

/* Replaces the walls (host array, copied; n_walls <= DEM_MAX_WALLS) and clears the
 * particle-wall tangential overlaps.  Forces are re-evaluated before the next step. */
dem_status dem_set_walls(dem_ctx* ctx, const dem_wall* walls, int32_t n_walls);

/* Batch contexts only (cfg.n_instances > 1): gives each instance its particle range,
 * materials and walls (host array of cfg.n_instances entries, copied).  Must be called
 * before the first dem_step; calling it again replaces the tables, clears the particle-
 * wall tangential overlaps and re-evaluates forces before the next step.  DEM_ERR_ARG if
 * the ranges are not increasing from 0, a wall count exceeds DEM_MAX_INSTANCE_WALLS or a
 * material is invalid; DEM_ERR_STATE on a context that is not a batch.  No counterpart
 * in the paper (it runs one system per process group). */
dem_status dem_set_instances(dem_ctx* ctx, const dem_instance* instances, int32_t n_instances);

/* Advances n_steps >= 0 time steps, asynchronously on the context's stream.  Returns
 * DEM_ERR_STATE if a sticky device error is already known on the host. */
dem_status dem_step(dem_ctx* ctx, int64_t n_steps);

/* Measurement entry point: advances n_steps >= 0 time steps with the same kernels as
 * dem_step, but launched one by one on the context's stream, with CUDA events around
 * every launch of the force-and-integration kernel and around every contact search; the
 * host waits for each step's search decision.  Outputs (any may be NULL): summed device
 * milliseconds of the step kernel and of the searches, the number of step-kernel
 * launches and of searches, and the summed milliseconds and number of inner-list builds
 * (mixed contexts; see dem_stats.inner_builds).  Synchronises. */
dem_status dem_step_profiled(dem_ctx* ctx, int64_t n_steps, double* step_kernel_ms, double* search_ms,
                             int64_t* step_launches, int64_t* searches, double* inner_ms, int64_t* inner_builds);

/* Blocks until the context's stream is idle; reports sticky device errors. */
dem_status dem_sync(dem_ctx* ctx);

/* Current state in the caller's particle order: x^n, v^n, w^n (full-step velocities)
 * and active flags.  Any pointer may be NULL.  Synchronises. */
dem_status dem_get_state(dem_ctx* ctx, double* x, double* v, double* w, uint8_t* active);

/* Replaces the state (NULL keeps that part), clears sticky errors, forces a contact
 * search and a force evaluation at the next dem_step.  Tangential overlaps of pairs
 * still in contact are kept. */
dem_status dem_set_state(dem_ctx* ctx, const double* x, const double* v, const double* w,
                         const uint8_t* active);

/* Contact force and torque sums ([n][3] FP64, caller order; gravity excluded) of the
 * last force evaluation.  Synchronises. */
dem_status dem_get_forces(dem_ctx* ctx, double* force, double* torque);

/* Current fine-search list as pairs (i, j), i < j, in caller indices, lexicographic
 * order; writes min(count, capacity) pairs ([capacity][2] int32) and the count. */
dem_status dem_get_pairs(dem_ctx* ctx, int32_t* pairs, int64_t capacity, int64_t* count);

/* Tangential overlaps: pairs (i < j, caller indices) with a non-zero overlap of the
 * (i, j) orientation, and the particle-wall overlaps [n][n_walls][3] (may be NULL). */
dem_status dem_get_history(dem_ctx* ctx, int32_t* pairs, double* dt_pair, int64_t capacity,
                           int64_t* count, double* dt_wall);
/* Sets the tangential overlaps (pairs given as (i, j) carry the (i, j) orientation);
 * they take effect at the next contact search, which is forced. */
dem_status dem_set_history(dem_ctx* ctx, int64_t n_pairs, const int32_t* pairs,
                           const double* dt_pair, const double* dt_wall);

dem_status dem_get_stats(dem_ctx* ctx, dem_stats* out);

/* Contact search for callers that cannot allocate device memory (an application whose
 * memory is entirely owned by its own pool allocator, or a loop that cannot afford the
 * device-wide synchronisation an allocation may cause).  The paper has no counterpart:
 * this is a service of the library, not a step of the method.
 *
 * Finds all pairs (i, j), i < j, of active particles with |x_j - x_i|^2 < cutoff^2 --
 * the same set, with the same rounding, as the fine search of a context with r_c =
 * cutoff -- using no workspace: only the caller's buffers and one fixed 10 MiB scratch
 * array that every GPU loading the library holds until the process exits.
 *   x       device, [n][3] FP64;  active: device uint8 [n] or NULL (all active)
 *   domain  host double[3] each: box of the cell grid (points outside are clamped)
 *   pairs   device int32 [capacity][2]: the first min(count, capacity) pairs, ordered by
 *           i, then by the cells sharing a vertex with i's cell, then by j within a cell;
 *           may be NULL when capacity is 0 (count only)
 *   count   host: total number of pairs
 * Limits: n <= DEM_STATIC_MAX_PARTICLES (else DEM_ERR_CAPACITY); grids finer than
 * DEM_STATIC_MAX_CELLS cells are coarsened; a total above DEM_STATIC_MAX_PAIRS returns
 * DEM_ERR_CAPACITY with `count` set to the total and nothing written.  The call reads the
 * total back to the host and synchronises `stream` (twice when pairs are written), so it
 * cannot be captured into a CUDA graph.  All calls share the scratch and it keeps the
 * last call's contents (the per-cell counters and the total are cleared by every call);
 * calls that overlap on the GPU race and must not be issued.  The first call on a device
 * looks up the scratch's device address on that device, which must be current. */
#define DEM_STATIC_MAX_PARTICLES 262144
#define DEM_STATIC_MAX_CELLS 524288
#define DEM_STATIC_MAX_PAIRS 2147483647
dem_status dem_find_pairs_static(const double* x, const uint8_t* active, int64_t n, double cutoff,
                                 const double* domain_lo, const double* domain_hi, int32_t* pairs,
                                 int64_t capacity, int64_t* count, void* stream);
/* Measurement aid (no counterpart in the paper): issue rates of the arithmetic pipes the
 * step kernels depend on, on the current device, in thread-level instructions per second:
 * rates[0] FP64 fused multiply-add, rates[1] FP64 add, rates[2] FP32 fused multiply-add,
 * rates[3] FP32 -> FP64 conversion (host array of 4).  Each from a kernel of independent
 * chains over 8 blocks of 256 threads per SM, timed with CUDA events on `stream` after a
 * warm-up launch; allocates nothing; synchronises.  The FP64 path's roofline is its FP64
 * instruction rate against rates[0]. */
dem_status dem_pipe_rates(double* rates, void* stream);
const char* dem_status_string(dem_status s);
void dem_destroy(dem_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
