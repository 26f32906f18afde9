// dem_device.cuh -- device-side data layout and helpers of the GB300 DEM hot path.
//
// Layout in HBM (all inside the caller's workspace; see dem_api.cu for the offsets):
//   per particle, cell-sorted order, structure of arrays
//     x[2], v[2], w[2]  FP64 [3][n]   ping-pong by time step (parity ctl->cur)
//     act[2]            uint8 [n]     1 = in the system; ping-pong with the state
//     rad[2], id[2]     FP32 / int32  reordered at each rebuild (parity ctl->sbuf)
//     xref              FP64 [3][n]   positions at the last contact search; in a mixed
//                                     context FP32 [6][n]: their hi parts, then lo parts
//     shadow[2]         float4 [n]    {hx, hy, hz, R} of each particle: written at each
//                                     contact search, read by its FP32 filters (the fine
//                                     search and the history restore); ping-pong with the state
//     render[2]         float4 [n][3] {hx, hy, hz, lx} {ly, lz, vx, vy} {vz, wx, wy, wz}
//                                     (mixed path): the FP32 copy that contact partners and
//                                     the inner-list build read, written by every step;
//                                     x = hx + lx to 2^-48; a particle out of the system has
//                                     hx = hy = hz = kFar; the radius is rad[]; ping-pong
//                                     with the state
//     mask[2]           uint64 [n]    bit k < 56: neighbour slot k has a tangential overlap;
//                                     bit 56+w: wall w has one (parity ctl->hc)
//     hist[2]           FP64 [32][3][n] tangential overlaps of the set bits, compact, in
//                                     bit order, in component planes (parity ctl->hc)
//     nbr               int32 [n][56] fine-search list (full list: each pair twice)
//     nbr_cnt           int32 [n]
//     inner, inner_cnt  uint8 [n][32], uint8 [n] (mixed path): the slots of the fine-search
//                                     list whose partner was within R_i + R_j + delta at the
//                                     last inner build, ascending (so in partner-id order)
//     inner_j           int32 [n][32] (mixed path) the partners of those slots
//     inner_lo, pslot   uint8 [n], int2 [32][n] (mixed path, one evaluation per pair): the
//                                     leading slots whose partner has the smaller id, and the
//                                     other (owned) slots packed as {j, k | m << 8}, m the own
//                                     position in the partner's row
//     rec, upart        float4 [32][n][2], float [6][n] (same): reactions pushed by owners to
//                                     their partners, and each owner's own partial sums
//     xin               FP32 [7][n]   (mixed path) positions at the last inner build, hi
//                                     parts then lo parts, then the distance of that position
//                                     from the search reference x_ref (rounded up)
//   per cell: cell_count, cell_start (int32 [n_cells + 2])
//   hash table of tangential overlaps used at rebuild: hkey uint64 [cap], hval FP64 [cap][3]
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dem.h"

namespace demgb {

constexpr int kMaxWalls = 8;
constexpr int kMaxNbr = 56;      // slots per particle in the fine-search list
constexpr int kHistStride = 32;  // simultaneous contacts per particle (particles + walls)
constexpr int kInnerMax = 32;    // entries of a particle's inner list (mixed path)
// Position of a particle out of the system in the FP32 copies of the mixed path: its
// square (1e36) is still finite in FP32.
constexpr float kFar = 1e18f;
// Tangential overlaps are stored in component planes: component d of entry r of every
// particle's compact list lies in plane 3 r + d, [kHistStride][3][n] doubles, so a warp's
// reads and writes of its particles' r-th entries are three contiguous runs of whole
// sectors (a partly written sector costs a DRAM read before its write-back; particles hold
// a few entries, the first planes are dense).  Component d of entry r of particle i:
// hist + i + hcomp(n, r, d).
__host__ __device__ __forceinline__ size_t hcomp(int n, int r, int d) {
  return ((size_t)r * 3 + (size_t)d) * (size_t)n;
}
constexpr unsigned long long kEmptyKey = 0xFFFFFFFFFFFFFFFFull;

// status bits (sticky, in Control::status)
constexpr unsigned kStCapacity = 1u, kStNonfinite = 2u, kStOverlap = 4u, kStTimeout = 8u;

struct WallDev {
  int kind;
  int translates;   // 1: point and c move with V (translational boundary motion)
  double p[3];      // point (plane), point on axis (cylinder), centre (annulus)
  double n[3];      // unit normal / axis
  double radius, inner;
  double Om[3];     // angular velocity vector of the surface
  double c[3];      // rotation origin
  double V[3];      // translation velocity of the surface
  double t_on, t_off;
};

// FP32 copies of the wall geometry for the conservative prefilter of the mixed path.
struct WallF {     // 32 bytes: the prefilter reads it for every particle
  float p[3], n[3], radius, inner;
};

// The mixed path's FP32 form of a plane or cylinder whose normal or axis is a coordinate
// axis (and that does not translate): the point and the radius as hi + lo pairs, so that
// the overlap comes out of double-float arithmetic as accurately as from FP64, and the
// rotation in FP32 for the wall's velocity at the contact point.  axis < 0: no such form,
// the FP64 geometry is used.
struct WallX {
  int axis;          // n = sign * e_axis, or -1
  float sign;
  float ph[3], pl[3];  // point = ph + pl
  float rh, rl;        // radius = rh + rl (cylinder)
  float Om[3], c[3], V[3];
};

// Material constants of one contact type pair (Table equation_parameters): effective Y
// and G, -2 sqrt(5/6) beta, sliding and rolling friction; particle-particle (_pp) and
// particle-wall (_pw).  MatF holds their FP32 copies for the mixed path.
// lin_den_* = 1 + (pi / ln e)^2 of Eq. linearetan (linear model).
struct MatD {
  double Ye_pp, Ge_pp, ceta_pp, mu_pp, mur_pp, lin_den_pp;
  double Ye_pw, Ge_pw, ceta_pw, mu_pw, mur_pw, lin_den_pw;
};
struct MatF {
  float Ye_pp, Ge_pp, ceta_pp, mu_pp, mur_pp, lin_den_pp;
  float Ye_pw, Ge_pw, ceta_pw, mu_pw, mur_pw, lin_den_pw;
};

// One member of a batch: its materials and walls (device table indexed by instance).
constexpr int kMaxInstWalls = 4;
struct InstDev {
  MatD md;
  MatF mf;
  int n_walls;
  int pad;
  WallDev walls[kMaxInstWalls];
  WallF wf[kMaxInstWalls];
  float wf_v[kMaxInstWalls][3];   // FP32 translation velocity of translating walls, else 0
  WallX wx[kMaxInstWalls];
};

// Device-resident control block: everything that changes from step to step.
struct Control {
  int cur;              // state parity holding the positions of the next force evaluation
  int sbuf;             // parity of rad/id (flips at rebuild)
  int hc;               // parity of mask/hist
  int need_rebuild;     // set by the step kernel when a displacement exceeds skin/2
  int init;             // 1: the next evaluation is the initial one (no overlap increment)
  int ran;              // 1: at least one evaluation has run since the state was set
  int last;             // 1: the current evaluation is the last of a dem_step call
  int hist_preloaded;   // 1: the hash table already holds overlaps given by the caller
  int n_act_sorted;     // particles [0, n_act_sorted) were active at the last rebuild
  int max_nbr_seen;
  unsigned wall_on;     // bit k: wall k exists at the time of the current evaluation
  int do_rebuild;       // decision of the current iteration (read by the host in eager mode)
  int flip_due;         // 1: a step kernel ran; its parity flip is not applied yet
  unsigned status;      // sticky error bits
  unsigned max_ovl_bits;  // float bits of max delta_n / R over the last step
  long long step;       // completed time steps
  long long since_rebuild;
  long long rebuilds;
  long long remaining;  // evaluations left in the current dem_step call
  // inner list (mixed path): a particle moved more than delta / 2 from its position at the
  // last inner build, the decision of the current iteration, and the number of builds
  int need_inner;
  int do_inner;
  long long inner_builds;
  unsigned long long n_touch_dir;   // directed particle-particle contacts, last step
  unsigned long long n_wall_touch;
  unsigned long long n_pairs_dir;   // directed fine-search entries at the last rebuild
  unsigned long long n_active;
  unsigned long long n_active_now;  // scratch of dem_get_stats
};

// Applies the parity flip a step kernel left due (see end_step): the state and history
// parities, and the end of the initial evaluation.  One thread.
__device__ __forceinline__ void apply_flip(Control* C) {
  if (C->flip_due) {
    C->cur ^= 1;
    C->hc ^= 1;
    C->init = 0;
    C->ran = 1;
    C->flip_due = 0;
  }
}

struct Params {
  int n;
  int n_walls;
  int precision;        // 0 FP64, 1 mixed
  int sm_count;         // SMs of the device the context runs on
  int step_block;       // threads per step-kernel block; 0 = step_block(n, sm_count)
  int rolling;          // 0 none, 1 constant, 2 viscous (Table rolling_torque)
  int contact_model;    // 0 non-linear, 1 linear (Eqs. linearkn, linearetan)
  int integrator;       // 0 velocity Verlet, 1 explicit Euler (Eq. integ_EE)
  int any_translating;  // some wall (of the context or of an instance) translates
  int pair_once;        // mixed path: each pair evaluated once by its owner (see below)
  double lin_V;         // characteristic impact velocity of Eq. linearkn
  float f_lin_V;
  int rebuild_every;
  int nc[3];
  int cell_tile_shift;   // cells are ordered in columns of 2^shift x 2^shift cells (cell_index)
  int n_cells;
  unsigned hcap_mask;   // hash capacity - 1 (power of two)
  double dt, half_dt;
  double g[3];
  double density;
  double rc2;           // fine-search threshold squared
  double disp_lim2;     // (skin/2)^2
  double z_sink;
  double max_overlap_ratio;
  double lo[3], inv_h[3];
  float wall_margin;    // FP32 prefilter margin for walls (m)
  MatD md;              // material constants of a single system
  WallDev walls[kMaxWalls];
  // FP32 copies of uniform constants (mixed path), computed once on the host
  float f_density, f_dt, f_g[3], f_disp_lim2, f_rc;
  // inner list: margin delta and (delta / 2)^2 (slightly reduced); skin / 2, below which
  // a particle cannot fire the search trigger
  float f_inner_margin, f_inner_lim2, f_disp_lim;
  MatF mf;
  long long z_sink_key;   // ordered-integer image of z_sink (exact comparison without FP64)
  WallF wf[kMaxWalls];
  float wf_v[kMaxWalls][3];   // FP32 translation velocity of translating walls, else 0
  WallX wx[kMaxWalls];
  // batch (n_inst > 1): per-instance materials and walls replace md, mf, walls, wf
  int n_inst;
  const InstDev* itab;  // [n_inst]
  int* inst[2];         // [n] instance of each particle, reordered with rad/id (parity sbuf)
  // buffers
  double* x[2];
  double* v[2];
  double* w[2];
  uint8_t* act[2];
  float* rad[2];
  int* id[2];
  unsigned long long* mask[2];
  double* hist[2];
  double* xref;
  float4* shadow[2];    // [n] FP32 {x_hi, R} (see the layout above)
  float4* render[2];    // [n][3] FP32 {x_hi, x_lo.x} {x_lo.y, x_lo.z, v.x, v.y} {v.z, w}
  int* nbr;
  int* nbr_cnt;
  uint8_t* nbr_lo;      // [n] entries of the fine-search list with a smaller partner id
  uint8_t* inner;       // [n][kInnerMax] (mixed path)
  int* inner_j;         // [n][kInnerMax] partner of each inner slot
  uint8_t* inner_cnt;   // [n]
  // one evaluation per pair (mixed path, pair_once): the pair belongs to its partner of
  // smaller id (the owner).  inner_lo: leading slots of a particle's inner list whose
  // partners own the pair; pslot: the owned slots, each with where the owner sits in the
  // partner's inner list; rec: slot-major [kInnerMax][n][2] the reaction an owner
  // computed for its partner {F, M_x}{M_y, M_z, 0, 0}; upart [6][n]: the owner's own sum
  // of its owned pairs and walls, same packing
  uint8_t* inner_lo;    // [n]
  int2* pslot;          // [kInnerMax][n] the owned slots, packed from entry 0 (slot-major):
                        //   {partner j, fine-list slot k | (position m in j's inner list) << 8}
  float4* rec;
  float* upart;
  float* xin;           // [4][n] hi parts of x at the last inner refresh, and |x_in - x_ref|
  unsigned* key;        // [n] cell key of the current (pre-sort) order
  int* local;           // [n] slot within the cell (order of the atomics)
  int* members;         // [n] particles grouped by cell, any order within a cell
  int* order;           // [n] sorted position -> previous position
  int* cell_count;      // [n_cells + 1]
  int* cell_start;      // [n_cells + 2]
  int* scan_tmp;        // block sums of the scan
  unsigned long long* hkey;
  double* hval;         // [cap][3]
  double* wall_tmp;     // [n][kMaxWalls][3] wall overlaps by particle id, at rebuild
  uint8_t* wall_tmp_mask;  // [n]
  double* out_v;        // [3][n] full-step velocities of the last step (sorted order)
  double* out_w;
  double* out_F;        // [3][n] contact force and torque sums of the last evaluation
  double* out_M;
  double* stage;        // [9][n] staging in caller order for state transfers
  Control* ctl;
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

// Squared distance dx*dx + dy*dy + dz*dz with dx = b - a, left to right, no contraction:
// the same rounding as the CPU reference of the contact search.
__device__ __forceinline__ double sqdist_exact(double ax, double ay, double az, double bx, double by,
                                               double bz) {
  double dx = dsub(bx, ax), dy = dsub(by, ay), dz = dsub(bz, az);
  double s = dmul(dx, dx);
  s = dadd(s, dmul(dy, dy));
  s = dadd(s, dmul(dz, dz));
  return s;
}

// Bound on the error of an FP32 distance between two particles computed from the hi
// parts of their positions (split_df truncates, |x - hi| < 2^-23 |x|): per axis the
// difference of the hi parts is off by less than 2^-23 (a_i + a_j) plus its own rounding
// (at most 2^-24 of a value below `reach`), so the distance is off by less than sqrt(3)
// times that.  a_i, a_j are the largest coordinate magnitudes of the two particles.
__device__ __forceinline__ float hi_distance_error(float a_i, float a_j, float reach) {
  return 1.7320509f * (1.1920929e-7f * (a_i + a_j) * 1.0001f + 5.9604645e-8f * reach) + 1e-30f;
}

__device__ __forceinline__ float max_abs3(float4 h) { return fmaxf(fmaxf(fabsf(h.x), fabsf(h.y)), fabsf(h.z)); }

// Position of cell (cx, cy, cz) in the sort order.  The grid is cut into columns of
// T x T cells in x and y (T = 2^shift) spanning all of z; columns are taken in row-major
// order, and inside a column x runs fastest, then y, then z.  A cell's 26 neighbours are
// then within about T^2 cells of it, except across column faces, so the step kernel
// finds most of a particle's neighbours still in L2 when it reads them.  With T at
// least the grid's x and y extents this is the plain x-fastest order.
__host__ __device__ __forceinline__ int cell_index(const int* nc, int shift, int cx, int cy, int cz) {
  const int tile = 1 << shift;
  const int tx = cx >> shift, ty = cy >> shift;
  const int ix = cx - (tx << shift), iy = cy - (ty << shift);
  const int wx = min(tile, nc[0] - (tx << shift)), hy = min(tile, nc[1] - (ty << shift));
  return ((ty << shift) * nc[0] + (tx << shift) * hy) * nc[2] + (cz * hy + iy) * wx + ix;
}

// Error-free transformations in FP32 (Knuth two-sum, FMA two-product).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// FP32 -> FP64 conversion with integer operations (exact for normal numbers; zero and
// subnormals map to signed zero; inf/NaN preserved).  Keeps conversions off the FP64
// pipe, which on this part issues at 1/72 of the FP32 rate.
__device__ __forceinline__ double f2d_int(float f) {
  unsigned u = __float_as_uint(f);
  unsigned sign = u & 0x80000000u;
  unsigned e = (u >> 23) & 0xFFu;
  unsigned m = u & 0x7FFFFFu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 255u) ? (sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 with integer operations, rounding half away from zero on the magnitude;
// results below the FP32 normal range flush to zero, above it saturate to infinity.
__device__ __forceinline__ float d2f_int(double d) {
  unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  unsigned sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FFu) - 896;
  unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned r = ((unsigned)(e > 0 ? e : 0) << 23) + m + ((lo >> 28) & 1u);
  r = (e <= 0) ? 0u : r;
  r = (e >= 255 || r >= 0x7F800000u) ? 0x7F800000u : r;
  return __uint_as_float(r | sign);
}

// Split x into hi + lo (FP32 each) with integer operations: hi keeps the leading 24
// significant bits of x (truncated), lo the next 24 (rounded); |x - hi - lo| <= 2^-48 |x|.
// Values below 2^-75 in magnitude collapse to (0, 0).
__device__ __forceinline__ void split_df(double x, float& h, float& l) {
  unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  unsigned sign = hw & 0x80000000u;
  int e = (int)((hw >> 20) & 0x7FFu);
  int ef = e - 896;
  unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  float hv = __uint_as_float(sign | ((unsigned)(ef > 0 ? ef : 0) << 23) | mh);
  unsigned ml = lw & 0x1FFFFFFFu;
  float scale = __uint_as_float((unsigned)(e > 948 ? e - 948 : 0) << 23);
  float lv = __fmul_rn(__uint2float_rn(ml), scale);
  lv = sign ? -lv : lv;
  bool ok = (ef > 0) && (ef < 255);
  h = ok ? hv : (ef >= 255 ? __double2float_rn(x) : 0.0f);
  l = ok ? lv : 0.0f;
}

// Leading 24 significant bits of x (truncated), as split_df's hi part, integer ops only.
__device__ __forceinline__ float hi_df(double x) {
  float h, l;
  split_df(x, h, l);
  return h;
}

// Writes the FP32 copy of a particle (render) from its split position (h, l) and its
// velocities.  A particle out of the system is put at kFar on every axis: its distance
// to any particle in the domain exceeds every contact and list reach, so no pair with it
// touches or enters an inner list.
__device__ __forceinline__ void write_render(float4* rd, const float* h, const float* l, const double* v,
                                            const double* w, bool active) {
  rd[0] = active ? make_float4(h[0], h[1], h[2], l[0]) : make_float4(kFar, kFar, kFar, 0.0f);
  rd[1] = make_float4(l[1], l[2], d2f_int(v[0]), d2f_int(v[1]));
  rd[2] = make_float4(d2f_int(v[2]), d2f_int(w[0]), d2f_int(w[1]), d2f_int(w[2]));
}

// b - a as an unevaluated FP32 pair (s, t), exact up to the rounding of the low parts.
__device__ __forceinline__ void df_diff(float ah, float al, float bh, float bl, float& s, float& t) {
  float e;
  two_sum(bh, -ah, s, e);
  t = __fadd_rn(__fsub_rn(bl, al), e);
}

// Upper bound on how far a particle has moved since the last inner-list refresh: its new
// position hn + ln against the hi parts of the refresh position (the lo parts are not
// kept; split_df truncates, so each was below 2^-23 of its coordinate, and together they
// add at most sqrt(3) 2^-23 max|x_in| to the distance).  The factor 1 + 1e-5 covers the
// FP32 rounding of the sum and the root.
__device__ __forceinline__ float moved_since_inner(const float* xin, int n, int i, const float* hn, const float* ln) {
  float d2 = 0.f, a = 0.f;
  for (int d = 0; d < 3; d++) {
    const float r = xin[(size_t)d * n + i];
    float s1, t1;
    df_diff(r, 0.0f, hn[d], ln[d], s1, t1);
    const float u = s1 + t1;
    d2 += u * u;
    a = fmaxf(a, fabsf(r));
  }
  return sqrtf(d2) * (1.0f + 1e-5f) + 1.7320509f * 1.1920929e-7f * 1.0001f * a;
}

// Monotone map of a double's bits to a signed integer (exact ordering, integer ops only).
__host__ __device__ __forceinline__ long long ordered_key(long long bits) {
  return bits ^ ((bits >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ unsigned long long pair_key(int a, int b) {
  unsigned lo = (unsigned)(a < b ? a : b), hi = (unsigned)(a < b ? b : a);
  return ((unsigned long long)lo << 32) | hi;
}
__device__ __forceinline__ unsigned hash_slot(unsigned long long k, unsigned mask) {
  unsigned long long h = k * 0x9E3779B97F4A7C15ull;
  return (unsigned)(h >> 32) & mask;
}

__device__ __forceinline__ int cell_coord(double xd, double lo, double inv_h, int nc) {
  double f = floor(dmul(dsub(xd, lo), inv_h));
  // NaN and negative map to 0, beyond the grid to the last cell
  return (f >= 0.0) ? (f < (double)nc ? (int)f : nc - 1) : 0;
}

// Launchers (host side), defined in the .cu files.
void launch_rebuild(const Params& P, cudaStream_t s);
void launch_inner(const Params& P, cudaStream_t s);
void launch_hist_clear(const Params& P, cudaStream_t s, int force);
void scan_exclusive_i32(const int* in, int n, int* out, int* partials, cudaStream_t s);
void launch_step_fp64(const Params& P, cudaStream_t s);
void launch_step_mixed(const Params& P, cudaStream_t s);
void launch_inner_mirror(const Params& P, cudaStream_t s);

constexpr int kStepBlock = 128;   // largest block of the step kernels

// Threads per block of a step kernel for n particles on sm_count SMs: 128 when the grid
// covers every SM at least twice, smaller blocks for smaller systems so that their
// particles spread over more SMs (the work per particle is long and latency-bound).
inline int step_block(int n, int sm_count) {
  if (n >= sm_count * 128 * 2) return 128;
  if (n >= sm_count * 64 * 2) return 64;
  return 32;
}

}  // namespace demgb
