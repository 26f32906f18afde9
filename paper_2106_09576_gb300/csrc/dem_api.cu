// dem_api.cu -- C ABI, workspace layout and step scheduling of the GB300 DEM hot path.
//
// A time step is one "iteration" on the device:
//   k_begin      decides whether a contact search is due (Sec. 3.1) and counts the step;
//   IF (due)     the rebuild sequence of dem_rebuild.cu;
//   k_step       forces, history, integration (dem_step_impl.cuh).
// dem_step(n) replays these iterations inside one CUDA graph: a WHILE conditional node
// around [k_begin -> IF conditional node -> k_step]; k_begin sets both conditions from
// device-resident counters, so the host never waits on the device between steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/dem.h"
#include "dem_device.cuh"

using namespace demgb;

struct dem_ctx {
  dem_config cfg;
  Params P;
  cudaStream_t stream = nullptr;
  int device = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  size_t stage_bytes = 0;
  int* io_cnt = nullptr;   // [n + 1] per-particle counts for ordered output
  int* io_off = nullptr;   // [n + 2]
  dem_wall walls[kMaxWalls];
  int n_walls = 0;
  cudaGraphExec_t exec = nullptr;
  bool eager = false;
  bool instances_set = false;  // batch contexts: dem_set_instances has been called
  unsigned sticky = 0;     // device status bits already reported on the host
};

namespace {

constexpr size_t kAlign = 256;
constexpr int kCellTileShift = 5;   // cell order: columns of 32 x 32 cells (cell_index)

struct Layout {
  size_t total = 0;
  size_t add(size_t bytes) {
    size_t off = (total + kAlign - 1) / kAlign * kAlign;
    total = off + bytes;
    return off;
  }
};

struct Derived {
  double dmax, rc, skin;
  int nc[3];
  int n_cells;
  size_t hcap;
};

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

bool valid_material(const dem_material& m) {
  return m.young > 0.0 && m.poisson > -1.0 && m.poisson < 0.5 && m.restitution > 0.0 && m.restitution <= 1.0 &&
         m.mu_slide >= 0.0 && m.mu_roll >= 0.0;
}

bool valid_wall(const dem_wall& W) {
  if (W.kind < 0 || W.kind > 2) return false;
  const double nn = std::sqrt(W.normal[0] * W.normal[0] + W.normal[1] * W.normal[1] + W.normal[2] * W.normal[2]);
  if (!(nn > 0.0)) return false;
  if (W.kind >= 1 && !(W.radius > 0.0)) return false;
  if (W.kind == 2 && !(W.inner_radius >= 0.0 && W.inner_radius < W.radius)) return false;
  return true;
}

dem_status derive(const dem_config* c, Derived* d) {
  if (!c || c->n <= 0 || c->n >= (1LL << 31) - 64) return DEM_ERR_ARG;
  if (!(c->density > 0.0) || !(c->radius_max > 0.0) || !(c->dt > 0.0)) return DEM_ERR_ARG;
  if (c->precision != DEM_PRECISION_FP64 && c->precision != DEM_PRECISION_MIXED) return DEM_ERR_ARG;
  if (c->rolling_model < 0 || c->rolling_model > 2) return DEM_ERR_ARG;
  if (c->contact_model < 0 || c->contact_model > 1 || c->integrator < 0 || c->integrator > 1) return DEM_ERR_ARG;
  if (c->contact_model == 1 && !(c->linear_velocity > 0.0 && std::isfinite(c->linear_velocity))) return DEM_ERR_ARG;
  if (c->n_instances < 0 || c->n_instances > c->n) return DEM_ERR_ARG;
  if (c->step_block != 0 && c->step_block != 32 && c->step_block != 64 && c->step_block != 128) return DEM_ERR_ARG;
  if (c->pair_eval != DEM_PAIR_EVAL_ONCE && c->pair_eval != DEM_PAIR_EVAL_BOTH) return DEM_ERR_ARG;
  if (!valid_material(c->particle) || !valid_material(c->wall)) return DEM_ERR_ARG;
  if (!finite3(c->gravity) || !finite3(c->domain_lo) || !finite3(c->domain_hi)) return DEM_ERR_ARG;
  // search threshold: r_c = d_max + skin, or factor * d_max (Sec. 3.2), same arithmetic
  // as the CPU statement of the method
  double dmax = 2.0 * (double)(float)c->radius_max;
  double rc, skin;
  if (c->skin > 0.0) {
    rc = dmax + c->skin;
    skin = c->skin;
  } else {
    if (!(c->neighbor_factor >= 1.0)) return DEM_ERR_ARG;
    rc = c->neighbor_factor * dmax;
    skin = rc - dmax;
  }
  d->dmax = dmax;
  d->rc = rc;
  d->skin = skin;
  // uniform grid, cell edge h >= r_c (1 + 1e-6) so that rounding in the cell index can
  // never separate two particles closer than r_c by more than one cell
  double hmin = rc * (1.0 + 1e-6);
  long long cells = 1;
  for (int a = 0; a < 3; a++) {
    double L = c->domain_hi[a] - c->domain_lo[a];
    if (!(L > 0.0)) return DEM_ERR_ARG;
    double k = std::floor(L / hmin);
    d->nc[a] = (int)std::max(1.0, std::min(k, 1.0e6));
  }
  // keep the cell count below the scan limit (4096 * 4096) by coarsening uniformly
  for (;;) {
    cells = (long long)d->nc[0] * d->nc[1] * d->nc[2];
    if (cells + 2 <= 4096LL * 4096LL) break;
    for (int a = 0; a < 3; a++) d->nc[a] = std::max(1, (int)(d->nc[a] * 0.9));
  }
  d->n_cells = (int)cells;
  size_t cap = 1024;
  while (cap < (size_t)c->n * 4) cap <<= 1;
  d->hcap = cap;
  return DEM_OK;
}

struct Offsets {
  size_t x[2], v[2], w[2], act[2], rad[2], id[2], mask[2], hist[2], shadow[2], render[2], inst[2], itab, xref, nbr, nbr_cnt,
      nbr_lo, inner_lo, pslot, rec, upart,
      inner, inner_j, inner_cnt, xin, key, local, members, order,
      cell_count, cell_start, scan_tmp, hkey, hval, wall_tmp, wall_tmp_mask, out_v, out_w, out_F, out_M,
      stage, ctl, io_cnt, io_off;
  size_t total;
  size_t stage_bytes;
};

Offsets layout(const dem_config* c, const Derived& d) {
  const size_t n = (size_t)c->n;
  Layout L;
  Offsets o;
  for (int b = 0; b < 2; b++) {
    o.x[b] = L.add(3 * n * 8);
    o.v[b] = L.add(3 * n * 8);
    o.w[b] = L.add(3 * n * 8);
    o.act[b] = L.add(n);
    o.rad[b] = L.add(n * 4);
    o.id[b] = L.add(n * 4);
    o.mask[b] = L.add(n * 8);
    o.hist[b] = L.add(n * kHistStride * 3 * 8);
    const bool mixed = c->precision == DEM_PRECISION_MIXED;   // FP32 copies for neighbours
    o.shadow[b] = L.add(n * 16);
    o.render[b] = L.add(mixed ? n * 48 : 0);
  }
  const size_t n_inst = c->n_instances > 1 ? (size_t)c->n_instances : 0;
  for (int b = 0; b < 2; b++) o.inst[b] = L.add(n_inst ? n * 4 : 0);
  o.itab = L.add(n_inst * sizeof(InstDev));
  o.xref = L.add(3 * n * 8);
  o.nbr = L.add(n * kMaxNbr * 4);
  o.nbr_cnt = L.add(n * 4);
  o.nbr_lo = L.add(n);
  {
    const bool mixed = c->precision == DEM_PRECISION_MIXED;   // the inner list of the mixed path
    o.inner = L.add(mixed ? n * kInnerMax : 0);
    o.inner_j = L.add(mixed ? n * kInnerMax * 4 : 0);
    o.inner_cnt = L.add(mixed ? n : 0);
    o.xin = L.add(mixed ? 4 * n * 4 : 0);
    // one evaluation per pair: partner positions, pushed reactions, owners' own sums
    const bool once = mixed && c->pair_eval == DEM_PAIR_EVAL_ONCE;
    o.inner_lo = L.add(once ? n : 0);
    o.pslot = L.add(once ? n * kInnerMax * 8 : 0);
    o.rec = L.add(once ? n * kInnerMax * 32 : 0);
    o.upart = L.add(once ? n * 24 : 0);
  }
  o.key = L.add(n * 4);
  o.local = L.add(n * 4);
  o.members = L.add(n * 4);
  o.order = L.add(n * 4);
  o.cell_count = L.add(((size_t)d.n_cells + 1) * 4);
  o.cell_start = L.add(((size_t)d.n_cells + 2) * 4);
  o.scan_tmp = L.add(4096 * 4);
  o.hkey = L.add(d.hcap * 8);
  o.hval = L.add(d.hcap * 24);
  o.wall_tmp = L.add(n * kMaxWalls * 24);
  o.wall_tmp_mask = L.add(n);
  o.out_v = L.add(3 * n * 8);
  o.out_w = L.add(3 * n * 8);
  o.out_F = L.add(3 * n * 8);
  o.out_M = L.add(3 * n * 8);
  o.stage_bytes = std::max<size_t>(n * kMaxWalls * 24, 4096);
  o.stage = L.add(o.stage_bytes);
  o.ctl = L.add(sizeof(Control));
  o.io_cnt = L.add((n + 1) * 4);
  o.io_off = L.add((n + 2) * 4);
  o.total = L.total + kAlign;
  return o;
}

// ------------------------------------------------------------------ small kernels
__global__ void k_begin(Params P, cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_reb,
                        cudaGraphConditionalHandle h_inner, int in_graph) {
  Control* C = P.ctl;
  apply_flip(C);   // the previous evaluation's parities
  const long long rem = C->remaining;
  C->last = rem <= 1 ? 1 : 0;
  C->remaining = rem - 1;
  if (!C->init) {
    C->step++;
    C->since_rebuild++;
  }
  const int need =
      (C->init || C->need_rebuild || (P.rebuild_every > 0 && C->since_rebuild >= P.rebuild_every)) ? 1 : 0;
  // the inner list (mixed path) is refreshed by every contact search, else when due
  const int inner = (P.precision == DEM_PRECISION_MIXED && C->need_inner && !need) ? 1 : 0;
  if (need || inner) C->need_inner = 0;
  C->do_rebuild = need;
  C->do_inner = inner;
  // walls present at the time of this evaluation (floating walls, Sec. 3.6)
  const double t = (double)C->step * P.dt;
  unsigned on = 0u;
  for (int k = 0; k < P.n_walls; k++)
    if (t >= P.walls[k].t_on && t < P.walls[k].t_off) on |= 1u << k;
  C->wall_on = on;
  C->n_touch_dir = 0ull;
  C->n_wall_touch = 0ull;
  C->n_active = 0ull;
  C->max_ovl_bits = 0u;
  if (in_graph) {
    cudaGraphSetConditional(h_reb, (unsigned)need);
    cudaGraphSetConditional(h_inner, (unsigned)inner);
    cudaGraphSetConditional(h_loop, rem - 1 > 0 ? 1u : 0u);
  }
}

// Closes a dem_step call: applies the last evaluation's parity flip.
__global__ void k_end(Params P) { apply_flip(P.ctl); }

__global__ void k_set_remaining(Control* C, long long n_steps) {
  C->remaining = n_steps + (C->init ? 1 : 0);
}

// caller order [n][3] (stage) -> sorted SoA of buffer `cur`, gathered through id
__global__ void k_in_vec(Params P, const double* src, int which, int identity) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  const int u = identity ? p : P.id[C->sbuf][p];
  double* dst = which == 0 ? P.x[C->cur] : (which == 1 ? P.v[C->cur] : P.w[C->cur]);
  for (int d = 0; d < 3; d++) dst[(size_t)d * P.n + p] = src[3 * (size_t)u + d];
}

__global__ void k_in_act(Params P, const uint8_t* src) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  P.act[C->cur][p] = src[P.id[C->sbuf][p]] ? 1 : 0;
}

// caller order (stage) -> instance of each sorted particle, gathered through id
__global__ void k_in_inst(Params P, const int* src) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const int sb = P.ctl->sbuf;
  P.inst[sb][p] = src[P.id[sb][p]];
}

__global__ void k_init_identity(Params P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  P.id[0][p] = p;
  P.act[0][p] = 1;
}

// sorted -> caller order [n][3] (stage).  what: 0 x, 1 v, 2 w, 3 F, 4 M
__global__ void k_out_vec(Params P, double* dst, int what) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  const int u = P.id[C->sbuf][p];
  const bool ran = C->ran != 0;
  const int prev = ran ? (C->cur ^ 1) : C->cur;
  const double* src;
  switch (what) {
    case 0: src = P.x[prev]; break;
    case 1: src = ran ? P.out_v : P.v[prev]; break;
    case 2: src = ran ? P.out_w : P.w[prev]; break;
    case 3: src = P.out_F; break;
    default: src = P.out_M; break;
  }
  for (int d = 0; d < 3; d++) dst[3 * (size_t)u + d] = src[(size_t)d * P.n + p];
}

__global__ void k_out_act(Params P, uint8_t* dst) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  const int prev = C->ran ? (C->cur ^ 1) : C->cur;
  dst[P.id[C->sbuf][p]] = P.act[prev][p];
}

__global__ void k_count_active(Params P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const Control* C = P.ctl;
  const int prev = C->ran ? (C->cur ^ 1) : C->cur;
  unsigned a = (p < P.n) ? P.act[prev][p] : 0u;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0 && a) atomicAdd(&P.ctl->n_active_now, (unsigned long long)a);
}

// Per-particle count of list entries (mode 0) or overlap entries (mode 1) with id_i < id_j.
__global__ void k_io_count(Params P, int* cnt, int mode) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  int c = 0;
  if (p < C->n_act_sorted) {
    const int* ids = P.id[C->sbuf];
    const int a = ids[p];
    const int* nb = P.nbr + (size_t)p * kMaxNbr;
    const unsigned long long m = P.mask[C->hc][p];
    for (int k = 0; k < P.nbr_cnt[p]; k++) {
      if (mode == 1 && !((m >> k) & 1ull)) continue;
      if (a < ids[nb[k]]) c++;
    }
  }
  cnt[p] = c;
}

// Writes entries with global index in [lo, hi) to out (pairs int32[2], then FP64[3] values
// for mode 1 at out + 2*(hi-lo) int32 ... kept as separate arrays below).
__global__ void k_io_emit(Params P, const int* off, long long lo, long long hi, int* pairs, double* vals,
                          int mode) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  if (p >= C->n_act_sorted) return;
  long long g = off[p];
  if (g >= hi || off[p + 1] <= lo) return;
  const int* ids = P.id[C->sbuf];
  const int a = ids[p];
  const int* nb = P.nbr + (size_t)p * kMaxNbr;
  const unsigned long long m = P.mask[C->hc][p];
  const double* H = P.hist[C->hc] + (size_t)p;
  for (int k = 0; k < P.nbr_cnt[p]; k++) {
    const bool has = (m >> k) & 1ull;
    if (mode == 1 && !has) continue;
    const int b = ids[nb[k]];
    if (!(a < b)) continue;
    if (g >= lo && g < hi) {
      pairs[2 * (g - lo)] = a;
      pairs[2 * (g - lo) + 1] = b;
      if (mode == 1) {
        const int r = __popcll(m & ((1ull << k) - 1ull));
        vals[3 * (g - lo)] = H[hcomp(P.n, r, 0)];
        vals[3 * (g - lo) + 1] = H[hcomp(P.n, r, 1)];
        vals[3 * (g - lo) + 2] = H[hcomp(P.n, r, 2)];
      }
    }
    g++;
  }
}

// Particle-wall overlaps in caller order [n][n_walls][3].
__global__ void k_out_wall_hist(Params P, double* dst, int nw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const Control* C = P.ctl;
  const int u = P.id[C->sbuf][p];
  const unsigned long long m = (p < C->n_act_sorted) ? P.mask[C->hc][p] : 0ull;
  const double* H = P.hist[C->hc] + (size_t)p;
  for (int w = 0; w < nw; w++) {
    const int bit = kMaxNbr + w;
    double v[3] = {0.0, 0.0, 0.0};
    if ((m >> bit) & 1ull) {
      const int r = __popcll(m & ((1ull << bit) - 1ull));
      v[0] = H[hcomp(P.n, r, 0)];
      v[1] = H[hcomp(P.n, r, 1)];
      v[2] = H[hcomp(P.n, r, 2)];
    }
    for (int d = 0; d < 3; d++) dst[((size_t)u * nw + w) * 3 + d] = v[d];
  }
}

// Inserts caller-given overlaps (pairs in caller ids, value of the (i, j) orientation).
__global__ void k_hist_insert_pairs(Params P, const int* pairs, const double* vals, long long count) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int a = pairs[2 * t], b = pairs[2 * t + 1];
  const unsigned long long key = pair_key(a, b);
  const double sg = a < b ? 1.0 : -1.0;
  unsigned h = hash_slot(key, P.hcap_mask);
  for (unsigned probe = 0; probe <= P.hcap_mask; probe++) {
    unsigned long long prev = atomicCAS(&P.hkey[h], kEmptyKey, key);
    if (prev == kEmptyKey || prev == key) {
      P.hval[3 * (size_t)h] = sg * vals[3 * t];
      P.hval[3 * (size_t)h + 1] = sg * vals[3 * t + 1];
      P.hval[3 * (size_t)h + 2] = sg * vals[3 * t + 2];
      return;
    }
    h = (h + 1) & P.hcap_mask;
  }
  atomicOr(&P.ctl->status, kStCapacity);
}

__global__ void k_hist_insert_walls(Params P, const double* src, int nw) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= P.n) return;
  uint8_t m = 0;
  for (int w = 0; w < nw; w++) {
    const double* s = src + ((size_t)u * nw + w) * 3;
    double* d = P.wall_tmp + ((size_t)u * kMaxWalls + w) * 3;
    d[0] = s[0];
    d[1] = s[1];
    d[2] = s[2];
    if (s[0] != 0.0 || s[1] != 0.0 || s[2] != 0.0) m |= (uint8_t)(1u << w);
  }
  P.wall_tmp_mask[u] = m;
}

__global__ void k_mark(Control* C, int init, int preloaded, int clear_status) {
  if (init) {
    C->init = 1;
    C->ran = 0;
    C->need_rebuild = 1;
  }
  if (preloaded >= 0) C->hist_preloaded = preloaded;
  if (clear_status) C->status = 0u;
}

__global__ void k_clear_wall_bits(Params P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const int hc = P.ctl->hc;
  P.mask[hc][p] &= (1ull << kMaxNbr) - 1ull;
}

__global__ void k_ctl_init(Control* C, int n) {
  memset(C, 0, sizeof(Control));
  C->init = 1;
  C->need_rebuild = 1;
  C->n_act_sorted = n;
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

dem_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DEM_OK : DEM_ERR_CUDA; }
#define CK(call)                                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return DEM_ERR_CUDA;  \
  } while (0)

// A truncated list or table leaves the steps that follow undefined (a record nobody
// wrote, a contact dropped), so the capacity error, the cause, is reported first.
dem_status status_from_bits(unsigned b) {
  if (b & kStCapacity) return DEM_ERR_CAPACITY;
  if (b & kStNonfinite) return DEM_ERR_NONFINITE;
  if (b & kStOverlap) return DEM_ERR_OVERLAP;
  if (b & kStTimeout) return DEM_ERR_TIMEOUT;
  return DEM_OK;
}

double eff_young(const dem_material& a, const dem_material& b) {
  return 1.0 / ((1.0 - a.poisson * a.poisson) / a.young + (1.0 - b.poisson * b.poisson) / b.young);
}
double eff_shear(const dem_material& a, const dem_material& b) {
  return 1.0 / (2.0 * (2.0 - a.poisson) * (1.0 + a.poisson) / a.young +
                2.0 * (2.0 - b.poisson) * (1.0 + b.poisson) / b.young);
}
// -2 sqrt(5/6) beta, beta = ln(e) / sqrt(ln(e)^2 + pi^2) (Table equation_parameters)
// 1 + (pi / ln e)^2, the denominator of Eq. linearetan (infinite for e = 1: no damping)
double linear_damping_den(double e) {
  const double q = 3.14159265358979323846 / std::log(e);
  return 1.0 + q * q;
}

double eta_coeff(double e) {
  double le = std::log(e);
  double beta = le / std::sqrt(le * le + 3.14159265358979323846 * 3.14159265358979323846);
  return -2.0 * std::sqrt(5.0 / 6.0) * beta;
}

void fill_materials(const dem_material& part, const dem_material& wall, MatD* md, MatF* mf) {
  md->Ye_pp = eff_young(part, part);
  md->Ge_pp = eff_shear(part, part);
  md->ceta_pp = eta_coeff(part.restitution);
  md->mu_pp = part.mu_slide;
  md->mur_pp = part.mu_roll;
  md->Ye_pw = eff_young(part, wall);
  md->Ge_pw = eff_shear(part, wall);
  md->ceta_pw = eta_coeff(wall.restitution);
  md->mu_pw = wall.mu_slide;
  md->mur_pw = wall.mu_roll;
  md->lin_den_pp = linear_damping_den(part.restitution);
  md->lin_den_pw = linear_damping_den(wall.restitution);
  mf->lin_den_pp = (float)md->lin_den_pp;
  mf->lin_den_pw = (float)md->lin_den_pw;
  mf->Ye_pp = (float)md->Ye_pp;
  mf->Ge_pp = (float)md->Ge_pp;
  mf->ceta_pp = (float)md->ceta_pp;
  mf->mu_pp = (float)md->mu_pp;
  mf->mur_pp = (float)md->mur_pp;
  mf->Ye_pw = (float)md->Ye_pw;
  mf->Ge_pw = (float)md->Ge_pw;
  mf->ceta_pw = (float)md->ceta_pw;
  mf->mu_pw = (float)md->mu_pw;
  mf->mur_pw = (float)md->mur_pw;
}

// A double as an FP32 pair h + l (h the nearest float, l the nearest float to the rest).
void split_host(double v, float* h, float* l) {
  *h = (float)v;
  *l = (float)(v - (double)*h);
}

void to_device_wall(const dem_wall& s, WallDev* W, WallF* F, float* fv, WallX* X) {
  std::memset(W, 0, sizeof(*W));
  std::memset(F, 0, sizeof(*F));
  std::memset(X, 0, sizeof(*X));
  W->kind = s.kind;
  W->translates = s.translates ? 1 : 0;
  double nn = std::sqrt(s.normal[0] * s.normal[0] + s.normal[1] * s.normal[1] + s.normal[2] * s.normal[2]);
  double na = std::sqrt(s.rot_axis[0] * s.rot_axis[0] + s.rot_axis[1] * s.rot_axis[1] + s.rot_axis[2] * s.rot_axis[2]);
  for (int d = 0; d < 3; d++) {
    W->p[d] = s.point[d];
    W->n[d] = s.normal[d] / nn;
    W->Om[d] = na > 0.0 ? s.omega * s.rot_axis[d] / na : 0.0;
    W->c[d] = s.rot_origin[d];
    W->V[d] = s.velocity[d];
  }
  W->radius = s.radius;
  W->inner = s.inner_radius;
  W->t_on = s.t_on;
  W->t_off = s.t_off;
  for (int d = 0; d < 3; d++) {
    F->p[d] = (float)W->p[d];
    F->n[d] = (float)W->n[d];
  }
  F->radius = (float)W->radius;
  F->inner = (float)W->inner;
  for (int d = 0; d < 3; d++) fv[d] = W->translates ? (float)W->V[d] : 0.0f;
  // the FP32 form: planes and cylinders along a coordinate axis that do not translate
  X->axis = -1;
  if ((W->kind == 0 || W->kind == 1) && !W->translates) {
    for (int a = 0; a < 3; a++) {
      const int b = (a + 1) % 3, c2 = (a + 2) % 3;
      if (std::fabs(W->n[a]) == 1.0 && W->n[b] == 0.0 && W->n[c2] == 0.0) {
        X->axis = a;
        X->sign = (float)W->n[a];
      }
    }
  }
  for (int d = 0; d < 3; d++) {
    split_host(W->p[d], &X->ph[d], &X->pl[d]);
    X->Om[d] = (float)W->Om[d];
    X->c[d] = (float)W->c[d];
    X->V[d] = (float)W->V[d];
  }
  split_host(W->radius, &X->rh, &X->rl);
}

void fill_walls(dem_ctx* c) {
  for (int k = 0; k < kMaxWalls; k++) {
    if (k < c->n_walls) {
      to_device_wall(c->walls[k], &c->P.walls[k], &c->P.wf[k], c->P.wf_v[k], &c->P.wx[k]);
    } else {
      std::memset(&c->P.walls[k], 0, sizeof(WallDev));
      std::memset(&c->P.wf[k], 0, sizeof(WallF));
      std::memset(&c->P.wx[k], 0, sizeof(WallX));
      c->P.wx[k].axis = -1;
      for (int d = 0; d < 3; d++) c->P.wf_v[k][d] = 0.0f;
    }
  }
  c->P.n_walls = c->n_walls;
  c->P.any_translating = 0;
  for (int k = 0; k < c->n_walls; k++)
    if (c->P.walls[k].translates) c->P.any_translating = 1;
}

void launch_step(const Params& P, cudaStream_t s) {
  if (P.precision == DEM_PRECISION_MIXED)
    launch_step_mixed(P, s);
  else
    launch_step_fp64(P, s);
}

void destroy_graph(dem_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  c->exec = nullptr;
}

// WHILE(loop) { k_begin -> IF(rebuild) { rebuild } -> IF(inner) { inner build } -> k_step } -> k_end
dem_status build_graph(dem_ctx* c) {
  destroy_graph(c);
  cudaGraph_t g = nullptr;
  cudaStream_t cs = nullptr;
  dem_status st = DEM_ERR_CUDA;
  do {
    if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle hl, hr, hi;
    if (cudaGraphConditionalHandleCreate(&hl, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    if (cudaGraphConditionalHandleCreate(&hr, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) break;
    if (cudaGraphConditionalHandleCreate(&hi, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hl;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp) != cudaSuccess) break;
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    k_begin<<<1, 1, 0, cs>>>(c->P, hl, hr, hi, 1);
    if (cudaStreamEndCapture(cs, &body) != cudaSuccess) break;
    size_t nn = 0;
    if (cudaGraphGetNodes(body, nullptr, &nn) != cudaSuccess || nn != 1) break;
    cudaGraphNode_t begin_node;
    if (cudaGraphGetNodes(body, &begin_node, &nn) != cudaSuccess) break;
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hr;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    if (cudaGraphAddNode(&inode, body, &begin_node, nullptr, 1, &ip) != cudaSuccess) break;
    cudaGraph_t rbody = ip.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, rbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    launch_rebuild(c->P, cs);
    if (cudaStreamEndCapture(cs, &rbody) != cudaSuccess) break;
    // IF(inner list due) { inner build } after the search's IF
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hi;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t nnode;
    if (cudaGraphAddNode(&nnode, body, &inode, nullptr, 1, &np) != cudaSuccess) break;
    cudaGraph_t ibody = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    launch_inner(c->P, cs);
    if (cudaStreamEndCapture(cs, &ibody) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, body, &nnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    launch_step(c->P, cs);
    if (cudaStreamEndCapture(cs, &body) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    k_end<<<1, 1, 0, cs>>>(c->P);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess) break;
    if (cudaGraphInstantiate(&c->exec, g, 0) != cudaSuccess) {
      c->exec = nullptr;
      break;
    }
    st = DEM_OK;
  } while (0);
  if (cs) cudaStreamDestroy(cs);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return st;
}

dem_status check_sticky(dem_ctx* c) {
  unsigned bits = 0;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(&bits, &c->P.ctl->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  c->sticky |= bits;
  return status_from_bits(c->sticky);
}

// Runs `iters` iterations eagerly (debug mode): the host reads the rebuild decision.
dem_status run_eager(dem_ctx* c, long long n_steps) {
  k_set_remaining<<<1, 1, 0, c->stream>>>(c->P.ctl, n_steps);
  long long rem = 0;
  CK(cudaMemcpyAsync(&rem, &c->P.ctl->remaining, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (long long it = 0; it < rem; it++) {
    k_begin<<<1, 1, 0, c->stream>>>(c->P, 0, 0, 0, 0);
    int need = 0, inner = 0;
    CK(cudaMemcpyAsync(&need, &c->P.ctl->do_rebuild, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&inner, &c->P.ctl->do_inner, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (need) launch_rebuild(c->P, c->stream);
    if (inner) launch_inner(c->P, c->stream);
    launch_step(c->P, c->stream);
  }
  k_end<<<1, 1, 0, c->stream>>>(c->P);
  CK(cudaGetLastError());
  return DEM_OK;
}

dem_status run_iterations(dem_ctx* c, long long n_steps) {
  if (c->eager) return run_eager(c, n_steps);
  if (!c->exec) {
    dem_status s = build_graph(c);
    if (s != DEM_OK) return s;
  }
  k_set_remaining<<<1, 1, 0, c->stream>>>(c->P.ctl, n_steps);
  CK(cudaGetLastError());
  CK(cudaGraphLaunch(c->exec, c->stream));
  return DEM_OK;
}

// Copies `bytes` from a host or device pointer into the stage area.
dem_status to_stage(dem_ctx* c, const void* src, size_t bytes, size_t off = 0) {
  CK(cudaMemcpyAsync((char*)c->P.stage + off, src, bytes, cudaMemcpyDefault, c->stream));
  return DEM_OK;
}
dem_status from_stage(dem_ctx* c, void* dst, size_t bytes, size_t off = 0) {
  CK(cudaMemcpyAsync(dst, (const char*)c->P.stage + off, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DEM_OK;
}

dem_status upload_vecs(dem_ctx* c, const double* x, const double* v, const double* w, int identity) {
  const size_t n = (size_t)c->P.n;
  const int T = 256;
  const double* src[3] = {x, v, w};
  for (int k = 0; k < 3; k++) {
    if (!src[k]) continue;
    dem_status s = to_stage(c, src[k], 3 * n * 8);
    if (s != DEM_OK) return s;
    k_in_vec<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, c->P.stage, k, identity);
  }
  CK(cudaGetLastError());
  return DEM_OK;
}

// Emits ordered list entries (mode 0) or overlaps (mode 1) to caller arrays in chunks.
dem_status emit(dem_ctx* c, int mode, int32_t* pairs, double* vals, int64_t capacity, int64_t* count) {
  const int n = c->P.n;
  const int T = 256;
  k_io_count<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, c->io_cnt, mode);
  scan_exclusive_i32(c->io_cnt, n, c->io_off, c->P.scan_tmp, c->stream);
  int total = 0;
  CK(cudaMemcpyAsync(&total, c->io_off + n, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = total;
  const long long want = std::min<long long>(total, capacity);
  const size_t per = mode == 1 ? 32 : 8;
  const long long chunk = (long long)(c->stage_bytes / per);
  for (long long lo = 0; lo < want; lo += chunk) {
    const long long hi = std::min(want, lo + chunk);
    int* sp = (int*)c->P.stage;
    double* sv = (double*)((char*)c->P.stage + (size_t)(hi - lo) * 8);
    k_io_emit<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, c->io_off, lo, hi, sp, sv, mode);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pairs + 2 * lo, sp, (size_t)(hi - lo) * 8, cudaMemcpyDefault, c->stream));
    if (mode == 1)
      CK(cudaMemcpyAsync(vals + 3 * lo, sv, (size_t)(hi - lo) * 24, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DEM_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

dem_status dem_workspace_bytes(const dem_config* cfg, size_t* bytes) {
  if (!bytes) return DEM_ERR_ARG;
  Derived d;
  dem_status s = derive(cfg, &d);
  if (s != DEM_OK) return s;
  *bytes = layout(cfg, d).total;
  return DEM_OK;
}

dem_status dem_create(const dem_config* cfg, const double* x, const double* v, const double* w,
                      const float* radius, void* workspace, size_t workspace_bytes, void* stream, dem_ctx** out) {
  if (!out || !x || !v || !w || !radius || !workspace) return DEM_ERR_ARG;
  *out = nullptr;
  Derived d;
  dem_status s = derive(cfg, &d);
  if (s != DEM_OK) return s;
  Offsets o = layout(cfg, d);
  if (workspace_bytes < o.total) return DEM_ERR_CAPACITY;
  dem_ctx* c = new dem_ctx();
  c->cfg = *cfg;
  c->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return DEM_ERR_CUDA;
  }
  char* base = (char*)(((uintptr_t)workspace + kAlign - 1) / kAlign * kAlign);
  c->ws = base;
  c->ws_bytes = workspace_bytes;
  c->stage_bytes = o.stage_bytes;
  Params& P = c->P;
  std::memset(&P, 0, sizeof(P));
  P.n = (int)cfg->n;
  P.precision = cfg->precision;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
    P.sm_count = sms;
  }
  P.rolling = cfg->rolling_model;
  P.contact_model = cfg->contact_model;
  P.integrator = cfg->integrator;
  P.lin_V = cfg->linear_velocity;
  P.f_lin_V = (float)cfg->linear_velocity;
  P.rebuild_every = cfg->rebuild_every;
  for (int a = 0; a < 3; a++) {
    P.nc[a] = d.nc[a];
    P.g[a] = cfg->gravity[a];
    P.lo[a] = cfg->domain_lo[a];
    P.inv_h[a] = (double)d.nc[a] / (cfg->domain_hi[a] - cfg->domain_lo[a]);
  }
  P.n_cells = d.n_cells;
  P.cell_tile_shift = kCellTileShift;
  P.hcap_mask = (unsigned)(d.hcap - 1);
  P.dt = cfg->dt;
  P.half_dt = 0.5 * cfg->dt;
  P.density = cfg->density;
  P.rc2 = d.rc * d.rc;
  {
    double half = 0.5 * d.skin;
    P.disp_lim2 = half * half;
  }
  P.z_sink = cfg->z_sink;
  P.max_overlap_ratio = cfg->max_overlap_ratio;
  {
    double ext = 0.0;
    for (int a = 0; a < 3; a++)
      ext = std::max(ext, std::max(std::fabs(cfg->domain_lo[a]), std::fabs(cfg->domain_hi[a])));
    P.wall_margin = (float)(1e-6 * std::max(1.0, ext) + 1e-9);
  }
  fill_materials(cfg->particle, cfg->wall, &P.md, &P.mf);
  P.f_density = (float)P.density;
  P.f_dt = (float)P.dt;
  for (int a = 0; a < 3; a++) P.f_g[a] = (float)P.g[a];
  P.f_disp_lim2 = (float)(P.disp_lim2 * (1.0 - 1e-5));   // conservative: rebuild slightly early
  {
    // inner list (mixed path): the pairs of the fine-search list within R_i + R_j + delta,
    // refreshed when a particle has moved delta / 2
    const double delta = std::min(0.1 * d.dmax, 0.25 * d.skin);
    P.f_inner_margin = (float)delta;
    P.f_inner_lim2 = (float)(0.25 * delta * delta * (1.0 - 1e-5));
    P.f_disp_lim = (float)(0.5 * d.skin);
  }
  P.f_rc = (float)d.rc;
  P.step_block = cfg->step_block;
  P.n_inst = cfg->n_instances > 1 ? cfg->n_instances : 0;
  {
    long long zb;
    double zs = cfg->z_sink;
    std::memcpy(&zb, &zs, 8);
    P.z_sink_key = ordered_key(zb);
  }
  for (int b = 0; b < 2; b++) {
    P.x[b] = (double*)(base + o.x[b]);
    P.v[b] = (double*)(base + o.v[b]);
    P.w[b] = (double*)(base + o.w[b]);
    P.act[b] = (uint8_t*)(base + o.act[b]);
    P.rad[b] = (float*)(base + o.rad[b]);
    P.id[b] = (int*)(base + o.id[b]);
    P.mask[b] = (unsigned long long*)(base + o.mask[b]);
    P.hist[b] = (double*)(base + o.hist[b]);
    P.shadow[b] = (float4*)(base + o.shadow[b]);
    P.render[b] = (float4*)(base + o.render[b]);
    P.inst[b] = (int*)(base + o.inst[b]);
  }
  P.itab = (const InstDev*)(base + o.itab);
  P.xref = (double*)(base + o.xref);
  P.nbr = (int*)(base + o.nbr);
  P.nbr_cnt = (int*)(base + o.nbr_cnt);
  P.nbr_lo = (uint8_t*)(base + o.nbr_lo);
  P.pair_once = (cfg->precision == DEM_PRECISION_MIXED && cfg->pair_eval == DEM_PAIR_EVAL_ONCE) ? 1 : 0;
  P.inner_lo = (uint8_t*)(base + o.inner_lo);
  P.pslot = (int2*)(base + o.pslot);
  P.rec = (float4*)(base + o.rec);
  P.upart = (float*)(base + o.upart);
  P.inner = (uint8_t*)(base + o.inner);
  P.inner_j = (int*)(base + o.inner_j);
  P.inner_cnt = (uint8_t*)(base + o.inner_cnt);
  P.xin = (float*)(base + o.xin);
  P.key = (unsigned*)(base + o.key);
  P.local = (int*)(base + o.local);
  P.members = (int*)(base + o.members);
  P.order = (int*)(base + o.order);
  P.cell_count = (int*)(base + o.cell_count);
  P.cell_start = (int*)(base + o.cell_start);
  P.scan_tmp = (int*)(base + o.scan_tmp);
  P.hkey = (unsigned long long*)(base + o.hkey);
  P.hval = (double*)(base + o.hval);
  P.wall_tmp = (double*)(base + o.wall_tmp);
  P.wall_tmp_mask = (uint8_t*)(base + o.wall_tmp_mask);
  P.out_v = (double*)(base + o.out_v);
  P.out_w = (double*)(base + o.out_w);
  P.out_F = (double*)(base + o.out_F);
  P.out_M = (double*)(base + o.out_M);
  P.stage = (double*)(base + o.stage);
  P.ctl = (Control*)(base + o.ctl);
  c->io_cnt = (int*)(base + o.io_cnt);
  c->io_off = (int*)(base + o.io_off);
  c->n_walls = 0;
  fill_walls(c);
  const char* ev = std::getenv("DEM_GB300_EAGER");
  c->eager = ev && ev[0] == '1';

  const int T = 256;
  const size_t n = (size_t)cfg->n;
  k_ctl_init<<<1, 1, 0, c->stream>>>(P.ctl, P.n);
  k_init_identity<<<blocks_for(n, T), T, 0, c->stream>>>(P);
  if (cudaMemsetAsync(P.mask[0], 0, n * 8, c->stream) != cudaSuccess ||
      cudaMemsetAsync(P.mask[1], 0, n * 8, c->stream) != cudaSuccess ||
      cudaMemsetAsync(P.nbr_cnt, 0, n * 4, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(P.rad[0], radius, n * 4, cudaMemcpyDefault, c->stream) != cudaSuccess ||
      upload_vecs(c, x, v, w, 1) != DEM_OK || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    delete c;
    return DEM_ERR_CUDA;
  }
  // every radius must be positive and no larger than radius_max
  std::vector<float> r(n);
  if (cudaMemcpy(r.data(), P.rad[0], n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    delete c;
    return DEM_ERR_CUDA;
  }
  const float rmax = (float)cfg->radius_max;
  for (size_t i = 0; i < n; i++)
    if (!(r[i] > 0.0f) || !(r[i] <= rmax)) {
      delete c;
      return DEM_ERR_ARG;
    }
  *out = c;
  return DEM_OK;
}

dem_status dem_set_walls(dem_ctx* c, const dem_wall* walls, int32_t n_walls) {
  if (!c || n_walls < 0 || n_walls > kMaxWalls || (n_walls > 0 && !walls)) return DEM_ERR_ARG;
  if (c->P.n_inst > 1) return DEM_ERR_STATE;   // a batch takes its walls per instance
  for (int k = 0; k < n_walls; k++)
    if (!valid_wall(walls[k])) return DEM_ERR_ARG;
  for (int k = 0; k < n_walls; k++) c->walls[k] = walls[k];
  c->n_walls = n_walls;
  fill_walls(c);
  destroy_graph(c);
  const int T = 256;
  k_clear_wall_bits<<<blocks_for(c->P.n, T), T, 0, c->stream>>>(c->P);
  k_mark<<<1, 1, 0, c->stream>>>(c->P.ctl, 1, -1, 0);
  return cuda_status(cudaGetLastError());
}

dem_status dem_set_instances(dem_ctx* c, const dem_instance* inst, int32_t n_instances) {
  if (!c || !inst) return DEM_ERR_ARG;
  if (c->P.n_inst <= 1) return DEM_ERR_STATE;
  if (n_instances != c->P.n_inst) return DEM_ERR_ARG;
  const long long n = c->P.n;
  std::vector<InstDev> tab((size_t)n_instances);
  int any_tr = 0;
  std::vector<int> of((size_t)n);
  for (int k = 0; k < n_instances; k++) {
    const dem_instance& I = inst[k];
    const long long lo = I.first, hi = k + 1 < n_instances ? inst[k + 1].first : n;
    if (lo < 0 || hi > n || lo > hi || (k == 0 && lo != 0)) return DEM_ERR_ARG;
    if (!valid_material(I.particle) || !valid_material(I.wall)) return DEM_ERR_ARG;
    if (I.n_walls < 0 || I.n_walls > kMaxInstWalls) return DEM_ERR_ARG;
    InstDev& D = tab[(size_t)k];
    std::memset(&D, 0, sizeof(D));
    fill_materials(I.particle, I.wall, &D.md, &D.mf);
    D.n_walls = I.n_walls;
    for (int w = 0; w < I.n_walls; w++) {
      if (!valid_wall(I.walls[w])) return DEM_ERR_ARG;
      to_device_wall(I.walls[w], &D.walls[w], &D.wf[w], D.wf_v[w], &D.wx[w]);
      if (D.walls[w].translates) any_tr = 1;
    }
    for (long long i = lo; i < hi; i++) of[(size_t)i] = k;
  }
  // the instance of each particle, gathered into the current sorted order through id
  if (n * 4 > (long long)c->stage_bytes) return DEM_ERR_CAPACITY;
  CK(cudaMemcpyAsync((void*)c->P.itab, tab.data(), tab.size() * sizeof(InstDev), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->P.stage, of.data(), (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
  const int T = 256;
  k_in_inst<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, (const int*)c->P.stage);
  k_clear_wall_bits<<<blocks_for(n, T), T, 0, c->stream>>>(c->P);
  k_mark<<<1, 1, 0, c->stream>>>(c->P.ctl, 1, -1, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));   // the host tables above go out of scope
  destroy_graph(c);
  c->P.any_translating = any_tr;
  c->instances_set = true;
  return DEM_OK;
}

dem_status dem_step(dem_ctx* c, int64_t n_steps) {
  if (!c || n_steps < 0) return DEM_ERR_ARG;
  if (c->sticky) return DEM_ERR_STATE;
  if (c->P.n_inst > 1 && !c->instances_set) return DEM_ERR_STATE;
  if (n_steps == 0) return DEM_OK;
  return run_iterations(c, n_steps);
}

dem_status dem_step_profiled(dem_ctx* c, int64_t n_steps, double* step_kernel_ms, double* search_ms,
                             int64_t* step_launches, int64_t* searches, double* inner_ms, int64_t* inner_builds) {
  if (c && c->P.n_inst > 1 && !c->instances_set) return DEM_ERR_STATE;
  if (!c || n_steps < 0) return DEM_ERR_ARG;
  if (c->sticky) return DEM_ERR_STATE;
  double ks = 0.0, ss = 0.0, is = 0.0;
  int64_t nk = 0, ns = 0, ni = 0;
  if (n_steps > 0) {
    cudaEvent_t e[6];
    for (auto& ev : e)
      if (cudaEventCreate(&ev) != cudaSuccess) return DEM_ERR_CUDA;
    dem_status st = DEM_OK;
    k_set_remaining<<<1, 1, 0, c->stream>>>(c->P.ctl, n_steps);
    long long rem = 0;
    if (cudaMemcpyAsync(&rem, &c->P.ctl->remaining, sizeof(long long), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      st = DEM_ERR_CUDA;
    for (long long it = 0; st == DEM_OK && it < rem; it++) {
      k_begin<<<1, 1, 0, c->stream>>>(c->P, 0, 0, 0, 0);
      int need = 0, inner = 0;
      if (cudaMemcpyAsync(&need, &c->P.ctl->do_rebuild, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
              cudaSuccess ||
          cudaMemcpyAsync(&inner, &c->P.ctl->do_inner, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        st = DEM_ERR_CUDA;
        break;
      }
      if (need) {
        cudaEventRecord(e[2], c->stream);
        launch_rebuild(c->P, c->stream);
        cudaEventRecord(e[3], c->stream);
      }
      if (inner) {
        cudaEventRecord(e[4], c->stream);
        launch_inner(c->P, c->stream);
        cudaEventRecord(e[5], c->stream);
      }
      cudaEventRecord(e[0], c->stream);
      launch_step(c->P, c->stream);
      cudaEventRecord(e[1], c->stream);
      if (cudaEventSynchronize(e[1]) != cudaSuccess) {
        st = DEM_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e[0], e[1]);
      ks += ms;
      nk++;
      if (need) {
        cudaEventElapsedTime(&ms, e[2], e[3]);
        ss += ms;
        ns++;
      }
      if (inner) {
        cudaEventElapsedTime(&ms, e[4], e[5]);
        is += ms;
        ni++;
      }
    }
    for (auto& ev : e) cudaEventDestroy(ev);
    if (st != DEM_OK) return st;
    k_end<<<1, 1, 0, c->stream>>>(c->P);
    CK(cudaGetLastError());
  }
  if (step_kernel_ms) *step_kernel_ms = ks;
  if (search_ms) *search_ms = ss;
  if (step_launches) *step_launches = nk;
  if (searches) *searches = ns;
  if (inner_ms) *inner_ms = is;
  if (inner_builds) *inner_builds = ni;
  return check_sticky(c);
}

dem_status dem_sync(dem_ctx* c) {
  if (!c) return DEM_ERR_ARG;
  return check_sticky(c);
}

dem_status dem_get_state(dem_ctx* c, double* x, double* v, double* w, uint8_t* active) {
  if (!c) return DEM_ERR_ARG;
  const size_t n = (size_t)c->P.n;
  const int T = 256;
  double* out[3] = {x, v, w};
  for (int k = 0; k < 3; k++) {
    if (!out[k]) continue;
    k_out_vec<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, c->P.stage, k);
    CK(cudaGetLastError());
    dem_status s = from_stage(c, out[k], 3 * n * 8);
    if (s != DEM_OK) return s;
  }
  if (active) {
    k_out_act<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, (uint8_t*)c->P.stage);
    CK(cudaGetLastError());
    dem_status s = from_stage(c, active, n);
    if (s != DEM_OK) return s;
  }
  return check_sticky(c);
}

dem_status dem_set_state(dem_ctx* c, const double* x, const double* v, const double* w, const uint8_t* active) {
  if (!c) return DEM_ERR_ARG;
  const size_t n = (size_t)c->P.n;
  const int T = 256;
  CK(cudaStreamSynchronize(c->stream));
  // After steps, the current state is x^n in buffer cur^1 and v^n, w^n in the outputs;
  // bring it into buffer cur, which the next contact search reads, then overwrite the
  // parts the caller gives.
  Control h;
  CK(cudaMemcpy(&h, c->P.ctl, sizeof(Control), cudaMemcpyDeviceToHost));
  if (h.ran) {
    const int cur = h.cur, prev = h.cur ^ 1;
    CK(cudaMemcpyAsync(c->P.x[cur], c->P.x[prev], 3 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.v[cur], c->P.out_v, 3 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.w[cur], c->P.out_w, 3 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->P.act[cur], c->P.act[prev], n, cudaMemcpyDeviceToDevice, c->stream));
  }
  dem_status s = upload_vecs(c, x, v, w, 0);
  if (s != DEM_OK) return s;
  if (active) {
    s = to_stage(c, active, n);
    if (s != DEM_OK) return s;
    k_in_act<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, (const uint8_t*)c->P.stage);
  }
  k_mark<<<1, 1, 0, c->stream>>>(c->P.ctl, 1, -1, 1);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->sticky = 0;
  return DEM_OK;
}

dem_status dem_get_forces(dem_ctx* c, double* force, double* torque) {
  if (!c) return DEM_ERR_ARG;
  int ran = 0;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(&ran, &c->P.ctl->ran, sizeof(int), cudaMemcpyDeviceToHost));
  if (!ran) {
    // forces before the first step: run the initial evaluation only
    if (c->sticky) return DEM_ERR_STATE;
    dem_status s = run_iterations(c, 0);
    if (s != DEM_OK) return s;
  }
  const size_t n = (size_t)c->P.n;
  const int T = 256;
  double* out[2] = {force, torque};
  for (int k = 0; k < 2; k++) {
    if (!out[k]) continue;
    k_out_vec<<<blocks_for(n, T), T, 0, c->stream>>>(c->P, c->P.stage, 3 + k);
    CK(cudaGetLastError());
    dem_status s = from_stage(c, out[k], 3 * n * 8);
    if (s != DEM_OK) return s;
  }
  return check_sticky(c);
}

dem_status dem_get_pairs(dem_ctx* c, int32_t* pairs, int64_t capacity, int64_t* count) {
  if (!c || !count || capacity < 0 || (capacity > 0 && !pairs)) return DEM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  int ran = 0;
  CK(cudaMemcpy(&ran, &c->P.ctl->ran, sizeof(int), cudaMemcpyDeviceToHost));
  if (!ran) {
    dem_status s = run_iterations(c, 0);
    if (s != DEM_OK) return s;
  }
  return emit(c, 0, pairs, nullptr, capacity, count);
}

dem_status dem_get_history(dem_ctx* c, int32_t* pairs, double* dt_pair, int64_t capacity, int64_t* count,
                           double* dt_wall) {
  if (!c || !count || capacity < 0 || (capacity > 0 && (!pairs || !dt_pair))) return DEM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  int ran = 0;
  CK(cudaMemcpy(&ran, &c->P.ctl->ran, sizeof(int), cudaMemcpyDeviceToHost));
  if (!ran) {
    dem_status s = run_iterations(c, 0);
    if (s != DEM_OK) return s;
  }
  dem_status s = emit(c, 1, pairs, dt_pair, capacity, count);
  if (s != DEM_OK) return s;
  if (dt_wall && c->n_walls > 0) {
    const int T = 256;
    k_out_wall_hist<<<blocks_for(c->P.n, T), T, 0, c->stream>>>(c->P, c->P.stage, c->n_walls);
    CK(cudaGetLastError());
    s = from_stage(c, dt_wall, (size_t)c->P.n * c->n_walls * 24);
    if (s != DEM_OK) return s;
  }
  return DEM_OK;
}

dem_status dem_set_history(dem_ctx* c, int64_t n_pairs, const int32_t* pairs, const double* dt_pair,
                           const double* dt_wall) {
  if (!c || n_pairs < 0 || (n_pairs > 0 && (!pairs || !dt_pair))) return DEM_ERR_ARG;
  const int T = 256;
  CK(cudaStreamSynchronize(c->stream));
  launch_hist_clear(c->P, c->stream, 1);
  const long long chunk = (long long)(c->stage_bytes / 32);
  for (long long lo = 0; lo < n_pairs; lo += chunk) {
    const long long hi = std::min<long long>(n_pairs, lo + chunk);
    dem_status s = to_stage(c, pairs + 2 * lo, (size_t)(hi - lo) * 8);
    if (s != DEM_OK) return s;
    s = to_stage(c, dt_pair + 3 * lo, (size_t)(hi - lo) * 24, (size_t)(hi - lo) * 8);
    if (s != DEM_OK) return s;
    k_hist_insert_pairs<<<blocks_for(hi - lo, T), T, 0, c->stream>>>(
        c->P, (const int*)c->P.stage, (const double*)((char*)c->P.stage + (hi - lo) * 8), hi - lo);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
  }
  if (dt_wall && c->n_walls > 0) {
    dem_status s = to_stage(c, dt_wall, (size_t)c->P.n * c->n_walls * 24);
    if (s != DEM_OK) return s;
    k_hist_insert_walls<<<blocks_for(c->P.n, T), T, 0, c->stream>>>(c->P, c->P.stage, c->n_walls);
  }
  k_mark<<<1, 1, 0, c->stream>>>(c->P.ctl, 1, 1, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return DEM_OK;
}

dem_status dem_get_stats(dem_ctx* c, dem_stats* out) {
  if (!c || !out) return DEM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  Control h;
  CK(cudaMemcpy(&h, c->P.ctl, sizeof(Control), cudaMemcpyDeviceToHost));
  // count the particles still in the system at the current step
  CK(cudaMemsetAsync(&c->P.ctl->n_active_now, 0, sizeof(unsigned long long), c->stream));
  k_count_active<<<blocks_for(c->P.n, 256), 256, 0, c->stream>>>(c->P);
  CK(cudaGetLastError());
  unsigned long long act = 0;
  CK(cudaMemcpyAsync(&act, &c->P.ctl->n_active_now, sizeof(act), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memset(out, 0, sizeof(*out));
  out->steps = h.step;
  out->rebuilds = h.rebuilds;
  out->n_pairs = (int64_t)(h.n_pairs_dir / 2);
  out->n_touch = (int64_t)(h.n_touch_dir / 2);
  out->n_wall_touch = (int64_t)h.n_wall_touch;
  out->n_active = (int64_t)act;
  out->time = (double)h.step * c->cfg.dt;
  float mo;
  std::memcpy(&mo, &h.max_ovl_bits, 4);
  out->max_overlap_ratio = mo;
  c->sticky |= h.status;
  out->status_bits = c->sticky;
  out->max_neighbors_seen = h.max_nbr_seen;
  out->inner_builds = h.inner_builds;
  dem_workspace_bytes(&c->cfg, &out->required_workspace);
  return DEM_OK;
}

const char* dem_status_string(dem_status s) {
  switch (s) {
    case DEM_OK: return "ok";
    case DEM_ERR_ARG: return "invalid argument";
    case DEM_ERR_CUDA: return "CUDA runtime error";
    case DEM_ERR_CAPACITY: return "capacity exceeded (workspace, neighbour slots, contacts or hash table)";
    case DEM_ERR_NONFINITE: return "non-finite position or velocity";
    case DEM_ERR_OVERLAP: return "normal overlap above max_overlap_ratio";
    case DEM_ERR_TIMEOUT: return "bounded device wait timed out";
    case DEM_ERR_STATE: return "call out of order or sticky device error";
    default: return "unknown status";
  }
}

void dem_destroy(dem_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  delete c;
}

}  // extern "C"
