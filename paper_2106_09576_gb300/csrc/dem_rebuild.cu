// dem_rebuild.cu -- contact search at a rebuild step (Sec. 3.1-3.2).
//
// Sequence (all on the context stream, inside a conditional graph node):
//   1. save the tangential overlaps of the old list into a hash table keyed by the
//      caller ids (id_min, id_max); particle-wall overlaps go to a per-id scratch;
//   2. cell key of every active particle over a uniform grid (cell edge >= r_c);
//      counting sort by key: per-cell counts (integer atomics), exclusive scan (the
//      cell ranges), scatter, then each cell's members ordered by previous position,
//      so the result is a stable sort and does not depend on atomic order;
//   3. permute the particle state into the other buffer (x_ref = x);
//   4. fine search: for each particle, the 27 cells sharing a vertex with its own
//      (the broad search), keep j with |x_j - x_i|^2 < r_c^2 (same rounding as the CPU
//      reference), and order the list by partner id;
//   5. for every new list entry look the pair up in the hash table and rebuild the
//      compact per-particle overlap storage and its bit mask.
#include "dem_device.cuh"

namespace demgb {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanBlock * kScanItems;

// ------------------------------------------------------------------ exclusive scan
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[kScanBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  int excl = x - v + (wid > 0 ? warp_sums[wid - 1] : 0);
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

__global__ void k_scan_partials(const int* in, int n, int* partials) {
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int s = 0;
  for (int k = 0; k < kScanItems; k++) s += (base + k < n) ? in[base + k] : 0;
  int total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void k_scan_partials_top(int* partials, int nb) {
  // one block; nb <= kScanTile
  int base = threadIdx.x * kScanItems;
  int vals[kScanItems];
  int s = 0;
  for (int k = 0; k < kScanItems; k++) {
    vals[k] = (base + k < nb) ? partials[base + k] : 0;
    s += vals[k];
  }
  int excl = block_exclusive_scan(s, nullptr);
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < nb) partials[base + k] = excl;
    excl += vals[k];
  }
}

// out[0..n] = exclusive scan of in[0..n-1]; out[n] = total
__global__ void k_scan_final(const int* in, int n, const int* partials, int* out) {
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int vals[kScanItems];
  int s = 0;
  for (int k = 0; k < kScanItems; k++) {
    vals[k] = (base + k < n) ? in[base + k] : 0;
    s += vals[k];
  }
  int total;
  int excl = block_exclusive_scan(s, &total) + partials[blockIdx.x];
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) out[base + k] = excl;
    excl += vals[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = partials[blockIdx.x] + total;
}

void scan_exclusive_i32(const int* in, int n, int* out, int* partials, cudaStream_t s) {
  int nb = (n + kScanTile - 1) / kScanTile;
  if (nb < 1) nb = 1;
  k_scan_partials<<<nb, kScanBlock, 0, s>>>(in, n, partials);
  k_scan_partials_top<<<1, kScanBlock, 0, s>>>(partials, nb);
  k_scan_final<<<nb, kScanBlock, 0, s>>>(in, n, partials, out);
}

// ------------------------------------------------------------------ 1. save history
__global__ void k_hist_save(Params P) {
  const Control* C = P.ctl;
  if (C->hist_preloaded) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C->n_act_sorted) return;
  const int cur = C->cur, sb = C->sbuf, hc = C->hc;
  if (!P.act[cur][i]) return;
  const unsigned long long m = P.mask[hc][i];
  if (!m) return;
  const int* ids = P.id[sb];
  const int a = ids[i];
  const double* H = P.hist[hc] + (size_t)i;
  const int* nb = P.nbr + (size_t)i * kMaxNbr;
  int rank = 0;
  for (int k = 0; k < 64; k++) {
    if (!((m >> k) & 1ull)) continue;
    if (k < kMaxNbr) {
      const int b = ids[nb[k]];
      if (a < b) {  // each unordered pair stored once, orientation (a, b)
        const unsigned long long key = pair_key(a, b);
        unsigned h = hash_slot(key, P.hcap_mask);
        bool done = false;
        for (unsigned probe = 0; probe <= P.hcap_mask; probe++) {
          unsigned long long prev = atomicCAS(&P.hkey[h], kEmptyKey, key);
          if (prev == kEmptyKey || prev == key) {
            P.hval[3 * (size_t)h] = H[hcomp(P.n, rank, 0)];
            P.hval[3 * (size_t)h + 1] = H[hcomp(P.n, rank, 1)];
            P.hval[3 * (size_t)h + 2] = H[hcomp(P.n, rank, 2)];
            done = true;
            break;
          }
          h = (h + 1) & P.hcap_mask;
        }
        if (!done) atomicOr(&P.ctl->status, kStCapacity);
      }
    } else {
      const int w = k - kMaxNbr;
      double* dst = P.wall_tmp + ((size_t)a * kMaxWalls + w) * 3;
      dst[0] = H[hcomp(P.n, rank, 0)];
      dst[1] = H[hcomp(P.n, rank, 1)];
      dst[2] = H[hcomp(P.n, rank, 2)];
      P.wall_tmp_mask[a] |= (uint8_t)(1u << w);
    }
    rank++;
  }
}

// ------------------------------------------------------------------ 2. cell sort
__global__ void k_cell_count(Params P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  const int cur = P.ctl->cur;
  const double* X = P.x[cur];
  const int n = P.n;
  unsigned key;
  if (P.act[cur][p]) {
    int cx = cell_coord(X[p], P.lo[0], P.inv_h[0], P.nc[0]);
    int cy = cell_coord(X[n + p], P.lo[1], P.inv_h[1], P.nc[1]);
    int cz = cell_coord(X[2 * n + p], P.lo[2], P.inv_h[2], P.nc[2]);
    key = (unsigned)cell_index(P.nc, P.cell_tile_shift, cx, cy, cz);
  } else {
    key = (unsigned)P.n_cells;  // bucket of particles that left the system
  }
  P.key[p] = key;
  P.local[p] = atomicAdd(&P.cell_count[key], 1);
}

__global__ void k_cell_scatter(Params P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  P.members[P.cell_start[P.key[p]] + P.local[p]] = p;
}

// Orders each cell's members by previous position: the sort becomes stable and
// independent of the order in which the atomics were served.  One thread per member: it
// counts the members of its cell with a smaller previous position and lands there, so a
// crowded cell costs each of its m members O(m) work (as the fine search over it does)
// and no thread sorts a whole cell.  The bucket of particles that left the system keeps
// any order.
__global__ void k_cell_order(Params P) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.n) return;
  const int p = P.members[s];
  const int c = P.key[p];
  if (c >= P.n_cells) {
    P.order[s] = p;
    return;
  }
  const int b = P.cell_start[c], e = P.cell_start[c + 1];
  int r = 0;
  for (int t = b; t < e; t++) r += P.members[t] < p ? 1 : 0;
  P.order[b + r] = p;
}

// ------------------------------------------------------------------ 3. permute
__global__ void k_permute(Params P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n;
  if (q >= n) return;
  const Control* C = P.ctl;
  const int cur = C->cur, nxt = cur ^ 1, sb = C->sbuf;
  const int p = P.order[q];
  double xv[3], vv[3], wv[3];
  for (int d = 0; d < 3; d++) {
    xv[d] = P.x[cur][d * n + p];
    vv[d] = P.v[cur][d * n + p];
    wv[d] = P.w[cur][d * n + p];
    P.x[nxt][d * n + q] = xv[d];
    P.v[nxt][d * n + q] = vv[d];
    P.w[nxt][d * n + q] = wv[d];
  }
  const float r = P.rad[sb][p];
  const uint8_t a = P.act[cur][p];
  float h[3], l[3];
  for (int d = 0; d < 3; d++) split_df(xv[d], h[d], l[d]);
  if (P.precision == DEM_PRECISION_MIXED) {
    float* xr = reinterpret_cast<float*>(P.xref);
    for (int d = 0; d < 3; d++) {
      xr[d * n + q] = h[d];
      xr[(3 + d) * n + q] = l[d];
    }
    write_render(P.render[nxt] + 3 * (size_t)q, h, l, vv, wv, a != 0);
  } else {
    for (int d = 0; d < 3; d++) P.xref[d * n + q] = xv[d];
  }
  P.shadow[nxt][q] = make_float4(h[0], h[1], h[2], r);
  P.act[nxt][q] = a;
  P.rad[sb ^ 1][q] = r;
  P.id[sb ^ 1][q] = P.id[sb][p];
  if (P.n_inst > 1) P.inst[sb ^ 1][q] = P.inst[sb][p];
}

// Particles out of the system sit after the active ones and are never touched by the
// step kernel: give both state buffers their values.  Separate from k_permute, whose
// threads still read the source buffer.
__global__ void k_mirror_inactive(Params P) {
  const int n = P.n;
  const int q = P.cell_start[P.n_cells] + blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int cur = P.ctl->cur, nxt = cur ^ 1;
  for (int d = 0; d < 3; d++) {
    P.x[cur][d * n + q] = P.x[nxt][d * n + q];
    P.v[cur][d * n + q] = P.v[nxt][d * n + q];
    P.w[cur][d * n + q] = P.w[nxt][d * n + q];
  }
  P.act[cur][q] = P.act[nxt][q];
  P.shadow[cur][q] = P.shadow[nxt][q];
  if (P.precision == DEM_PRECISION_MIXED)
    for (int k = 0; k < 3; k++) P.render[cur][3 * (size_t)q + k] = P.render[nxt][3 * (size_t)q + k];
}

// ------------------------------------------------------------------ 4. fine search
// The list under construction (partner indices and their ids) lives in shared memory, one
// row per thread (odd row stride: no bank conflicts between rows), so keeping it ordered by
// partner id compares against ids already at hand instead of reloading them from global
// memory; the finished row is copied out once.
constexpr int kNbrBlock = 64;
constexpr int kNbrRow = kMaxNbr + 1;

__global__ void __launch_bounds__(kNbrBlock) k_neighbors(Params P) {
  __shared__ int s_idx[kNbrBlock * kNbrRow];
  __shared__ int s_id[kNbrBlock * kNbrRow];
  int* ri = s_idx + threadIdx.x * kNbrRow;
  int* rd = s_id + threadIdx.x * kNbrRow;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n;
  const int nact = P.cell_start[P.n_cells];
  if (q >= nact) {
    if (q < n) P.nbr_cnt[q] = 0;
    return;
  }
  const int nxt = P.ctl->cur ^ 1, sb1 = P.ctl->sbuf ^ 1;
  const double* X = P.x[nxt];
  const float4* SH = P.shadow[nxt];
  const int* ids = P.id[sb1];
  const double xi = X[q], yi = X[n + q], zi = X[2 * n + q];
  // FP32 decision from the hi parts where it is certain; the exact FP64 test otherwise
  const float4 hi = SH[q];
  const float ai = max_abs3(hi);
  const float rcf = P.f_rc;
  // in a batch, particles of different instances never interact
  const int* inst = P.n_inst > 1 ? P.inst[sb1] : nullptr;
  const int my_inst = inst ? inst[q] : 0;
  const int cx = cell_coord(xi, P.lo[0], P.inv_h[0], P.nc[0]);
  const int cy = cell_coord(yi, P.lo[1], P.inv_h[1], P.nc[1]);
  const int cz = cell_coord(zi, P.lo[2], P.inv_h[2], P.nc[2]);
  int* out = P.nbr + (size_t)q * kMaxNbr;
  int cnt = 0;
  bool overflow = false;
  for (int dz = -1; dz <= 1; dz++) {
    const int z = cz + dz;
    if (z < 0 || z >= P.nc[2]) continue;
    for (int dy = -1; dy <= 1; dy++) {
      const int y = cy + dy;
      if (y < 0 || y >= P.nc[1]) continue;
      for (int dx = -1; dx <= 1; dx++) {
        const int x = cx + dx;
        if (x < 0 || x >= P.nc[0]) continue;
        const int c = cell_index(P.nc, P.cell_tile_shift, x, y, z);
        const int b = P.cell_start[c], e = P.cell_start[c + 1];
        for (int j = b; j < e; j++) {
          if (j == q) continue;
          if (inst && inst[j] != my_inst) continue;
          const float4 hj = SH[j];
          const float ex = hj.x - hi.x, ey = hj.y - hi.y, ez = hj.z - hi.z;
          const float d2 = ex * ex + ey * ey + ez * ez;
          const float err = hi_distance_error(ai, max_abs3(hj), 2.0f * rcf) + rcf * 1.2e-7f;
          const float lo = fmaxf(rcf - err, 0.0f), up = rcf + err;
          bool inside;
          if (d2 < lo * lo * (1.0f - 1e-6f)) inside = true;
          else if (d2 > up * up * (1.0f + 1e-6f)) inside = false;
          else inside = sqdist_exact(xi, yi, zi, X[j], X[n + j], X[2 * n + j]) < P.rc2;
          if (inside) {
            if (cnt < kMaxNbr) {
              // insertion by partner id keeps the list ordered as a serial pair loop
              const int idj = ids[j];
              int k = cnt - 1;
              while (k >= 0 && rd[k] > idj) {
                ri[k + 1] = ri[k];
                rd[k + 1] = rd[k];
                k--;
              }
              ri[k + 1] = j;
              rd[k + 1] = idj;
              cnt++;
            } else {
              overflow = true;
            }
          }
        }
      }
    }
  }
  int nlo = 0;   // the list is ordered by partner id: its partners of smaller id lead
  for (int k = 0; k < cnt; k++) {
    out[k] = ri[k];
    nlo += rd[k] < ids[q] ? 1 : 0;
  }
  P.nbr_cnt[q] = cnt;
  P.nbr_lo[q] = (uint8_t)nlo;
  if (overflow) atomicOr(&P.ctl->status, kStCapacity);
  // one atomic per warp for the search statistics (not two per particle on two words)
  const unsigned act = __activemask();
  const unsigned wmax = __reduce_max_sync(act, (unsigned)(cnt + (overflow ? 1 : 0)));
  const unsigned wsum = __reduce_add_sync(act, (unsigned)cnt);
  if ((threadIdx.x & 31) == __ffs(act) - 1) {
    atomicMax(&P.ctl->max_nbr_seen, (int)wmax);
    atomicAdd(&P.ctl->n_pairs_dir, (unsigned long long)wsum);
  }
}

// ------------------------------------------------------------------ 5. restore history
__global__ void k_hist_load(Params P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n;
  if (q >= n) return;
  const Control* C = P.ctl;
  const int nact = P.cell_start[P.n_cells];
  const int hn = C->hc ^ 1, sb1 = C->sbuf ^ 1;
  if (q >= nact) {
    P.mask[0][q] = 0ull;
    P.mask[1][q] = 0ull;
    return;
  }
  const int* ids = P.id[sb1];
  const int a = ids[q];
  const int* nb = P.nbr + (size_t)q * kMaxNbr;
  const int cnt = P.nbr_cnt[q];
  double* H = P.hist[hn] + (size_t)q;
  unsigned long long m = 0ull;
  int rank = 0;
  // Only pairs that touch now can keep an overlap: the first force evaluation after this
  // search drops the others.  The FP32 test below is widened by its error bound, so it
  // never skips a touching pair.
  const float4* SH = P.shadow[C->cur ^ 1];
  const float4 hi = SH[q];
  const float ai = max_abs3(hi);
  for (int k = 0; k < cnt; k++) {
    const int j = nb[k];
    const float4 hj = SH[j];
    const float ex = hj.x - hi.x, ey = hj.y - hi.y, ez = hj.z - hi.z;
    const float reach = hi.w + hj.w;
    const float up = reach + hi_distance_error(ai, max_abs3(hj), 2.0f * reach);
    if (ex * ex + ey * ey + ez * ez > up * up * (1.0f + 1e-6f)) continue;
    const int b = ids[j];
    if (P.pair_once && b < a) continue;   // one evaluation per pair: the owner keeps the overlap
    const unsigned long long key = pair_key(a, b);
    unsigned h = hash_slot(key, P.hcap_mask);
    for (unsigned probe = 0; probe <= P.hcap_mask; probe++) {
      const unsigned long long kk = P.hkey[h];
      if (kk == kEmptyKey) break;
      if (kk == key) {
        if (rank < kHistStride) {
          const double sg = a < b ? 1.0 : -1.0;
          H[hcomp(P.n, rank, 0)] = sg * P.hval[3 * (size_t)h];
          H[hcomp(P.n, rank, 1)] = sg * P.hval[3 * (size_t)h + 1];
          H[hcomp(P.n, rank, 2)] = sg * P.hval[3 * (size_t)h + 2];
          m |= 1ull << k;
          rank++;
        } else {
          atomicOr(&P.ctl->status, kStCapacity);
        }
        break;
      }
      h = (h + 1) & P.hcap_mask;
    }
  }
  const uint8_t wm = P.wall_tmp_mask[a];
  for (int w = 0; w < kMaxWalls; w++) {
    if (!((wm >> w) & 1u)) continue;
    if (rank < kHistStride) {
      const double* src = P.wall_tmp + ((size_t)a * kMaxWalls + w) * 3;
      H[hcomp(P.n, rank, 0)] = src[0];
      H[hcomp(P.n, rank, 1)] = src[1];
      H[hcomp(P.n, rank, 2)] = src[2];
      m |= 1ull << (kMaxNbr + w);
      rank++;
    } else {
      atomicOr(&P.ctl->status, kStCapacity);
    }
  }
  P.mask[hn][q] = m;
}

// ------------------------------------------------------------------ 6. inner list (mixed)
// The slots k of each particle's fine-search list whose partner lies within
// R_i + R_j + delta, decided on the FP32 hi parts with the test widened by their error
// bound (so no such pair is dropped), in ascending k, i.e. in partner-id order.  The
// particle's position becomes the reference of the next refresh, stored with its distance
// from the search reference (rounded up): the step kernel bounds a particle's move since
// the search by that distance plus its move since the refresh, and tests the search
// trigger exactly only when the bound comes near skin / 2.
__global__ void k_inner_build(Params P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  Control* C = P.ctl;
  if (blockIdx.x == 0 && threadIdx.x == 0) C->inner_builds++;
  const int n = P.n;
  if (q >= n) return;
  if (q >= C->n_act_sorted) {
    P.inner_cnt[q] = 0;
    return;
  }
  const int cur = C->cur;
  const float4* RD = P.render[cur];
  const float* RAD = P.rad[C->sbuf];
  const float4 q0 = RD[3 * (size_t)q], q1 = RD[3 * (size_t)q + 1];
  const float4 hi = make_float4(q0.x, q0.y, q0.z, RAD[q]);
  const float ai = max_abs3(hi);
  const int* nb = P.nbr + (size_t)q * kMaxNbr;
  const int cnt = P.nbr_cnt[q];
  uint8_t* row = P.inner + (size_t)q * kInnerMax;
  int* rowj = P.inner_j + (size_t)q * kInnerMax;
  int m = 0, mlo = 0;
  const int nlo = P.nbr_lo[q];
  bool overflow = false;
  for (int k = 0; k < cnt; k++) {
    const int j = nb[k];
    const float4 hj = RD[3 * (size_t)j];   // x_hi
    if (hj.x == kFar) continue;             // out of the system: never a contact
    const float ex = hj.x - hi.x, ey = hj.y - hi.y, ez = hj.z - hi.z;
    const float reach = hi.w + RAD[j] + P.f_inner_margin;
    const float up = reach + hi_distance_error(ai, max_abs3(hj), 2.0f * reach);
    if (ex * ex + ey * ey + ez * ez > up * up * (1.0f + 1e-6f)) continue;
    if (m < kInnerMax) {
      row[m] = (uint8_t)k;
      rowj[m] = j;
      m++;
      mlo += k < nlo ? 1 : 0;
    } else {
      overflow = true;
    }
  }
  P.inner_cnt[q] = (uint8_t)m;
  if (P.pair_once) P.inner_lo[q] = (uint8_t)mlo;
  if (overflow) atomicOr(&C->status, kStCapacity);
  const float* xr = reinterpret_cast<const float*>(P.xref);
  const float h[3] = {hi.x, hi.y, hi.z}, l[3] = {q0.w, q1.x, q1.y};
  float d2 = 0.0f;
  for (int d = 0; d < 3; d++) {
    float s1, t1;
    df_diff(xr[d * n + q], xr[(3 + d) * n + q], h[d], l[d], s1, t1);
    const float u = s1 + t1;
    d2 += u * u;
    P.xin[d * n + q] = h[d];
  }
  P.xin[3 * n + q] = sqrtf(d2) * (1.0f + 1e-5f);
}

// One evaluation per pair: for every slot of a particle's inner list whose pair it owns
// (partner of larger id), the position of the particle in the partner's inner list, where
// the step pushes the reaction; the owned slots are packed from entry 0 as {j, k | m << 8}
// so that the step reads one 8-byte entry per owned pair.  The inner test is symmetric
// (the same FP32 operations on both sides), so the partner's row holds the owner among
// its leading, foreign-owned slots; a row truncated at kInnerMax has already raised the
// capacity error, and a slot whose owner is not found is marked m = 255 and never written.
__global__ void k_inner_mirror(Params P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.ctl->n_act_sorted) return;
  const int cnt = P.inner_cnt[q], lo = P.inner_lo[q];
  const uint8_t* row = P.inner + (size_t)q * kInnerMax;
  const int* rowj = P.inner_j + (size_t)q * kInnerMax;
  int2* ps = P.pslot + q;   // slot-major: entry t at ps[t * n]
  bool missing = false;
  for (int s = lo; s < cnt; s++) {
    const int j = rowj[s];
    const int* pj = P.inner_j + (size_t)j * kInnerMax;
    const int jlo = P.inner_lo[j];
    int m = 255;
    for (int t = 0; t < jlo; t++)
      if (pj[t] == q) {
        m = t;
        break;
      }
    missing |= m == 255;
    ps[(size_t)(s - lo) * P.n] = make_int2(j, (int)row[s] | (m << 8));
  }
  if (missing) atomicOr(&P.ctl->status, kStCapacity);
}

void launch_inner(const Params& P, cudaStream_t s) {
  if (P.precision != DEM_PRECISION_MIXED) return;
  const int T = 256;
  k_inner_build<<<(P.n + T - 1) / T, T, 0, s>>>(P);
  if (P.pair_once) k_inner_mirror<<<(P.n + T - 1) / T, T, 0, s>>>(P);
}

__global__ void k_rebuild_begin(Params P) {
  Control* C = P.ctl;
  C->max_nbr_seen = 0;
  C->n_pairs_dir = 0ull;
}

__global__ void k_rebuild_end(Params P) {
  Control* C = P.ctl;
  C->cur ^= 1;
  C->sbuf ^= 1;
  C->hc ^= 1;
  C->n_act_sorted = P.cell_start[P.n_cells];
  C->need_rebuild = 0;
  C->since_rebuild = 0;
  C->rebuilds++;
  C->hist_preloaded = 0;
}

// Clearing of the hash table and the wall scratch runs before k_hist_save; it is
// separate so that dem_set_history can clear, then fill, then mark them preloaded.
__global__ void k_hist_clear(Params P, int force) {
  if (!force && P.ctl->hist_preloaded) return;
  const size_t cap = (size_t)P.hcap_mask + 1;
  for (size_t h = blockIdx.x * (size_t)blockDim.x + threadIdx.x; h < cap; h += (size_t)gridDim.x * blockDim.x)
    P.hkey[h] = kEmptyKey;
  for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < (size_t)P.n;
       a += (size_t)gridDim.x * blockDim.x)
    P.wall_tmp_mask[a] = 0;
}

void launch_hist_clear(const Params& P, cudaStream_t s, int force) {
  k_hist_clear<<<152 * 8, 256, 0, s>>>(P, force);
}

void launch_rebuild(const Params& P, cudaStream_t s) {
  const int T = 256;
  const int nb = (P.n + T - 1) / T;
  k_rebuild_begin<<<1, 1, 0, s>>>(P);
  // 1. the hash table and the wall scratch are cleared unless the caller preloaded them
  //    (dem_set_history clears and fills them itself and sets hist_preloaded)
  launch_hist_clear(P, s, 0);
  k_hist_save<<<nb, T, 0, s>>>(P);
  // 2. counting sort by cell key
  cudaMemsetAsync(P.cell_count, 0, sizeof(int) * (P.n_cells + 1), s);
  k_cell_count<<<nb, T, 0, s>>>(P);
  scan_exclusive_i32(P.cell_count, P.n_cells + 1, P.cell_start, P.scan_tmp, s);
  k_cell_scatter<<<nb, T, 0, s>>>(P);
  k_cell_order<<<nb, T, 0, s>>>(P);
  // 3. permutation
  k_permute<<<nb, T, 0, s>>>(P);
  k_mirror_inactive<<<nb, T, 0, s>>>(P);
  // 4. fine search
  k_neighbors<<<(P.n + kNbrBlock - 1) / kNbrBlock, kNbrBlock, 0, s>>>(P);
  // 5. history
  k_hist_load<<<nb, T, 0, s>>>(P);
  k_rebuild_end<<<1, 1, 0, s>>>(P);
  // 6. the inner list of the mixed path, drawn from the new list
  launch_inner(P, s);
}

}  // namespace demgb
