// dem_static_pairs.cu -- contact search that allocates nothing: dem_find_pairs_static.
//
// For callers that cannot allocate device memory themselves -- an application whose
// device memory is entirely owned by its own pool allocator and refuses foreign
// cudaMalloc calls, or a loop that cannot afford the device-wide synchronisation an
// allocation may cause -- this entry point finds the same pairs as the fine search of a
// context, using only the caller's input and output buffers plus one fixed scratch array
// that is part of the library image.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes (10 MiB): every GPU
// on which the library is loaded holds it until the process exits.  It bounds the
// problem to DEM_STATIC_MAX_PARTICLES particles; grids with more than
// DEM_STATIC_MAX_CELLS cells are coarsened (cells stay at least as large as the cutoff).
// The pair total is counted in 64 bits first; a total above DEM_STATIC_MAX_PAIRS is
// refused before any pair is written, so the 32-bit per-particle offsets never wrap.
// All calls share the array and it keeps the last call's contents: the per-cell counters
// and the pair total are cleared at the start of every call, everything else is
// overwritten before it is read.  Calls whose work overlaps on the GPU (two streams, or
// two host threads) race on the array and must not be issued.
//
// Host code cannot use the array's name as a device address: the first call on each
// device looks the address up with cudaGetSymbolAddress while that device is current,
// and later calls on that device reuse it.  Every call reads the pair total back to the
// host and synchronises its stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/dem.h"
#include "dem_device.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 10u << 20;
constexpr size_t kRegionAlign = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_pair_scratch[kStaticScratchBytes];

struct ScratchLayout {
  size_t count, start, key, local, order, pcount, poff, partials, pairs64, total;
};

constexpr size_t align_up(size_t v) { return (v + kRegionAlign - 1) / kRegionAlign * kRegionAlign; }

constexpr ScratchLayout make_layout(size_t cells, size_t n) {
  ScratchLayout L{};
  size_t o = 0;
  L.count = o;    o = align_up(o + (cells + 1) * 4);
  L.start = o;    o = align_up(o + (cells + 2) * 4);
  L.key = o;      o = align_up(o + n * 4);
  L.local = o;    o = align_up(o + n * 4);
  L.order = o;    o = align_up(o + n * 4);
  L.pcount = o;   o = align_up(o + n * 4);
  L.poff = o;     o = align_up(o + (n + 1) * 4);
  L.partials = o; o = align_up(o + 4096 * 4);
  L.pairs64 = o;  o = align_up(o + 8);
  L.total = o;
  return L;
}
static_assert(make_layout(DEM_STATIC_MAX_CELLS, DEM_STATIC_MAX_PARTICLES).total <= kStaticScratchBytes,
              "static scratch too small for the advertised limits");

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

struct Grid {
  double lo[3], inv_h[3];
  int nc[3];
  int cells;
};

__device__ __forceinline__ int sp_cell(const Grid& g, double xd, int a) {
  return demgb::cell_coord(xd, g.lo[a], g.inv_h[a], g.nc[a]);
}

__global__ void k_sp_key(const double* x, const uint8_t* active, int n, Grid g, int* key, int* local, int* count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int k = g.cells;  // particles out of the system go to the last bucket
  if (!active || active[p]) {
    const int cx = sp_cell(g, x[3 * (size_t)p], 0);
    const int cy = sp_cell(g, x[3 * (size_t)p + 1], 1);
    const int cz = sp_cell(g, x[3 * (size_t)p + 2], 2);
    k = (cz * g.nc[1] + cy) * g.nc[0] + cx;
  }
  key[p] = k;
  local[p] = atomicAdd(&count[k], 1);
}

__global__ void k_sp_scatter(int n, const int* key, const int* local, const int* start, int* order) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  order[start[key[p]] + local[p]] = p;
}

// Each cell's members in increasing particle index, written to `sorted`: the member at
// scatter position s (any order, from the atomics of k_sp_key) goes to the cell start plus
// the number of members with a smaller index.  One thread per particle, so a crowded
// cell costs each of its m members O(m) work -- the same as the pair search over that
// cell -- and no thread ever sorts a whole cell.  The out-of-system bucket is not used.
__global__ void k_sp_rank(int n, int cells, const int* key, const int* start, const int* order, int* sorted) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int p = order[s];
  const int c = key[p];
  if (c >= cells) return;
  const int b = start[c], e = start[c + 1];
  int r = 0;
  for (int t = b; t < e; t++) r += order[t] < p ? 1 : 0;
  sorted[b + r] = p;
}

// Pairs (i, j), i < j, |x_j - x_i|^2 < rc^2 (same rounding as the context's fine search).
// mode 0: count per i, and the 64-bit total; mode 1: write at off[i] (the caller has
// checked that the total, hence every offset, fits in 32 bits).
__global__ void k_sp_pairs(const double* x, const uint8_t* active, int n, Grid g, double rc2, const int* start,
                           const int* order, int* pcount, const int* poff, int* pairs, long long capacity, int mode,
                           unsigned long long* total) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (active && !active[i]) {
    if (mode == 0) pcount[i] = 0;
    return;
  }
  const double xi = x[3 * (size_t)i], yi = x[3 * (size_t)i + 1], zi = x[3 * (size_t)i + 2];
  const int cx = sp_cell(g, xi, 0), cy = sp_cell(g, yi, 1), cz = sp_cell(g, zi, 2);
  long long out = mode == 1 ? poff[i] : 0;
  int c = 0;
  for (int dz = -1; dz <= 1; dz++) {
    const int z = cz + dz;
    if (z < 0 || z >= g.nc[2]) continue;
    for (int dy = -1; dy <= 1; dy++) {
      const int y = cy + dy;
      if (y < 0 || y >= g.nc[1]) continue;
      for (int dx = -1; dx <= 1; dx++) {
        const int xx = cx + dx;
        if (xx < 0 || xx >= g.nc[0]) continue;
        const int cell = (z * g.nc[1] + y) * g.nc[0] + xx;
        for (int s = start[cell]; s < start[cell + 1]; s++) {
          const int j = order[s];
          if (j <= i) continue;
          const double s2 = demgb::sqdist_exact(xi, yi, zi, x[3 * (size_t)j], x[3 * (size_t)j + 1],
                                                x[3 * (size_t)j + 2]);
          if (!(s2 < rc2)) continue;
          if (mode == 1 && out >= 0 && out < capacity) {
            pairs[2 * out] = i;
            pairs[2 * out + 1] = j;
          }
          out++;
          c++;
        }
      }
    }
  }
  if (mode == 0) {
    pcount[i] = c;
    const unsigned act = __activemask();
    const unsigned long long ws = __reduce_add_sync(act, (unsigned)c);
    if ((threadIdx.x & 31) == __ffs(act) - 1 && ws) atomicAdd(total, ws);
  }
}

}  // namespace

extern "C" dem_status dem_find_pairs_static(const double* x, const uint8_t* active, int64_t n, double cutoff,
                                            const double* domain_lo, const double* domain_hi, int32_t* pairs,
                                            int64_t capacity, int64_t* count, void* stream) {
  if (!x || !count || !domain_lo || !domain_hi || n < 0 || capacity < 0 || (capacity > 0 && !pairs))
    return DEM_ERR_ARG;
  if (!(cutoff > 0.0) || !std::isfinite(cutoff)) return DEM_ERR_ARG;
  if (n > DEM_STATIC_MAX_PARTICLES) return DEM_ERR_CAPACITY;
  *count = 0;
  if (n == 0) return DEM_OK;
  // uniform grid with cell edge >= cutoff (1 + 1e-6), at most DEM_STATIC_MAX_CELLS cells
  Grid g;
  const double hmin = cutoff * (1.0 + 1e-6);
  for (int a = 0; a < 3; a++) {
    const double L = domain_hi[a] - domain_lo[a];
    if (!(L > 0.0) || !std::isfinite(L)) return DEM_ERR_ARG;
    g.nc[a] = (int)std::max(1.0, std::min(std::floor(L / hmin), 1.0e6));
  }
  while ((long long)g.nc[0] * g.nc[1] * g.nc[2] > DEM_STATIC_MAX_CELLS)
    for (int a = 0; a < 3; a++) g.nc[a] = std::max(1, (int)(g.nc[a] * 0.9));
  for (int a = 0; a < 3; a++) {
    g.lo[a] = domain_lo[a];
    g.inv_h[a] = (double)g.nc[a] / (domain_hi[a] - domain_lo[a]);
  }
  g.cells = g.nc[0] * g.nc[1] * g.nc[2];

  // device address of the static scratch: looked up once per device, with it current
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DEM_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_pair_scratch) != cudaSuccess || !p) return DEM_ERR_CUDA;
      g_scratch_addr[dev] = (unsigned char*)p;
    }
    base = g_scratch_addr[dev];
  }
  const ScratchLayout L = make_layout((size_t)g.cells, (size_t)n);
  int* cnt = (int*)(base + L.count);
  int* start = (int*)(base + L.start);
  int* key = (int*)(base + L.key);
  int* local = (int*)(base + L.local);
  int* order = (int*)(base + L.order);
  int* pcount = (int*)(base + L.pcount);
  int* poff = (int*)(base + L.poff);
  int* partials = (int*)(base + L.partials);
  unsigned long long* total64 = (unsigned long long*)(base + L.pairs64);
  cudaStream_t s = (cudaStream_t)stream;
  const int T = 256;
  const int nb = (int)((n + T - 1) / T);
  const double rc2 = cutoff * cutoff;

  if (cudaMemsetAsync(cnt, 0, ((size_t)g.cells + 1) * 4, s) != cudaSuccess ||
      cudaMemsetAsync(total64, 0, 8, s) != cudaSuccess)
    return DEM_ERR_CUDA;
  k_sp_key<<<nb, T, 0, s>>>(x, active, (int)n, g, key, local, cnt);
  demgb::scan_exclusive_i32(cnt, g.cells + 1, start, partials, s);
  k_sp_scatter<<<nb, T, 0, s>>>((int)n, key, local, start, order);
  // `local` is free after the scatter: it receives the cell-ordered members
  k_sp_rank<<<nb, T, 0, s>>>((int)n, g.cells, key, start, order, local);
  int* sorted = local;
  k_sp_pairs<<<nb, T, 0, s>>>(x, active, (int)n, g, rc2, start, sorted, pcount, nullptr, nullptr, 0, 0, total64);
  unsigned long long total = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&total, total64, sizeof(total), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DEM_ERR_CUDA;
  *count = (int64_t)total;
  if (total > (unsigned long long)DEM_STATIC_MAX_PAIRS) return DEM_ERR_CAPACITY;   // nothing written
  if (capacity == 0) return DEM_OK;
  demgb::scan_exclusive_i32(pcount, (int)n, poff, partials, s);
  k_sp_pairs<<<nb, T, 0, s>>>(x, active, (int)n, g, rc2, start, sorted, pcount, poff, pairs, capacity, 1, total64);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return DEM_ERR_CUDA;
  return DEM_OK;
}
