// surrogate.cu -- the learned surrogate of the DEM drum (include/surrogate.h): a
// message-passing network on the contact graph, trained and run with BF16 tensor-core
// products (tcgen05 for the 128-wide products of the forward pass and the data gradients,
// mma.sync m16n8k16 for the rest; FP32 accumulation) and deterministic segment sums.
//
// The other products -- the weight gradients, where the long dimension (edges or nodes) is
// the reduction, and the decoder's 8-wide ones -- go through one tiled mma.sync GEMM kernel
// whose A operand is read through an accessor: the concatenation [S0[g(r)] | S1[r]] of two
// BF16 row blocks (g an optional row gather), either as A or transposed (weight gradients,
// split over blocks with FP32 partial sums reduced in a fixed order).  Aggregations over the receiver-sorted CSR are segment sums, so
// forward and backward results do not depend on thread timing (no float atomics).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/surrogate.h"
#include "surrogate_tc.cuh"

namespace {

constexpr int H = SURR_HIDDEN;
constexpr int FIN = SURR_NODE_IN;
constexpr int EIN = SURR_EDGE_IN;
constexpr int NOUT = SURR_OUT;
constexpr int kSplit = 64;   // reduction chunks of a weight-gradient product
constexpr float kAgg = SURR_AGG_SCALE;

__device__ float g_mse_part[256];   // partial sums of surr_mse (one call at a time per device)

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------ parameters
struct Layout {
  int64_t W[6], b[6], total;
  int in[6], out[6];
};

Layout make_layout() {
  Layout L;
  const int ins[6] = {FIN, H + EIN, 2 * H, 2 * H, 2 * H, H};
  const int outs[6] = {H, H, H, H, H, NOUT};
  int64_t o = 0;
  for (int l = 0; l < 6; l++) {
    L.in[l] = ins[l];
    L.out[l] = outs[l];
    L.W[l] = o;
    o += (int64_t)ins[l] * outs[l];
    L.b[l] = o;
    o += outs[l];
  }
  L.total = o;
  return L;
}

// ------------------------------------------------------------------ operand accessors
// A(m, k) of an [M][K] operand that is the concatenation [S0[g0(m)] (w0 columns) | S1[m]].
struct CatA {
  const bf16* s0;
  const int* g0;   // row gather of S0 (null: identity)
  int w0;
  const bf16* s1;  // null if w0 == K
  int w1;
  __device__ __forceinline__ bf16 at(int64_t m, int k) const {
    if (k < w0) {
      const int64_t r = g0 ? g0[m] : m;
      return s0[r * w0 + k];
    }
    return s1[m * w1 + (k - w0)];
  }
};

// B(k, n): a row-major [K][N] matrix (trans = 0) or the transpose of a row-major [N][K] one.
struct MatB {
  const bf16* p;
  int ld;
  int trans;
  __device__ __forceinline__ bf16 at(int64_t k, int64_t n) const { return trans ? p[n * ld + k] : p[k * ld + n]; }
};

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------------------ the GEMM kernel
// C = opA(A) B over the reduction range [r0, r1) of the k index, block tile 64 x 64, k step
// 16, 4 warps of 32 x 32.  transA: opA(A)(m, k) = A(k, m) (A read through CatA with its
// row index k), used for weight gradients, where the reduction runs over the rows of A.
// Out-of-range rows and columns are read as zero and not written.
constexpr int BM = 64, BN = 64, BK = 16;

template <bool kTransA>
__global__ void __launch_bounds__(128) k_gemm(CatA A, MatB B, int64_t M, int64_t N, int64_t K, int64_t kchunk,
                                              float* C, int64_t ldc) {
  __shared__ bf16 As[BM][BK + 2];
  __shared__ bf16 Bs[BK][BN + 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int64_t k_lo = (int64_t)blockIdx.z * kchunk;
  const int64_t k_hi = k_lo + kchunk < K ? k_lo + kchunk : K;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 4; j++)
      for (int q = 0; q < 4; q++) acc[i][j][q] = 0.0f;
  const bf16 zero = __float2bfloat16(0.0f);
  for (int64_t k0 = k_lo; k0 < k_hi; k0 += BK) {
    // A tile [64][16] and B tile [16][64]: 1024 elements each, 8 per thread
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = e / BK, c = e % BK;
      const int64_t m = m0 + r, k = k0 + c;
      bf16 v = zero;
      if (m < M && k < k_hi) v = kTransA ? A.at(k, (int)m) : A.at(m, (int)k);
      As[r][c] = v;
    }
    for (int e = tid; e < BK * BN; e += 128) {
      const int r = e / BN, c = e % BN;
      const int64_t k = k0 + r, n = n0 + c;
      Bs[r][c] = (k < k_hi && n < N) ? B.at(k, n) : zero;
    }
    __syncthreads();
    const int g = lane >> 2, t = lane & 3;
    uint32_t a[2][4], b[4][2];
    for (int i = 0; i < 2; i++) {
      const int r = wm + i * 16 + g;
      a[i][0] = pack2(As[r][2 * t], As[r][2 * t + 1]);
      a[i][1] = pack2(As[r + 8][2 * t], As[r + 8][2 * t + 1]);
      a[i][2] = pack2(As[r][2 * t + 8], As[r][2 * t + 9]);
      a[i][3] = pack2(As[r + 8][2 * t + 8], As[r + 8][2 * t + 9]);
    }
    for (int j = 0; j < 4; j++) {
      const int c = wn + j * 8 + g;
      b[j][0] = pack2(Bs[2 * t][c], Bs[2 * t + 1][c]);
      b[j][1] = pack2(Bs[2 * t + 8][c], Bs[2 * t + 9][c]);
    }
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 4; j++) mma16816(acc[i][j], a[i], b[j]);
    __syncthreads();
  }
  // C (or this split's partial) rows m, columns n
  float* Cz = C + (int64_t)blockIdx.z * M * ldc;
  const int g = lane >> 2, t = lane & 3;
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 4; j++)
      for (int q = 0; q < 4; q++) {
        const int64_t m = m0 + wm + i * 16 + g + (q >= 2 ? 8 : 0);
        const int64_t n = n0 + wn + j * 8 + 2 * t + (q & 1);
        if (m < M && n < N) Cz[m * ldc + n] = acc[i][j][q];
      }
}

// ------------------------------------------------------------------ elementwise kernels
// z = C + bias; u = relu(z) (or z when relu = 0); out = (res ? res + u : u).  Writes u and
// out in BF16 (either may be null) and out in FP32 when outf is given.
__global__ void k_epilogue(const float* C, const float* bias, int64_t M, int N, int relu, const bf16* res, bf16* u_out,
                           bf16* out, float* outf) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int n = (int)(e % N);
  float z = C[e] + bias[n];
  const float u = relu ? fmaxf(z, 0.0f) : z;
  const float o = res ? __bfloat162float(res[e]) + u : u;
  if (u_out) u_out[e] = __float2bfloat16(u);
  if (out) out[e] = __float2bfloat16(o);
  if (outf) outf[e] = o;
}

// Y = h W5 + b5 for the 8 outputs: one thread per row, W5 (128 x 8) in shared memory, FP32
// accumulation.  Eight columns are too narrow for a tensor-core tile.
__global__ void __launch_bounds__(128) k_decoder(const bf16* h, const bf16* W, const float* b, int64_t n, float* Y) {
  __shared__ float Ws[H * NOUT];
  for (int e = threadIdx.x; e < H * NOUT; e += blockDim.x) Ws[e] = __bfloat162float(W[e]);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc[NOUT];
  for (int o = 0; o < NOUT; o++) acc[o] = b[o];
  const uint4* hr = reinterpret_cast<const uint4*>(h + i * H);
  for (int q = 0; q < H / 8; q++) {
    const uint4 u = hr[q];
    const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
    for (int p2 = 0; p2 < 4; p2++) {
      const int k = 8 * q + 2 * p2;
      const float x0 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w4[p2] & 0xFFFFu)));
      const float x1 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w4[p2] >> 16)));
      for (int o = 0; o < NOUT; o++) acc[o] = fmaf(x1, Ws[(k + 1) * NOUT + o], fmaf(x0, Ws[k * NOUT + o], acc[o]));
    }
  }
  float4* yo = reinterpret_cast<float4*>(Y + i * NOUT);
  yo[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  yo[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

// The same for a count that is a multiple of 8, 8 values per thread (16-byte stores).
__global__ void k_to_bf16_x8(const float4* src, uint4* dst, int64_t count8) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count8) return;
  const float4 a = src[2 * e], b = src[2 * e + 1];
  auto pk = [](float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(hi)) << 16);
  };
  dst[e] = make_uint4(pk(a.x, a.y), pk(a.z, a.w), pk(b.x, b.y), pk(b.z, b.w));
}

__global__ void k_to_bf16(const float* src, bf16* dst, int64_t count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) dst[e] = __float2bfloat16(src[e]);
}

// out[i] = sum over the CSR row i of src[g(e)] (g = col for a neighbour sum, the edge
// itself for an edge sum), source rows ld_src apart; FP32 accumulation in row order; one
// warp per row, 4 of the H columns per lane.  Writes BF16 and/or FP32 (adding to the FP32
// output when `accumulate` is set), times `scale` (SURR_AGG_SCALE for the network's sums).
__global__ void k_segsum(const int* row_ptr, const int* col, const bf16* src_b, const float* src_f, int64_t ld_src,
                         int64_t n, bf16* out_b, float* out_f, int accumulate, float scale) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  float s[4] = {0.f, 0.f, 0.f, 0.f};
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
    const int64_t r = col ? col[e] : e;
    for (int q = 0; q < 4; q++) {
      const int64_t idx = r * ld_src + lane * 4 + q;
      s[q] += src_b ? __bfloat162float(src_b[idx]) : src_f[idx];
    }
  }
  for (int q = 0; q < 4; q++) {
    const int64_t idx = i * H + lane * 4 + q;
    const float v = scale * s[q];
    if (out_b) out_b[idx] = __float2bfloat16(v);
    if (out_f) out_f[idx] = accumulate ? out_f[idx] + v : v;
  }
}

// dz[e][h] = da[recv[e]][h] * relu'(u[e][h] > 0): the gradient of the edge messages (each
// message enters only the sum at its receiver)
__global__ void k_gather_mask(const float* da, const int32_t* recv, const bf16* u, int64_t nE, bf16* dz_b,
                              float* dz_f) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE * H) return;
  const int64_t m = e / H;
  const int h = (int)(e % H);
  float d = kAgg * da[(int64_t)recv[m] * H + h];
  if (!(__bfloat162float(u[e]) > 0.0f)) d = 0.0f;
  dz_b[e] = __float2bfloat16(d);
  dz_f[e] = d;
}

// dz = dout * relu'(u > 0) (u is the stored activation), in BF16 for the next product and
// FP32 for the bias gradient.  cols: width of dout rows; dout may have a row stride.
__global__ void k_relu_back(const float* dout, int64_t ld_dout, const bf16* u, int64_t M, int N, int relu,
                            bf16* dz_b, float* dz_f) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int64_t m = e / N;
  const int n = (int)(e % N);
  float d = dout[m * ld_dout + n];
  if (relu && !(__bfloat162float(u[e]) > 0.0f)) d = 0.0f;
  dz_b[e] = __float2bfloat16(d);
  dz_f[e] = d;
}

// dst[m][n] += src[m * lds + n] for the first N columns (FP32)
// Block c0 of W^T for a data gradient: Wt[c][j] = W[c0 + j][c], W row-major [K][H] (rows
// c0 .. c0 + H - 1 used), so that dz Wt is columns c0 .. c0 + H - 1 of dz W^T.
__global__ void k_wt_block(const bf16* W, int c0, bf16* Wt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= H * H) return;
  const int c = t / H, j = t % H;
  Wt[t] = W[(int64_t)(c0 + j) * H + c];
}

__global__ void k_add_cols(float* dst, const float* src, int64_t lds, int64_t M, int N) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int64_t m = e / N;
  const int n = (int)(e % N);
  dst[e] += src[m * lds + n];
}

// out[k][n] = sum over the splits of part[z][k][n] (fixed order)
__global__ void k_reduce_splits(const float* part, int splits, int64_t count, float* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  float s = 0.0f;
  for (int z = 0; z < splits; z++) s += part[(int64_t)z * count + e];
  out[e] = s;
}

// column sums of an [M][N] FP32 matrix (bias gradients): one block per column, fixed tree
__global__ void k_colsum(const float* a, int64_t M, int N, float* out) {
  __shared__ float sh[256];
  const int n = blockIdx.x;
  float s = 0.0f;
  for (int64_t m = threadIdx.x; m < M; m += blockDim.x) s += a[m * N + n];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = sh[0];
}

__global__ void k_mse(const float* Y, const float* T, const float* w, int64_t n, float* part, float* dY) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NOUT; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % NOUT);
    float d = 0.0f;
    if (c < 6) {
      const float r = Y[e] - T[(e / NOUT) * 6 + c];
      s += w[c] * r * r;
      d = 2.0f * w[c] * r / (float)(n * 6);
    }
    dY[e] = d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mse_final(const float* part, int nb, int64_t n, float* loss) {
  float s = 0.0f;
  for (int b = 0; b < nb; b++) s += part[b];
  *loss = s / (float)(n * 6);
}

__global__ void k_adam(float* p, bf16* pb, const float* g, float* m, float* v, int64_t count, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.0f - b1) * gi;
  const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[e] -= upd;
  pb[e] = __float2bfloat16(p[e]);
}

// CSR of an undirected graph from pairs (i < j): count, scan, fill (rows sorted by sender)
__global__ void k_csr_count(const int32_t* pairs, int64_t np, int32_t* deg) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  atomicAdd(&deg[pairs[2 * k]], 1);
  atomicAdd(&deg[pairs[2 * k + 1]], 1);
}

__global__ void k_scan_serial_blocks(const int32_t* deg, int64_t n, int32_t* row_ptr) {
  // one block: row_ptr = exclusive scan of deg (n + 1 entries), chunked per thread
  __shared__ int32_t part[1024];
  const int T = blockDim.x;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t lo = threadIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  int32_t s = 0;
  for (int64_t i = lo; i < hi; i++) s += deg[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int t = 0; t < T; t++) {
      const int32_t v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int32_t run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; i++) {
    row_ptr[i] = run;
    run += deg[i];
  }
  if (hi == n && lo < hi) row_ptr[n] = run;
  if (n == 0 && threadIdx.x == 0) row_ptr[0] = 0;
}

__global__ void k_csr_fill(const int32_t* pairs, int64_t np, const int32_t* row_ptr, int32_t* fill, int32_t* col) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int32_t a = pairs[2 * k], b = pairs[2 * k + 1];
  col[row_ptr[a] + atomicAdd(&fill[a], 1)] = b;
  col[row_ptr[b] + atomicAdd(&fill[b], 1)] = a;
}

// each row in increasing sender order, so the sums do not depend on the atomic order above
__global__ void k_csr_sort_rows(const int32_t* row_ptr, int64_t n, int32_t* col) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = row_ptr[i] + 1; a < row_ptr[i + 1]; a++) {
    const int32_t v = col[a];
    int k = a - 1;
    while (k >= row_ptr[i] && col[k] > v) {
      col[k + 1] = col[k];
      k--;
    }
    col[k + 1] = v;
  }
}

__global__ void k_receivers(const int32_t* row_ptr, int64_t n, int32_t* recv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) recv[e] = (int32_t)i;
}

// ------------------------------------------------------------------ workspace
struct WS {
  bf16 *Xb, *Eb, *h0, *u1, *a, *u2, *h1, *s1, *u3, *h2, *s2, *u4, *h3;
  bf16 *dzb;     // [max(nE, n)][H]
  float *C;      // [max(nE, n)][2H] FP32 product / gradient scratch
  float *dzf;    // [max(nE, n)][H]
  float *dh;     // [n][H]
  float *dh2;    // [n][H]
  float *part;   // [kSplit][2H][H]
  bf16 *wt;      // [7][H][H] transposed weight blocks of the data gradients (layers 4, 3, 2: two each; 1: one)
  int32_t* recv; // [nE]
  float* mse;    // [1024]
  size_t total;
};

size_t al(size_t v) { return (v + 255) / 256 * 256; }

WS layout_ws(char* base, int64_t n, int64_t nE) {
  WS w;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = al(o + bytes);
    return base ? base + r : nullptr;
  };
  const int64_t mx = nE > n ? nE : n;
  w.Xb = (bf16*)take(n * FIN * 2);
  w.Eb = (bf16*)take(nE * EIN * 2);
  w.h0 = (bf16*)take(n * H * 2);
  w.u1 = (bf16*)take(nE * H * 2);
  w.a = (bf16*)take(n * H * 2);
  w.u2 = (bf16*)take(n * H * 2);
  w.h1 = (bf16*)take(n * H * 2);
  w.s1 = (bf16*)take(n * H * 2);
  w.u3 = (bf16*)take(n * H * 2);
  w.h2 = (bf16*)take(n * H * 2);
  w.s2 = (bf16*)take(n * H * 2);
  w.u4 = (bf16*)take(n * H * 2);
  w.h3 = (bf16*)take(n * H * 2);
  w.dzb = (bf16*)take(mx * H * 2);
  w.C = (float*)take(mx * 2 * H * 4);
  w.dzf = (float*)take(mx * H * 4);
  w.dh = (float*)take(n * H * 4);
  w.dh2 = (float*)take(n * H * 4);
  w.part = (float*)take((size_t)kSplit * 2 * H * H * 4);
  w.wt = (bf16*)take((size_t)7 * H * H * 2);
  w.recv = (int32_t*)take(nE * 4);
  w.mse = (float*)take(1024 * 4);
  w.total = o;
  return w;
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// C[M][N] = opA(A) B: full product (kTransA false) or a weight gradient (true, M = width of
// A's columns, K = rows of A, reduced over kSplit chunks into out).
void gemm(const CatA& A, const MatB& B, int64_t M, int64_t N, int64_t K, float* C, cudaStream_t s) {
  dim3 grid(nblk(N, BN), nblk(M, BM), 1);
  k_gemm<false><<<grid, 128, 0, s>>>(A, B, M, N, K, K, C, N);
}

void gemm_wgrad(const CatA& A, const MatB& B, int64_t M, int64_t N, int64_t K, float* part, float* out,
                cudaStream_t s) {
  int64_t chunk = (K + kSplit - 1) / kSplit;
  chunk = (chunk + BK - 1) / BK * BK;
  const int splits = (int)((K + chunk - 1) / chunk);
  dim3 grid(nblk(N, BN), nblk(M, BM), splits > 0 ? splits : 1);
  k_gemm<true><<<grid, 128, 0, s>>>(A, B, M, N, K, chunk, part, N);
  k_reduce_splits<<<nblk(M * N, 256), 256, 0, s>>>(part, splits > 0 ? splits : 1, M * N, out);
}

// ------------------------------------------------------------------ features and rollout
// geometry g: {cx, y0, cz, Rd, L, d0, vs, 0}: drum axis along y through (cx, cz) from y0 to
// y0 + L, radius Rd; d0 the length scale (largest diameter), vs the velocity scale.
__global__ void k_node_features(const double* x, const double* v, const double* w, const float* rad, int64_t n,
                                const double* g, float* X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double cx = g[0], y0 = g[1], cz = g[2], Rd = g[3], L = g[4], d0 = g[5], vs = g[6];
  const double R = rad[i];
  const double px = x[3 * i] - cx, py = x[3 * i + 1] - y0, pz = x[3 * i + 2] - cz;
  const double rho = sqrt(px * px + pz * pz);
  float* o = X + i * FIN;
  for (int d = 0; d < 3; d++) {
    o[d] = (float)(v[3 * i + d] / vs);
    o[3 + d] = (float)(w[3 * i + d] * R / vs);
  }
  o[6] = (float)(2.0 * R / d0);
  o[7] = (float)(px / Rd);
  o[8] = (float)(pz / Rd);
  o[9] = (float)(py / L - 0.5);
  o[10] = (float)fmin(fmax((Rd - rho) / d0, 0.0), 5.0);
  o[11] = (float)fmin(fmax(fmin(py, L - py) / d0, 0.0), 5.0);
  o[12] = 1.0f;
  o[13] = o[14] = o[15] = 0.0f;
}

__global__ void k_edge_features(const double* x, const double* v, const double* w, const float* rad,
                                const int32_t* recv, const int32_t* col, int64_t nE, const double* g, float* E) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  const double d0 = g[5], vs = g[6];
  const int64_t i = recv[e], j = col[e];
  double dx[3], r2 = 0.0;
  for (int d = 0; d < 3; d++) {
    dx[d] = x[3 * j + d] - x[3 * i + d];
    r2 += dx[d] * dx[d];
  }
  const double r = sqrt(r2);
  float* o = E + e * EIN;
  for (int d = 0; d < 3; d++) {
    o[d] = (float)(dx[d] / d0);
    o[5 + d] = (float)((v[3 * j + d] - v[3 * i + d]) / vs);
    o[8 + d] = (float)((w[3 * j + d] * rad[j] - w[3 * i + d] * rad[i]) / vs);
  }
  o[3] = (float)(r / d0);
  o[4] = (float)(100.0 * fmax((double)rad[i] + (double)rad[j] - r, 0.0) / d0);   // overlap, in 0.01 d0
  for (int d = 11; d < EIN; d++) o[d] = 0.0f;
}

// targets: the velocity and spin increments over the k steps, scaled like the outputs
__global__ void k_targets(const double* v0, const double* w0, const double* v1, const double* w1, const float* rad,
                          int64_t n, const double* g, const float* sc, float* T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double vs = g[6], R = rad[i];
  for (int d = 0; d < 3; d++) {
    T[6 * i + d] = (float)((v1[3 * i + d] - v0[3 * i + d]) / vs / sc[d]);
    T[6 * i + 3 + d] = (float)((w1[3 * i + d] - w0[3 * i + d]) * R / vs / sc[3 + d]);
  }
}

// one surrogate step of k DEM steps: v += dv, w += dw, x += (v_old + v_new) / 2 * k dt
__global__ void k_apply(double* x, double* v, double* w, const float* rad, int64_t n, const float* Y, const double* g,
                        const float* sc, double kdt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double vs = g[6], R = rad[i];
  for (int d = 0; d < 3; d++) {
    const double dv = (double)Y[NOUT * i + d] * sc[d] * vs;
    const double dw = (double)Y[NOUT * i + 3 + d] * sc[3 + d] * vs / R;
    const double vo = v[3 * i + d];
    v[3 * i + d] = vo + dv;
    w[3 * i + d] += dw;
    x[3 * i + d] += 0.5 * (vo + v[3 * i + d]) * kdt;
  }
}

}  // namespace

// ================================================================== C ABI
extern "C" int surr_params(surr_param_layout* out) {
  if (!out) return 1;
  const Layout L = make_layout();
  for (int l = 0; l < 6; l++) {
    out->W[l] = L.W[l];
    out->b[l] = L.b[l];
  }
  out->total = L.total;
  return 0;
}

extern "C" int surr_workspace_bytes(int64_t n, int64_t n_edges, size_t* bytes) {
  if (!bytes || n < 0 || n_edges < 0) return 1;
  *bytes = layout_ws(nullptr, n, n_edges).total + 256;
  return 0;
}

extern "C" int surr_build_csr(const int32_t* pairs, int64_t n_pairs, int64_t n, int32_t* row_ptr, int32_t* col,
                              int32_t* scratch, void* stream) {
  if (n < 0 || n_pairs < 0 || !row_ptr || !scratch || (n_pairs > 0 && (!pairs || !col))) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* deg = scratch;
  int32_t* fill = scratch + n + 1;
  if (cudaMemsetAsync(deg, 0, (size_t)(2 * n + 1) * 4, s) != cudaSuccess) return 2;
  if (n_pairs > 0) k_csr_count<<<nblk(n_pairs, 256), 256, 0, s>>>(pairs, n_pairs, deg);
  k_scan_serial_blocks<<<1, 1024, 0, s>>>(deg, n, row_ptr);
  if (n_pairs > 0) {
    k_csr_fill<<<nblk(n_pairs, 256), 256, 0, s>>>(pairs, n_pairs, row_ptr, fill, col);
    k_csr_sort_rows<<<nblk(n, 256), 256, 0, s>>>(row_ptr, n, col);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_params_to_bf16(const float* params, void* params_bf16, int64_t count, void* stream) {
  if (!params || !params_bf16 || count < 0) return 1;
  k_to_bf16<<<nblk(count, 256), 256, 0, (cudaStream_t)stream>>>(params, (bf16*)params_bf16, count);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_forward(const void* params_bf16, const float* params, const float* X, const float* E,
                            const int32_t* row_ptr, const int32_t* col, int64_t n, int64_t nE, void* workspace,
                            float* Y, void* stream) {
  if (!params_bf16 || !params || !X || !row_ptr || !workspace || !Y || n <= 0 || nE < 0 || (nE > 0 && (!E || !col)))
    return 1;
  if (((uintptr_t)X & 15u) || (nE > 0 && ((uintptr_t)E & 15u)) || ((uintptr_t)Y & 15u)) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = make_layout();
  const bf16* Pb = (const bf16*)params_bf16;
  char* base = (char*)(((uintptr_t)workspace + 255) / 256 * 256);
  WS w = layout_ws(base, n, nE);
  const int T = 256;
  k_to_bf16_x8<<<nblk(n * FIN / 8, T), T, 0, s>>>((const float4*)X, (uint4*)w.Xb, n * FIN / 8);
  if (nE > 0) k_to_bf16_x8<<<nblk(nE * EIN / 8, T), T, 0, s>>>((const float4*)E, (uint4*)w.Eb, nE * EIN / 8);
  k_receivers<<<nblk(n, T), T, 0, s>>>(row_ptr, n, w.recv);
  // node encoder and the 128-wide layers on the tensor cores (tcgen05), epilogues fused
  const bf16* W = Pb;
  auto tc = [&](const bf16* s0, const int32_t* g0, int w0, const bf16* s1, int w1, int l, const bf16* res,
                bf16* u_out, bf16* out, int64_t M) {
    surrtc::Args a{s0, g0, w0, s1, w1, W + L.W[l], params + L.b[l], 1, res, u_out, out, nullptr, M};
    return surrtc::launch(a, s);
  };
  bool ok = tc(w.Xb, nullptr, FIN, nullptr, 0, 0, nullptr, nullptr, w.h0, n);
  // edge messages and their sum at each receiver
  if (nE > 0) ok = ok && tc(w.h0, w.recv, H, w.Eb, EIN, 1, nullptr, nullptr, w.u1, nE);
  k_segsum<<<nblk(n * 32, T), T, 0, s>>>(row_ptr, nullptr, w.u1, nullptr, H, n, w.a, nullptr, 0, kAgg);
  ok = ok && tc(w.h0, nullptr, H, w.a, H, 2, w.h0, w.u2, w.h1, n);
  // two node layers on neighbour sums
  k_segsum<<<nblk(n * 32, T), T, 0, s>>>(row_ptr, col, w.h1, nullptr, H, n, w.s1, nullptr, 0, kAgg);
  ok = ok && tc(w.h1, nullptr, H, w.s1, H, 3, w.h1, w.u3, w.h2, n);
  k_segsum<<<nblk(n * 32, T), T, 0, s>>>(row_ptr, col, w.h2, nullptr, H, n, w.s2, nullptr, 0, kAgg);
  ok = ok && tc(w.h2, nullptr, H, w.s2, H, 4, w.h2, w.u4, w.h3, n);
  if (!ok) return 2;
  // decoder
  k_decoder<<<nblk(n, 128), 128, 0, s>>>(w.h3, Pb + L.W[5], params + L.b[5], n, Y);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_backward(const void* params_bf16, const float* dY, const int32_t* row_ptr, const int32_t* col,
                             int64_t n, int64_t nE, void* workspace, float* grad, void* stream) {
  if (!params_bf16 || !dY || !row_ptr || !workspace || !grad || n <= 0 || nE < 0 || (nE > 0 && !col)) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = make_layout();
  const bf16* Pb = (const bf16*)params_bf16;
  char* base = (char*)(((uintptr_t)workspace + 255) / 256 * 256);
  WS w = layout_ws(base, n, nE);
  const int T = 256;
  // ---- decoder, Y = h3 W5 + b5: dW5 = h3^T dY, db5, dh3 = dY W5^T
  k_relu_back<<<nblk(n * NOUT, T), T, 0, s>>>(dY, NOUT, nullptr, n, NOUT, 0, w.dzb, w.dzf);
  gemm_wgrad(CatA{w.h3, nullptr, H, nullptr, 0}, MatB{w.dzb, NOUT, 0}, H, NOUT, n, w.part, grad + L.W[5], s);
  k_colsum<<<NOUT, 256, 0, s>>>(w.dzf, n, NOUT, grad + L.b[5]);
  gemm(CatA{w.dzb, nullptr, NOUT, nullptr, 0}, MatB{Pb + L.W[5], NOUT, 1}, n, H, NOUT, w.dh, s);
  // The data gradients dz W^T of the 128-wide layers run on the tensor cores (the forward
  // pass's tcgen05 product, no bias and no activation, FP32 out), one 128-column block of
  // W^T at a time: blocks of layers 4, 3, 2 (two each) and 1 (the h0[recv] rows only: the
  // edge features need no gradient).
  const int wt_layer[7] = {4, 4, 3, 3, 2, 2, 1};
  for (int b = 0; b < 7; b++)
    k_wt_block<<<nblk(H * H, T), T, 0, s>>>(Pb + L.W[wt_layer[b]], (b & 1) ? H : 0, w.wt + (size_t)b * H * H);
  auto dgrad = [&](int b, int64_t M, float* out) {
    surrtc::Args a{w.dzb, nullptr, H, nullptr, 0, w.wt + (size_t)b * H * H, nullptr, 0, nullptr, nullptr, nullptr,
                   out, M};
    return surrtc::launch(a, s);
  };
  bool ok = true;
  float* C0 = w.C;                  // [M][H]: columns 0 .. H - 1 of dz W^T
  float* C1 = w.C + (size_t)n * H;  // [n][H]: columns H .. 2H - 1
  // ---- node layers: h_out = h_in + u, u = relu([h_in | s] W + b), s = neighbour sum of h_in
  const bf16* hin[2] = {w.h1, w.h2};
  const bf16* sin[2] = {w.s1, w.s2};
  const bf16* uin[2] = {w.u3, w.u4};
  for (int l = 4; l >= 3; l--) {
    const int q = l - 3;
    k_relu_back<<<nblk(n * H, T), T, 0, s>>>(w.dh, H, uin[q], n, H, 1, w.dzb, w.dzf);
    gemm_wgrad(CatA{hin[q], nullptr, H, sin[q], H}, MatB{w.dzb, H, 0}, 2 * H, H, n, w.part, grad + L.W[l], s);
    k_colsum<<<H, 256, 0, s>>>(w.dzf, n, H, grad + L.b[l]);
    // d[h_in | s] = dz W^T; dh_in = dh_out + d[:, :H] + (neighbour sum of d[:, H:]) -- the
    // graph is symmetric, so the transpose of the neighbour sum is the neighbour sum
    ok = ok && dgrad(2 * (4 - l), n, C0) && dgrad(2 * (4 - l) + 1, n, C1);
    k_add_cols<<<nblk(n * H, T), T, 0, s>>>(w.dh, C0, H, n, H);
    k_segsum<<<nblk(n * 32, T), T, 0, s>>>(row_ptr, col, nullptr, C1, H, n, nullptr, w.dh, 1, kAgg);
  }
  // ---- layer 2: h1 = h0 + u2, u2 = relu([h0 | a] W2 + b2), a = sum of the edge messages
  k_relu_back<<<nblk(n * H, T), T, 0, s>>>(w.dh, H, w.u2, n, H, 1, w.dzb, w.dzf);
  gemm_wgrad(CatA{w.h0, nullptr, H, w.a, H}, MatB{w.dzb, H, 0}, 2 * H, H, n, w.part, grad + L.W[2], s);
  k_colsum<<<H, 256, 0, s>>>(w.dzf, n, H, grad + L.b[2]);
  ok = ok && dgrad(4, n, C0) && dgrad(5, n, C1);
  k_add_cols<<<nblk(n * H, T), T, 0, s>>>(w.dh, C0, H, n, H);                // dh0 (so far)
  // da = d[:, H:] (dense FP32 copy)
  k_relu_back<<<nblk(n * H, T), T, 0, s>>>(C1, H, nullptr, n, H, 0, w.dzb, w.dh2);
  // ---- layer 1 (edges): u1 = relu([h0[recv] | E] W1 + b1)
  if (nE > 0) {
    k_gather_mask<<<nblk(nE * H, T), T, 0, s>>>(w.dh2, w.recv, w.u1, nE, w.dzb, w.dzf);
    gemm_wgrad(CatA{w.h0, w.recv, H, w.Eb, EIN}, MatB{w.dzb, H, 0}, H + EIN, H, nE, w.part, grad + L.W[1], s);
    k_colsum<<<H, 256, 0, s>>>(w.dzf, nE, H, grad + L.b[1]);
    ok = ok && dgrad(6, nE, C0);
    // dh0[i] += sum over the edges into i of d[e, :H]
    k_segsum<<<nblk(n * 32, T), T, 0, s>>>(row_ptr, nullptr, nullptr, C0, H, n, nullptr, w.dh, 1, 1.0f);
  } else {
    cudaMemsetAsync(grad + L.W[1], 0, (size_t)(L.b[1] - L.W[1] + H) * 4, s);
  }
  // ---- encoder: h0 = relu(X W0 + b0)
  k_relu_back<<<nblk(n * H, T), T, 0, s>>>(w.dh, H, w.h0, n, H, 1, w.dzb, w.dzf);
  gemm_wgrad(CatA{w.Xb, nullptr, FIN, nullptr, 0}, MatB{w.dzb, H, 0}, FIN, H, n, w.part, grad + L.W[0], s);
  k_colsum<<<H, 256, 0, s>>>(w.dzf, n, H, grad + L.b[0]);
  if (!ok) return 2;
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_mse(const float* Y, const float* Tt, const float* wts, int64_t n, float* loss, float* dY,
                        void* stream) {
  if (!Y || !Tt || !wts || !loss || !dY || n <= 0) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  // a fixed 256-block grid writes its partial sums into a file-scope device array
  float* pp = nullptr;
  if (cudaGetSymbolAddress((void**)&pp, g_mse_part) != cudaSuccess) return 2;
  k_mse<<<256, 256, 0, s>>>(Y, Tt, wts, n, pp, dY);
  k_mse_final<<<1, 1, 0, s>>>(pp, 256, n, loss);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_adam(float* params, void* params_bf16, const float* grad, float* m, float* v, int64_t count,
                         float lr, float beta1, float beta2, float eps, int64_t step, void* stream) {
  if (!params || !params_bf16 || !grad || !m || !v || count < 0 || step < 1) return 1;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_adam<<<nblk(count, 256), 256, 0, (cudaStream_t)stream>>>(params, (bf16*)params_bf16, grad, m, v, count, lr,
                                                              beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_gemm_bf16(const void* A, const void* B, float* C, int64_t M, int64_t K, int64_t N, void* stream) {
  if (!A || !B || !C || M < 0 || K <= 0 || N <= 0 || K % 16 || N % 8) return 1;
  gemm(CatA{(const bf16*)A, nullptr, (int)K, nullptr, 0}, MatB{(const bf16*)B, (int)N, 0}, M, N, K, C,
       (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_gemm_bf16_tc(const void* A, const void* B, float* C, int64_t M, int64_t K, void* stream) {
  if (!A || !B || !C || M < 0 || K < 16 || K > 256 || K % 16) return 1;
  surrtc::Args a{(const bf16*)A, nullptr, (int)K, nullptr, 0, (const bf16*)B, nullptr, 0, nullptr, nullptr, nullptr,
                 C, M};
  return surrtc::launch(a, (cudaStream_t)stream) ? 0 : 2;
}

extern "C" int surr_tc_wait_probe(int* gave_up, int* timed_out) {
  if (!gave_up || !timed_out) return 1;
  return surrtc::wait_probe(gave_up, timed_out) ? 0 : 2;
}

extern "C" int surr_tc_timeouts(int* count) {
  if (!count) return 1;
  *count = surrtc::timeouts();
  return *count < 0 ? 2 : 0;
}

extern "C" int surr_features(const double* x, const double* v, const double* w, const float* radius, int64_t n,
                             const int32_t* row_ptr, const int32_t* col, int64_t n_edges, const double* geom,
                             int32_t* recv_scratch, float* X, float* E, void* stream) {
  if (!x || !v || !w || !radius || !row_ptr || !geom || !X || n <= 0 || n_edges < 0 ||
      (n_edges > 0 && (!col || !E || !recv_scratch)))
    return 1;
  cudaStream_t s = (cudaStream_t)stream;
  k_node_features<<<nblk(n, 256), 256, 0, s>>>(x, v, w, radius, n, geom, X);
  if (n_edges > 0) {
    k_receivers<<<nblk(n, 256), 256, 0, s>>>(row_ptr, n, recv_scratch);
    k_edge_features<<<nblk(n_edges, 256), 256, 0, s>>>(x, v, w, radius, recv_scratch, col, n_edges, geom, E);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_targets(const double* v0, const double* w0, const double* v1, const double* w1,
                            const float* radius, int64_t n, const double* geom, const float* out_scale, float* T,
                            void* stream) {
  if (!v0 || !w0 || !v1 || !w1 || !radius || !geom || !out_scale || !T || n <= 0) return 1;
  k_targets<<<nblk(n, 256), 256, 0, (cudaStream_t)stream>>>(v0, w0, v1, w1, radius, n, geom, out_scale, T);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int surr_apply(double* x, double* v, double* w, const float* radius, int64_t n, const float* Y,
                          const double* geom, const float* out_scale, double kdt, void* stream) {
  if (!x || !v || !w || !radius || !Y || !geom || !out_scale || n <= 0) return 1;
  k_apply<<<nblk(n, 256), 256, 0, (cudaStream_t)stream>>>(x, v, w, radius, n, Y, geom, out_scale, kdt);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
