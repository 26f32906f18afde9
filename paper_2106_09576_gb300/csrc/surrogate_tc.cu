// surrogate_tc.cu -- the surrogate's 128-wide layer products on the 5th-generation tensor
// cores: tcgen05.mma (BF16 operands, FP32 accumulator in tensor memory), operands staged in
// shared memory in the 128-byte-swizzled K-major layout, accumulators read back with
// tcgen05.ld into a fused epilogue (bias, ReLU, residual, BF16 stores).
//
// A CTA of 160 threads works through 128 x 128 output tiles (persistent over tiles).
// The weights (K x 128, at most 64 KB) are loaded once per CTA; the rows of A stream
// through a ring of 2 to 4 stages of 64 K-columns (16 KB) with cp.async, continuing across
// the CTA's tiles, so the copies of the next stages overlap the products and the epilogue
// of the current one.  A row of A may be gathered (the receiver's node state
// for an edge message), so A is copied per 16-byte chunk rather than as one tensor tile.
// Four warps copy and run the epilogue, one thread of a fifth warp issues the products;
// they hand stages and accumulators to each other through mbarriers (see k_gemm_tc); every
// wait is bounded.
//
// Layers this narrow (N = 128) are bound by HBM, not by the tensor cores: a row of A of
// K BF16 values feeds 256 K flops, i.e. 64 to 128 flops per byte moved, below the ~330
// flops per byte at which the tensor cores would become the limit.
#include "surrogate_tc.cuh"

namespace surrtc {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128;                 // rows of a tile (M of the instruction)
constexpr int TN = 128;                 // output columns (N of the instruction)
constexpr int TK = 64;                  // K columns per stage: one 128-byte swizzle row
constexpr int kThreads = 128;
constexpr int kStageBytes = TM * TK * 2;    // 16 KB
constexpr int kMaxK = 256;
constexpr int kMaxKStages = kMaxK / TK;
constexpr int kMaxStages = 4;              // A stages in flight at most
constexpr long long kSpinLimit = 1ll << 18;  // try_wait calls per wait (each may sleep)

__device__ int g_timeouts;
__device__ int g_probe[2];   // wait_probe's results (one probe at a time per device)

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of 16-byte chunk c (0..7) of row r in a stage of 128-byte rows, 128-byte
// swizzle: the chunk index is XORed with the row index within its group of 8 rows.
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// Shared-memory matrix descriptor of a K-major operand with the 128-byte swizzle: start
// address >> 4 (bits 0-13), leading byte offset 16 (unused by this layout, bits 16-29),
// stride byte offset 1024 = one group of 8 rows (bits 32-45), descriptor version 1
// (bits 46-47), swizzle mode 2 = 128 bytes (bits 61-63).  The stage base is 1024-aligned;
// the k-th slice of 16 columns starts 32 k bytes further.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity; gives up after kSpinLimit attempts, or at once
// when another thread of the CTA has given up (so a broken pipeline unwinds quickly), and
// counts the timeout in *counter.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* counter = &g_timeouts) {
  for (long long it = 0; it < kSpinLimit; it++) {
    if (mbar_try(b, parity)) return true;
    if (*abort) return false;
  }
  *abort = 1;
  atomicAdd(counter, 1);
  return false;
}

// Self-test of the bound: 128 threads wait on an mbarrier that nothing arrives on; every
// wait must give up (by the bound, or through the abort flag once a thread has) and the
// kernel must return.  out[0]: waits that gave up, out[1]: timeouts counted (the threads
// that reached the bound before seeing the flag, at least one).
__global__ void k_wait_probe(int* out) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u, &abort_flag, out + 1);
  if (!ok) atomicAdd(out, 1);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's lane of tensor memory.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(hi)) << 16);
}

// Epilogue of 32 columns [c0, c0 + 32) of one row.
__device__ __forceinline__ void epilogue32(const Args& a, int64_t row, int c0, float* z) {
  const size_t o = (size_t)row * TN + c0;
#pragma unroll
  for (int i = 0; i < 32; i++) {
    if (a.bias) z[i] += a.bias[c0 + i];
    if (a.relu) z[i] = fmaxf(z[i], 0.0f);
  }
  if (a.u_out) {
    uint4* d = reinterpret_cast<uint4*>(a.u_out + o);
#pragma unroll
    for (int q = 0; q < 4; q++)
      d[q] = make_uint4(pack_bf16(z[8 * q], z[8 * q + 1]), pack_bf16(z[8 * q + 2], z[8 * q + 3]),
                        pack_bf16(z[8 * q + 4], z[8 * q + 5]), pack_bf16(z[8 * q + 6], z[8 * q + 7]));
  }
  if (a.res) {
    const uint4* rs = reinterpret_cast<const uint4*>(a.res + o);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint4 u = rs[q];
      const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int h = 0; h < 4; h++) {
        z[8 * q + 2 * h] += __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[h] & 0xFFFFu)));
        z[8 * q + 2 * h + 1] += __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[h] >> 16)));
      }
    }
  }
  if (a.out) {
    uint4* d = reinterpret_cast<uint4*>(a.out + o);
#pragma unroll
    for (int q = 0; q < 4; q++)
      d[q] = make_uint4(pack_bf16(z[8 * q], z[8 * q + 1]), pack_bf16(z[8 * q + 2], z[8 * q + 3]),
                        pack_bf16(z[8 * q + 4], z[8 * q + 5]), pack_bf16(z[8 * q + 6], z[8 * q + 7]));
  }
  if (a.outf) {
    float4* d = reinterpret_cast<float4*>(a.outf + o);
#pragma unroll
    for (int q = 0; q < 8; q++) d[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
  }
}

// Roles: warps 0-3 (128 threads) copy A into the stage ring and run the epilogue (warp w
// reads tensor-memory lanes 32 w .. 32 w + 31, i.e. rows 32 w .. of the tile); lane 0 of
// warp 4 issues the products.  Barriers (parities follow the use count of each):
//   full[b]      128 arrivals: every copier's copies of the stage in buffer b have landed
//                (cp.async.mbarrier.arrive.noinc, no thread blocks on its own copies)
//   empty[b]     tcgen05.commit after the products that read buffer b
//   acc_full[a]  tcgen05.commit after the last products of a tile into accumulator a
//   acc_empty[a] 128 arrivals: the epilogue has read accumulator a
// Two accumulators (256 tensor-memory columns) let the products of tile t + 1 run during
// the epilogue of tile t.
__global__ void __launch_bounds__(kThreads + 32, 1) k_gemm_tc(const __grid_constant__ Args a, int ns) {
  extern __shared__ uint8_t dyn[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~(uintptr_t)1023);
  uint8_t* Bs = base;                                   // nkb stages of W
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = a.w0 + a.w1, nkb = (K + TK - 1) / TK;
  uint8_t* As = base + (size_t)nkb * kStageBytes;      // ns stages of A
  const int64_t tiles = (a.M + TM - 1) / TM;
  const int64_t my_tiles = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t Q = my_tiles * nkb;                    // stages this CTA streams

  if (warp == 0) {   // 256 columns of tensor memory: two 128 x 128 FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < ns; b++) {
      mbar_init(&full[b], kThreads);
      mbar_init(&empty[b], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kThreads);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // W (K x 128, N contiguous) into K-major stages: stage s, row n, chunk c holds
  // W[64 s + 8 c .. + 7][n]; columns past K are zero.
  for (int it = tid; it < nkb * TN * 8; it += blockDim.x) {
    const int s = it / (TN * 8), rem = it - s * (TN * 8), nr = rem >> 3, c = rem & 7;
    uint32_t w4[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k0 = s * TK + c * 8 + 2 * q;
      const uint32_t lo = k0 < K ? __bfloat16_as_ushort(a.W[(int64_t)k0 * TN + nr]) : 0u;
      const uint32_t hi = k0 + 1 < K ? __bfloat16_as_ushort(a.W[(int64_t)(k0 + 1) * TN + nr]) : 0u;
      w4[q] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4*>(Bs + (size_t)s * kStageBytes + sw128(nr, c)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* abort = &abort_flag;

  if (warp < 4) {
    // ---------------- copiers and epilogue
    bool ok = true;
    // gathered rows: the source rows of this thread's 8 rows of the tile being copied
    // (gidx), and those of the CTA's next tile, fetched while the current one is copied
    // (pidx), so that no copy waits on a dependent index load
    int gidx[8], pidx[8];
    int64_t gtile = -1, ptile = -1;
    auto fetch_idx = [&](int64_t t, int* dst) {
      const int64_t m0 = (blockIdx.x + t * gridDim.x) * TM;
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int64_t m = m0 + (tid >> 3) + 16 * j;
        dst[j] = m < a.M ? a.g0[m] : 0;
      }
    };
    // stage q (stage q % nkb of this CTA's tile q / nkb) into buffer q % ns, then an
    // arrival on full[] once this thread's copies have landed
    auto load = [&](int64_t q) {
      const int64_t t = q / nkb;
      const int64_t ti = blockIdx.x + t * gridDim.x;
      const int s = (int)(q % nkb), buf = (int)(q % ns);
      if (q >= ns) ok = mbar_wait(&empty[buf], (uint32_t)((q / ns - 1) & 1), abort) && ok;
      const int64_t m0 = ti * TM;
      const int len = min(TK, K - s * TK);
      const int c = tid & 7;
      if (a.g0 && gtile != t) {
        if (ptile == t) {
#pragma unroll
          for (int j = 0; j < 8; j++) gidx[j] = pidx[j];
        } else {
          fetch_idx(t, gidx);
        }
        gtile = t;
      }
      if (c * 8 < len) {
        const int col = s * TK + c * 8;
        const uint32_t dst0 = smem_u32(As + (size_t)buf * kStageBytes);
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int r = (tid >> 3) + 16 * j;
          const int64_t m = m0 + r;
          const bf16* src = a.s0;
          int bytes = 0;
          if (m < a.M) {
            bytes = 16;
            if (col < a.w0) {
              const int64_t row = a.g0 ? (int64_t)gidx[j] : m;
              src = a.s0 + row * a.w0 + col;
            } else {
              src = a.s1 + m * a.w1 + (col - a.w0);
            }
          }
          cp16(dst0 + sw128(r, c), src, bytes);
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&full[buf])) : "memory");
      if (a.g0 && s == 0 && ptile != t + 1 && t + 1 < my_tiles) {
        fetch_idx(t + 1, pidx);
        ptile = t + 1;
      }
    };
    for (int64_t q = 0; q < ns - 1 && q < Q; q++) load(q);
    for (int64_t q = 0; q < Q; q++) {
      if (q + ns - 1 < Q) load(q + ns - 1);
      if ((int)(q % nkb) == nkb - 1) {   // epilogue of the tile that stage q ends
        const int64_t t = q / nkb;
        const int acc = (int)(t & 1);
        ok = mbar_wait(&acc_full[acc], (uint32_t)((t >> 1) & 1), abort) && ok;
        tc_fence_after();
        const int64_t row = (blockIdx.x + t * gridDim.x) * TM + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 32) {
          float z[32];
          tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * TN + c0), z);
          if (ok && row < a.M) epilogue32(a, row, c0, z);
        }
        tc_fence_before();
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(
                         smem_u32(&acc_empty[acc]))
                     : "memory");
      }
    }
    cp_wait_all();
  } else {
    // ---------------- the issuer of the products: the whole warp waits, lane 0 issues
    for (int64_t t = 0; t < my_tiles; t++) {
      const int acc = (int)(t & 1);
      if (t >= 2) mbar_wait(&acc_empty[acc], (uint32_t)(((t >> 1) - 1) & 1), abort);
      tc_fence_after();
      for (int s = 0; s < nkb; s++) {
        const int64_t q = t * nkb + s;
        const int b = (int)(q % ns);
        mbar_wait(&full[b], (uint32_t)((q / ns) & 1), abort);
        fence_async_smem();   // the copiers' writes, acquired through full[b], to the tensor cores
        tc_fence_after();
        if (lane == 0) {
          const int len = min(TK, K - s * TK);
          const uint64_t ad = desc_sw128(smem_u32(As + (size_t)b * kStageBytes));
          const uint64_t bd = desc_sw128(smem_u32(Bs + (size_t)s * kStageBytes));
          for (int kk = 0; kk < len / 16; kk++)
            mma_bf16(tmem + (uint32_t)(acc * TN), ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk),
                     (s > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&empty[b]);
        }
        __syncwarp();
      }
      if (lane == 0) mma_commit(&acc_full[acc]);
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem) : "memory");
  }
}

// SMs of the current device (queried on every launch: the library may serve several GPUs).
int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess || sms <= 0)
    sms = 1;
  return sms;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bool launch(const Args& a, cudaStream_t s) {
  const int K = a.w0 + a.w1;
  if (a.M < 0 || K < 16 || K > kMaxK || K % 16 || a.w0 % 8 || a.w1 % 8 || a.w0 <= 0 || !a.s0 || !a.W ||
      (a.w1 > 0 && !a.s1) || !aligned16(a.s0) || (a.s1 && !aligned16(a.s1)) || (a.res && !aligned16(a.res)) ||
      (a.u_out && !aligned16(a.u_out)) || (a.out && !aligned16(a.out)) || (a.outf && !aligned16(a.outf)))
    return false;
  if (a.M == 0) return true;
  const int nkb = (K + TK - 1) / TK;
  // as many A stages (2 to 4) as leave room for two CTAs per SM next to the resident W
  const size_t per_sm = 227 * 1024;
  int ns = kMaxStages;
  while (ns > 2 && 2 * (1024 + (size_t)(nkb + ns) * kStageBytes + 1024 + 64) > per_sm) ns--;
  // at least 80 KB, so that no more than two CTAs (512 columns of tensor memory) share an SM
  size_t smem = 1024 + (size_t)(nkb + ns) * kStageBytes;
  if (smem < 80 * 1024) smem = 80 * 1024;
  // the attribute belongs to the current device's copy of the kernel: set it on every launch
  if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           1024 + (kMaxKStages + kMaxStages) * kStageBytes) != cudaSuccess)
    return false;
  const int64_t tiles = (a.M + TM - 1) / TM;
  const int64_t cap = 2 * (int64_t)sm_count();
  const int grid = (int)(tiles < cap ? tiles : cap);
  k_gemm_tc<<<grid, kThreads + 32, smem, s>>>(a, ns);
  return cudaGetLastError() == cudaSuccess;
}

bool wait_probe(int* gave_up, int* timed_out) {
  int* d = nullptr;
  int h[2] = {0, 0};
  bool ok = cudaGetSymbolAddress((void**)&d, g_probe) == cudaSuccess &&
            cudaMemset(d, 0, 2 * sizeof(int)) == cudaSuccess;
  if (ok) {
    k_wait_probe<<<1, kThreads>>>(d);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
         cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  *gave_up = h[0];
  *timed_out = h[1];
  return ok;
}

int timeouts() {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_timeouts, sizeof(int)) != cudaSuccess) return -1;
  return h;
}

}  // namespace surrtc
