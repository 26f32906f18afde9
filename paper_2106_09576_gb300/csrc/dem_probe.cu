// dem_probe.cu -- measured issue rates of the arithmetic pipes the step kernels lean on.
//
// The FP64 path is bound by FP64 arithmetic, and the mixed path is designed around the
// ratio of FP64 to FP32 rates on this part (FP64 work kept to the integration and the
// tangential-overlap sums, conversions done with integer operations).  This probe gives
// those rates as measured numbers: thread-level instructions per second of FP64 fused
// multiply-add, FP64 add, FP32 fused multiply-add and FP32 -> FP64 conversion, each from
// a kernel of many independent chains (no dependency stalls) over every SM, timed with
// CUDA events after a warm-up launch.  Not a step of the method: a measurement aid for
// the rooflines of the step kernels.
#include <cuda_runtime.h>

#include "../../include/dem.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeBlock = 256;

// op 0: DFMA, 1: DADD, 2: FFMA, 3: F2F.F64.F32 (cvt.f64.f32).  Each iteration issues
// kChains instructions of the probed kind on independent registers; the results feed a
// store guarded by `iters < 0`, which the caller never passes but the compiler cannot
// rule out, so nothing is eliminated and the (null) sink is never touched.
template <int kOp>
__global__ void __launch_bounds__(kProbeBlock) k_pipe_probe(int iters, double seed, double* sink) {
  const double s = seed + threadIdx.x * 1e-9;
  if (kOp == 0 || kOp == 1) {
    double a[kChains];
    for (int k = 0; k < kChains; k++) a[k] = s + k;
    const double m = 1.0 - 1e-12, c = 1e-9;
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = (kOp == 0) ? fma(a[k], m, c) : __dadd_rn(a[k], c);
    }
    double t = 0.0;
    for (int k = 0; k < kChains; k++) t += a[k];
    if (iters < 0) sink[threadIdx.x] = t;
  } else if (kOp == 2) {
    float a[kChains];
    for (int k = 0; k < kChains; k++) a[k] = (float)s + k;
    const float m = 1.0f - 1e-7f, c = 1e-6f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], m, c);
    }
    float t = 0.0f;
    for (int k = 0; k < kChains; k++) t += a[k];
    if (iters < 0) sink[threadIdx.x] = t;
  } else {
    // conversions of varying FP32 values; the FP32 value advances by an integer add and
    // the FP64 result is folded in with integer adds, so the conversion is the only
    // non-integer instruction in the loop
    unsigned u[kChains], acc = 0u;
    for (int k = 0; k < kChains; k++) u[k] = __float_as_uint((float)s + k);
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int k = 0; k < kChains; k++) {
        const double d = (double)__uint_as_float(u[k]);
        acc += (unsigned)__double2loint(d) ^ (unsigned)__double2hiint(d);
        u[k] += 1u;
      }
    }
    if (iters < 0) sink[threadIdx.x] = (double)acc;
  }
}

template <int kOp>
double time_probe(int blocks, int iters, double* sink, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, bool* ok) {
  k_pipe_probe<kOp><<<blocks, kProbeBlock, 0, s>>>(iters, 1.0, sink);   // warm-up
  cudaEventRecord(e0, s);
  k_pipe_probe<kOp><<<blocks, kProbeBlock, 0, s>>>(iters, 1.0, sink);
  cudaEventRecord(e1, s);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
    *ok = false;
    return 0.0;
  }
  return (double)blocks * kProbeBlock * (double)iters * kChains / (ms * 1e-3);
}

}  // namespace

extern "C" dem_status dem_pipe_rates(double* rates, void* stream) {
  if (!rates) return DEM_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess || sms <= 0)
    return DEM_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  double* sink = nullptr;   // never written: the kernels' stores need iters < 0
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DEM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return DEM_ERR_CUDA;
  }
  const int blocks = sms * 8;
  bool ok = true;
  rates[0] = time_probe<0>(blocks, 4096, sink, s, e0, e1, &ok);
  rates[1] = time_probe<1>(blocks, 4096, sink, s, e0, e1, &ok);
  rates[2] = time_probe<2>(blocks, 65536, sink, s, e0, e1, &ok);
  rates[3] = time_probe<3>(blocks, 4096, sink, s, e0, e1, &ok);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || !ok) return DEM_ERR_CUDA;
  return DEM_OK;
}
