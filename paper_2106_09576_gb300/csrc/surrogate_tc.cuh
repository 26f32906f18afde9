// surrogate_tc.cuh -- interface between the surrogate's forward pass (surrogate.cu) and its
// 5th-generation tensor-core product (surrogate_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace surrtc {

// out(m, :) = epilogue(A(m, :) W) for the 128-wide layers of the network, where
//   A(m, :) = [S0[g0 ? g0[m] : m] (w0 columns) | S1[m] (w1 columns)]   (BF16, row-major rows)
//   W       = [K][128] BF16 row-major (K = w0 + w1, a multiple of 16, at most 256)
//   z = A W + bias (FP32, accumulated in tensor memory); u = relu ? max(z, 0) : z;
//   o = res ? res + u : u;  writes u (BF16) to u_out, o (BF16) to out and o (FP32) to outf,
//   each when not null, all [M][128] row-major.
// w0 and w1 are multiples of 8 and every row starts on a 16-byte boundary.
struct Args {
  const __nv_bfloat16* s0;
  const int32_t* g0;
  int w0;
  const __nv_bfloat16* s1;
  int w1;
  const __nv_bfloat16* W;
  const float* bias;
  int relu;
  const __nv_bfloat16* res;
  __nv_bfloat16* u_out;
  __nv_bfloat16* out;
  float* outf;
  int64_t M;
};

// Launches the product on `s`; returns false for arguments outside the limits above.
bool launch(const Args& a, cudaStream_t s);

// Number of waits on the tensor cores that ran out of their iteration limit since the
// library was loaded (0 unless something is badly wrong; the outputs of such a tile are
// not written).
int timeouts();

// Self-test of the wait bound (see surr_tc_wait_probe).  False on a CUDA error.
bool wait_probe(int* gave_up, int* timed_out);

}  // namespace surrtc
