/*
 * surrogate.h -- C ABI of the learned surrogate of the DEM drum: a message-passing network
 * on the radius-1.2 d contact graph that predicts the velocity and spin increments of every
 * particle over k DEM steps.  The paper has no counterpart (it is the learned part this
 * project adds beside the method); plain DEM is its reference and its fallback.
 *
 * Network (hidden width H = 128, BF16 weights and activations, FP32 accumulation):
 *   h0 = relu(X W0 + b0)                          node encoder, X [N][16]
 *   m  = relu([h0[i] | E] W1 + b1)                 per directed edge i <- j, E [nE][16]
 *   a  = c * sum over the edges into i of m        (segment sum over a receiver-sorted CSR)
 *   h1 = h0 + relu([h0 | a] W2 + b2)
 *   s  = c * sum over neighbours j of h1[j];  h2 = h1 + relu([h1 | s] W3 + b3)
 *   s  = c * sum over neighbours j of h2[j];  h3 = h2 + relu([h2 | s] W4 + b4)
 * with c = SURR_AGG_SCALE, so that sums over a dozen neighbours keep the activations' size.
 *   Y  = h3 W5 + b5                                Y [N][8] (6 outputs used)
 * Parameters live in one FP32 array (the master copy the optimiser updates) and one BF16
 * copy for the tensor-core products, both at the offsets of surr_param_layout.
 * All pointers are device pointers; every call runs on `stream`; nothing is allocated.
 * Return value: 0 ok, 1 bad argument, 2 CUDA error.
 */
#ifndef SURROGATE_H
#define SURROGATE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SURR_HIDDEN 128
#define SURR_NODE_IN 16
#define SURR_EDGE_IN 16
#define SURR_OUT 8
#define SURR_AGG_SCALE 0.125f

/* Offsets (in elements) of the parameter tensors in the flat arrays, and the total:
 * W0 [16][128] b0 [128] W1 [144][128] b1 [128] W2 [256][128] b2 [128] W3 [256][128] b3 [128]
 * W4 [256][128] b4 [128] W5 [128][8] b5 [8]; weights row-major [in][out]. */
typedef struct {
  int64_t W[6], b[6];
  int64_t total;
} surr_param_layout;
int surr_params(surr_param_layout* out);

/* Bytes of device scratch for a graph of n nodes and n_edges directed edges. */
int surr_workspace_bytes(int64_t n, int64_t n_edges, size_t* bytes);

/* Receiver-sorted CSR of the undirected graph given as pairs (i < j): row_ptr [n + 1],
 * col [2 n_pairs] (the sender of each edge).  `scratch` holds n + 1 + n ints. */
int surr_build_csr(const int32_t* pairs, int64_t n_pairs, int64_t n, int32_t* row_ptr, int32_t* col,
                   int32_t* scratch, void* stream);

/* Converts the FP32 parameters to the BF16 copy. */
int surr_params_to_bf16(const float* params, void* params_bf16, int64_t count, void* stream);

/* Forward pass: X [n][16], E [n_edges][16] (FP32), Y [n][8] (FP32), each 16-byte aligned.
 * The 128-wide layers run on the 5th-generation tensor cores (see surr_gemm_bf16_tc).  The
 * workspace keeps the activations the backward pass needs. */
int surr_forward(const void* params_bf16, const float* params, const float* X, const float* E,
                 const int32_t* row_ptr, const int32_t* col, int64_t n, int64_t n_edges, void* workspace,
                 float* Y, void* stream);

/* Backward pass of the last forward on the same workspace: dY [n][8] in, grad [total] out
 * (FP32, overwritten).  The data gradients of the 128-wide layers (dz W^T, one 128-column
 * block of W^T at a time) run on the 5th-generation tensor cores; the weight gradients,
 * reductions over the node or edge dimension, on the warp-level product. */
int surr_backward(const void* params_bf16, const float* dY, const int32_t* row_ptr, const int32_t* col,
                  int64_t n, int64_t n_edges, void* workspace, float* grad, void* stream);

/* Mean squared error over the first 6 outputs of n rows (with per-column weights w[6]):
 * loss (one float) and dY = dLoss/dY. */
int surr_mse(const float* Y, const float* T, const float* w, int64_t n, float* loss, float* dY, void* stream);

/* One Adam step on `count` FP32 parameters (moments m, v), then the BF16 copy. */
int surr_adam(float* params, void* params_bf16, const float* grad, float* m, float* v, int64_t count, float lr,
              float beta1, float beta2, float eps, int64_t step, void* stream);

/* Inputs of the network from a drum state (caller order [n][3] FP64, radius FP32):
 * geom = {cx, y0, cz, Rd, L, d0, vs, 0} -- the drum axis along y through (cx, cz) from y0 to
 * y0 + L, radius Rd, length scale d0, velocity scale vs.  Node features X [n][16]: v / vs,
 * w R / vs, 2R / d0, position in the drum frame, distances to the mantle and the caps
 * (in d0, clipped to 5), 1.  Edge features E [n_edges][16]: (x_j - x_i) / d0, |x_j - x_i| /
 * d0, the overlap max(R_i + R_j - |x_j - x_i|, 0) in units of 0.01 d0, (v_j - v_i) / vs,
 * (w_j R_j - w_i R_i) / vs.
 * recv_scratch holds n_edges ints (the receiver of each edge). */
int surr_features(const double* x, const double* v, const double* w, const float* radius, int64_t n,
                  const int32_t* row_ptr, const int32_t* col, int64_t n_edges, const double* geom,
                  int32_t* recv_scratch, float* X, float* E, void* stream);

/* Training targets T [n][6]: the velocity and spin increments between two states k steps
 * apart, (v1 - v0) / vs and (w1 - w0) R / vs, divided by out_scale[6]. */
int surr_targets(const double* v0, const double* w0, const double* v1, const double* w1, const float* radius,
                 int64_t n, const double* geom, const float* out_scale, float* T, void* stream);

/* One surrogate step standing for k DEM steps (kdt = k dt): with dv = Y[:, 0:3] out_scale vs
 * and dw = Y[:, 3:6] out_scale vs / R, v += dv, w += dw, x += (v_old + v_new) / 2 kdt. */
int surr_apply(double* x, double* v, double* w, const float* radius, int64_t n, const float* Y, const double* geom,
               const float* out_scale, double kdt, void* stream);

/* C[M][N] = A[M][K] B[K][N] with A, B BF16 row-major, C FP32: the warp-level tensor-core
 * product (mma.sync) used by the weight gradients and the decoder, exposed for its own test.
 * M any, K a multiple of 16, N a multiple of 8. */
int surr_gemm_bf16(const void* A, const void* B, float* C, int64_t M, int64_t K, int64_t N, void* stream);

/* The same product for N = 128 on the 5th-generation tensor cores (tcgen05.mma, FP32
 * accumulator in tensor memory), which the forward pass uses for its 128-wide layers:
 * C [M][128] (FP32) = A [M][K] B [K][128] (BF16, row-major, 16-byte aligned rows); K a
 * multiple of 16 from 16 to 256. */
int surr_gemm_bf16_tc(const void* A, const void* B, float* C, int64_t M, int64_t K, void* stream);

/* Waits on the tensor cores that ran out of their iteration limit since the library was
 * loaded (synchronises the device; 0 in normal operation). */
int surr_tc_timeouts(int* count);

/* Self-test of the bound on the tensor-core kernel's waits: one CTA of 128 threads waits on
 * a barrier that nothing arrives on.  Every wait gives up (gave_up = 128) after the bound or
 * through the CTA's abort flag, the threads that reached the bound first are counted
 * (timed_out >= 1), and the kernel returns; the counter of surr_tc_timeouts is not touched.
 * Results pass through a file-scope device array (one probe at a time per device);
 * synchronises the device. */
int surr_tc_wait_probe(int* gave_up, int* timed_out);

#ifdef __cplusplus
}
#endif
#endif
