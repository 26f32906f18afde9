// dem_step_mixed.cu -- mixed-precision instantiation of the step kernel: FP32 contact
// law, FP64 positions, velocities, integration and tangential-overlap accumulation.
#include "dem_step_impl.cuh"

namespace demgb {
void launch_step_mixed(const Params& P, cudaStream_t s) {
  const int blocks = (P.n + kStepBlock - 1) / kStepBlock;
  k_step<true><<<blocks, kStepBlock, 0, s>>>(P);
}
}  // namespace demgb
