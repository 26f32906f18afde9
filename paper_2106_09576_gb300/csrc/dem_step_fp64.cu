// dem_step_fp64.cu -- FP64 instantiation of the step kernel.  Built with -fmad=false so
// that every product and sum rounds separately, as in the serial CPU statement.
#include "dem_step_impl.cuh"

namespace demgb {
void launch_step_fp64(const Params& P, cudaStream_t s) {
  const int blocks = (P.n + kStepBlock - 1) / kStepBlock;
  k_step<false><<<blocks, kStepBlock, 0, s>>>(P);
}
}  // namespace demgb
