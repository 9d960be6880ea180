// mc_batch_split.cu -- instantiations of the batched survey kernel for the split form (FP64 geodesic,
// FP32 rest), which the FP64 pipe bounds like the FP64 form.
#include "mc_batch.cuh"

namespace mcgb {

// register caps 255 and 168 (minimum 1 and 3 resident CTAs per SM); with the network one variant
BatchKernel batch_kernel_split(bool sur, int minb) {
  if (sur) return k_batch<2, true, 1>;
  return minb == 1 ? k_batch<2, false, 1> : k_batch<2, false, 3>;
}

}  // namespace mcgb
