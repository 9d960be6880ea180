// mc_batch_fp64.cu -- instantiations of the batched survey kernel for the plain FP64 form.
#include "mc_batch.cuh"

namespace mcgb {

// register caps 255, 168, 128 (minimum 1, 3, 4 resident CTAs per SM)
BatchKernel batch_kernel_fp64(bool, int minb) {
  return minb == 1 ? k_batch<0, false, 1> : minb == 3 ? k_batch<0, false, 3> : k_batch<0, false, 4>;
}

}  // namespace mcgb
