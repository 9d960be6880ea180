// mc_batch_mixed.cu -- instantiations of the batched survey kernel for the mixed (double-float) form.
#include "mc_batch.cuh"

namespace mcgb {

// register caps 255, 168, 128, 80, 64 (minimum 1, 3, 4, 6, 8 resident CTAs per SM; 6 and 8 read the
// model descriptors through L1); with the network one variant (tensor memory: one CTA per SM)
BatchKernel batch_kernel_mixed(bool sur, int minb) {
  if (sur) return k_batch<1, true, 1>;
  return minb == 1   ? k_batch<1, false, 1>
         : minb == 3 ? k_batch<1, false, 3>
         : minb == 4 ? k_batch<1, false, 4>
         : minb == 6 ? k_batch<1, false, 6>
                     : k_batch<1, false, 8>;
}

}  // namespace mcgb
