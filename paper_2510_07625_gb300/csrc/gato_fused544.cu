// Instantiations of the fused SQP kernel with 544 threads per CTA.
#include "gato_kernels.cuh"

namespace gato {

cudaError_t launch_fused_544(const FusedLaunch& a, size_t smem, bool sb, cudaStream_t s) {
  return sb ? launch_fused_t<544, true>(a, smem, s) : launch_fused_t<544, false>(a, smem, s);
}

}  // namespace gato
