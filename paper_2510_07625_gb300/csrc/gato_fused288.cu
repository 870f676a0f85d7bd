// Instantiations of the fused SQP kernel with 288 threads per CTA.
#include "gato_kernels.cuh"

namespace gato {

cudaError_t launch_fused_288(const FusedLaunch& a, size_t smem, bool sb, cudaStream_t s) {
  return sb ? launch_fused_t<288, true>(a, smem, s) : launch_fused_t<288, false>(a, smem, s);
}

}  // namespace gato
