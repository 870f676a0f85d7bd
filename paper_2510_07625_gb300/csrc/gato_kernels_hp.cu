// The high-precision instantiations of the fused kernel: their own
// translation unit, compiled beside the FP32 one.
#include "gato_kernels.cuh"

namespace gato {

cudaError_t launch_fused_hp(const FusedLaunch& a, size_t smem, cudaStream_t s, bool reg) {
  return reg ? launch_kernel<true, true>(a, smem, s) : launch_kernel<false, true>(a, smem, s);
}

cudaError_t configure_fused_hp(size_t smem) {
  cudaError_t e = configure_kernel<true, true>(smem);
  if (e == cudaSuccess) e = configure_kernel<false, true>(smem);
  return e;
}

}  // namespace gato
