// Launchers of the batched SQP kernels (plain form and dispatch of the fused form).
#include "gato_kernels.cuh"

namespace gato {

int fused_threads_for(int nmax) { return nmax <= 35 ? 288 : 544; }

size_t fused_smem_bytes(int nmax) {
  return smem_floats(nmax, nmax <= SMEM_BLOCKS_NMAX) * sizeof(float);
}

cudaError_t launch_fused(const FusedLaunch& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const bool sb = a.nmax <= SMEM_BLOCKS_NMAX;
  const int nt = a.threads > 0 ? a.threads : fused_threads_for(a.nmax);
  const size_t smem = smem_floats(a.nmax, sb) * sizeof(float);
  if (smem > SMEM_LIMIT_BYTES) return cudaErrorInvalidValue;
  if (nt == 288) return launch_fused_288(a, smem, sb, s);
  return launch_fused_544(a, smem, sb, s);
}
cudaError_t launch_plain(const ProbDesc* probs, const DevModel* models, Result* results, int b,
                         float* ws, const WsLayout& L, int nmax, int iters, const Params& prm,
                         int stop_stage, cudaStream_t s) {
  PlainArgs a;
  a.probs = probs;
  a.models = models;
  a.results = results;
  a.ws = ws;
  a.layout = L;
  a.b = b;
  a.nmax = nmax;
  a.iters = iters;
  a.prm = prm;
  a.it = 0;
  const int nt = fused_threads_for(nmax);
  auto go = [&](int stage) -> cudaError_t {
    if (nt == 288)
      sqp_plain_stage<288><<<1, 288, 0, s>>>(stage, a);
    else
      sqp_plain_stage<544><<<1, 544, 0, s>>>(stage, a);
    return cudaGetLastError();
  };
  cudaError_t e = go(PS_LOAD);
  if (e != cudaSuccess) return e;
  for (int it = 0;; ++it) {
    a.it = it;
    if (it == iters && !(prm.kkt_tol > 0.f)) break;
    for (int st = PS_MASS; st <= PS_KKT; ++st) {
      if ((e = go(st)) != cudaSuccess) return e;
      if (stop_stage == st) return cudaSuccess;
    }
    if (it == iters) break;
    for (int st = PS_SCHUR; st <= PS_ACCEPT; ++st) {
      if ((e = go(st)) != cudaSuccess) return e;
      if (stop_stage == st) return cudaSuccess;
    }
  }
  return go(PS_STORE);
}

}  // namespace gato
