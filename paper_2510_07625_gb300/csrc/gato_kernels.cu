// The batched SQP kernels and their launchers.
#include <algorithm>
#include <numeric>
#include <vector>

#include "gato_kernels.cuh"

namespace gato {

size_t fused_smem_bytes(int nmax, int csize) {
  return smem_floats(kpc_for(nmax, csize)) * sizeof(float);
}

int cluster_size(int N, int knots_per_cta, int cluster) {
  int c = cluster_for(N);
  if (knots_per_cta >= 2) c = std::max(c, (N + 1 + knots_per_cta - 1) / knots_per_cta);
  if (cluster > 0) c = std::max(c, cluster);
  c = std::min(c, 8);
  c = std::max(cluster_for(N), std::min(c, std::max(1, (N + 1) / 2)));  // at least 2 knots per CTA
  // every CTA but the last holds kpc >= 2 knots, the last at least one
  const int kpc = kpc_for(N, c);
  return (N + 1 + kpc - 1) / kpc;
}

void order_solves(const int* N_of, int n, int* order, const LaunchPlan& plan) {
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    const int ca = cluster_size(N_of[a], plan.knots_per_cta, plan.cluster);
    const int cb = cluster_size(N_of[b], plan.knots_per_cta, plan.cluster);
    if (ca != cb) return ca > cb;
    return N_of[a] > N_of[b];
  });
  for (int i = 0; i < n; ++i) order[i] = idx[i];
}

int num_sms() {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 1;
  }
  return sms[dev];
}

static size_t g_configured[2][64] = {};

template <bool REG>
static cudaError_t configure_t(size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  size_t& done = g_configured[REG ? 0 : 1][dev];
  if (smem > done) {
    e = cudaFuncSetAttribute(sqp_fused<REG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    done = smem;
  }
  return cudaSuccess;
}

cudaError_t configure_fused(size_t smem) {
  if (smem > SMEM_LIMIT_BYTES) return cudaErrorInvalidValue;
  cudaError_t e = configure_t<true>(smem);
  if (e != cudaSuccess) return e;
  num_sms();
  return configure_t<false>(smem);
}

template <bool REG>
static cudaError_t launch_fused_t(const FusedLaunch& a, size_t smem, cudaStream_t s) {
  cudaError_t e = configure_t<REG>(smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n * a.csize));
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sqp_fused<REG>, a);
}

template <bool REG>
static cudaError_t active_clusters_t(int csize, size_t smem, int* out) {
  cudaError_t e = configure_t<REG>(smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(csize * num_sms()));
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, sqp_fused<REG>, &cfg);
}

cudaError_t fused_active_clusters(int nmax, int csize, bool reg, int* out) {
  *out = 0;
  if (csize < 1 || csize > 8) return cudaErrorInvalidValue;
  const size_t smem = fused_smem_bytes(nmax, csize);
  if (smem > SMEM_LIMIT_BYTES) return cudaErrorInvalidValue;
  return reg ? active_clusters_t<true>(csize, smem, out) : active_clusters_t<false>(csize, smem, out);
}

bool use_throughput_variant(int n, int csize, int variant, size_t smem) {
  (void)n;
  (void)csize;
  (void)smem;
  // automatic = the latency form: with the halo knots recomputed in the
  // cluster it is faster than two CTAs per SM at every batch size and horizon
  // measured (B 1..256, N 32..128); the throughput form is kept on request
  return variant == 2;
}

cudaError_t launch_fused(const FusedLaunch& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.csize < 1 || a.csize > 8) return cudaErrorInvalidValue;
  const size_t smem = fused_smem_bytes(a.nmax, a.csize);
  if (smem > SMEM_LIMIT_BYTES) return cudaErrorInvalidValue;
  if (use_throughput_variant(a.n, a.csize, a.variant, smem)) return launch_fused_t<false>(a, smem, s);
  return launch_fused_t<true>(a, smem, s);
}

cudaError_t launch_fused_grouped(FusedLaunch base, const int* order_host, const int* order_dev,
                                 const int* N_of, int n, cudaStream_t s, const LaunchPlan& plan) {
  struct Group { int g0, g1, c; };
  Group groups[8];
  int ng = 0;
  for (int g0 = 0; g0 < n;) {
    const int c = cluster_size(N_of[order_host[g0]], plan.knots_per_cta, plan.cluster);
    int g1 = g0 + 1;
    while (g1 < n && cluster_size(N_of[order_host[g1]], plan.knots_per_cta, plan.cluster) == c) ++g1;
    if (ng == 8) return cudaErrorInvalidValue;  // sizes are distinct and in 1..8
    groups[ng++] = {g0, g1, c};
    g0 = g1;
  }
  base.variant = plan.variant;
  const bool fork = ng > 1 && plan.n_aux > 0 && plan.aux && plan.ev;
  cudaError_t e;
  if (fork) {
    e = cudaEventRecord(plan.ev[plan.n_aux], s);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < ng; ++i) {
    FusedLaunch a = base;
    a.order = order_dev + groups[i].g0;
    a.n = groups[i].g1 - groups[i].g0;
    a.csize = groups[i].c;
    a.nmax = N_of[order_host[groups[i].g0]];
    // the first group stays on the caller's stream, the others fork off it
    cudaStream_t si = s;
    if (fork && i > 0 && i - 1 < plan.n_aux) {
      si = plan.aux[i - 1];
      e = cudaStreamWaitEvent(si, plan.ev[plan.n_aux], 0);
      if (e != cudaSuccess) return e;
    }
    e = launch_fused(a, si);
    if (e != cudaSuccess) return e;
    if (si != s) {
      e = cudaEventRecord(plan.ev[i - 1], si);
      if (e != cudaSuccess) return e;
      e = cudaStreamWaitEvent(s, plan.ev[i - 1], 0);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_plain(const ProbDesc* probs, const DevModel* models, Result* results, int b,
                         int N_b, float* ws, const WsLayout& L, int nmax, int iters, const Params& prm,
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
  a.redo = 0;
  a.csize = cluster_for(N_b);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.csize);
  cfg.blockDim = dim3(NTHR);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto go = [&](int stage) -> cudaError_t { return cudaLaunchKernelEx(&cfg, sqp_plain_stage, stage, a); };
  cudaError_t e = go(PS_LOAD);
  if (e != cudaSuccess) return e;
  for (int it = 0;; ++it) {
    a.it = it;
    if (it == iters && !(prm.kkt_tol > 0.f)) break;
    for (int st = PS_MASS; st <= PS_KKT; ++st) {
      if ((e = go(st)) != cudaSuccess) return e;
      if (stop_stage == st) return cudaSuccess;
    }
    if (it == iters) {
      if (prm.escalate && prm.kkt_tol > 0.f) {
        // a convergence test passed in FP32 is repeated in the high-precision mode
        a.redo = 1;
        for (int st = PS_MASS; st <= PS_KKT; ++st)
          if ((e = go(st)) != cudaSuccess) return e;
        a.redo = 0;
      }
      break;
    }
    for (int st = PS_SCHUR; st <= PS_ACCEPT; ++st) {
      if ((e = go(st)) != cudaSuccess) return e;
      if (stop_stage == st) return cudaSuccess;
    }
    if (prm.escalate && prm.kkt_tol > 0.f) {
      // the pass that repeats the iteration in the high-precision mode when its
      // FP32 line search found no decrease (each launch returns at once otherwise)
      a.redo = 1;
      for (int st = PS_MASS; st <= PS_ACCEPT; ++st)
        if ((e = go(st)) != cudaSuccess) return e;
      a.redo = 0;
    }
  }
  return go(PS_STORE);
}

}  // namespace gato
