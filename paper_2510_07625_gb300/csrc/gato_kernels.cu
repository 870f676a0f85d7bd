// The batched SQP kernels and their launchers.
#include <algorithm>
#include <numeric>
#include <vector>

#include "gato_kernels.cuh"

namespace gato {

// ----------------------------------------------------------------- plain form

struct PlainArgs {
  const ProbDesc* probs;
  const DevModel* models;
  Result* results;
  float* ws;
  WsLayout layout;
  int b, nmax, iters, it, csize;
  int redo;  // 1: the pass that repeats an iteration in the high-precision mode
  Params prm;
};

__global__ void __launch_bounds__(NTHR, 1) sqp_plain_stage(int stage, PlainArgs a) {
  __shared__ __align__(16) float red[2 * RED_SLOTS * RED_W];
  __shared__ float zeros196[196];
  for (int i = threadIdx.x; i < 196; i += NTHR) zeros196[i] = 0.f;
  __syncthreads();
  const int csize = a.csize;
  const int rank = csize > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const ProbDesc P = a.probs[a.b];
  const size_t K = (size_t)a.nmax + 1;
  Ctx C;
  bind_problem(C, P, a.models + P.model);
  bind_workspace(C, a.ws, a.layout);
  bind_partition(C, rank, csize);
  C.Dm = a.ws + a.layout.Dm;
  C.Lm = a.ws + a.layout.Lm;
  C.Pm = a.ws + a.layout.Pm;
  C.bk0 = 0;
  C.Lz = zeros196;
  C.vb = a.ws + a.layout.vec;
  C.vstride = (int)((K + 2) * VW);
  C.vk0 = -1;
  C.vbl = C.vbr = nullptr;
  C.vk0l = C.vk0r = 0;
  C.scal = C.vb + NVEC * C.vstride;
  C.xs = C.scal + SCAL_FLOATS;
  C.red = red;
  C.tm = nullptr;
  const Params& prm = a.prm;
  int* rflags = reinterpret_cast<int*>(C.scal + S_RFLAGS);
  int rbuf = 0;
  if (stage == PS_LOAD) {
    if (rank == 0 && threadIdx.x < SCAL_FLOATS) {
      const int t = threadIdx.x;
      C.scal[t] = t == S_RHO ? P.w[5]
                : (t == S_FEXT ? P.fext[0] : (t == S_FEXT + 1 ? P.fext[1] : (t == S_FEXT + 2 ? P.fext[2] : 0.f)));
      if (t == S_HP) C.scal[t] = a.prm.high ? 1.f : 0.f;
    }
    load_iterate(C, P);
    return;
  }
  if (a.prm.rho_adapt) C.w[5] = C.scal[S_RHO];  // the adapted rho of this SQP iteration
  C.hp = C.scal[S_HP] != 0.f;
  if (stage == PS_STORE) {
    store_iterate(C, P);
    if (rank == 0 && threadIdx.x == 0) {
      Result* out = a.results + a.b;
      out->flags = *rflags;
      out->sqp_iters = (int)C.scal[S_NSQP];
      out->pcg_iters = (int)C.scal[S_NPCG];
      out->kkt = C.scal[S_KKT];
      out->merit = C.scal[S_MERITF];
    }
    return;
  }
  if (C.scal[S_DONE] != 0.f) return;
  if (a.redo && C.scal[S_REDO] == 0.f) return;  // no escalation in this iteration
  // an escalation decided at the KKT stage skips the rest of the first pass
  if (!a.redo && stage > PS_KKT && C.scal[S_REDO] != 0.f) return;
  const bool lead = rank == 0 && threadIdx.x == 0;
  switch (stage) {
    case PS_MASS: st_mass_bias(C); break;
    case PS_FD: st_forward_dynamics(C); break;
    case PS_VALUE: st_value_and_cost(C); break;
    case PS_TANGENT: st_tangents(C); break;
    case PS_JAC: st_dyn_jacobians(C); break;
    case PS_KKT: {
      st_kkt_merit(C, prm.mu, rbuf);
      if (a.it == 0 || a.redo) st_line_search(C, prm.mu, prm.beta, prm.n_alpha, rbuf, true);  // the iterate's merit
      const bool bad = *reinterpret_cast<volatile int*>(C.scal + S_FLAGS) != 0;
      if (lead) {
        C.scal[S_MERITF] = C.scal[S_MERIT0];
        int f = *rflags;
        bool done = false;
        if (bad) {
          f |= F_NONFINITE;
          done = true;
        } else if (prm.kkt_tol > 0.f && C.scal[S_KKT] <= prm.kkt_tol && prm.escalate && !C.hp) {
          // confirm convergence with the high-precision residual (the pass
          // that repeats this iteration in that mode)
          C.scal[S_HP] = 1.f;
          C.scal[S_REDO] = 1.f;
        } else if (prm.kkt_tol > 0.f && C.scal[S_KKT] <= prm.kkt_tol) {
          f |= F_CONVERGED;
          done = true;
        } else if (a.it == a.iters) {
          f |= F_MAXITER;
          done = true;
        }
        *rflags = f;
        if (done) C.scal[S_DONE] = 1.f;
      }
      break;
    }
    case PS_SCHUR: st_schur(C); break;
    case PS_BINV:
      st_block_inverse(C);
      csync(C);
      if (lead && *reinterpret_cast<volatile int*>(C.scal + S_FLAGS)) {
        *rflags |= F_NONFINITE;
        C.scal[S_DONE] = 1.f;
      }
      break;
    case PS_PCG: {
      if (prm.linsolve == 1) {
        st_direct(C);
        csync(C);
        if (lead && *reinterpret_cast<volatile int*>(C.scal + S_FLAGS)) {
          *rflags |= F_NONFINITE;
          C.scal[S_DONE] = 1.f;
        }
        break;
      }
      bool hit = false;
      const int n = st_pcg<true>(C, prm.pcg_eps, prm.pcg_max, prm.precond, &hit, rbuf);
      if (lead) {
        C.scal[S_NPCG] += (float)n;
        if (hit) *rflags |= F_PCGMAX;
      }
      break;
    }
    case PS_RECOVER:
      st_recover(C);
      csync(C);
      if (lead && *reinterpret_cast<volatile int*>(C.scal + S_FLAGS)) {
        *rflags |= F_NONFINITE;
        C.scal[S_DONE] = 1.f;
      }
      break;
    case PS_LS: st_line_search(C, prm.mu, prm.beta, prm.n_alpha, rbuf); break;
    case PS_ACCEPT: {
      const int choice = st_accept(C, prm.beta, prm.n_alpha);
      if (choice < 0 && prm.escalate && prm.kkt_tol > 0.f && !C.hp) {
        // repeat this iteration in the high-precision mode (the next pass)
        if (lead) {
          C.scal[S_HP] = 1.f;
          C.scal[S_REDO] = 1.f;
        }
        break;
      }
      if (lead) C.scal[S_REDO] = 0.f;
      if (lead && prm.rho_adapt) C.scal[S_RHO] = rho_next(C.w[5], choice);
      if (lead) {
        if (choice >= 0)
          C.scal[S_MERITF] = C.scal[S_MERITS + choice];
        else
          *rflags |= F_LSFAIL;
        C.scal[S_NSQP] += 1.f;
      }
      break;
    }
    default: break;
  }
}

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

cudaError_t configure_fused(size_t smem) {
  if (smem > SMEM_LIMIT_BYTES) return cudaErrorInvalidValue;
  cudaError_t e = configure_kernel<true, false>(smem);
  if (e == cudaSuccess) e = configure_kernel<false, false>(smem);
  if (e == cudaSuccess) e = configure_fused_hp(smem);
  num_sms();
  return e;
}

template <bool REG>
static cudaError_t active_clusters_t(int csize, size_t smem, int* out) {
  cudaError_t e = configure_kernel<REG, false>(smem);
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
  return cudaOccupancyMaxActiveClusters(out, sqp_fused<REG, false>, &cfg);
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
  const bool reg = !use_throughput_variant(a.n, a.csize, a.variant, smem);
  if (a.prm.high) return launch_fused_hp(a, smem, s, reg);
  cudaError_t e = reg ? launch_kernel<true, false>(a, smem, s) : launch_kernel<false, false>(a, smem, s);
  if (e != cudaSuccess || !(a.prm.escalate && a.prm.kkt_tol > 0.f)) return e;
  // the solves that escalated continue in the high-precision kernel
  FusedLaunch r = a;
  r.resume = 1;
  return launch_fused_hp(r, smem, s, reg);
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
