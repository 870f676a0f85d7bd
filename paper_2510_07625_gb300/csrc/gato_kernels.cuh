// Kernel templates of the batched SQP solver (GATO, arXiv 2510.07625, Alg. 1).
//
// sqp_fused: the persistent fused form.  One thread-block cluster per solve
//   runs every SQP iteration of that solve (linearise -> Schur -> PCG ->
//   recover -> line search) with the PCG working set on chip (block rows in
//   registers, vectors in shared memory) and exits on its own convergence.
//   Clusters are launched longest horizon first.
// The plain form (sqp_plain_stage, gato_kernels.cu) is the comparison
// baseline: the same stage functions, but each stage of each SQP iteration of
// one solve is a separate launch and every array lives in global memory.
#pragma once

#include "gato_internal.h"
#include "gato_phases.cuh"

namespace gato {

__device__ __forceinline__ void bind_workspace(Ctx& C, float* ws, const WsLayout& L) {
  C.X = ws + L.X;
  C.U = ws + L.U;
  C.dX = ws + L.dX;
  C.dU = ws + L.dU;
  C.Fq = ws + L.Fq;
  C.Fv = ws + L.Fv;
  C.Mi = ws + L.Mi;
  C.qdd = ws + L.qdd;
  C.dT = ws + L.dT;
  C.Qi = ws + L.Qi;
  C.Ri = ws + L.Ri;
  C.qg = ws + L.qg;
  C.rg = ws + L.rg;
  C.cv = ws + L.cv;
  C.Jk = ws + L.Jk;
  C.Dx = ws + L.Dx;
  C.Du = ws + L.Du;
  C.nu = ws + L.nu;
  C.Xlo = ws + L.Xlo;
  C.Ulo = ws + L.Ulo;
  C.LV = reinterpret_cast<LinkRec*>(ws + L.LV);
}

__device__ __forceinline__ void bind_problem(Ctx& C, const ProbDesc& P, const DevModel* M) {
  C.N = P.N;
  C.dof = P.dof;
  C.cost_kind = P.cost_kind;
  C.h = P.dt;
#pragma unroll
  for (int i = 0; i < 6; ++i) C.w[i] = P.w[i];
  C.x_ref = P.x_ref;
  C.ee_ref = P.ee_ref;
  C.M = M;
}

// Knot range of cluster rank r for a solve of horizon N on csize CTAs.
__device__ __forceinline__ void bind_partition(Ctx& C, int rank, int csize) {
  const int kpc = kpc_for(C.N, csize);
  const int K = C.N + 1;
  C.rank = rank;
  C.csize = csize;
  C.k0 = min(rank * kpc, K);
  C.k1 = min(C.k0 + kpc, K);
}

// Hand-over record of an escalating solve (ints in the solve's workspace at
// WsLayout::hand): the FP32 kernel stops where a solve escalates and the
// high-precision kernel, launched after it, resumes that iteration from the
// workspace.  The two instantiations keep the high-precision stages out of
// the FP32 kernel entirely, so they add no register pressure to its PCG.
enum : int {
  H_PENDING = 0,  // 1: the solve escalated and waits for the high-precision kernel
  H_IT,           // the SQP iteration to repeat
  H_SQP,          // SQP iterations completed
  H_PCG,          // PCG iterations so far
  H_FLAGS,        // result flags so far
  H_PCG_AT,       // PCG iterations when iteration H_IT began (for its log record)
  H_RHO,          // the solve's (possibly adapted) rho, float bits
  H_COUNT
};

// The whole SQP loop of one solve (Sec. II-A Steps 1-3, repeated).  HP
// false: FP32 throughout; where the precision mode asks to escalate, the
// solve's state goes to `hand` and the loop stops without a result.  HP true:
// the high-precision mode throughout, either from the start or, with
// `resume`, from the hand-over record of an escalated solve (a solve without
// one returns at once).
template <bool REG, bool HP>
__device__ void sqp_solve(Ctx& C, const ProbDesc& P, const Params& prm, int iters, Result* out, int* hand,
                          bool resume, int* itlog = nullptr, int itlog_iters = 0) {
  int rbuf = 0;
  long long tl = C.tm ? clock64() : 0;
  const bool logging = itlog && C.rank == 0 && threadIdx.x == 0;
  C.hp = HP ? 1 : 0;
  int flags = 0, sqp = 0, pcg_total = 0;
  float kkt = 0.f, merit = 0.f;
  bool base_stale = true;  // the iterate's own merit is due (first iteration, or after escalating)
  int pcg_at_start = 0;    // pcg_total when the iteration began (for the log)
  int it = 0;
  if (HP && resume) {
    // every thread of the cluster reads the same record: the exit is uniform
    const volatile int* h = hand;
    if (h[H_PENDING] == 0) return;
    it = h[H_IT];
    sqp = h[H_SQP];
    pcg_total = h[H_PCG];
    flags = h[H_FLAGS];
    pcg_at_start = h[H_PCG_AT];
    C.w[5] = __int_as_float(h[H_RHO]);
    // the iterate, multipliers and low parts (zero in FP32) stay in the
    // workspace; only x_s is shared-memory state (padded, as load_iterate
    // leaves it: the padding rows of the knot-0 defect read it)
    if (threadIdx.x < VS) C.xs[threadIdx.x] = 0.f;
    __syncthreads();
    if (threadIdx.x < 2 * C.dof) C.xs[pad_state(threadIdx.x, C.dof)] = P.x_s[threadIdx.x];
    csync(C);
  } else {
    if (logging)
      for (int i = 0; i < itlog_iters * ITLOG_W; ++i) itlog[i] = (i % ITLOG_W == 0) ? -2 : 0;
    if (!HP && C.rank == 0 && threadIdx.x == 0) hand[H_PENDING] = 0;
    load_iterate(C, P);
    csync(C);
  }
  tstamp(C, T_LOAD, tl);
  bool escalated = false;     // FP32 kernel: the solve's state went to the hand-over record
  bool resuming = HP && resume;  // the first pass repeats the hand-over iteration
  for (;; ++it) {
    if (!resuming) {
      if (it == iters && !(prm.kkt_tol > 0.f)) break;
      pcg_at_start = pcg_total;
    }
    resuming = false;
    st_mass_bias(C);
    __syncthreads();
    tstamp(C, T_MASS, tl);
    st_forward_dynamics(C);
    __syncthreads();
    tstamp(C, T_FD, tl);
    st_value_and_cost(C);
    __syncthreads();
    tstamp(C, T_VALUE, tl);
    st_tangents(C);
    __syncthreads();
    tstamp(C, T_TANGENT, tl);
    st_dyn_jacobians(C);
    csync(C);  // defect c_k0 comes from the neighbour's last knot
    tstamp(C, T_JAC, tl);
    st_kkt_merit(C, prm.mu, rbuf);
    if (base_stale) {  // the iterate's merit, by the code that evaluates the trial merits
      st_line_search(C, prm.mu, prm.beta, prm.n_alpha, rbuf, true);
      base_stale = false;
    }
    tstamp(C, T_KKT, tl);
    kkt = C.scal[S_KKT];
    merit = C.scal[S_MERIT0];
    // the KKT stage left the cluster-wide non-finite flag in every CTA
    if (*reinterpret_cast<volatile int*>(C.scal + S_FLAGS)) {
      flags |= F_NONFINITE;
      break;
    }
    if (prm.kkt_tol > 0.f && kkt <= prm.kkt_tol) {
      if (!HP && prm.escalate) {
        // confirm convergence with the high-precision residual: the FP32
        // dual residual carries the kappa(M)-amplified error of A_k
        escalated = true;
        break;
      }
      flags |= F_CONVERGED;
      break;
    }
    if (it == iters) {
      flags |= F_MAXITER;
      break;
    }
    st_schur(C);
    __syncthreads();
    tstamp(C, T_SCHUR, tl);
    if (prm.linsolve == 1) {  // direct block elimination instead of PCG
      st_direct(C);
      if (cluster_flag(C, rbuf)) {
        flags |= F_NONFINITE;
        break;
      }
      tstamp(C, T_BINV, tl);
    } else {
      st_block_inverse(C);
      if (cluster_flag(C, rbuf)) {
        flags |= F_NONFINITE;
        break;
      }
      tstamp(C, T_BINV, tl);
      bool hit = false;
      pcg_total += st_pcg<REG, HP>(C, prm.pcg_eps, prm.pcg_max, prm.precond, &hit, rbuf);
      if (hit) flags |= F_PCGMAX;
    }
    if (C.tm && C.rank == 0 && threadIdx.x == 0) tl = clock64();
    st_recover(C);
    if (cluster_flag(C, rbuf)) {
      flags |= F_NONFINITE;
      break;
    }
    tstamp(C, T_RECOVER, tl);
    st_line_search(C, prm.mu, prm.beta, prm.n_alpha, rbuf);
    tstamp(C, T_LS, tl);
    const float m_base[2] = {C.scal[S_MDF], C.scal[S_MDF + 1]};
    const float m_full[2] = {C.scal[S_MDF + 2], C.scal[S_MDF + 3]};
    const int choice = st_accept(C, prm.beta, prm.n_alpha);
    csync(C);
    if (!HP && choice < 0 && prm.escalate && prm.kkt_tol > 0.f) {
      // the FP32 line search found no decrease: repeat this iteration in the
      // high-precision mode (every thread takes the same branch)
      escalated = true;
      break;
    }
    if (logging && it < itlog_iters) {
      int* r = itlog + it * ITLOG_W;
      r[0] = choice;
      r[1] = pcg_total - pcg_at_start;
      r[2] = __float_as_int(kkt);
      r[3] = C.hp;
      r[4] = __float_as_int(m_base[0]);
      r[5] = __float_as_int(m_base[1]);
      r[6] = __float_as_int(m_full[0]);
      r[7] = __float_as_int(m_full[1]);
    }
    if (prm.rho_adapt) C.w[5] = rho_next(C.w[5], choice);  // every thread, the same choice
    tstamp(C, T_ACCEPT, tl);
    if (choice >= 0)
      merit = C.scal[S_MERITS + choice];
    else
      flags |= F_LSFAIL;
    ++sqp;
  }
  csync(C);
  if (!HP && escalated) {
    if (C.rank == 0 && threadIdx.x == 0) {
      hand[H_IT] = it;
      hand[H_SQP] = sqp;
      hand[H_PCG] = pcg_total;
      hand[H_FLAGS] = flags;
      hand[H_PCG_AT] = pcg_at_start;
      hand[H_RHO] = __float_as_int(C.w[5]);
      hand[H_PENDING] = 1;
    }
    return;
  }
  store_iterate(C, P);
  if (C.rank == 0 && threadIdx.x == 0) {
    out->flags = flags;
    out->sqp_iters = sqp;
    out->pcg_iters = pcg_total;
    out->kkt = kkt;
    out->merit = merit;
  }
}

// REG = true: 1 CTA per SM, all PCG block rows in registers (latency);
// REG = false: 2 CTAs per SM, off-diagonal rows read from shared memory (throughput).
// HP = false: the FP32 solve (escalating solves stop at a hand-over record);
// HP = true: the high-precision mode, from the start or (a.resume) resuming
// the hand-over records of the FP32 launch before it on the same stream.
template <bool REG, bool HP>
__global__ void __launch_bounds__(NTHR, REG ? 1 : 2) sqp_fused(FusedLaunch a) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int csize = a.csize;
  const int rank = csize > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int b = a.order ? a.order[blockIdx.x / csize] : blockIdx.x / csize;
  const ProbDesc P = a.probs[b];
  static_assert(sizeof(DevModel) <= 96 * sizeof(float), "model slot");
  for (int i = threadIdx.x; i < (int)(sizeof(DevModel) / sizeof(float)); i += NTHR)
    sm[i] = reinterpret_cast<const float*>(a.models + P.model)[i];
  float* scal = sm + 96;
  float* red = scal + SCAL_FLOATS;
  float* xs = red + 2 * RED_SLOTS * RED_W;
  float* vb = xs + 16;
  const int kpc = kpc_for(a.nmax, csize);
  const int vstride = (kpc + 4) * VW;  // knots k0-2 .. k1+1
  float* blocks = vb + NVEC * vstride;
  float* zblock = blocks + (3 * kpc + 1) * BS;  // 196 zeros (L_{N+1})
  float* ws = a.ws + (size_t)b * a.ws_stride;
  Ctx C;
  bind_problem(C, P, reinterpret_cast<const DevModel*>(sm));
  bind_workspace(C, ws, a.layout);
  bind_partition(C, rank, csize);
  C.xs = xs;
  C.red = red;
  C.scal = scal;
  // stage counters accumulate in shared memory (thread 0 of rank 0) and are
  // added to the solve's global counters once at the end
  __shared__ long long tm_sh[T_COUNT];
  if (threadIdx.x < T_COUNT) tm_sh[threadIdx.x] = 0;
  C.tm = a.timing ? tm_sh : nullptr;
  C.Dm = blocks;
  C.Lm = blocks + kpc * BS;
  C.Pm = blocks + (2 * kpc + 1) * BS;
  C.bk0 = C.k0;
  C.Lz = zblock;
  C.vb = vb;
  C.vstride = vstride;
  C.vk0 = C.k0 - 2;
  C.vbl = nullptr;
  C.vbr = nullptr;
  C.vk0l = C.vk0r = 0;
  C.hrep = REG && csize > 1;
  if (csize > 1) {
    cg::cluster_group cl = cg::this_cluster();
    const int skpc = kpc_for(C.N, csize);
    if (rank > 0 && C.k0 > 0 && C.k0 < C.k1) {
      C.vbl = cl.map_shared_rank(vb, rank - 1);
      C.vk0l = min((rank - 1) * skpc, C.N + 1) - 2;
    }
    if (rank < csize - 1 && C.k1 <= C.N && C.k0 < C.k1) {
      C.vbr = cl.map_shared_rank(vb, rank + 1);
      C.vk0r = C.k1 - 2;
    }
  }
  if (threadIdx.x < SCAL_FLOATS) {  // the force read from the descriptor in memory, not P's copy
    const int t = threadIdx.x - S_FEXT;
    scal[threadIdx.x] = (t >= 0 && t < 3) ? a.probs[b].fext[t] : 0.f;
  }
  for (int i = threadIdx.x; i < 196; i += NTHR) zblock[i] = 0.f;
  __syncthreads();
  sqp_solve<REG, HP>(C, P, a.prm, a.iters, a.results + b, reinterpret_cast<int*>(ws + a.layout.hand),
                     a.resume != 0, a.itlog ? a.itlog + (size_t)b * a.itlog_iters * ITLOG_W : nullptr,
                     a.itlog_iters);
  if (a.timing) {
    __syncthreads();
    if (rank == 0 && threadIdx.x < T_COUNT) a.timing[(size_t)b * T_COUNT + threadIdx.x] += tm_sh[threadIdx.x];
  }
}

// Shared-memory attribute of one fused instantiation, set once per device for
// launches of up to `smem` bytes.
template <bool REG, bool HP>
cudaError_t configure_kernel(size_t smem) {
  static size_t done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (smem > done[dev]) {
    e = cudaFuncSetAttribute(sqp_fused<REG, HP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    done[dev] = smem;
  }
  return cudaSuccess;
}

// One launch of a fused instantiation: a.n clusters of a.csize CTAs.
template <bool REG, bool HP>
cudaError_t launch_kernel(const FusedLaunch& a, size_t smem, cudaStream_t s) {
  cudaError_t e = configure_kernel<REG, HP>(smem);
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
  return cudaLaunchKernelEx(&cfg, sqp_fused<REG, HP>, a);
}

}  // namespace gato
