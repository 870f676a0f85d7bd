// Kernel templates of the batched SQP solver (GATO, arXiv 2510.07625, Alg. 1).
//
// sqp_fused: the persistent fused form.  One thread-block cluster per solve
//   runs every SQP iteration of that solve (linearise -> Schur -> PCG ->
//   recover -> line search) with the PCG working set on chip (block rows in
//   registers, vectors in shared memory) and exits on its own convergence.
//   Clusters are launched longest horizon first.
// sqp_plain_stage: the plain form used as the comparison baseline.  The same
//   stage functions, but each stage of each SQP iteration of one solve is a
//   separate launch and every array lives in global memory.
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

// The whole SQP loop of one solve (Sec. II-A Steps 1-3, repeated).
template <bool REG>
__device__ void sqp_solve(Ctx& C, const ProbDesc& P, const Params& prm, int iters, Result* out,
                          int* itlog = nullptr, int itlog_iters = 0) {
  int rbuf = 0;
  long long tl = C.tm ? clock64() : 0;
  const bool logging = itlog && C.rank == 0 && threadIdx.x == 0;
  C.hp = prm.high ? 1 : 0;
  if (logging)
    for (int i = 0; i < itlog_iters * ITLOG_W; ++i) itlog[i] = (i % ITLOG_W == 0) ? -2 : 0;
  load_iterate(C, P);
  csync(C);
  tstamp(C, T_LOAD, tl);
  int flags = 0, sqp = 0, pcg_total = 0;
  float kkt = 0.f, merit = 0.f;
  bool base_stale = true;  // the iterate's own merit is due (first iteration, or after escalating)
  int pcg_at_start = 0;    // pcg_total when the iteration began (for the log)
  for (int it = 0;; ++it) {
    if (it == iters && !(prm.kkt_tol > 0.f)) break;
    pcg_at_start = pcg_total;
  retry:
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
      if (prm.escalate && !C.hp) {
        // confirm convergence with the high-precision residual: the FP32
        // dual residual carries the kappa(M)-amplified error of A_k
        C.hp = 1;
        base_stale = true;
        goto retry;
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
      pcg_total += st_pcg<REG>(C, prm.pcg_eps, prm.pcg_max, prm.precond, &hit, rbuf);
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
    if (choice < 0 && prm.escalate && prm.kkt_tol > 0.f && !C.hp) {
      // the FP32 line search found no decrease: repeat this iteration in the
      // high-precision mode (every thread takes the same branch)
      C.hp = 1;
      base_stale = true;
      goto retry;
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
template <bool REG>
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
  sqp_solve<REG>(C, P, a.prm, a.iters, a.results + b,
                 a.itlog ? a.itlog + (size_t)b * a.itlog_iters * ITLOG_W : nullptr, a.itlog_iters);
  if (a.timing) {
    __syncthreads();
    if (rank == 0 && threadIdx.x < T_COUNT) a.timing[(size_t)b * T_COUNT + threadIdx.x] += tm_sh[threadIdx.x];
  }
}

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

}  // namespace gato
