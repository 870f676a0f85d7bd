// Kernel templates of the batched SQP solver (GATO, arXiv 2510.07625, Alg. 1).
//
// sqp_fused: the persistent fused form.  One CTA per solve runs every SQP
//   iteration of that solve (linearise -> Schur -> PCG -> recover -> line
//   search) with the PCG working set in shared memory, and exits on its own
//   convergence.  Blocks are launched longest horizon first.
// sqp_plain_stage: the plain form used as the comparison baseline.  The same
//   stage functions, but each stage of each SQP iteration of one solve is a
//   separate single-CTA launch and every array lives in global memory.
#pragma once

#include "gato_internal.h"

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
  C.Li = ws + L.Li;
  C.Dx = ws + L.Dx;
  C.Du = ws + L.Du;
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

__device__ __forceinline__ void bind_vectors(Ctx& C, float* v, size_t VV) {
  C.nu = v;
  C.rr = v + VV;
  C.pb0 = v + 2 * VV;
  C.pb1 = v + 3 * VV;
  C.qv = v + 4 * VV;
  C.yv = v + 5 * VV;
  C.wv = v + 6 * VV;
  C.zv = v + 7 * VV;
  C.rhs = v + 8 * VV;
  C.dnu = v + 9 * VV;
}

__device__ __forceinline__ int sflags(const Ctx& C) {
  return *reinterpret_cast<volatile int*>(C.scal + S_FLAGS);
}

// The whole SQP loop of one solve (Sec. II-A Steps 1-3, repeated).
template <int NT>
__device__ void sqp_solve(Ctx& C, const ProbDesc& P, const Params& prm, int iters, Result* out) {
  load_iterate<NT>(C, P);
  int flags = 0, sqp = 0, pcg_total = 0;
  float kkt = 0.f, merit = 0.f;
  for (int it = 0;; ++it) {
    if (it == iters && !(prm.kkt_tol > 0.f)) break;
    st_mass_bias<NT>(C);
    __syncthreads();
    st_forward_dynamics<NT>(C);
    __syncthreads();
    st_value_and_cost<NT>(C);
    __syncthreads();
    st_tangents<NT>(C);
    __syncthreads();
    st_dyn_jacobians<NT>(C);
    __syncthreads();
    st_kkt_merit<NT>(C, prm.mu);
    kkt = C.scal[S_KKT];
    merit = C.scal[S_MERIT0];
    if (sflags(C)) {
      flags |= F_NONFINITE;
      break;
    }
    if (prm.kkt_tol > 0.f && kkt <= prm.kkt_tol) {
      flags |= F_CONVERGED;
      break;
    }
    if (it == iters) {
      flags |= F_MAXITER;
      break;
    }
    st_schur<NT>(C);
    __syncthreads();
    st_block_inverse<NT>(C);
    __syncthreads();
    if (sflags(C)) {
      flags |= F_NONFINITE;
      break;
    }
    bool hit = false;
    pcg_total += st_pcg<NT>(C, prm.pcg_eps, prm.pcg_max, prm.precond, &hit);
    if (hit) flags |= F_PCGMAX;
    st_recover<NT>(C);
    __syncthreads();
    if (sflags(C)) {
      flags |= F_NONFINITE;
      break;
    }
    st_line_search<NT>(C, prm.mu, prm.beta, prm.n_alpha);
    const int choice = st_accept<NT>(C, prm.beta, prm.n_alpha);
    if (choice >= 0)
      merit = C.scal[S_MERITS + choice];
    else
      flags |= F_LSFAIL;
    ++sqp;
  }
  __syncthreads();
  store_iterate<NT>(C, P);
  if (threadIdx.x == 0) {
    out->flags = flags;
    out->sqp_iters = sqp;
    out->pcg_iters = pcg_total;
    out->kkt = kkt;
    out->merit = merit;
  }
}

template <int NT, bool SB>
__global__ void __launch_bounds__(NT, 1) sqp_fused(FusedLaunch a) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int b = a.order ? a.order[blockIdx.x] : blockIdx.x;
  const ProbDesc P = a.probs[b];
  static_assert(sizeof(DevModel) <= 96 * sizeof(float), "model slot");
  for (int i = threadIdx.x; i < (int)(sizeof(DevModel) / sizeof(float)); i += NT)
    sm[i] = reinterpret_cast<const float*>(a.models + P.model)[i];
  float* scal = sm + 96;
  float* red = scal + 64;
  float* xs = red + 128;
  float* vec = xs + 16;
  const size_t K = (size_t)a.nmax + 1, VV = K * VS;
  float* ws = a.ws + (size_t)b * a.ws_stride;
  Ctx C;
  bind_problem(C, P, reinterpret_cast<const DevModel*>(sm));
  bind_workspace(C, ws, a.layout);
  bind_vectors(C, vec, VV);
  if (SB) {
    float* blocks = vec + NVEC_SMEM * VV;
    C.Dm = blocks;
    C.Lm = blocks + K * BS;
    C.Pm = blocks + 2 * K * BS;
  } else {
    C.Dm = ws + a.layout.Dm;
    C.Lm = ws + a.layout.Lm;
    C.Pm = ws + a.layout.Pm;
  }
  C.xs = xs;
  C.red = red;
  C.scal = scal;
  if (threadIdx.x < 64) scal[threadIdx.x] = 0.f;
  __syncthreads();
  sqp_solve<NT>(C, P, a.prm, a.iters, a.results + b);
}

// ----------------------------------------------------------------- plain form

struct PlainArgs {
  const ProbDesc* probs;
  const DevModel* models;
  Result* results;
  float* ws;
  WsLayout layout;
  int b, nmax, iters, it;
  Params prm;
};

enum : int { S_DONE = 12, S_NSQP = 13, S_NPCG = 14, S_RFLAGS = 15 };

template <int NT>
__global__ void __launch_bounds__(NT, 1) sqp_plain_stage(int stage, PlainArgs a) {
  __shared__ float red[128];
  const ProbDesc P = a.probs[a.b];
  const size_t K = (size_t)a.nmax + 1, VV = K * VS;
  Ctx C;
  bind_problem(C, P, a.models + P.model);
  bind_workspace(C, a.ws, a.layout);
  float* vec = a.ws + a.layout.vec;
  bind_vectors(C, vec, VV);
  C.Dm = a.ws + a.layout.Dm;
  C.Lm = a.ws + a.layout.Lm;
  C.Pm = a.ws + a.layout.Pm;
  C.scal = vec + 12 * VV;
  C.xs = C.scal + 64;
  C.red = red;
  const Params& prm = a.prm;
  int* rflags = reinterpret_cast<int*>(C.scal + S_RFLAGS);
  if (stage == PS_LOAD) {
    if (threadIdx.x < 64) C.scal[threadIdx.x] = 0.f;
    __syncthreads();
    load_iterate<NT>(C, P);
    return;
  }
  if (stage == PS_STORE) {
    store_iterate<NT>(C, P);
    if (threadIdx.x == 0) {
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
  switch (stage) {
    case PS_MASS: st_mass_bias<NT>(C); break;
    case PS_FD: st_forward_dynamics<NT>(C); break;
    case PS_VALUE: st_value_and_cost<NT>(C); break;
    case PS_TANGENT: st_tangents<NT>(C); break;
    case PS_JAC: st_dyn_jacobians<NT>(C); break;
    case PS_KKT: {
      st_kkt_merit<NT>(C, prm.mu);
      if (threadIdx.x == 0) {
        C.scal[S_MERITF] = C.scal[S_MERIT0];
        int f = *rflags;
        bool done = false;
        if (sflags(C)) {
          f |= F_NONFINITE;
          done = true;
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
    case PS_SCHUR: st_schur<NT>(C); break;
    case PS_BINV:
      st_block_inverse<NT>(C);
      __syncthreads();
      if (threadIdx.x == 0 && sflags(C)) {
        *rflags |= F_NONFINITE;
        C.scal[S_DONE] = 1.f;
      }
      break;
    case PS_PCG: {
      bool hit = false;
      const int n = st_pcg<NT>(C, prm.pcg_eps, prm.pcg_max, prm.precond, &hit);
      if (threadIdx.x == 0) {
        C.scal[S_NPCG] += (float)n;
        if (hit) *rflags |= F_PCGMAX;
      }
      break;
    }
    case PS_RECOVER:
      st_recover<NT>(C);
      __syncthreads();
      if (threadIdx.x == 0 && sflags(C)) {
        *rflags |= F_NONFINITE;
        C.scal[S_DONE] = 1.f;
      }
      break;
    case PS_LS: st_line_search<NT>(C, prm.mu, prm.beta, prm.n_alpha); break;
    case PS_ACCEPT: {
      const int choice = st_accept<NT>(C, prm.beta, prm.n_alpha);
      if (threadIdx.x == 0) {
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

// Launches one instantiation of the fused kernel.
template <int NT, bool SB>
cudaError_t launch_fused_t(const FusedLaunch& a, size_t smem, cudaStream_t s) {
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(sqp_fused<NT, SB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  sqp_fused<NT, SB><<<a.n, NT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused_288(const FusedLaunch& a, size_t smem, bool sb, cudaStream_t s);
cudaError_t launch_fused_544(const FusedLaunch& a, size_t smem, bool sb, cudaStream_t s);

}  // namespace gato
