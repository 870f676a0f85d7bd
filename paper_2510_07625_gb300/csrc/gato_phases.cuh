// The stages of one SQP iteration (GATO, arXiv 2510.07625, Alg. 1) as
// block-level device functions.  One thread block works on one solve.
//
// Thread mapping for knot-row work: each warp covers 4 knots with 7 lanes per
// knot (lanes 28..31 idle); lane j of a knot owns state rows j (q_j) and j+7
// (qd_j) of every block row of that knot.  The 7 lanes of a knot share a warp,
// so dependencies inside one knot need only __syncwarp; dependencies between
// knots and the dot-product reductions use __syncthreads.
//
// Storage: a solve's hot arrays (Schur blocks, preconditioner blocks, PCG
// vectors) are addressed through the Ctx pointers, which the fused kernel
// points at shared memory and the plain form at global memory.  Blocks are
// 14x14 column-major with stride BS; vectors use stride VS per knot.
#pragma once

#include "gato_device.cuh"

namespace gato {

struct Ctx {
  int N, dof, cost_kind;
  float h;
  float w[6];
  const float* x_ref;   // user layout, (N+1) x 2*dof
  const float* ee_ref;  // (N+1) x 3
  const DevModel* M;
  float* xs;            // padded x_s [VS]
  // global workspace
  float *X, *U, *dX, *dU, *Fq, *Fv, *Mi, *qdd, *dT, *Qi, *Ri, *qg, *rg, *cv, *Jk, *Li;
  float *Dx, *Du;       // dual residual d = g + C^T nu at the current linearisation
  LinkRec* LV;
  // hot arrays (shared or global)
  float *Dm, *Lm, *Pm, *nu, *rr, *pb0, *pb1, *qv, *yv, *wv, *zv, *rhs, *dnu;
  // reductions (always shared): red[2][32][2], scal[64]
  float* red;
  float* scal;
};

// scal[] slots
enum : int {
  S_KKT = 0, S_MERIT0, S_CMAX, S_GMAX, S_DMAX, S_ALPHA, S_FLAGS, S_PCG, S_ITERS, S_MERITF,
  S_CHOICE, S_REDBUF, S_MERITS = 16  // S_MERITS..S_MERITS+15: trial merits
};

// Per-knot strides of the global workspace arrays.
constexpr int FQS = 49, QIS = 56, DTS = 14 * 8, LIS = 196;

struct WsLayout {
  size_t X, U, dX, dU, Fq, Fv, Mi, qdd, dT, Qi, Ri, qg, rg, cv, Jk, Li, LV, Dm, Lm, Pm, vec, Dx, Du,
      total;
};

__host__ __device__ inline size_t align32(size_t n) { return (n + 31) & ~size_t(31); }

// Offsets (floats) of one solve's workspace for horizon up to Nmax.  Blocks and
// vectors are included only when `global_hot` (plain form or long horizons).
__host__ __device__ inline WsLayout ws_layout(int Nmax, bool global_blocks, bool global_vecs) {
  WsLayout L;
  size_t o = 0;
  const size_t K = Nmax + 1;
  L.X = o; o += align32(K * VS);
  L.U = o; o += align32(Nmax * US);
  L.dX = o; o += align32(K * VS);
  L.dU = o; o += align32(Nmax * US);
  L.Fq = o; o += align32(Nmax * FQS);
  L.Fv = o; o += align32(Nmax * FQS);
  L.Mi = o; o += align32(Nmax * FQS);
  L.qdd = o; o += align32(Nmax * US);
  L.dT = o; o += align32(Nmax * DTS);
  L.Qi = o; o += align32(K * QIS);
  L.Ri = o; o += align32(Nmax * US);
  L.qg = o; o += align32(K * VS);
  L.rg = o; o += align32(Nmax * US);
  L.cv = o; o += align32(K * VS);
  L.Jk = o; o += align32(K);
  L.Li = o; o += align32(K * LIS);
  L.LV = o; o += align32(Nmax * QM * LVS);
  L.Dx = o; o += align32(K * VS);
  L.Du = o; o += align32(Nmax * US);
  if (global_blocks) {
    L.Dm = o; o += align32(K * BS);
    L.Lm = o; o += align32(K * BS);
    L.Pm = o; o += align32(K * BS);
  } else {
    L.Dm = L.Lm = L.Pm = 0;
  }
  if (global_vecs) {
    L.vec = o; o += align32(12 * K * VS + 128);
  } else {
    L.vec = 0;
  }
  L.total = align32(o);
  return L;
}

// Vector slots of the fused kernel's shared-memory layout.
constexpr int NVEC_SMEM = 10;

// Shared-memory floats of the fused kernel for horizon Nmax.
__host__ __device__ inline size_t smem_floats(int Nmax, bool smem_blocks) {
  const size_t K = Nmax + 1;
  size_t f = 96 /*model*/ + 64 /*scal*/ + 128 /*red*/ + 16 /*xs*/;
  f += NVEC_SMEM * K * VS;  // nu rr p0 p1 q y w z rhs + 1 spare
  if (smem_blocks) f += 3 * K * BS;
  return align32(f);
}

// ------------------------------------------------------------ small helpers

__device__ __forceinline__ int pad_state(int ui, int dof) { return ui < dof ? ui : QM + (ui - dof); }

__device__ __forceinline__ float& blk(float* base, int k, int r, int c) { return base[k * BS + c * XM + r]; }

__device__ __forceinline__ float xref_at(const Ctx& C, int k, int i) {
  const int nx = 2 * C.dof;
  const int ii = i < QM ? i : i - QM;
  if (ii >= C.dof) return 0.f;
  return C.x_ref[k * nx + (i < QM ? ii : C.dof + ii)];
}

// Element (r, c) of A_k = [[I + h^2 Fq, hI + h^2 Fv], [h Fq, I + h Fv]].
__device__ __forceinline__ float A_elem(const float* Fq, const float* Fv, float h, int r, int c) {
  if (r < QM) {
    if (c < QM) return (r == c ? 1.f : 0.f) + h * h * Fq[r * QM + c];
    return (r == c - QM ? h : 0.f) + h * h * Fv[r * QM + c - QM];
  }
  if (c < QM) return h * Fq[(r - QM) * QM + c];
  return (r == c ? 1.f : 0.f) + h * Fv[(r - QM) * QM + c - QM];
}

// c_r = h (h v_r + v_{7+r}): the common factor of A^T v and B^T v.
__device__ __forceinline__ void at_factor(const float* v, float h, float* cfac) {
#pragma unroll
  for (int r = 0; r < QM; ++r) cfac[r] = h * (h * v[r] + v[QM + r]);
}

// (A^T v)_i for rows i = j and j+7, given c_r.
__device__ __forceinline__ void at_rows(const float* Fq, const float* Fv, const float* v,
                                        const float* cfac, float h, int j, float& o0, float& o1) {
  float a0 = v[j], a1 = h * v[j] + v[QM + j];
#pragma unroll
  for (int r = 0; r < QM; ++r) {
    a0 += Fq[r * QM + j] * cfac[r];
    a1 += Fv[r * QM + j] * cfac[r];
  }
  o0 = a0;
  o1 = a1;
}

// (B^T v)_j with B = [h^2 Minv; h Minv] (Minv symmetric).
__device__ __forceinline__ float bt_row(const float* Mi, const float* cfac, int j) {
  float a = 0.f;
#pragma unroll
  for (int r = 0; r < QM; ++r) a += Mi[r * QM + j] * cfac[r];
  return a;
}

__device__ __forceinline__ float Qinv_elem(const float* Qi, int r, int c) {
  if (r < QM && c < QM) return Qi[r * QM + c];
  if (r >= QM && c >= QM) return r == c ? Qi[49 + r - QM] : 0.f;
  return 0.f;
}

template <int NT>
__device__ __forceinline__ DF block_df_sum(const Ctx& C, DF v) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int buf = (int)C.scal[S_REDBUF];
  v = warp_df_sum(v);
  __syncthreads();  // everyone has read S_REDBUF
  if (lane == 0) {
    C.red[(buf * 32 + warp) * 2] = v.hi;
    C.red[(buf * 32 + warp) * 2 + 1] = v.lo;
  }
  if (threadIdx.x == 0) C.scal[S_REDBUF] = (float)(buf ^ 1);
  __syncthreads();
  // every warp reduces the per-warp partials with the same shuffle tree, so all
  // threads hold the same (deterministic) total without another barrier
  DF s = lane < NW ? DF{C.red[(buf * 32 + lane) * 2], C.red[(buf * 32 + lane) * 2 + 1]} : df_zero();
  return warp_df_sum(s);
}

template <int NT>
__device__ __forceinline__ float block_max(const Ctx& C, float v, int slot) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) C.red[(slot * 32 + warp) * 2] = v;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < NW; ++w) m = fmaxf(m, C.red[(slot * 32 + w) * 2]);
  return m;
}

#define KNOT_LOOP(NT_, NLAST)                                                     \
  const int lane_ = threadIdx.x & 31, warp_ = threadIdx.x >> 5;                   \
  const int slot_ = lane_ / 7, j = lane_ - 7 * (lane_ / 7);                       \
  for (int kb_ = 4 * warp_; kb_ <= (NLAST); kb_ += 4 * ((NT_) / 32))              \
    for (int k = kb_ + slot_, once_ = 1; once_; once_ = 0)                        \
      for (const bool act = (lane_ < 28) && (k <= (NLAST)); once_; once_ = 0)

// ------------------------------------------------------------------ loading

// Copies the solve's iterate from user layout into the padded workspace.
template <int NT>
__device__ void load_iterate(const Ctx& C, const ProbDesc& P) {
  const int N = C.N, dof = C.dof, nx = 2 * dof;
  for (int i = threadIdx.x; i < (N + 1) * VS; i += NT) C.X[i] = 0.f;
  for (int i = threadIdx.x; i < N * US; i += NT) C.U[i] = 0.f;
  for (int i = threadIdx.x; i < (N + 1) * VS; i += NT) C.nu[i] = 0.f;
  if (threadIdx.x < VS) C.xs[threadIdx.x] = 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < (N + 1) * nx; i += NT) {
    const int k = i / nx, ui = i - k * nx;
    C.X[k * VS + pad_state(ui, dof)] = P.X[i];
    if (P.lam) C.nu[k * VS + pad_state(ui, dof)] = P.lam[i];
  }
  for (int i = threadIdx.x; i < N * dof; i += NT) {
    const int k = i / dof, ui = i - k * dof;
    C.U[k * US + ui] = P.U[i];
  }
  if (threadIdx.x < nx) C.xs[pad_state(threadIdx.x, dof)] = P.x_s[threadIdx.x];
  __syncthreads();
}

template <int NT>
__device__ void store_iterate(const Ctx& C, const ProbDesc& P) {
  const int N = C.N, dof = C.dof, nx = 2 * dof;
  for (int i = threadIdx.x; i < (N + 1) * nx; i += NT) {
    const int k = i / nx, ui = i - k * nx;
    P.X[i] = C.X[k * VS + pad_state(ui, dof)];
    if (P.lam) P.lam[i] = C.nu[k * VS + pad_state(ui, dof)];
  }
  for (int i = threadIdx.x; i < N * dof; i += NT) {
    const int k = i / dof, ui = i - k * dof;
    P.U[i] = C.U[k * US + ui];
  }
}

// --------------------------------------------------- stage 1: linearisation

// Mass-matrix columns (unit-acceleration RNEA) and bias forces per knot.
template <int NT>
__device__ void st_mass_bias(const Ctx& C) {
  const int N = C.N;
  const DevModel& M = *C.M;
  for (int it = threadIdx.x; it < N * 8; it += NT) {
    const int k = it >> 3, col = it & 7;
    float sq[QM], cq[QM], qd[QM], acc[QM], tau[QM];
    const float* x = C.X + k * VS;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      sincosf(x[i], &sq[i], &cq[i]);
      qd[i] = (col == 7) ? x[QM + i] : 0.f;
      acc[i] = (i == col) ? 1.f : 0.f;
    }
    rnea_value(M, sq, cq, qd, acc, col == 7 ? M.g : 0.f, tau, nullptr);
    if (col < 7) {
#pragma unroll
      for (int r = 0; r < QM; ++r) C.Mi[k * FQS + r * QM + col] = tau[r];
    } else {
#pragma unroll
      for (int r = 0; r < QM; ++r) C.qdd[k * US + r] = tau[r];
    }
  }
}

// Cholesky of M, explicit M^-1, qdd = M^-1 (u - bias), dynamics defects.
template <int NT>
__device__ void st_forward_dynamics(const Ctx& C) {
  const int N = C.N;
  const float h = C.h;
  for (int k = threadIdx.x; k <= N; k += NT) {
    if (k == N) {
#pragma unroll
      for (int i = 0; i < XM; ++i) C.cv[i] = C.xs[i] - C.X[i];
      continue;
    }
    float Ml[28];
#pragma unroll
    for (int i = 0; i < QM; ++i)
#pragma unroll
      for (int j2 = 0; j2 <= i; ++j2)
        Ml[i * (i + 1) / 2 + j2] = 0.5f * (C.Mi[k * FQS + i * QM + j2] + C.Mi[k * FQS + j2 * QM + i]);
#pragma unroll
    for (int i = 0; i < QM; ++i)
      if (i >= C.dof) Ml[i * (i + 1) / 2 + i] = 1.f;
    const bool ok = chol7(Ml);
    if (!ok) atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
    float b[QM];
#pragma unroll
    for (int i = 0; i < QM; ++i) b[i] = C.U[k * US + i] - C.qdd[k * US + i];
    chol7_solve(Ml, b);
    const float* x = C.X + k * VS;
    const float* xn = C.X + (k + 1) * VS;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      C.qdd[k * US + i] = b[i];
      const float qdn = x[QM + i] + h * b[i];
      const float qn = x[i] + h * qdn;
      C.cv[(k + 1) * VS + i] = qn - xn[i];
      C.cv[(k + 1) * VS + QM + i] = qdn - xn[QM + i];
    }
#pragma unroll
    for (int j2 = 0; j2 < QM; ++j2) {
      float e[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) e[i] = (i == j2) ? 1.f : 0.f;
      chol7_solve(Ml, e);
#pragma unroll
      for (int i = 0; i < QM; ++i) C.Mi[k * FQS + i * QM + j2] = e[i];
    }
  }
}

// Knot cost, its gradient and the inverse of its (Gauss-Newton) Hessian.
__device__ __forceinline__ void knot_cost(const Ctx& C, int k) {
  const int N = C.N;
  const float s = (k == N) ? C.w[3] : 1.f;
  const float wq = C.w[0], wqd = C.w[1], wr = C.w[2], wee = C.w[4], rho = C.w[5];
  const float* x = C.X + k * VS;
  float* qg = C.qg + k * VS;
  float* Qi = C.Qi + k * QIS;
  float J = 0.f;
  if (C.cost_kind == 0) {
#pragma unroll
    for (int i = 0; i < XM; ++i) {
      const float wi = i < QM ? wq : wqd;
      const float d = x[i] - xref_at(C, k, i);
      J += 0.5f * s * wi * d * d;
      qg[i] = s * wi * d;
    }
#pragma unroll
    for (int i = 0; i < 49; ++i) Qi[i] = 0.f;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      Qi[i * QM + i] = 1.f / (s * wq + rho);
      Qi[49 + i] = 1.f / (s * wqd + rho);
    }
  } else {
    float p[3], Jp[3 * QM];
    fk_ee(*C.M, x, p, Jp);
    const float* pr = C.ee_ref + 3 * k;
    const float d0 = p[0] - pr[0], d1 = p[1] - pr[1], d2 = p[2] - pr[2];
    J += 0.5f * s * wee * (d0 * d0 + d1 * d1 + d2 * d2);
    float Hl[28];
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      qg[i] = s * wee * (Jp[i] * d0 + Jp[QM + i] * d1 + Jp[2 * QM + i] * d2);
#pragma unroll
      for (int j2 = 0; j2 <= i; ++j2)
        Hl[i * (i + 1) / 2 + j2] = s * wee * (Jp[i] * Jp[j2] + Jp[QM + i] * Jp[QM + j2] +
                                              Jp[2 * QM + i] * Jp[2 * QM + j2]) +
                                   (i == j2 ? rho : 0.f);
    }
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      const float v = x[QM + i];
      J += 0.5f * s * wqd * v * v;
      qg[QM + i] = s * wqd * v;
      Qi[49 + i] = 1.f / (s * wqd + rho);
    }
    if (!chol7(Hl)) atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
#pragma unroll
    for (int j2 = 0; j2 < QM; ++j2) {
      float e[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) e[i] = (i == j2) ? 1.f : 0.f;
      chol7_solve(Hl, e);
#pragma unroll
      for (int i = 0; i < QM; ++i) Qi[i * QM + j2] = e[i];
    }
  }
  if (k < N) {
    const float* u = C.U + k * US;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      J += 0.5f * wr * u[i] * u[i];
      C.rg[k * US + i] = wr * u[i];
      C.Ri[k * US + i] = 1.f / wr;
    }
  }
  C.Jk[k] = J;
}

// Value RNEA at the dynamics solution (stored for the tangent pass) + costs.
template <int NT>
__device__ void st_value_and_cost(const Ctx& C) {
  const int N = C.N;
  for (int it = threadIdx.x; it < 2 * N + 1; it += NT) {
    if (it < N) {
      const int k = it;
      float sq[QM], cq[QM], tau[QM];
      const float* x = C.X + k * VS;
#pragma unroll
      for (int i = 0; i < QM; ++i) sincosf(x[i], &sq[i], &cq[i]);
      rnea_value(*C.M, sq, cq, x + QM, C.qdd + k * US, C.M->g, tau, C.LV + k * QM);
    } else {
      knot_cost(C, it - N);
    }
  }
}

// Directional derivatives of ID along every q_j and qd_j.
template <int NT>
__device__ void st_tangents(const Ctx& C) {
  const int N = C.N;
  for (int it = threadIdx.x; it < N * 14; it += NT) {
    const int k = it / 14, d = it - 14 * k;
    float dtau[QM];
    rnea_tangent(*C.M, C.LV + k * QM, C.X + k * VS + QM, d >= QM, d % QM, dtau);
#pragma unroll
    for (int i = 0; i < QM; ++i) C.dT[k * DTS + d * 8 + i] = dtau[i];
  }
}

// dqdd/dq = -M^-1 dID/dq, dqdd/dqd = -M^-1 dID/dqd.
template <int NT>
__device__ void st_dyn_jacobians(const Ctx& C) {
  const int N = C.N;
  for (int it = threadIdx.x; it < N * 98; it += NT) {
    const int k = it / 98, e = it - 98 * k;
    const int which = e / 49, r = (e % 49) / QM, c = e % QM;
    const float* Mi = C.Mi + k * FQS + r * QM;
    const float* col = C.dT + k * DTS + (which * QM + c) * 8;
    float a = 0.f;
#pragma unroll
    for (int l = 0; l < QM; ++l) a += Mi[l] * col[l];
    (which ? C.Fv : C.Fq)[k * FQS + r * QM + c] = -a;
  }
}

// KKT residual (reading c17) and the merit of the current iterate (Eq. 3).
// Also stores the dual residual d = g + C^T nu, accumulated with compensated
// sums: near convergence d is a small difference of O(|nu|) terms, and the
// step is recovered from it through G^-1 (R^-1 = 1/w_u amplifies its error).
template <int NT>
__device__ void st_kkt_merit(const Ctx& C, float mu) {
  const int N = C.N;
  const float h = C.h, h2 = C.h * C.h;
  float cmax = 0.f, gmax = 0.f, dmax = 0.f;
  bool bad = false;
  DF jsum = df_zero(), csum = df_zero();
  KNOT_LOOP(NT, N) {
    if (act) {
      const float* nu = C.nu + k * VS;
      DF d0 = df_add(df_add(df_zero(), C.qg[k * VS + j]), nu[j]);
      DF d1 = df_add(df_add(df_zero(), C.qg[k * VS + j + QM]), nu[j + QM]);
      DF du = df_zero();
      if (k < N) {
        const float* n1 = C.nu + (k + 1) * VS;
        const float* Fq = C.Fq + k * FQS;
        const float* Fv = C.Fv + k * FQS;
        const float* Mi = C.Mi + k * FQS;
        // A^T n1: rows j (q) and j+7 (qd) of [[I + h^2 Fq, hI + h^2 Fv], [h Fq, I + h Fv]]^T
        d0 = df_add(d0, -n1[j]);
        d1 = df_fma(d1, -h, n1[j]);
        d1 = df_add(d1, -n1[j + QM]);
        du = df_add(du, C.rg[k * US + j]);
#pragma unroll
        for (int r = 0; r < QM; ++r) {
          d0 = df_fma(d0, -h2 * Fq[r * QM + j], n1[r]);
          d0 = df_fma(d0, -h * Fq[r * QM + j], n1[QM + r]);
          d1 = df_fma(d1, -h2 * Fv[r * QM + j], n1[r]);
          d1 = df_fma(d1, -h * Fv[r * QM + j], n1[QM + r]);
          du = df_fma(du, -h2 * Mi[r * QM + j], n1[r]);
          du = df_fma(du, -h * Mi[r * QM + j], n1[QM + r]);
        }
      }
      const float dv[2] = {df_val(d0), df_val(d1)};
      C.Dx[k * VS + j] = dv[0];
      C.Dx[k * VS + j + QM] = dv[1];
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        const float cvi = C.cv[k * VS + i];
        cmax = fmaxf(cmax, fabsf(cvi));
        csum = df_add(csum, fabsf(cvi));
        const float g = C.qg[k * VS + i];
        gmax = fmaxf(gmax, fabsf(g));
        dmax = fmaxf(dmax, fabsf(dv[t]));
        bad = bad || !isfinite(cvi) || !isfinite(dv[t]);
      }
      if (k < N) {
        const float g = C.rg[k * US + j];
        const float duv = df_val(du);
        C.Du[k * US + j] = duv;
        gmax = fmaxf(gmax, fabsf(g));
        dmax = fmaxf(dmax, fabsf(duv));
        bad = bad || !isfinite(duv);
      }
      if (j == 0) {
        jsum = df_add(jsum, C.Jk[k]);
        bad = bad || !isfinite(C.Jk[k]);
      }
    }
  }
  // fmaxf drops NaN, so non-finite values are flagged separately
  const float badf = block_max<NT>(C, bad ? 1.f : 0.f, 0);
  cmax = block_max<NT>(C, cmax, 1);
  gmax = block_max<NT>(C, gmax, 0);
  dmax = block_max<NT>(C, dmax, 1);
  const float J = df_val(block_df_sum<NT>(C, jsum));
  const float c1 = df_val(block_df_sum<NT>(C, csum));
  if (threadIdx.x == 0) {
    C.scal[S_KKT] = fmaxf(cmax, dmax / fmaxf(1.f, gmax));
    C.scal[S_MERIT0] = J + mu * c1;
    if (badf > 0.f || !isfinite(J))
      atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
  }
  __syncthreads();
}

// ------------------------------------------------------ stage 2: Schur form

// Eq. 5-6 blocks (reading c1/c3 signs):  L_k = phi_{k-1} = -A_{k-1} Q_{k-1}^-1,
// D_k = theta_{k-1} = A Q^-1 A^T + B R^-1 B^T + Q_k^-1 (D_0 = Q_0^-1).
// Right-hand side for the multiplier correction dnu = nu - nu_0: zeta_k and
// gamma of Eq. 5 with the gradient g replaced by the dual residual
// d = g + C^T nu_0, i.e. rhs = -c - C G^-1 d = gamma - S nu_0, the initial
// residual of the warm-started PCG, formed without cancellation.
template <int NT>
__device__ void st_schur(const Ctx& C) {
  const int N = C.N;
  const float h = C.h;
  KNOT_LOOP(NT, N) {
    const int kk = k - 1;  // the dynamics knot feeding block row k
    if (act && k == 0) {
      const float* Qi = C.Qi;
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        float acc = 0.f;
        for (int c = 0; c < XM; ++c) {
          const float qv = Qinv_elem(Qi, i, c);
          blk(C.Dm, 0, i, c) = qv;
          acc += qv * C.Dx[c];
          blk(C.Lm, 0, i, c) = 0.f;
        }
        C.rhs[i] = -C.cv[i] - acc;
      }
    }
    if (act && k > 0) {
      const float* Fq = C.Fq + kk * FQS;
      const float* Fv = C.Fv + kk * FQS;
      const float* Qi = C.Qi + kk * QIS;
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        float Arow[XM];
#pragma unroll
        for (int l = 0; l < XM; ++l) Arow[l] = A_elem(Fq, Fv, h, i, l);
#pragma unroll
        for (int c = 0; c < XM; ++c) {
          float a;
          if (c < QM) {
            a = 0.f;
#pragma unroll
            for (int l = 0; l < QM; ++l) a += Arow[l] * Qi[l * QM + c];
          } else {
            a = Arow[c] * Qi[49 + c - QM];
          }
          blk(C.Lm, k, i, c) = -a;
        }
      }
    }
    __syncwarp();
    if (act && k > 0) {
      const float* Fq = C.Fq + kk * FQS;
      const float* Fv = C.Fv + kk * FQS;
      const float* Mi = C.Mi + kk * FQS;
      const float* Ri = C.Ri + kk * US;
      const float* Qi1 = C.Qi + k * QIS;
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        float Arow[XM];
#pragma unroll
        for (int l = 0; l < XM; ++l) Arow[l] = A_elem(Fq, Fv, h, i, l);
        const float si = t == 0 ? h * h : h;
        float BRrow[QM];
#pragma unroll
        for (int m = 0; m < QM; ++m) BRrow[m] = si * Mi[j * QM + m] * Ri[m];
        for (int c = 0; c < XM; ++c) {
          // theta = -A L^T + B R^-1 B^T + Q_{k}^-1   (A Q^-1 A^T = -A L^T)
          float a = 0.f;
#pragma unroll
          for (int l = 0; l < XM; ++l) a -= Arow[l] * blk(C.Lm, k, c, l);
          const int cm = c < QM ? c : c - QM;
          const float sc = c < QM ? h * h : h;
          float bb = 0.f;
#pragma unroll
          for (int m = 0; m < QM; ++m) bb += BRrow[m] * Mi[cm * QM + m];
          blk(C.Dm, k, i, c) = a + sc * bb + Qinv_elem(Qi1, i, c);
        }
        // zeta with d: L_k d_{k-1} - B R^-1 d_u,{k-1} + Q_k^-1 d_k
        float z = 0.f;
#pragma unroll
        for (int l = 0; l < XM; ++l) z += blk(C.Lm, k, i, l) * C.Dx[kk * VS + l];
#pragma unroll
        for (int m = 0; m < QM; ++m) z -= BRrow[m] * C.Du[kk * US + m];
#pragma unroll
        for (int l = 0; l < XM; ++l) z += Qinv_elem(Qi1, i, l) * C.Dx[k * VS + l];
        C.rhs[k * VS + i] = -C.cv[k * VS + i] - z;
      }
    }
  }
}

// D_k^-1 by Cholesky: the 7 lanes of a knot factor D_k in place in Pm, invert
// the factor column by column into Li, and form L^-T L^-1.
template <int NT>
__device__ void st_block_inverse(const Ctx& C) {
  const int N = C.N;
  bool bad = false;
  KNOT_LOOP(NT, N) {
    float* P = C.Pm;
    float* Li = C.Li + (act ? k : 0) * LIS;
    if (act)
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        for (int c = 0; c < XM; ++c) blk(P, k, i, c) = blk(C.Dm, k, i, c);
      }
    __syncwarp();
    for (int c = 0; c < XM; ++c) {
      if (act && (c % QM) == j) {
        const float d2 = blk(P, k, c, c);
        bad = bad || !(d2 > 0.f);
        blk(P, k, c, c) = sqrtf(fmaxf(d2, 1e-30f));
      }
      __syncwarp();
      if (act) {
        const float d = blk(P, k, c, c);
        for (int t = 0; t < 2; ++t) {
          const int i = j + QM * t;
          if (i > c) blk(P, k, i, c) = blk(P, k, i, c) / d;
        }
      }
      __syncwarp();
      if (act) {
        for (int t = 0; t < 2; ++t) {
          const int i = j + QM * t;
          if (i > c) {
            const float lic = blk(P, k, i, c);
            for (int l = c + 1; l <= i; ++l) blk(P, k, i, l) -= lic * blk(P, k, l, c);
          }
        }
      }
      __syncwarp();
    }
    // columns j and j+7 of L^-1 (lower triangular, column-major in Li)
    if (act)
      for (int t = 0; t < 2; ++t) {
        const int cc = j + QM * t;
        for (int i = 0; i < cc; ++i) Li[cc * XM + i] = 0.f;
        Li[cc * XM + cc] = 1.f / blk(P, k, cc, cc);
        for (int i = cc + 1; i < XM; ++i) {
          float s = 0.f;
          for (int l = cc; l < i; ++l) s += blk(P, k, i, l) * Li[cc * XM + l];
          Li[cc * XM + i] = -s / blk(P, k, i, i);
        }
      }
    __syncwarp();
    if (act)
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        for (int c = 0; c < XM; ++c) {
          float s = 0.f;
          for (int l = (i > c ? i : c); l < XM; ++l) s += Li[i * XM + l] * Li[c * XM + l];
          blk(P, k, i, c) = s;
        }
      }
    __syncwarp();
  }
  if (bad) atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
}

// ------------------------------------------------------------ stage 3: PCG

// Rows j, j+7 of (S v)_k, where v_k' is produced by `vf(k', c)`.
template <class VF>
__device__ __forceinline__ void s_rows(const Ctx& C, int N, int k, int j, VF vf, float& o0, float& o1) {
  float a0 = 0.f, a1 = 0.f;
  const int i0 = j, i1 = j + QM;
#pragma unroll 2
  for (int c = 0; c < XM; ++c) {
    const float v0 = vf(k, c);
    a0 += blk(C.Dm, k, i0, c) * v0;
    a1 += blk(C.Dm, k, i1, c) * v0;
    if (k > 0) {
      const float vm = vf(k - 1, c);
      a0 += blk(C.Lm, k, i0, c) * vm;
      a1 += blk(C.Lm, k, i1, c) * vm;
    }
    if (k < N) {
      const float vp = vf(k + 1, c);
      a0 += blk(C.Lm, k + 1, c, i0) * vp;
      a1 += blk(C.Lm, k + 1, c, i1) * vp;
    }
  }
  o0 = a0;
  o1 = a1;
}

// Rows j, j+7 of (O v)_k: the off-diagonal part of S only.
__device__ __forceinline__ void o_rows(const Ctx& C, int N, int k, int j, const float* v, float& o0,
                                       float& o1) {
  float a0 = 0.f, a1 = 0.f;
  const int i0 = j, i1 = j + QM;
#pragma unroll 2
  for (int c = 0; c < XM; ++c) {
    if (k > 0) {
      const float vm = v[(k - 1) * VS + c];
      a0 += blk(C.Lm, k, i0, c) * vm;
      a1 += blk(C.Lm, k, i1, c) * vm;
    }
    if (k < N) {
      const float vp = v[(k + 1) * VS + c];
      a0 += blk(C.Lm, k + 1, c, i0) * vp;
      a1 += blk(C.Lm, k + 1, c, i1) * vp;
    }
  }
  o0 = a0;
  o1 = a1;
}

__device__ __forceinline__ void p_rows(const Ctx& C, int k, int j, const float* v, float& o0, float& o1) {
  float a0 = 0.f, a1 = 0.f;
#pragma unroll 2
  for (int c = 0; c < XM; ++c) {
    const float vc = v[k * VS + c];
    a0 += blk(C.Pm, k, j, c) * vc;
    a1 += blk(C.Pm, k, j + QM, c) * vc;
  }
  o0 = a0;
  o1 = a1;
}

// Preconditioned CG (Sec. II-B, III-B) for the multiplier correction
// S dnu = rhs, started from dnu = 0; nu_0 + dnu equals the warm-started PCG
// iterate on S nu = gamma.  Stair preconditioner (Eq. 6) applied as
// D^-1 - D^-1 O D^-1 (reading c4).  Stops when sqrt(eta / eta_0) <= eps
// (reading c8).  Returns iterations.
template <int NT>
__device__ int st_pcg(const Ctx& C, float eps, int maxit, int precond, bool* hit_max) {
  const int N = C.N;
  const bool stair = (precond == 0);
  *hit_max = false;
  // dnu = 0, r = rhs ; y = D^-1 r
  {
    KNOT_LOOP(NT, N) {
      if (act) {
        C.dnu[k * VS + j] = 0.f;
        C.dnu[k * VS + j + QM] = 0.f;
        C.rr[k * VS + j] = C.rhs[k * VS + j];
        C.rr[k * VS + j + QM] = C.rhs[k * VS + j + QM];
      }
      __syncwarp();
      if (act) {
        float y0, y1;
        p_rows(C, k, j, C.rr, y0, y1);
        C.yv[k * VS + j] = y0;
        C.yv[k * VS + j + QM] = y1;
        if (!stair) {
          C.zv[k * VS + j] = y0;
          C.zv[k * VS + j + QM] = y1;
        }
      }
    }
  }
  __syncthreads();
  DF part = df_zero();
  {
    KNOT_LOOP(NT, N) {
      if (act && stair) {
        float w0, w1;
        o_rows(C, N, k, j, C.yv, w0, w1);
        C.wv[k * VS + j] = w0;
        C.wv[k * VS + j + QM] = w1;
      }
      __syncwarp();
      if (act) {
        if (stair) {
          float t0, t1;
          p_rows(C, k, j, C.wv, t0, t1);
          C.zv[k * VS + j] = C.yv[k * VS + j] - t0;
          C.zv[k * VS + j + QM] = C.yv[k * VS + j + QM] - t1;
        }
        part = df_fma(part, C.rr[k * VS + j], C.zv[k * VS + j]);
        part = df_fma(part, C.rr[k * VS + j + QM], C.zv[k * VS + j + QM]);
      }
    }
  }
  float eta = df_val(block_df_sum<NT>(C, part));
  const float eta0 = eta;
  if (!(eta0 > 1e-30f)) return 0;
  int it = 0;
  float beta = 0.f;
  bool first = true;
  float* pold = C.pb0;
  float* pnew = C.pb1;
  while (true) {
    // q = S p_new with p_new = z + beta p_old computed on the fly
    DF pq = df_zero();
    {
      const float* zv = C.zv;
      KNOT_LOOP(NT, N) {
        if (act) {
          auto pf = [&](int kk, int c) {
            return first ? zv[kk * VS + c] : zv[kk * VS + c] + beta * pold[kk * VS + c];
          };
          float s0, s1;
          s_rows(C, N, k, j, pf, s0, s1);
          const float p0 = pf(k, j), p1 = pf(k, j + QM);
          pnew[k * VS + j] = p0;
          pnew[k * VS + j + QM] = p1;
          C.qv[k * VS + j] = s0;
          C.qv[k * VS + j + QM] = s1;
          pq = df_fma(pq, p0, s0);
          pq = df_fma(pq, p1, s1);
        }
      }
    }
    const float pqv = df_val(block_df_sum<NT>(C, pq));
    const float alpha = eta / pqv;
    DF rz = df_zero();
    {
      KNOT_LOOP(NT, N) {
        if (act) {
          for (int t = 0; t < 2; ++t) {
            const int i = k * VS + j + QM * t;
            C.dnu[i] += alpha * pnew[i];
            C.rr[i] -= alpha * C.qv[i];
          }
        }
        __syncwarp();
        if (act) {
          float y0, y1;
          p_rows(C, k, j, C.rr, y0, y1);
          C.yv[k * VS + j] = y0;
          C.yv[k * VS + j + QM] = y1;
          if (!stair) {
            C.zv[k * VS + j] = y0;
            C.zv[k * VS + j + QM] = y1;
            rz = df_fma(rz, C.rr[k * VS + j], y0);
            rz = df_fma(rz, C.rr[k * VS + j + QM], y1);
          }
        }
      }
    }
    if (stair) {
      __syncthreads();
      KNOT_LOOP(NT, N) {
        if (act) {
          float w0, w1;
          o_rows(C, N, k, j, C.yv, w0, w1);
          C.wv[k * VS + j] = w0;
          C.wv[k * VS + j + QM] = w1;
        }
        __syncwarp();
        if (act) {
          float t0, t1;
          p_rows(C, k, j, C.wv, t0, t1);
          const float z0 = C.yv[k * VS + j] - t0, z1 = C.yv[k * VS + j + QM] - t1;
          C.zv[k * VS + j] = z0;
          C.zv[k * VS + j + QM] = z1;
          rz = df_fma(rz, C.rr[k * VS + j], z0);
          rz = df_fma(rz, C.rr[k * VS + j + QM], z1);
        }
      }
    }
    const float eta_new = df_val(block_df_sum<NT>(C, rz));
    ++it;
    if (!(eta_new > 0.f) || sqrtf(eta_new / eta0) <= eps) break;
    if (it >= maxit) {
      *hit_max = true;
      break;
    }
    beta = eta_new / eta;
    eta = eta_new;
    first = false;
    float* t = pold;
    pold = pnew;
    pnew = t;
  }
  __syncthreads();
  return it;
}

// ------------------------------------------------- stage 4: step recovery

// dx_k = -Q_k^-1 (q_k + nu_k - A_k^T nu_{k+1}), du_k = -R_k^-1 (r_k - B_k^T nu_{k+1})
// (Eq. 4, reading c1), evaluated as -G^-1 (d + C^T dnu); then nu += dnu.
template <int NT>
__device__ void st_recover(const Ctx& C) {
  const int N = C.N;
  const float h = C.h;
  bool bad = false;
  KNOT_LOOP(NT, N) {
    float bt = 0.f;
    if (act) {
      float at0 = 0.f, at1 = 0.f;
      if (k < N) {
        float cf[QM];
        at_factor(C.dnu + (k + 1) * VS, h, cf);
        at_rows(C.Fq + k * FQS, C.Fv + k * FQS, C.dnu + (k + 1) * VS, cf, h, j, at0, at1);
        bt = bt_row(C.Mi + k * FQS, cf, j);
      }
      C.wv[k * VS + j] = C.Dx[k * VS + j] + C.dnu[k * VS + j] - at0;
      C.wv[k * VS + j + QM] = C.Dx[k * VS + j + QM] + C.dnu[k * VS + j + QM] - at1;
    }
    __syncwarp();
    if (act) {
      const float* Qi = C.Qi + k * QIS;
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < QM; ++l) a += Qi[j * QM + l] * C.wv[k * VS + l];
      const float dx0 = -a;
      const float dx1 = -Qi[49 + j] * C.wv[k * VS + j + QM];
      C.dX[k * VS + j] = dx0;
      C.dX[k * VS + j + QM] = dx1;
      bad = bad || !isfinite(dx0) || !isfinite(dx1);
      if (k < N) {
        const float du = -C.Ri[k * US + j] * (C.Du[k * US + j] - bt);
        C.dU[k * US + j] = du;
        bad = bad || !isfinite(du);
      }
      C.nu[k * VS + j] += C.dnu[k * VS + j];
      C.nu[k * VS + j + QM] += C.dnu[k * VS + j + QM];
    }
  }
  if (bad) atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
}

// ------------------------------------------------- stage 5: line search

__device__ __forceinline__ float trial_cost(const Ctx& C, int k, const float* x, const float* u) {
  const int N = C.N;
  const float s = (k == N) ? C.w[3] : 1.f;
  const float wq = C.w[0], wqd = C.w[1], wr = C.w[2], wee = C.w[4];
  float J = 0.f;
  if (C.cost_kind == 0) {
#pragma unroll
    for (int i = 0; i < XM; ++i) {
      const float wi = i < QM ? wq : wqd;
      const float d = x[i] - xref_at(C, k, i);
      J += 0.5f * s * wi * d * d;
    }
  } else {
    float p[3];
    fk_ee(*C.M, x, p, nullptr);
    const float* pr = C.ee_ref + 3 * k;
    const float d0 = p[0] - pr[0], d1 = p[1] - pr[1], d2 = p[2] - pr[2];
    J += 0.5f * s * wee * (d0 * d0 + d1 * d1 + d2 * d2);
#pragma unroll
    for (int i = 0; i < QM; ++i) J += 0.5f * s * wqd * x[QM + i] * x[QM + i];
  }
  if (u) {
#pragma unroll
    for (int i = 0; i < QM; ++i) J += 0.5f * wr * u[i] * u[i];
  }
  return J;
}

// Merit (Eq. 3) of Z + alpha_i dZ for alpha_i = beta^-i (Eq. 7), i < n_alpha:
// one thread per (alpha, knot), contributions reduced per alpha in a fixed order.
template <int NT>
__device__ void st_line_search(const Ctx& C, float mu, float beta, int n_alpha) {
  const int N = C.N, K = N + 1;
  float* contrib = C.yv;  // [n_alpha][K] (free during the line search)
  for (int it = threadIdx.x; it < n_alpha * K; it += NT) {
    const int a = it / K, k = it - a * K;
    float alpha = 1.f;
    for (int i = 0; i < a; ++i) alpha /= beta;
    float x[XM], u[QM];
#pragma unroll
    for (int i = 0; i < XM; ++i) x[i] = C.X[k * VS + i] + alpha * C.dX[k * VS + i];
    float v;
    if (k < N) {
#pragma unroll
      for (int i = 0; i < QM; ++i) u[i] = C.U[k * US + i] + alpha * C.dU[k * US + i];
      float qdd[QM];
      forward_dynamics(*C.M, x, x + QM, u, qdd);
      float c1 = 0.f;
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        const float qdn = x[QM + i] + C.h * qdd[i];
        const float qn = x[i] + C.h * qdn;
        c1 += fabsf(qn - (C.X[(k + 1) * VS + i] + alpha * C.dX[(k + 1) * VS + i]));
        c1 += fabsf(qdn - (C.X[(k + 1) * VS + QM + i] + alpha * C.dX[(k + 1) * VS + QM + i]));
      }
      v = trial_cost(C, k, x, u) + mu * c1;
    } else {
      float c0 = 0.f;
#pragma unroll
      for (int i = 0; i < XM; ++i) {
        const float x0 = C.X[i] + alpha * C.dX[i];
        c0 += fabsf(C.xs[i] - x0);
      }
      v = trial_cost(C, k, x, nullptr) + mu * c0;
    }
    contrib[a * K + k] = v;
  }
  __syncthreads();
  // warp a sums the contributions of alpha_a in knot order (lane-strided, then a fixed tree)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  for (int a = warp; a < n_alpha; a += NW) {
    DF s = df_zero();
    for (int k = lane; k < K; k += 32) s = df_add(s, contrib[a * K + k]);
    s = warp_df_sum(s);
    if (lane == 0) {
      const float m = df_val(s);
      C.scal[S_MERITS + a] = isfinite(m) ? m : INFINITY;
    }
  }
  __syncthreads();
}

// Argmin with ties to the smallest index; accept only a strict decrease (c7).
template <int NT>
__device__ int st_accept(const Ctx& C, float beta, int n_alpha) {
  const int N = C.N;
  int best = 0;
  for (int a = 1; a < n_alpha; ++a)
    if (C.scal[S_MERITS + a] < C.scal[S_MERITS + best]) best = a;
  const float m0 = C.scal[S_MERIT0];
  const int choice = (C.scal[S_MERITS + best] < m0) ? best : -1;
  if (choice >= 0) {
    float alpha = 1.f;
    for (int i = 0; i < choice; ++i) alpha /= beta;
    for (int i = threadIdx.x; i < (N + 1) * VS; i += NT) C.X[i] += alpha * C.dX[i];
    for (int i = threadIdx.x; i < N * US; i += NT) C.U[i] += alpha * C.dU[i];
  }
  __syncthreads();
  return choice;
}

}  // namespace gato
