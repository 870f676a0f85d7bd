// The stages of one SQP iteration (GATO, arXiv 2510.07625, Alg. 1) as
// device functions run by a thread-block cluster that owns one solve.
//
// Partition: the cluster's C CTAs split the block rows (knots) 0..N of the
// solve into contiguous ranges [k0, k1) of at most KPC_MAX knots; a CTA does
// every per-knot computation of its own range.  Inside a CTA each warp covers
// 4 knots with 7 lanes per knot (lanes 28..31 idle); lane j owns rows j (q_j)
// and j+7 (qd_j) of every block row of its knot, so dependencies inside a knot
// need only __syncwarp.  Dependencies between knots and the reductions use
// cluster barriers (block barriers when C = 1).
//
// PCG working set: each thread keeps its two rows of D_k, L_k, L_{k+1}^T and
// D_k^-1 (112 floats) in registers for the whole solve; vectors live in a
// per-CTA window of knots [k0-1, k1] whose halo knots are written by the
// neighbour CTAs through distributed shared memory (the plain form keeps every
// vector in global memory and skips the pushes).
//
// Reductions are compensated (double-float) and deterministic: each warp's
// partial goes to a slot of every CTA of the cluster, and every warp then
// reduces all slots with the same fixed tree.
#pragma once

#include <cooperative_groups.h>

#include "gato_device.cuh"

namespace gato {

namespace cg = cooperative_groups;

constexpr int NWARP = 9;             // warps per CTA
constexpr int NTHR = 32 * NWARP;     // threads per CTA
constexpr int KPC_MAX = 4 * (NWARP - 1) + 1;  // knots per CTA: 33 (the PCG runs them on 8 warps)
constexpr int NVEC = 9;              // vector slots
constexpr int RED_SLOTS = 8 * NWARP; // per-warp partial slots (up to 8 CTAs)
constexpr int RED_W = 8;             // floats per slot

enum : int { V_RR = 0, V_P0, V_P1, V_Q, V_Y, V_W, V_Z, V_RHS, V_DNU };
// Knot stride of the vector windows: 18 floats, so that the four knots a warp
// reads with one instruction fall in four different shared-memory banks
// (with 16 the first and third knot collide).
constexpr int VW = 18;
static_assert(VW % 2 == 0, "window rows must stay 8-byte aligned for pair loads");

struct Ctx {
  int N, dof, cost_kind;
  float h;
  float w[6];
  const float* x_ref;   // user layout, (N+1) x 2*dof
  const float* ee_ref;  // (N+1) x 3
  const DevModel* M;
  // cluster partition
  int rank, csize, k0, k1;
  // global workspace
  float *X, *U, *dX, *dU, *Fq, *Fv, *Mi, *qdd, *dT, *Qi, *Ri, *qg, *rg, *cv, *Jk;
  float *Dx, *Du;       // dual residual d = g + C^T nu at the current linearisation
  float* nu;            // multiplier (global, all knots)
  // low parts of the iterate (X + Xlo, U + Ulo as double-float pairs); zero
  // until the solve escalates to the high-precision mode
  float *Xlo, *Ulo;
  // 1 once the solve has escalated: double-float mass matrix and bias,
  // refined dynamics solves, double-float iterate and trial merits
  int hp = 0;
  LinkRec* LV;
  float* xs;            // padded x_s [VS]
  // Schur / preconditioner blocks: knot k at index k - bk0
  float *Dm, *Lm, *Pm;
  int bk0;
  const float* Lz;  // a 14x14 block of zeros (stands for L_{N+1})
  // vectors: slot s of knot k at vb + s * vstride + (k - vk0) * VW
  float* vb;
  int vstride, vk0;
  float* vbl;  // left neighbour's window (distributed shared memory) or null
  int vk0l;
  float* vbr;  // right neighbour's window or null
  int vk0r;
  // PCG halo knots recomputed locally (fused latency form, clusters): the
  // window then spans [k0-2, k1+1] and only w rows cross CTAs
  bool hrep = false;
  // reductions: red[2][RED_SLOTS][RED_W] in this CTA's shared memory
  float* red;
  float* scal;
  // optional per-stage cycle counters (rank 0, thread 0), see TimingSlot
  long long* tm;
};

// Slots of the per-stage cycle counters.
enum TimingSlot : int {
  T_LOAD = 0, T_MASS, T_FD, T_VALUE, T_TANGENT, T_JAC, T_KKT, T_SCHUR, T_BINV, T_PCG_INIT, T_PCG_S,
  T_PCG_Y, T_PCG_WZ, T_RECOVER, T_LS, T_ACCEPT, T_COUNT
};

// Adds the cycles since *last to counter `slot` (rank 0, thread 0 only).
__device__ __forceinline__ void tstamp(const Ctx& C, int slot, long long& last) {
  if (C.tm && C.rank == 0 && threadIdx.x == 0) {
    const long long t = clock64();
    C.tm[slot] += t - last;
    last = t;
  }
}

// scal[] slots (SCAL_FLOATS floats); from S_MDF on the merits as normalised
// (hi, lo) pairs: the base merit, then trial i at S_MDF + 2 + 2i
constexpr int SCAL_FLOATS = 128;  // S_MDF + 2 + 2 * MAX_ALPHA = 98 used
constexpr int S_MDF = 64;
static_assert(S_MDF + 2 + 2 * MAX_ALPHA <= SCAL_FLOATS, "merit pairs fit the scalar block");
enum : int {
  S_KKT = 0, S_MERIT0, S_CMAX, S_GMAX, S_DMAX, S_ALPHA, S_FLAGS, S_PCG, S_ITERS, S_MERITF,
  S_CHOICE, S_REDBUF, S_DONE, S_NSQP, S_NPCG, S_RFLAGS, S_MERITS = 16,  // S_MERITS..+15
  S_RHO = 32,  // the adapted rho between the plain form's launches
  S_FEXT = 33, // S_FEXT..+2: the solve's end-effector force (base frame)
  S_HP = 36,   // plain form: 1 once the solve is in the high-precision mode
  S_REDO = 37  // plain form: 1 while an iteration is to be repeated in that mode
};

// The solve's constant end-effector force (Sec. IV-D's disturbance hypotheses).
__device__ __forceinline__ V3 ee_force(const Ctx& C) {
  return v3(C.scal[S_FEXT], C.scal[S_FEXT + 1], C.scal[S_FEXT + 2]);
}

// rho after an SQP iteration (Sec. IV-C adjusts it from the line search's
// outcome): / 3 after an accepted step, * 2 after a rejected one, within
// [1e-8, 1e1].
__device__ __forceinline__ float rho_next(float rho, int choice) {
  return choice >= 0 ? fmaxf(rho / 3.f, 1e-8f) : fminf(rho * 2.f, 1e1f);
}

// One record of the per-iteration log (int32 each): the line search's choice
// (alpha index, -1 rejected; -2 for an iteration not reached), the PCG
// iterations of the iteration, the KKT residual at its linearisation (float
// bits), 1 if it ran in the high-precision mode, then the merit of the
// iterate and the merit of the full step's trial point as (hi, lo) float bits.
constexpr int ITLOG_W = 8;

// Per-knot strides of the global workspace arrays.
constexpr int FQS = 49, QIS = 56, DTS = 14 * 8, LIS = 196;

struct WsLayout {
  size_t X, U, dX, dU, Fq, Fv, Mi, qdd, dT, Qi, Ri, qg, rg, cv, Jk, Li, LV, Dm, Lm, Pm, vec, Dx, Du,
      nu, Xlo, Ulo, hand, total;
};

__host__ __device__ inline size_t align32(size_t n) { return (n + 31) & ~size_t(31); }

// Offsets (floats) of one solve's workspace for horizon up to Nmax.  Blocks and
// vectors are included only for the plain form (everything global).
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
  L.Li = o;  // (no longer used: the block inverse keeps its rows in registers)
  L.LV = o; o += align32(Nmax * QM * LVS);
  L.Dx = o; o += align32(K * VS);
  L.Du = o; o += align32(Nmax * US);
  L.nu = o; o += align32(K * VS);
  L.Xlo = o; o += align32(K * VS);
  L.Ulo = o; o += align32(Nmax * US);
  L.hand = o; o += 32;  // hand-over record of an escalating solve (ints)
  if (global_blocks) {
    L.Dm = o; o += align32(K * BS);
    L.Lm = o; o += align32(K * BS);
    L.Pm = o; o += align32(K * BS);
  } else {
    L.Dm = L.Lm = L.Pm = 0;
  }
  if (global_vecs) {
    L.vec = o; o += align32(NVEC * (K + 2) * VW + SCAL_FLOATS + 16);
  } else {
    L.vec = 0;
  }
  L.total = align32(o);
  return L;
}

// Shared-memory floats of one fused CTA owning at most `kpc` knots.
__host__ __device__ inline size_t smem_floats(int kpc) {
  size_t f = 96 /*model*/ + SCAL_FLOATS + 2 * RED_SLOTS * RED_W + 16 /*xs*/;
  f += NVEC * (size_t)(kpc + 4) * VW;  // windows over knots k0-2 .. k1+1
  f += (size_t)(3 * kpc + 1) * BS + 196;  // blocks + a zero block
  return align32(f);
}

// Cluster size for horizon N: the fewest CTAs with at most KPC_MAX knots each.
__host__ __device__ inline int cluster_for(int N) { return (N + 1 + KPC_MAX - 1) / KPC_MAX; }
__host__ __device__ inline int kpc_for(int N, int C) { return (N + 1 + C - 1) / C; }

// ------------------------------------------------------------ small helpers

__device__ __forceinline__ int pad_state(int ui, int dof) { return ui < dof ? ui : QM + (ui - dof); }

__device__ __forceinline__ float& blk(float* base, int k, int r, int c) { return base[k * BS + c * XM + r]; }
__device__ __forceinline__ float& bD(const Ctx& C, int k, int r, int c) { return blk(C.Dm, k - C.bk0, r, c); }
__device__ __forceinline__ float& bL(const Ctx& C, int k, int r, int c) { return blk(C.Lm, k - C.bk0, r, c); }
__device__ __forceinline__ float& bP(const Ctx& C, int k, int r, int c) { return blk(C.Pm, k - C.bk0, r, c); }

// Entries 2m, 2m+1 of a window row (8-byte aligned: the window base, its
// slot stride and VW are even).
__device__ __forceinline__ float2 ld2(const float* v, int m) { return reinterpret_cast<const float2*>(v)[m]; }

__device__ __forceinline__ float* vec(const Ctx& C, int s, int k) {
  return C.vb + s * C.vstride + (k - C.vk0) * VW;
}

__device__ __forceinline__ void csync(const Ctx& C) {
  if (C.csize > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
}

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

__device__ __forceinline__ void flag_nonfinite(const Ctx& C) {
  atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
}

// ------------------------------------------------------------- reductions

// Each warp contributes `nv` floats; lane 0 writes them into slot
// [buf][rank * NWARP + warp] of every CTA in the cluster.
__device__ __forceinline__ void red_publish(const Ctx& C, int buf, const float* v, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    const int slot = (buf * RED_SLOTS + C.rank * NWARP + warp) * RED_W;
    if (C.csize > 1) {
      cg::cluster_group cl = cg::this_cluster();
      for (int r = 0; r < C.csize; ++r) {
        float* dst = cl.map_shared_rank(C.red, r);
        for (int i = 0; i < nv; ++i) dst[slot + i] = v[i];
      }
    } else {
      for (int i = 0; i < nv; ++i) C.red[slot + i] = v[i];
    }
  }
}

// Cluster-wide compensated sum; every thread returns the same value.
__device__ __forceinline__ DF cluster_df_sum(const Ctx& C, DF v, int& buf) {
  const int lane = threadIdx.x & 31;
  v = warp_df_sum(v);
  const float pv[2] = {v.hi, v.lo};
  red_publish(C, buf, pv, 2);
  csync(C);
  const int ns = C.csize * NWARP;
  DF s = df_zero();
  for (int i = lane; i < ns; i += 32) {
    const float* p = C.red + (buf * RED_SLOTS + i) * RED_W;
    s = df_addd(s, DF{p[0], p[1]});
  }
  buf ^= 1;
  return warp_df_sum(s);
}

// Cluster-wide maxima of 4 values and compensated sums of 2 values.
__device__ __forceinline__ void cluster_max4_sum2(const Ctx& C, float* mx, DF* sm, int& buf) {
  const int lane = threadIdx.x & 31;
  float v[RED_W];
  for (int i = 0; i < 4; ++i) v[i] = warp_max(mx[i]);
  for (int i = 0; i < 2; ++i) {
    const DF t = warp_df_sum(sm[i]);
    v[4 + 2 * i] = t.hi;
    v[5 + 2 * i] = t.lo;
  }
  red_publish(C, buf, v, RED_W);
  csync(C);
  const int ns = C.csize * NWARP;
  float m[4] = {0.f, 0.f, 0.f, 0.f};
  DF s[2] = {df_zero(), df_zero()};
  for (int i = lane; i < ns; i += 32) {
    const float* p = C.red + (buf * RED_SLOTS + i) * RED_W;
    for (int q = 0; q < 4; ++q) m[q] = fmaxf(m[q], p[q]);
    for (int q = 0; q < 2; ++q) s[q] = df_addd(s[q], DF{p[4 + 2 * q], p[5 + 2 * q]});
  }
  for (int q = 0; q < 4; ++q) mx[q] = warp_max(m[q]);
  for (int q = 0; q < 2; ++q) sm[q] = warp_df_sum(s[q]);
  buf ^= 1;
}

// Cluster-wide OR of the non-finite flag (every CTA takes the same branch).
__device__ __forceinline__ bool cluster_flag(const Ctx& C, int& buf) {
  float mx[4] = {0.f, 0.f, 0.f, 0.f};
  DF sm[2] = {df_zero(), df_zero()};
  if (*reinterpret_cast<volatile int*>(C.scal + S_FLAGS)) mx[0] = 1.f;
  cluster_max4_sum2(C, mx, sm, buf);
  return mx[0] > 0.f;
}

// The knot a thread owns in knot-row work: k = k0 + 4 warp + lane / 7.
#define OWN_KNOT(Cx)                                                           \
  const int lane_ = threadIdx.x & 31, warp_ = threadIdx.x >> 5;                \
  const int j = lane_ - 7 * (lane_ / 7);                                       \
  const int k = (Cx).k0 + 4 * warp_ + lane_ / 7;                               \
  const bool act = (lane_ < 28) && (k < (Cx).k1)

// ------------------------------------------------------------------ loading

// Copies the CTA's knots of the iterate from user layout into the padded
// workspace and the multiplier into the global nu.
__device__ inline void load_iterate(const Ctx& C, const ProbDesc& P) {
  const int N = C.N, dof = C.dof, nx = 2 * dof;
  const int ke = C.k1 < N ? C.k1 : N;  // dynamics knots [k0, ke)
  for (int i = threadIdx.x; i < (C.k1 - C.k0) * VS; i += NTHR) {
    C.X[C.k0 * VS + i] = 0.f;
    C.Xlo[C.k0 * VS + i] = 0.f;
    C.nu[C.k0 * VS + i] = 0.f;
  }
  for (int i = threadIdx.x; i < (ke - C.k0) * US; i += NTHR) {
    C.U[C.k0 * US + i] = 0.f;
    C.Ulo[C.k0 * US + i] = 0.f;
  }
  if (threadIdx.x < VS) C.xs[threadIdx.x] = 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < (C.k1 - C.k0) * nx; i += NTHR) {
    const int k = C.k0 + i / nx, ui = i % nx;
    C.X[k * VS + pad_state(ui, dof)] = P.X[k * nx + ui];
    if (P.lam) C.nu[k * VS + pad_state(ui, dof)] = P.lam[k * nx + ui];
  }
  for (int i = threadIdx.x; i < (ke - C.k0) * dof; i += NTHR) {
    const int k = C.k0 + i / dof, ui = i % dof;
    C.U[k * US + ui] = P.U[k * dof + ui];
  }
  if (threadIdx.x < nx) C.xs[pad_state(threadIdx.x, dof)] = P.x_s[threadIdx.x];
}

__device__ inline void store_iterate(const Ctx& C, const ProbDesc& P) {
  const int N = C.N, dof = C.dof, nx = 2 * dof;
  const int ke = C.k1 < N ? C.k1 : N;
  for (int i = threadIdx.x; i < (C.k1 - C.k0) * nx; i += NTHR) {
    const int k = C.k0 + i / nx, ui = i % nx;
    P.X[k * nx + ui] = C.X[k * VS + pad_state(ui, dof)] + C.Xlo[k * VS + pad_state(ui, dof)];
    if (P.lam) P.lam[k * nx + ui] = C.nu[k * VS + pad_state(ui, dof)];
  }
  for (int i = threadIdx.x; i < (ke - C.k0) * dof; i += NTHR) {
    const int k = C.k0 + i / dof, ui = i % dof;
    P.U[k * dof + ui] = C.U[k * US + ui] + C.Ulo[k * US + ui];
  }
}

// --------------------------------------------------- stage 1: linearisation

// ---- high-precision mode (a solve escalates to it when its FP32 line search
// finds no decrease; see sqp_solve)
//
// For the rod arms M's smallest eigenvalue (a thin link turning about its own
// axis, m r^2 / 2) is about 1/3000 of its largest, while the RNEA rounds every
// entry of M and of the bias at the scale of the largest forces in the chain;
// solving M qdd = tau - b amplifies that rounding by kappa(M) (in FP32: ~1e-5
// relative in A_k and in qdd, measured against the FP64 oracle).  Near a
// solution that noise, and the FP32 rounding of the iterate itself, are larger
// than the merit decrease of a step, so the FP32 line search stalls with a
// KKT residual of 1e-6..1e-4.  The high-precision mode removes both: M and the
// bias in double-float (dfl), each dynamics solve refined once against them,
// the iterate as double-float (hi, lo) pairs, the trial merits in double-float.
// Double-float runs on the FP32 pipe; only sin and cos of q use FP64.
//
// The stages below run as out-of-line calls with their fields passed by
// value, so that their registers do not enter the allocation of the kernel
// that calls them.

// Mass-matrix columns and bias in double-float (dfl; sin and cos of q by
// FP64) at q = X + Xlo, one (knot, column) per thread.  Each value is stored as an (hi, lo) float pair: hi in Mi (the bias
// in qdd), lo in the tangent array dT (column c at dT + c * 8, the bias at
// dT + 56), which is free until the tangent stage.
struct MassView {
  const DevModel* M;
  const float *X, *Xlo;
  float *Mi, *qdd, *dT;
  float fx, fy, fz;
  int k0, ke;
};

static __device__ __noinline__ void st_mass_bias_hp(MassView v) {
  const DevModel& M = *v.M;
  // one (knot, column) per thread, one round (8 KPC_MAX <= NTHR); the knot's
  // eight threads share a warp, each forms sin and cos of one joint and the
  // others take them by shuffles (idle threads join the shuffles)
  const int it = threadIdx.x;
  const bool act = it < (v.ke - v.k0) * 8;
  const int k = v.k0 + (act ? it >> 3 : 0), col = it & 7;
  const int base = (it & 31) & ~7;
  const float* x = v.X + k * VS;
  const float* xl = v.Xlo + k * VS;
  dfl sj(0), cj(1);
  if (act && col < QM) sincos(dfl(x[col], xl[col]), &sj, &cj);
  dfl sq[QM], cq[QM], qd[QM], acc[QM], tau[QM];
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    sq[i] = dfl(__shfl_sync(0xffffffffu, sj.hi, base + i), __shfl_sync(0xffffffffu, sj.lo, base + i));
    cq[i] = dfl(__shfl_sync(0xffffffffu, cj.hi, base + i), __shfl_sync(0xffffffffu, cj.lo, base + i));
    qd[i] = (col == 7) ? dfl(x[QM + i], xl[QM + i]) : dfl(0);
    acc[i] = (i == col) ? dfl(1) : dfl(0);
  }
  if (!act) return;
  const Vec3<dfl> fw = col == 7 ? v3t<dfl>(dfl(v.fx), dfl(v.fy), dfl(v.fz)) : vzero<dfl>();
  rnea_value<dfl>(M, sq, cq, qd, acc, col == 7 ? dfl(M.g) : dfl(0), fw, tau, nullptr);
  float* lo = v.dT + k * DTS + col * 8;
#pragma unroll
  for (int r = 0; r < QM; ++r) {
    lo[r] = tau[r].lo;
    if (col < 7) v.Mi[k * FQS + r * QM + col] = tau[r].hi;
    else v.qdd[k * US + r] = tau[r].hi;
  }
}

// Mass-matrix columns (unit-acceleration RNEA) and bias forces per knot.
__device__ inline void st_mass_bias(const Ctx& C) {
  const int ke = C.k1 < C.N ? C.k1 : C.N;
  if (C.hp) {
    MassView v;
    v.M = C.M;
    v.X = C.X;
    v.Xlo = C.Xlo;
    v.Mi = C.Mi;
    v.qdd = C.qdd;
    v.dT = C.dT;
    const V3 fw = ee_force(C);
    v.fx = fw.x;
    v.fy = fw.y;
    v.fz = fw.z;
    v.k0 = C.k0;
    v.ke = ke;
    st_mass_bias_hp(v);
    return;
  }
  const DevModel& M = *C.M;
  for (int it = threadIdx.x; it < (ke - C.k0) * 8; it += NTHR) {
    const int k = C.k0 + (it >> 3), col = it & 7;
    float sq[QM], cq[QM], qd[QM], acc[QM], tau[QM];
    const float* x = C.X + k * VS;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      sincosf(x[i], &sq[i], &cq[i]);
      qd[i] = (col == 7) ? x[QM + i] : 0.f;
      acc[i] = (i == col) ? 1.f : 0.f;
    }
    rnea_value(M, sq, cq, qd, acc, col == 7 ? M.g : 0.f, col == 7 ? ee_force(C) : vzero(), tau, nullptr);
    if (col < 7) {
#pragma unroll
      for (int r = 0; r < QM; ++r) C.Mi[k * FQS + r * QM + col] = tau[r];
    } else {
#pragma unroll
      for (int r = 0; r < QM; ++r) C.qdd[k * US + r] = tau[r];
    }
  }
}

// High-precision forward dynamics: M^-1 and qdd = M^-1 (u - bias) with one
// step of iterative refinement each (the residual of the FP32 solution against
// the (hi, lo) matrix, formed in double-float and solved with the same FP32
// factor: the refined error is ~kappa(M) eps_32 times the first one), and the
// defects of the double-float iterate formed in double-float from differences
// of the iterates, e = (qd_k - qd_{k+1}) + h qdd, so that their rounding
// scales with e itself rather than with the state.
struct FdView {
  const float *X, *Xlo, *U, *Ulo, *xs;
  float *Mi, *qdd, *dT, *cv, *scal;
  float h;
  int N, dof, k0, k1;
};

static __device__ __noinline__ void st_forward_dynamics_hp(FdView v) {
  const int N = v.N;
  const int ke = v.k1 < N ? v.k1 : N;
  const int nk = ke - v.k0;
  const int it = threadIdx.x;
  const int k = v.k0 + (it >> 3), col = it & 7;
  const bool act = it < 8 * nk;
  float Ml[28];
  if (act) {
#pragma unroll
    for (int i = 0; i < QM; ++i)
#pragma unroll
      for (int j2 = 0; j2 <= i; ++j2)
        Ml[i * (i + 1) / 2 + j2] = 0.5f * (v.Mi[k * FQS + i * QM + j2] + v.Mi[k * FQS + j2 * QM + i]);
#pragma unroll
    for (int i = 0; i < QM; ++i)
      if (i >= v.dof) Ml[i * (i + 1) / 2 + i] = 1.f;
  }
  // the double-float right-hand side and the residual of the first solve
  // against the (hi, lo) matrix, both read before any column of M^-1
  // overwrites M
  dfl res[QM];
  float x[QM];
  bool ok = true;
  if (act) {
    const float* lo = v.dT + k * DTS;
    dfl rhs[QM];
#pragma unroll
    for (int i = 0; i < QM; ++i)
      rhs[i] = col == 7 ? dfl(v.U[k * US + i], v.Ulo[k * US + i]) - dfl(v.qdd[k * US + i], lo[56 + i])
                        : dfl(i == col ? 1 : 0);
    ok = chol7(Ml);
#pragma unroll
    for (int i = 0; i < QM; ++i) x[i] = rhs[i].hi;
    chol7_solve(Ml, x);
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      dfl r = rhs[i];
#pragma unroll
      for (int j2 = 0; j2 < QM; ++j2) {
        dfl m;
        if (i >= v.dof || j2 >= v.dof) {
          m = dfl(i == j2 ? 1 : 0);
        } else {
          m = dfl(0.5f) * (dfl(v.Mi[k * FQS + i * QM + j2], lo[j2 * 8 + i]) +
                           dfl(v.Mi[k * FQS + j2 * QM + i], lo[i * 8 + j2]));
        }
        r -= m * dfl(x[j2]);
      }
      res[i] = r;
    }
  }
  __syncthreads();  // every M_k is read before a column of M_k^-1 overwrites it
  if (act) {
    float d[QM];
#pragma unroll
    for (int i = 0; i < QM; ++i) d[i] = res[i].hi;
    chol7_solve(Ml, d);
    if (col == 7) {
      if (!ok) atomicOr(reinterpret_cast<int*>(v.scal + S_FLAGS), F_NONFINITE);
      const float* xk = v.X + k * VS;
      const float* xkl = v.Xlo + k * VS;
      const float* xn = v.X + (k + 1) * VS;
      const float* xnl = v.Xlo + (k + 1) * VS;
      const dfl h(v.h), h2 = h * h;
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        const dfl a = dfl_sum(x[i], d[i]);
        v.qdd[k * US + i] = a.hi;
        // qd+ = qd + h qdd, q+ = q + h qd+ = q + h qd + h^2 qdd
        const dfl dqd = (dfl(xk[QM + i]) - dfl(xn[QM + i])) + (dfl(xkl[QM + i]) - dfl(xnl[QM + i]));
        const dfl dq = (dfl(xk[i]) - dfl(xn[i])) + (dfl(xkl[i]) - dfl(xnl[i]));
        const dfl qdk(xk[QM + i], xkl[QM + i]);
        v.cv[(k + 1) * VS + QM + i] = (dqd + h * a).hi;
        v.cv[(k + 1) * VS + i] = (dq + h * qdk + h2 * a).hi;
      }
    } else {
#pragma unroll
      for (int i = 0; i < QM; ++i) v.Mi[k * FQS + i * QM + col] = dfl_sum(x[i], d[i]).hi;
    }
  }
  if (it == 8 * nk && v.k0 == 0) {  // c_0 = x_s - x_0, by the CTA owning knot 0
#pragma unroll
    for (int i = 0; i < XM; ++i) v.cv[i] = ((dfl(v.xs[i]) - dfl(v.X[i])) - dfl(v.Xlo[i])).hi;
  }
}

// Cholesky of M, explicit M^-1, qdd = M^-1 (u - bias), dynamics defects.
// One (knot, right-hand side) per thread: column c < 7 of M^-1 or, for c = 7,
// qdd and the defects; every thread of a knot factors M_k itself (the same
// bits), so the eight triangular solves run side by side.
__device__ inline void st_forward_dynamics(const Ctx& C) {
  const int N = C.N;
  if (C.hp) {
    FdView v;
    v.X = C.X;
    v.Xlo = C.Xlo;
    v.U = C.U;
    v.Ulo = C.Ulo;
    v.xs = C.xs;
    v.Mi = C.Mi;
    v.qdd = C.qdd;
    v.dT = C.dT;
    v.cv = C.cv;
    v.scal = C.scal;
    v.h = C.h;
    v.N = N;
    v.dof = C.dof;
    v.k0 = C.k0;
    v.k1 = C.k1;
    st_forward_dynamics_hp(v);
    return;
  }
  const int ke = C.k1 < N ? C.k1 : N;
  const float h = C.h;
  const int nk = ke - C.k0;  // 8 * nk + 1 <= 8 * KPC_MAX + 1 < NTHR: one round
  static_assert(8 * KPC_MAX + 1 <= NTHR, "one (knot, column) per thread");
  const int it = threadIdx.x;
  const int k = C.k0 + (it >> 3), col = it & 7;
  const bool act = it < 8 * nk;
  float Ml[28];
  if (act) {
#pragma unroll
    for (int i = 0; i < QM; ++i)
#pragma unroll
      for (int j2 = 0; j2 <= i; ++j2)
        Ml[i * (i + 1) / 2 + j2] = 0.5f * (C.Mi[k * FQS + i * QM + j2] + C.Mi[k * FQS + j2 * QM + i]);
#pragma unroll
    for (int i = 0; i < QM; ++i)
      if (i >= C.dof) Ml[i * (i + 1) / 2 + i] = 1.f;
  }
  __syncthreads();  // every M_k is read before a column of M_k^-1 overwrites it
  if (act) {
    const bool ok = chol7(Ml);
    if (col == 7) {
      if (!ok) flag_nonfinite(C);
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
    } else {
      float e[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) e[i] = (i == col) ? 1.f : 0.f;
      chol7_solve(Ml, e);
#pragma unroll
      for (int i = 0; i < QM; ++i) C.Mi[k * FQS + i * QM + col] = e[i];
    }
  }
  if (it == 8 * nk && C.k0 == 0) {  // c_0 = x_s - x_0, by the CTA owning knot 0
#pragma unroll
    for (int i = 0; i < XM; ++i) C.cv[i] = C.xs[i] - C.X[i];
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
      const float d = C.hp ? (x[i] - xref_at(C, k, i)) + C.Xlo[k * VS + i] : x[i] - xref_at(C, k, i);
      J += 0.5f * s * wi * d * d;
      qg[i] = s * wi * d;
    }
#pragma unroll
    for (int i = 0; i < 49; ++i) Qi[i] = 0.f;
    // products and sums rounded explicitly: a multiply-add contracted in one
    // kernel and not in another would round these differently at small rho
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      Qi[i * QM + i] = 1.f / __fadd_rn(__fmul_rn(s, wq), rho);
      Qi[49 + i] = 1.f / __fadd_rn(__fmul_rn(s, wqd), rho);
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
        Hl[i * (i + 1) / 2 + j2] = __fadd_rn(__fmul_rn(s * wee, Jp[i] * Jp[j2] + Jp[QM + i] * Jp[QM + j2] +
                                                                  Jp[2 * QM + i] * Jp[2 * QM + j2]),
                                             i == j2 ? rho : 0.f);
    }
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      const float v = x[QM + i];
      J += 0.5f * s * wqd * v * v;
      qg[QM + i] = s * wqd * (C.hp ? v + C.Xlo[k * VS + QM + i] : v);
      Qi[49 + i] = 1.f / __fadd_rn(__fmul_rn(s, wqd), rho);
    }
    if (C.hp) {  // p(q + q_lo) = p(q) + J_p q_lo to first order: the gradient gains J_p^T J_p q_lo
      const float* xl = C.Xlo + k * VS;
      float dp[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int i = 0; i < QM; ++i) dp[r] += Jp[r * QM + i] * xl[i];
#pragma unroll
      for (int i = 0; i < QM; ++i)
        qg[i] += s * wee * (Jp[i] * dp[0] + Jp[QM + i] * dp[1] + Jp[2 * QM + i] * dp[2]);
    }
    // the packed Q_qq, inverted column by column in the next phase
#pragma unroll
    for (int i = 0; i < 28; ++i) Qi[i] = Hl[i];
  }
  if (k < N) {
    const float* u = C.U + k * US;
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      J += 0.5f * wr * u[i] * u[i];
      C.rg[k * US + i] = wr * (C.hp ? u[i] + C.Ulo[k * US + i] : u[i]);
      C.Ri[k * US + i] = 1.f / wr;
    }
  }
  C.Jk[k] = J;
}


// Value RNEA at the dynamics solution (stored for the tangent pass) + costs.
// End-effector cost: Q_qq^-1 by one (knot, column) per thread, each thread
// factoring its knot's packed Q_qq (the same bits), seven solves side by side.
__device__ inline void st_value_and_cost(const Ctx& C) {
  const int ke = C.k1 < C.N ? C.k1 : C.N;
  const int nd = ke - C.k0, nc = C.k1 - C.k0;
  for (int it = threadIdx.x; it < nd + nc; it += NTHR) {
    if (it < nd) {
      const int k = C.k0 + it;
      float sq[QM], cq[QM], tau[QM];
      const float* x = C.X + k * VS;
#pragma unroll
      for (int i = 0; i < QM; ++i) sincosf(x[i], &sq[i], &cq[i]);
      rnea_value(*C.M, sq, cq, x + QM, C.qdd + k * US, C.M->g, ee_force(C), tau, C.LV + k * QM);
    } else {
      knot_cost(C, C.k0 + it - nd);
    }
  }
  if (C.cost_kind != 0) {
    static_assert(QM * KPC_MAX <= NTHR, "one (knot, column) per thread");
    __syncthreads();  // every packed Q_qq is stored
    const int it = threadIdx.x;
    const int k = C.k0 + it / QM, col = it % QM;
    const bool act = it < QM * nc;
    float Hl[28];
    float* Qi = C.Qi + k * QIS;
    if (act) {
#pragma unroll
      for (int i = 0; i < 28; ++i) Hl[i] = Qi[i];
    }
    __syncthreads();  // every Q_qq is read before a column of its inverse overwrites it
    if (act) {
      const bool ok = chol7(Hl);
      if (!ok && col == 0) atomicOr(reinterpret_cast<int*>(C.scal + S_FLAGS), F_NONFINITE);
      float e[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) e[i] = (i == col) ? 1.f : 0.f;
      chol7_solve(Hl, e);
#pragma unroll
      for (int i = 0; i < QM; ++i) Qi[i * QM + col] = e[i];
    }
  }
}

// Directional derivatives of ID along every q_j and qd_j.
__device__ inline void st_tangents(const Ctx& C) {
  const int ke = C.k1 < C.N ? C.k1 : C.N;
  const V3 fw = ee_force(C);
  for (int it = threadIdx.x; it < (ke - C.k0) * 14; it += NTHR) {
    const int k = C.k0 + it / 14, d = it % 14;
    float dtau[QM];
    rnea_tangent(*C.M, C.LV + k * QM, C.X + k * VS + QM, d >= QM, d % QM, fw, dtau);
#pragma unroll
    for (int i = 0; i < QM; ++i) C.dT[k * DTS + d * 8 + i] = dtau[i];
  }
}

// dqdd/dq = -M^-1 dID/dq, dqdd/dqd = -M^-1 dID/dqd: one (knot, which, row r)
// per thread, the seven entries of row r from one read of M^-1's row.
__device__ inline void st_dyn_jacobians(const Ctx& C) {
  const int ke = C.k1 < C.N ? C.k1 : C.N;
  for (int it = threadIdx.x; it < (ke - C.k0) * 14; it += NTHR) {
    const int k = C.k0 + it / 14, e = it % 14;
    const int which = e / QM, r = e % QM;
    float mrow[QM];
#pragma unroll
    for (int l = 0; l < QM; ++l) mrow[l] = C.Mi[k * FQS + r * QM + l];
    float* out = (which ? C.Fv : C.Fq) + k * FQS + r * QM;
#pragma unroll
    for (int c = 0; c < QM; ++c) {
      const float* col = C.dT + k * DTS + (which * QM + c) * 8;
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < QM; ++l) a += mrow[l] * col[l];
      out[c] = -a;
    }
  }
}

// KKT residual max(||c||_inf, ||g + C^T nu||_inf / max(1, ||g||_inf)) at this
// linearisation with the last multiplier, and the merit of the current iterate (Eq. 3).
// Also stores the dual residual d = g + C^T nu, accumulated with compensated
// sums: near convergence d is a small difference of O(|nu|) terms, and the
// step is recovered from it through G^-1 (R^-1 = 1/w_u amplifies its error).
__device__ inline void st_kkt_merit(const Ctx& C, float mu, int& rbuf) {
  const int N = C.N;
  const float h = C.h, h2 = C.h * C.h;
  float mx[4] = {0.f, 0.f, 0.f, 0.f};  // |c|, |g|, |d|, non-finite
  DF sm[2] = {df_zero(), df_zero()};   // J, ||c||_1
  {
    OWN_KNOT(C);
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
      bool bad = false;
      for (int t = 0; t < 2; ++t) {
        const int i = j + QM * t;
        const float cvi = C.cv[k * VS + i];
        mx[0] = fmaxf(mx[0], fabsf(cvi));
        sm[1] = df_add(sm[1], fabsf(cvi));
        const float g = C.qg[k * VS + i];
        mx[1] = fmaxf(mx[1], fabsf(g));
        mx[2] = fmaxf(mx[2], fabsf(dv[t]));
        bad = bad || !isfinite(cvi) || !isfinite(dv[t]);
      }
      if (k < N) {
        const float g = C.rg[k * US + j];
        const float duv = df_val(du);
        C.Du[k * US + j] = duv;
        mx[1] = fmaxf(mx[1], fabsf(g));
        mx[2] = fmaxf(mx[2], fabsf(duv));
        bad = bad || !isfinite(duv);
      }
      if (j == 0) {
        sm[0] = df_add(sm[0], C.Jk[k]);
        bad = bad || !isfinite(C.Jk[k]);
      }
      if (bad) mx[3] = 1.f;
    }
  }
  if (*reinterpret_cast<volatile int*>(C.scal + S_FLAGS)) mx[3] = 1.f;
  cluster_max4_sum2(C, mx, sm, rbuf);
  const float J = df_val(sm[0]), c1 = df_val(sm[1]);
  if (threadIdx.x == 0) {
    C.scal[S_KKT] = fmaxf(mx[0], mx[2] / fmaxf(1.f, mx[1]));
    // (the merit itself comes from the line search's evaluation of the iterate)
    if (mx[3] > 0.f || !isfinite(J) || !isfinite(c1)) flag_nonfinite(C);
  }
  __syncthreads();
}

// ------------------------------------------------------ stage 2: Schur form

// Eq. 5-6 blocks (S = C G^-1 C^T, the SPD sign; the overall minus signs
// printed on S and Phi^-1 cancel):  L_k = phi_{k-1} = -A_{k-1} Q_{k-1}^-1,
// D_k = theta_{k-1} = A Q^-1 A^T + B R^-1 B^T + Q_k^-1 (D_0 = Q_0^-1).
// Right-hand side for the multiplier correction dnu = nu - nu_0: zeta_k and
// gamma of Eq. 5 with the gradient g replaced by the dual residual
// d = g + C^T nu_0, i.e. rhs = -c - C G^-1 d = gamma - S nu_0, the initial
// residual of the warm-started PCG, formed without cancellation.  A CTA also
// forms L_{k1} (the block its last row multiplies by L^T) from its own knot.
__device__ inline void st_schur(const Ctx& C) {
  const int N = C.N;
  const float h = C.h;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane - 7 * (lane / 7);
  const int k = C.k0 + 4 * warp + lane / 7;
  const bool act = (lane < 28) && (k < C.k1);
  const bool actL = (lane < 28) && (k <= C.k1) && (k <= N) && (k > 0);
  const int kk = k - 1;  // the dynamics knot feeding block row k
  // Every entry is accumulated in double-float and rounded once: B R^-1 B^T
  // reaches ~1e4 (R^-1 = 1e3, h |M^-1| ~ 4) while theta's entries along M's
  // well-conditioned directions are O(1), so FP32 partial sums would leave
  // ~eps_32 1e4 of cancellation error in them.
  if (act && k == 0) {
    const float* Qi = C.Qi;
    for (int t = 0; t < 2; ++t) {
      const int i = j + QM * t;
      DF acc = df_zero();
      for (int c = 0; c < XM; ++c) {
        const float qv = Qinv_elem(Qi, i, c);
        bD(C, 0, i, c) = qv;
        acc = df_fma(acc, qv, C.Dx[c]);
        bL(C, 0, i, c) = 0.f;
      }
      vec(C, V_RHS, 0)[i] = df_val(df_add(DF{-acc.hi, -acc.lo}, -C.cv[i]));
    }
  }
  if (actL) {
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
          DF s = df_zero();
#pragma unroll
          for (int l = 0; l < QM; ++l) s = df_fma(s, Arow[l], Qi[l * QM + c]);
          a = df_val(s);
        } else {
          a = Arow[c] * Qi[49 + c - QM];
        }
        bL(C, k, i, c) = -a;
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
    // B R^-1 B^T = si sc K with K = M^-1 R^-1 M^-1 and the row and column
    // factors si, sc (h^2 on q rows, h on qd rows): row j of K once, each
    // term (M^-1[j, m] R^-1[m]) M^-1[c, m] formed exactly as a (hi, lo) pair
    DF Kr[QM];
#pragma unroll
    for (int cm = 0; cm < QM; ++cm) {
      DF sk = df_zero();
#pragma unroll
      for (int m = 0; m < QM; ++m) {
        const float p = __fmul_rn(Mi[j * QM + m], Ri[m]);
        const float pe = __fmaf_rn(Mi[j * QM + m], Ri[m], -p);
        const float mi = Mi[cm * QM + m];
        const float q = __fmul_rn(p, mi);
        sk = df_addd(sk, DF{q, __fmaf_rn(p, mi, -q) + pe * mi});
      }
      Kr[cm] = sk;
    }
    for (int t = 0; t < 2; ++t) {
      const int i = j + QM * t;
      float Arow[XM];
#pragma unroll
      for (int l = 0; l < XM; ++l) Arow[l] = A_elem(Fq, Fv, h, i, l);
      const float si = t == 0 ? h * h : h;
      // row i of B R^-1 = si M^-1[j, :] R^-1 as exact (hi, lo) pairs
      float BRrow[QM], BRlo[QM];
#pragma unroll
      for (int m = 0; m < QM; ++m) {
        const float p1 = __fmul_rn(si, Mi[j * QM + m]);
        const float e1 = __fmaf_rn(si, Mi[j * QM + m], -p1);
        BRrow[m] = __fmul_rn(p1, Ri[m]);
        BRlo[m] = __fmaf_rn(p1, Ri[m], -BRrow[m]) + e1 * Ri[m];
      }
      for (int c = 0; c < XM; ++c) {
        // theta = -A L^T + B R^-1 B^T + Q_{k}^-1   (A Q^-1 A^T = -A L^T)
        DF a = df_zero();
#pragma unroll
        for (int l = 0; l < XM; ++l) a = df_fma(a, -Arow[l], bL(C, k, c, l));
        const int cm = c < QM ? c : c - QM;
        const float sc = c < QM ? h * h : h;
        DF kv = Kr[0];  // K[j][cm] (a select: cm is not a compile-time index)
#pragma unroll
        for (int m = 1; m < QM; ++m) kv = (cm == m) ? Kr[m] : kv;
        // (si sc) K[j][cm], both products exact to double-float accuracy
        const float f = __fmul_rn(si, sc);
        const float fe = __fmaf_rn(si, sc, -f);
        const float ph = __fmul_rn(f, kv.hi);
        const DF sbb = DF{ph, __fmaf_rn(f, kv.hi, -ph) + (f * kv.lo + fe * kv.hi)};
        bD(C, k, i, c) = df_val(df_add(df_addd(a, sbb), Qinv_elem(Qi1, i, c)));
      }
      // zeta with d: L_k d_{k-1} - B R^-1 d_u,{k-1} + Q_k^-1 d_k
      DF z = df_zero();
#pragma unroll
      for (int l = 0; l < XM; ++l) z = df_fma(z, bL(C, k, i, l), C.Dx[kk * VS + l]);
#pragma unroll
      for (int m = 0; m < QM; ++m) {
        z = df_fma(z, -BRrow[m], C.Du[kk * US + m]);
        z = df_add(z, -BRlo[m] * C.Du[kk * US + m]);
      }
#pragma unroll
      for (int l = 0; l < XM; ++l) z = df_fma(z, Qinv_elem(Qi1, i, l), C.Dx[k * VS + l]);
      vec(C, V_RHS, k)[i] = df_val(df_add(DF{-z.hi, -z.lo}, -C.cv[k * VS + i]));
    }
  }
}

// D_k^-1 by in-place Gauss-Jordan elimination without pivoting: D_k is
// symmetric positive definite, so every pivot is a positive diagonal of a
// Schur complement of D_k.  The 7 lanes of a knot hold rows j and j+7 in
// registers; at step c the owner of row c broadcasts it by shuffles, every
// lane eliminates column c from its rows and row c becomes the scaled pivot
// row, so after 14 steps the registers hold D_k^-1.  A non-positive or
// non-finite pivot flags the solve.
__device__ inline void st_block_inverse(const Ctx& C) {
  bool bad = false;
  OWN_KNOT(C);
  const int lane = threadIdx.x & 31;
  const int base = lane - j;  // first lane of this knot's group
  float a0[XM], a1[XM];       // rows j and j+7
#pragma unroll
  for (int c = 0; c < XM; ++c) {
    a0[c] = act ? bD(C, k, j, c) : (c == j ? 1.f : 0.f);
    a1[c] = act ? bD(C, k, j + QM, c) : (c == j + QM ? 1.f : 0.f);
  }
#pragma unroll
  for (int c = 0; c < XM; ++c) {
    const int owner = (base + (c % QM)) & 31;
    float pr[XM];
#pragma unroll
    for (int l = 0; l < XM; ++l) pr[l] = __shfl_sync(0xffffffffu, c < QM ? a0[l] : a1[l], owner);
    const float piv = pr[c];
    bad = bad || !(piv > 0.f) || !isfinite(piv);
    const float inv = 1.f / piv;
    const bool p0 = (j == c), p1 = (j + QM == c);  // this lane holds the pivot row
    const float f0 = a0[c], f1 = a1[c];
#pragma unroll
    for (int l = 0; l < XM; ++l) {
      if (l == c) continue;
      const float pl = pr[l] * inv;
      a0[l] = p0 ? pl : a0[l] - f0 * pl;
      a1[l] = p1 ? pl : a1[l] - f1 * pl;
    }
    a0[c] = p0 ? inv : -f0 * inv;
    a1[c] = p1 ? inv : -f1 * inv;
  }
  if (act) {
#pragma unroll
    for (int c = 0; c < XM; ++c) {
      bP(C, k, j, c) = a0[c];
      bP(C, k, j + QM, c) = a1[c];
    }
    if (bad) flag_nonfinite(C);
  }
  __syncwarp();
}

// ------------------------------------------------------------ stage 3: PCG

// Two rows of the off-diagonal blocks of S and of D^-1.  With REG = true all
// of them live in registers (the latency variant, 1 CTA per SM); with
// REG = false only the D^-1 rows do and L_k / L_{k+1}^T are read from their
// blocks (the throughput variant, 2 CTAs per SM).  The diagonal blocks D_k,
// used once per iteration, are always read from their block.  Values and
// arithmetic order are the same in both, so the results are bitwise equal.
template <bool REG>
struct RowRegs;

template <>
struct RowRegs<true> {
  float L0[XM], L1[XM];  // rows j, j+7 of L_k (zero for k = 0)
  float U0[XM], U1[XM];  // columns j, j+7 of L_{k+1} (zero for k = N)
  float P0[XM], P1[XM];  // rows j, j+7 of D_k^-1
  __device__ __forceinline__ float l0(int c) const { return L0[c]; }
  __device__ __forceinline__ float l1(int c) const { return L1[c]; }
  __device__ __forceinline__ float u0(int c) const { return U0[c]; }
  __device__ __forceinline__ float u1(int c) const { return U1[c]; }
  __device__ __forceinline__ void load(const Ctx& C, int k, int j, bool act) {
    load_from(C.Lm, C.Pm, C.bk0, C.N, k, j, act, true);
  }
  // Rows of knot k from block arrays whose first block is knot bk0 (this
  // CTA's or, through distributed shared memory, a neighbour's); lu = false
  // leaves the L and L^T rows zero.
  __device__ __forceinline__ void load_from(const float* Lm, const float* Pm, int bk0, int N, int k, int j,
                                            bool act, bool lu) {
    const int i0 = j, i1 = j + QM;
    const float* Lk = Lm + (k - bk0) * BS;
    const float* Pk = Pm + (k - bk0) * BS;
#pragma unroll
    for (int c = 0; c < XM; ++c) {
      L0[c] = (act && lu && k > 0) ? Lk[c * XM + i0] : 0.f;
      L1[c] = (act && lu && k > 0) ? Lk[c * XM + i1] : 0.f;
      U0[c] = (act && lu && k < N) ? Lk[BS + i0 * XM + c] : 0.f;
      U1[c] = (act && lu && k < N) ? Lk[BS + i1 * XM + c] : 0.f;
      P0[c] = act ? Pk[c * XM + i0] : 0.f;
      P1[c] = act ? Pk[c * XM + i1] : 0.f;
    }
  }
};

template <>
struct RowRegs<false> {
  const float* Lr;  // &L_k(j, 0): element (j, c) at Lr[c * XM], row j+7 at +7
  const float* Ur;  // &L_{k+1}(0, j): element (c, j) at Ur[c], column j+7 at +7 * XM
  float P0[XM], P1[XM];
  __device__ __forceinline__ float l0(int c) const { return Lr[c * XM]; }
  __device__ __forceinline__ float l1(int c) const { return Lr[c * XM + QM]; }
  __device__ __forceinline__ float u0(int c) const { return Ur[c]; }
  __device__ __forceinline__ float u1(int c) const { return Ur[QM * XM + c]; }
  __device__ __forceinline__ void load(const Ctx& C, int k, int j, bool act) {
    // k = 0 has L_0 = 0 stored; k = N reads the zero block L_{N+1} slot below
    const int kk = act ? k : C.k0;
    Lr = &bL(C, kk, j, 0);
    Ur = (act && k < C.N) ? &bL(C, k + 1, 0, j) : C.Lz + j * XM;
#pragma unroll
    for (int c = 0; c < XM; ++c) {
      P0[c] = act ? bP(C, k, j, c) : 0.f;
      P1[c] = act ? bP(C, k, j + QM, c) : 0.f;
    }
  }
};

__device__ __forceinline__ DF shfl_xor_df(DF v, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ DF shfl_df(DF v, int src) {
  return DF{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// Cluster-wide compensated sums of three values (one reduction for all),
// summed over the PCG's working warps 0..NWARP-2 of every CTA.  Inside a warp
// the three sums are reduce-scattered: the first level leaves a and b on the
// lower half-warp and c on the upper, the second a on lanes 0-7 and b on
// 8-15, so each level exchanges one value instead of three.  Lanes 0, 8 and
// 16 write the warp's partials into every CTA of the cluster; then every warp
// sums them in the same fixed order (lane 8q + i takes partials i, i + 8, ...
// of value q) and copies the totals from lanes 0, 8 and 16.
static_assert(NWARP - 1 == 8, "partials are indexed rank * 8 + working warp");
static_assert(3 * 64 * 2 <= RED_SLOTS * RED_W, "three values x 64 partials x 2 floats per buffer");
__device__ __forceinline__ void cluster_df_sum3(float* red, int rank, int csize, DF& a, DF& b, DF& c,
                                                int& buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* const base = red + buf * (RED_SLOTS * RED_W);
  if (warp < NWARP - 1) {
    const bool lower = lane < 16, hi8 = (lane & 8) != 0;
    DF k0 = df_addd(lower ? a : c, shfl_xor_df(lower ? c : a, 16));
    const DF k1 = df_addd(b, shfl_xor_df(b, 16));  // used on the lower half only
    DF v = lower ? (hi8 ? k1 : k0) : k0;
    const DF snd = lower ? (hi8 ? k0 : k1) : k0;
    v = df_addd(v, shfl_xor_df(snd, 8));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v = df_addd(v, shfl_xor_df(v, o));
    if ((lane & 7) == 0 && lane < 24) {
      const int off = ((lane >> 3) * 64 + rank * 8 + warp) * 2;
      const float2 val = make_float2(v.hi, v.lo);
      if (csize > 1) {
        cg::cluster_group cl = cg::this_cluster();
        for (int r = 0; r < csize; ++r) *reinterpret_cast<float2*>(cl.map_shared_rank(base, r) + off) = val;
      } else {
        *reinterpret_cast<float2*>(base + off) = val;
      }
    }
  }
  if (csize > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
  DF v = df_zero();
  if (lane < 24) {
    const float* src = base + (lane >> 3) * 128;
    for (int j = lane & 7; j < 8 * csize; j += 8) {
      const float2 t = *reinterpret_cast<const float2*>(src + 2 * j);
      v = df_addd(v, DF{t.x, t.y});
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = df_addd(v, shfl_xor_df(v, o));
  a = shfl_df(v, 0);
  b = shfl_df(v, 8);
  c = shfl_df(v, 16);
  buf ^= 1;
}

// Preconditioned CG (Sec. II-B, III-B) for the multiplier correction
// S dnu = rhs, started from dnu = 0; nu_0 + dnu equals the warm-started PCG
// iterate on S nu = gamma.  Stair preconditioner (Eq. 6) applied as
// D^-1 - D^-1 O D^-1 (Eq. 6 written exactly in factored form).  Stops when
// sqrt(eta / eta_0) <= eps with eta = r'u and eta_0 from the warm start, none
// when eta_0 < 1e-30.  Returns iterations.
//
// Evaluation order: a single-reduction arrangement of PCG whose iterates
// equal standard PCG's in exact arithmetic.  S is applied to u = Phi r
// (w = S u) and s = S p is carried by s = w + beta s.  One compensated
// reduction per iteration gives r'u, w'u and p_old'w; the new direction's
// curvature is expanded exactly, p'Sp = w'u + 2 beta p_old'w + beta^2
// (p'Sp)_old, and alpha = r'u / p'Sp.  (The Chronopoulos-Gear form instead
// assumes p_old'w = -r'u / alpha_old, which holds only while the FP32
// directions stay conjugate; on the end-effector workload it then stalled at
// the iteration cap where standard PCG takes ~250 iterations.)  Three barriers
// per iteration: the y halo (stair only), the u halo, the reduction.  Every
// address and scalar the loop needs is set up before it.
template <bool REG, bool HREP>
__device__ inline int st_pcg_t(const Ctx& C, float eps, int maxit, int precond, bool* hit_max, int& rbuf) {
  const bool stair = (precond == 0);
  *hit_max = false;
  long long tlast = C.tm ? clock64() : 0;
  // PCG lane map: warps 0-7 carry 4 knots each on lanes 0-27 (slots 0-7,
  // then 9-32); knot slot 8 uses the spare lanes 28-31 of warp 0 (rows 0-3)
  // and 28-30 of warp 1 (rows 4-6) -- slot 8, because its window rows fall in
  // other shared-memory banks than those of slots 0-7 (slots 16 apart share
  // banks).  The last warp does no PCG arithmetic, only barriers and
  // reductions, so no SM sub-partition issues for three working warps.
  const int lane_ = threadIdx.x & 31, warp_ = threadIdx.x >> 5;
  const int rank = C.rank, csize = C.csize;
  // warps 0..wown-1 hold own knots (slots 0-7 on warps 0-1, slot 8 on their
  // spare lanes, slot s > 8 on warp (s-1)/4); the others skip the arithmetic
  const int nown = C.k1 - C.k0;
  const int wown = nown <= 8 ? (nown + 3) / 4 : (nown == 9 ? 2 : (nown - 2) / 4 + 1);
  const bool pwarp = warp_ < wown;
  const bool spare = lane_ >= 28;
  const bool lane_ok = pwarp && (!spare || warp_ == 0 || (warp_ == 1 && lane_ < 31));
  // Halo knots (clusters, latency form): y of the neighbours' knots k0-2,
  // k0-1, k1, k1+1 and t, u of k0-1 and k1 are recomputed here from the
  // neighbours' block rows and their pushed w rows, with the same arithmetic
  // as the owners, so the values are bitwise the owners'.  Then no y or u
  // rows cross CTAs and the reduction's cluster barrier is the only one per
  // iteration.  The CTA's halo knots, in the order k0-2, k0-1, k1, k1+1 (the
  // ones that exist), take halo slots 0..3.  If a warp below the last has no
  // own knots (compact: at most 29 own knots), slot h sits on its lanes
  // 7h..7h+6.  Otherwise slot h < 3 sits on the spare lanes 28-31 of warp
  // 2h+2 (rows 0-3) and 28-30 of warp 2h+3 (rows 4-6), slot 3 on lanes 0-6 of
  // the last warp: a CTA with one neighbour (both CTAs of a two-CTA cluster)
  // has two halo knots on spare lanes of warps that issue their own knots'
  // instructions anyway.  Either way no SM sub-partition issues for three
  // warps unless a middle CTA holds 30 or more knots.
  constexpr bool hrep = REG && HREP;
  const bool hasL = rank > 0, hasR1 = rank < csize - 1 && C.k1 <= C.N, hasR2 = hasR1 && C.k1 + 1 <= C.N;
  const bool compact = wown < NWARP - 1;
  const int hslot = !hrep ? -1
                    : compact ? (warp_ == wown && lane_ < 28 ? lane_ / 7 : -1)
                    : (warp_ >= 2 && warp_ < NWARP - 1 && lane_ >= 28 && !((warp_ & 1) && lane_ == 31))
                          ? (warp_ - 2) / 2
                          : (warp_ == NWARP - 1 && lane_ < 7 ? 3 : -1);
  const int hs = hasL ? hslot : hslot + 2;  // 0: k0-2, 1: k0-1, 2: k1, 3: k1+1
  const bool hact = hslot >= 0 && hs <= 3 && (hs < 2 ? hasL : (hs == 2 ? hasR1 : hasR2));
  const int khalo = hs == 0 ? C.k0 - 2 : (hs == 1 ? C.k0 - 1 : (hs == 2 ? C.k1 : C.k1 + 1));
  const bool htu = hs == 1 || hs == 2;  // halo knots whose t and u are needed
  // a warp whose lanes carry halo knots only
  const bool hw = hrep && (compact ? warp_ == wown : (warp_ == NWARP - 1 && hasL && hasR2));
  // rows j, j+7 with j in 0..6 for every lane (idle lanes use row 0), so that
  // all block and vector addresses stay inside their 14x14 blocks and rows
  const int hrow = compact ? lane_ - 7 * (lane_ / 7)
                            : (warp_ == NWARP - 1 ? lane_ : lane_ - 28 + ((warp_ & 1) ? 4 : 0));
  const int j = lane_ok ? (spare ? lane_ - 28 + (warp_ == 1 ? 4 : 0) : lane_ - 7 * (lane_ / 7))
                        : (hslot >= 0 ? hrow : 0);
  const int slot = spare ? 8 : 4 * warp_ + lane_ / 7 + (4 * warp_ + lane_ / 7 >= 8 ? 1 : 0);
  const int k = hslot >= 0 ? khalo : C.k0 + slot;
  const bool act = lane_ok && k < C.k1;  // own knot
  const bool acty = act || hact;         // y of this lane's knot is stored
  const bool acttu = act || (hact && htu);
  RowRegs<REG> R;
  R.load(C, k, j, act);
  // zero every vector slot of the window (halos at the ends stay zero)
  for (int i = threadIdx.x; i < NVEC * C.vstride; i += NTHR) {
    const int s = i / C.vstride;
    if (s != V_RHS) C.vb[i] = 0.f;
  }
  float* const red = C.red;
  const int ka = acty ? k : C.k0;  // a valid knot for the address set-up of idle lanes
  const int kd = act ? k : C.k0;
  const int vstr = C.vstride;
  float* const wb = vec(C, 0, ka);  // slot s of this knot at wb + s * vstr
#define SLOT(s) (wb + (s) * vstr)
  // neighbour window of this knot's rows (slot s at pb + s * vstr), boundary knots only
  float* pbd = nullptr;
  if (act && C.vbl && k == C.k0) pbd = C.vbl + (k - C.vk0l) * VW;
  if (act && C.vbr && k == C.k1 - 1) pbd = C.vbr + (k - C.vk0r) * VW;
  float* const pb = hrep ? nullptr : pbd;  // y and u rows cross CTAs only without halo knots
  // with halo knots: w rows of the first two and last two knots go to the
  // neighbours' halo slots (V_P0 + iteration parity)
  float* const pwl = (hrep && act && C.vbl && k <= C.k0 + 1) ? C.vbl + (k - C.vk0l) * VW : nullptr;
  float* const pwr = (hrep && act && C.vbr && k >= C.k1 - 2) ? C.vbr + (k - C.vk0r) * VW : nullptr;
#define PUSH(s, a, b)                     \
  if (pb) {                               \
    pb[(s) * vstr + J] = (a);             \
    pb[(s) * vstr + J7] = (b);            \
  }
  const float* const Drow0 = &bD(C, kd, j, 0);  // D_k row j: element c at Drow0[c * XM]
  float* const rr = SLOT(V_RR);
  float* const yv = SLOT(V_Y);
  float* const uv = SLOT(V_Z);
  float* const tv = SLOT(V_W);
  float* const dn = SLOT(V_DNU);
  const int J = j, J7 = j + QM;
  // p, s and the own rows of u, w, r and dnu stay in registers (r and dnu
  // also in the window: y reads all rows of the knot's r, the recovery dnu)
  float p0 = 0.f, p1 = 0.f, s0 = 0.f, s1 = 0.f, u0 = 0.f, u1 = 0.f, w0 = 0.f, w1 = 0.f;
  float rv0 = 0.f, rv1 = 0.f, dv0 = 0.f, dv1 = 0.f;
  if (csize > 1) cg::this_cluster().sync(); else __syncthreads();
  if (act) {
    rv0 = SLOT(V_RHS)[J];
    rv1 = SLOT(V_RHS)[J7];
    rr[J] = rv0;
    rr[J7] = rv1;
  }
  if constexpr (REG) {
    if (hslot >= 0) {
      // the halo knot's rows and right-hand side, from the neighbour that owns it
      // (its blocks and window are final: the barrier above)
      cg::cluster_group cl = cg::this_cluster();
      const int nb = hs < 2 ? rank - 1 : rank + 1;
      const int nk0 = hs < 2 ? C.k0 - kpc_for(C.N, csize) : C.k1;  // the neighbour's first knot
      const int nbs = hact ? nb : rank;
      R.load_from(cl.map_shared_rank(C.Lm, nbs), cl.map_shared_rank(C.Pm, nbs), nk0, C.N, k, j, hact, htu);
      if (hact) {
        const float* rhs = cl.map_shared_rank(C.vb, nb) + V_RHS * vstr + (k - (nk0 - 2)) * VW;
        rv0 = rhs[J];
        rv1 = rhs[J7];
        rr[J] = rv0;
        rr[J7] = rv1;
      }
    }
  }
  int it = 0;
  float gamma0 = 0.f, alpha = 0.f, inv_gamma = 0.f, psp = 0.f;
  const float eps2 = eps * eps;
  while (true) {
    // u = Phi r: y = D^-1 r; u = y - D^-1 (O y).  Idle lanes (act false) run
    // the same straight-line code on a valid knot with zero block rows, so
    // the warp never branches on act; only their stores are predicated off.
    // (Block barrier: knot slot 8's rows span warps 0 and 1.)
    __syncthreads();
    if (pwarp || hw) {
      float y0 = 0.f, y1 = 0.f;
#pragma unroll
      for (int m = 0; m < XM / 2; ++m) {
        const float2 v = ld2(rr, m);
        y0 += R.P0[2 * m] * v.x;
        y1 += R.P1[2 * m] * v.x;
        y0 += R.P0[2 * m + 1] * v.y;
        y1 += R.P1[2 * m + 1] * v.y;
      }
      u0 = y0;
      u1 = y1;
      float* const dst = stair ? yv : uv;
      if (acty) {
        dst[J] = y0;
        dst[J7] = y1;
      }
      PUSH(stair ? V_Y : V_Z, y0, y1);
    }
    if (stair) {
      if (csize > 1 && !hrep) cg::this_cluster().sync(); else __syncthreads();
      tstamp(C, T_PCG_Y, tlast);
      if (pwarp || hw) {
        float t0 = 0.f, t1 = 0.f;
#pragma unroll
        for (int m = 0; m < XM / 2; ++m) {
          const float2 vm = ld2(yv - VW, m), vp = ld2(yv + VW, m);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = 2 * m + h;
            const float a = h ? vm.y : vm.x, b = h ? vp.y : vp.x;
            t0 += R.l0(c) * a;
            t1 += R.l1(c) * a;
            t0 += R.u0(c) * b;
            t1 += R.u1(c) * b;
          }
        }
        if (acttu) {
          tv[J] = t0;
          tv[J7] = t1;
        }
      }
      __syncthreads();
      if (pwarp || hw) {
        float q0 = 0.f, q1 = 0.f;
#pragma unroll
        for (int m = 0; m < XM / 2; ++m) {
          const float2 v = ld2(tv, m);
          q0 += R.P0[2 * m] * v.x;
          q1 += R.P1[2 * m] * v.x;
          q0 += R.P0[2 * m + 1] * v.y;
          q1 += R.P1[2 * m + 1] * v.y;
        }
        u0 -= q0;
        u1 -= q1;
        if (acttu) {
          uv[J] = u0;
          uv[J7] = u1;
        }
        PUSH(V_Z, u0, u1);
      }
    }
    if (csize > 1 && !hrep) cg::this_cluster().sync(); else __syncthreads();
    // w = S u
    DF ru = df_zero(), wu = df_zero(), pw = df_zero();
    if (pwarp) {
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int m = 0; m < XM / 2; ++m) {
        const float2 v2 = ld2(uv, m), vm2 = ld2(uv - VW, m), vp2 = ld2(uv + VW, m);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * m + h;
          const float v0 = h ? v2.y : v2.x;
          a0 += Drow0[c * XM] * v0;
          a1 += Drow0[c * XM + QM] * v0;
          const float vm = h ? vm2.y : vm2.x;
          a0 += R.l0(c) * vm;
          a1 += R.l1(c) * vm;
          const float vp = h ? vp2.y : vp2.x;
          a0 += R.u0(c) * vp;
          a1 += R.u1(c) * vp;
        }
      }
      w0 = a0;
      w1 = a1;
      const int wsl = (V_P0 + (it & 1)) * vstr;  // the neighbours' halo w slot of this iteration
      if (pwl) {
        pwl[wsl + J] = w0;
        pwl[wsl + J7] = w1;
      }
      if (pwr) {
        pwr[wsl + J] = w0;
        pwr[wsl + J7] = w1;
      }
      const DF ru1 = df_fma(df_fma(ru, rv0, u0), rv1, u1);
      const DF wu1 = df_fma(df_fma(wu, w0, u0), w1, u1);
      const DF pw1 = df_fma(df_fma(pw, p0, w0), p1, w1);  // p still holds the previous direction
      ru = act ? ru1 : ru;
      wu = act ? wu1 : wu;
      pw = act ? pw1 : pw;
    }
    tstamp(C, T_PCG_S, tlast);
    cluster_df_sum3(red, rank, csize, ru, wu, pw, rbuf);
    tstamp(C, T_PCG_WZ, tlast);
    // scalars: one division on the critical path; 1/gamma for the next
    // iteration is formed off it, and the stopping rule
    // sqrt(gamma / gamma_0) <= eps is tested as gamma <= eps^2 gamma_0
    const float gnew = df_val(ru), wu_f = df_val(wu), pw_f = df_val(pw);
    float beta;
    if (it == 0) {
      gamma0 = gnew;
      if (!(gamma0 > 1e-30f)) break;
      beta = 0.f;
      psp = wu_f;
    } else {
      if (!(gnew > 0.f) || gnew <= eps2 * gamma0) break;
      if (it >= maxit) {
        *hit_max = true;
        break;
      }
      beta = gnew * inv_gamma;
      psp = wu_f + beta * (2.f * pw_f + beta * psp);
    }
    alpha = gnew / psp;
    inv_gamma = 1.f / gnew;
    if (hslot >= 0) {  // the owner's w rows of this halo knot, pushed before the reduction
      const float* wh = SLOT(V_P0 + (it & 1));
      w0 = wh[J];
      w1 = wh[J7];
    }
    // p = u + beta p; s = w + beta s; dnu += alpha p; r -= alpha s (halo
    // knots: s and r only, the same expressions as their owners')
    p0 = u0 + beta * p0;
    p1 = u1 + beta * p1;
    s0 = w0 + beta * s0;
    s1 = w1 + beta * s1;
    {
      const float d0 = dv0 + alpha * p0, d1 = dv1 + alpha * p1;
      const float r0 = rv0 - alpha * s0, r1 = rv1 - alpha * s1;
      dv0 = d0;
      dv1 = d1;
      rv0 = r0;
      rv1 = r1;
      if (acty) {
        rr[J] = r0;
        rr[J7] = r1;
      }
    }
    ++it;
  }
  // the correction into the window (once, after the loop) and its boundary
  // rows to the neighbours for the recovery
  if (act) {
    dn[J] = dv0;
    dn[J7] = dv1;
  }
  if (act && pbd) {
    pbd[V_DNU * vstr + J] = dv0;
    pbd[V_DNU * vstr + J7] = dv1;
  }
  if (csize > 1) cg::this_cluster().sync(); else __syncthreads();
  return it;
#undef PUSH
#undef SLOT
}

// Out-of-line form of the loop, with the context passed by value: its
// registers are allocated on their own, so a caller whose other stages hold
// many live values (the high-precision kernel) cannot push the loop's
// register-resident block rows into local memory.  (In a caller without that
// pressure the inlined loop is faster: the call boundary costs it ~8 % per
// iteration.)
struct PcgOut {
  int it, hit, rbuf;
};

template <bool REG, bool HREP>
static __device__ __noinline__ PcgOut st_pcg_call(const Ctx C, float eps, int maxit, int precond, int rbuf) {
  bool hit = false;
  const int it = st_pcg_t<REG, HREP>(C, eps, maxit, precond, &hit, rbuf);
  return PcgOut{it, hit ? 1 : 0, rbuf};
}

// The loop with halo knots (C.hrep: fused latency form in a cluster) and
// without are separate instantiations, so the one-CTA loop carries none of
// the halo logic.  OOL: the out-of-line form above.
template <bool REG, bool OOL = false>
__device__ inline int st_pcg(const Ctx& C, float eps, int maxit, int precond, bool* hit_max, int& rbuf) {
  if constexpr (OOL) {
    const PcgOut o = (REG && C.hrep) ? st_pcg_call<REG, true>(C, eps, maxit, precond, rbuf)
                                     : st_pcg_call<REG, false>(C, eps, maxit, precond, rbuf);
    *hit_max = o.hit != 0;
    rbuf = o.rbuf;
    return o.it;
  } else {
    if constexpr (REG) {
      if (C.hrep) return st_pcg_t<true, true>(C, eps, maxit, precond, hit_max, rbuf);
    }
    return st_pcg_t<REG, false>(C, eps, maxit, precond, hit_max, rbuf);
  }
}

// ------------------------------------------------- stage 4: step recovery

// --------------------------------------- stage 3b: direct linear solve
//
// The direct alternative to PCG that Sec. II-B sets against iterative
// methods, for the same system S dnu = rhs, by block elimination from both
// ends of the horizon towards the knot m = floor((N+1)/2):
//   from the top, k < m:     D~_0 = D_0,  D~_k = D_k - L_k D~_{k-1}^-1 L_k^T,
//                            y~_k = rhs_k - L_k D~_{k-1}^-1 y~_{k-1};
//   from the bottom, k >= m: D^_N = D_N,  D^_k = D_k - L_{k+1}^T D^_{k+1}^-1 L_{k+1},
//                            y^_k = rhs_k - L_{k+1}^T D^_{k+1}^-1 y^_{k+1};
//   at m both meet:          G_m = D^_m - L_m D~_{m-1}^-1 L_m^T,
//                            g_m = y^_m - L_m D~_{m-1}^-1 y~_{m-1},  dnu_m = G_m^-1 g_m;
//   then outwards:           dnu_k = D~_k^-1 (y~_k - L_{k+1}^T dnu_{k+1})  (k < m),
//                            dnu_k = D^_k^-1 (y^_k - L_k dnu_{k-1})        (k > m).
// (Eliminating the last equation into the one above gives the bottom
// recursion; G_m is what is left of row m after both.)  The chain is about
// N/2 knots long when the two halves sit on different CTAs of a cluster, and
// m depends on N only, so every knot's arithmetic, and the result, is the
// same for any split of the knots over CTAs.  Inside a knot the work is
// parallel over the 14x14 block (one element per thread, block barriers
// between the products); the inverses by Gauss-Jordan on 2x2 pivot blocks
// without pivoting (every eliminated block is a Schur complement of the SPD
// S, so SPD; a pivot block that is not positive definite flags the solve).  Stage s of the sweeps runs rank s from
// the top and rank C-1-s from the bottom; the back substitution starts at the
// rank holding m and moves one rank outwards per stage.  Hand-overs go
// through distributed shared memory with one cluster barrier per stage;
// inverses go to the preconditioner's block slot, y~ / y^ to the y window,
// and the reduction slots are the scratch.
__device__ __forceinline__ void st_direct_body(const Ctx& C) {
  constexpr int BB = XM * XM;
  static_assert(5 * BB + 4 * XM <= 2 * RED_SLOTS * RED_W, "scratch in the reduction slots");
  static_assert(BB + XM <= NTHR, "one block element per thread");
  const int t = threadIdx.x;
  const int i = t % XM, j = t / XM;  // element (i, j) of a column-major block, t < BB
  const bool el = t < BB;
  // the vector part of a step runs on warp 7, which holds no block element
  // (warp 6 holds elements 192-195)
  constexpr int YT = 7 * 32;
  static_assert(BB <= YT && YT + XM <= NTHR, "vector part on its own warp");
  float* const W = C.red;
  float* const G0 = W + BB;
  float* const G1 = G0 + BB;
  float* const cF = G1 + BB;       // from the left neighbour: [BB] D~_{k0-1}^-1, [XM] y~_{k0-1}
  float* const cB = cF + BB + XM;  // from the right neighbour: [BB] D^_{k1}^-1, [XM] y^_{k1}
  float* const dL = cB + BB + XM;  // dnu_{k0-1} from the left neighbour
  float* const dR = dL + XM;       // dnu_{k1} from the right neighbour
  const int N = C.N, m = (N + 1) / 2;
  const int rm = m / kpc_for(N, C.csize);  // the rank holding m
  const bool own = C.k0 < C.k1;
  csync(C);  // every CTA has finished reading the reduction slots of earlier stages

  // G0 (SPD) inverted into Pk by Gauss-Jordan on 2x2 pivot blocks: with
  // P = {p, p+1} and Pi = A[P,P]^-1, the pivot block becomes Pi, pivot rows
  // Pi A[P,j], pivot columns -A[i,P] Pi, the rest A - A[:,P] Pi A[P,:] (seven
  // block barriers for 14 pivots; every leading block of an SPD matrix is SPD)
  static_assert(XM % 2 == 0, "pivot pairs");
  auto invert_into = [&](float* Pk) {
    float* A = G0;
    float* B = G1;
    for (int p = 0; p < XM; p += 2) {
      const int q = p + 1;
      if (el) {
        // element (r, c) at c * XM + r
        const float a = A[p * XM + p], b = A[q * XM + p], c = A[p * XM + q], d = A[q * XM + q];
        const float det = a * d - b * c;
        const float id = 1.f / det;
        const float P00 = d * id, P01 = -b * id, P10 = -c * id, P11 = a * id;
        const bool ip = (i == p || i == q), jp = (j == p || j == q);
        // every class's value (pivot block, pivot rows, pivot columns, the
        // rest) by its own expressions, then one select: the elements of a
        // warp fall in all four classes, so branches would run one by one
        const float apj = A[j * XM + p], aqj = A[j * XM + q], aip = A[p * XM + i], aiq = A[q * XM + i];
        const float v0 = P00 * apj + P01 * aqj, v1 = P10 * apj + P11 * aqj;  // Pi A[P, j]
        const float piv = (i == p) ? (j == p ? P00 : P01) : (j == p ? P10 : P11);
        const float row = (i == p) ? v0 : v1;
        const float col = (j == p) ? -(aip * P00 + aiq * P10) : -(aip * P01 + aiq * P11);
        const float rest = A[t] - (aip * v0 + aiq * v1);
        const float out = ip ? (jp ? piv : row) : (jp ? col : rest);
        (p == XM - 2 ? Pk : B)[t] = out;
        if (t == 0 && !(a > 0.f && det > 0.f && det < INFINITY)) flag_nonfinite(C);
      }
      __syncthreads();
      float* const tmp = A;
      A = B;
      B = tmp;
    }
  };
  // G0 = Ds - L_k Pp L_k^T, y_k = rs - L_k Pp yp (a step from the top; Ds / rs
  // may be the knot's own D^ / y^ slots at the meeting knot)
  auto from_top = [&](int k, const float* Ds, const float* rs, const float* Pp, const float* yp) {
    const float* Lk = &bL(C, k, 0, 0);
    float* yk = vec(C, V_Y, k);
    if (el) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < XM; ++l) a += Lk[l * XM + i] * Pp[j * XM + l];
      W[t] = a;
    }
    __syncthreads();
    if (el) {
      float a = Ds[t];
#pragma unroll
      for (int l = 0; l < XM; ++l) a -= W[l * XM + i] * Lk[l * XM + j];
      G0[t] = a;
    } else if (t >= YT && t < YT + XM) {
      const int r = t - YT;
      float a = rs[r];
#pragma unroll
      for (int l = 0; l < XM; ++l) a -= W[l * XM + r] * yp[l];
      yk[r] = a;
    }
    __syncthreads();
  };
  // G0 = D_k - L_{k+1}^T Pn L_{k+1}, y_k = rhs_k - L_{k+1}^T Pn yn (a step from the bottom)
  auto from_bottom = [&](int k, const float* Pn, const float* yn) {
    const float* Ln = &bL(C, k + 1, 0, 0);  // (L_{k+1}^T)(i, l) = L_{k+1}(l, i)
    const float* Dk = &bD(C, k, 0, 0);
    const float* rk = vec(C, V_RHS, k);
    float* yk = vec(C, V_Y, k);
    if (el) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < XM; ++l) a += Ln[i * XM + l] * Pn[j * XM + l];
      W[t] = a;
    }
    __syncthreads();
    if (el) {
      float a = Dk[t];
#pragma unroll
      for (int l = 0; l < XM; ++l) a -= W[l * XM + i] * Ln[j * XM + l];
      G0[t] = a;
    } else if (t >= YT && t < YT + XM) {
      const int r = t - YT;
      float a = rk[r];
#pragma unroll
      for (int l = 0; l < XM; ++l) a -= W[l * XM + r] * yn[l];
      yk[r] = a;
    }
    __syncthreads();
  };
  // the block as it is: D_k, rhs_k (the first knot from either end)
  auto as_is = [&](int k) {
    if (el) G0[t] = bD(C, k, i, j);
    else if (t >= YT && t < YT + XM) vec(C, V_Y, k)[t - YT] = vec(C, V_RHS, k)[t - YT];
    __syncthreads();
  };

  // sweeps from both ends
  for (int s = 0; s < C.csize; ++s) {
    if (C.rank == s && own) {  // from the top: knots [k0, min(k1, m))
      const int ke = min(C.k1, m);
      for (int k = C.k0; k < ke; ++k) {
        if (k == 0)
          as_is(k);
        else
          from_top(k, &bD(C, k, 0, 0), vec(C, V_RHS, k), k == C.k0 ? cF : &bP(C, k - 1, 0, 0),
                   k == C.k0 ? cF + BB : vec(C, V_Y, k - 1));
        invert_into(&bP(C, k, 0, 0));
      }
      if (C.k1 <= m && C.rank + 1 < C.csize) {  // D~^-1 and y~ of the last knot to the next CTA
        float* dst = cg::this_cluster().map_shared_rank(cF, C.rank + 1);
        if (el)
          dst[t] = bP(C, C.k1 - 1, i, j);
        else if (t < BB + XM)
          dst[t] = vec(C, V_Y, C.k1 - 1)[t - BB];
      }
    }
    if (C.rank == C.csize - 1 - s && own && C.k1 > m) {  // from the bottom: knots [max(k0, m), k1)
      const int kb = max(C.k0, m);
      for (int k = C.k1 - 1; k >= kb; --k) {
        if (k == N)
          as_is(k);
        else
          from_bottom(k, k == C.k1 - 1 ? cB : &bP(C, k + 1, 0, 0), k == C.k1 - 1 ? cB + BB : vec(C, V_Y, k + 1));
        if (k > m) {
          invert_into(&bP(C, k, 0, 0));
        } else {  // D^_m is kept as it is for the meeting step
          if (el) bP(C, k, i, j) = G0[t];
          __syncthreads();
        }
      }
      if (C.k0 > m && C.rank > 0) {  // D^^-1 and y^ of the first knot to the previous CTA
        float* dst = cg::this_cluster().map_shared_rank(cB, C.rank - 1);
        if (el)
          dst[t] = bP(C, C.k0, i, j);
        else if (t < BB + XM)
          dst[t] = vec(C, V_Y, C.k0)[t - BB];
      }
    }
    csync(C);
  }
  // the meeting knot: G_m^-1 and dnu_m; dnu_m goes at once to a neighbour
  // whose first (last) knot is next to m
  const int kpc = kpc_for(N, C.csize);
  const int k0m = rm * kpc, k1m = min(k0m + kpc, N + 1);
  if (own && C.rank == rm) {
    const bool loc = m - 1 >= C.k0;
    from_top(m, &bP(C, m, 0, 0), vec(C, V_Y, m), loc ? &bP(C, m - 1, 0, 0) : cF, loc ? vec(C, V_Y, m - 1) : cF + BB);
    invert_into(&bP(C, m, 0, 0));
    if (t < XM) W[t] = vec(C, V_Y, m)[t];
    __syncthreads();
    if (t < XM) {
      const float* Pm = &bP(C, m, 0, 0);
      float x = 0.f;
#pragma unroll
      for (int l = 0; l < XM; ++l) x += Pm[l * XM + t] * W[l];
      vec(C, V_DNU, m)[t] = x;
      if (m == C.k1 - 1 && C.rank + 1 < C.csize && C.k1 <= N)
        cg::this_cluster().map_shared_rank(dL, C.rank + 1)[t] = x;
      if (m == C.k0 && C.rank > 0) cg::this_cluster().map_shared_rank(dR, C.rank - 1)[t] = x;
    }
  }
  csync(C);
  // back substitution outwards: rank rm at stage 0, its neighbours one stage
  // later (at once when dnu_m reached them above), and so on
  const int sdown = rm - C.rank - (m == k0m ? 1 : 0);  // stage of a rank below rm
  const int sup = C.rank - rm - (m == k1m - 1 ? 1 : 0);  // stage of a rank above rm
  for (int s = 0; s < C.csize; ++s) {
    const bool mid = own && C.rank == rm && s == 0;
    const bool down = mid || (own && C.rank < rm && s == sdown);
    const bool up = mid || (own && C.rank > rm && s == sup);
    // the substitution runs on lanes 0-13 of warp 0 (warp barriers); the
    // other warps wait at the stage's cluster barrier
    if (down && t < 32) {  // k from m-1 (rank rm) or k1-1 down to k0
      for (int k = (C.rank == rm ? m - 1 : C.k1 - 1); k >= C.k0; --k) {
        if (t < XM) {
          float b = vec(C, V_Y, k)[t];
          const float* xn = (k == C.k1 - 1) ? dR : vec(C, V_DNU, k + 1);
          const float* Ln = &bL(C, k + 1, 0, 0);  // (L_{k+1}^T)(t, l) = L_{k+1}(l, t)
#pragma unroll
          for (int l = 0; l < XM; ++l) b -= Ln[t * XM + l] * xn[l];
          W[t] = b;
        }
        __syncwarp();
        if (t < XM) {
          const float* Pk = &bP(C, k, 0, 0);
          float x = 0.f;
#pragma unroll
          for (int l = 0; l < XM; ++l) x += Pk[l * XM + t] * W[l];
          vec(C, V_DNU, k)[t] = x;
        }
        __syncwarp();
      }
      // the first dnu to the previous CTA (unless dnu_m went there already)
      if (t < XM && C.rank > 0 && !(C.rank == rm && m == C.k0))
        cg::this_cluster().map_shared_rank(dR, C.rank - 1)[t] = vec(C, V_DNU, C.k0)[t];
    }
    if (up && t < 32) {  // k from m+1 (rank rm) or k0 up to k1-1
      for (int k = (C.rank == rm ? m + 1 : C.k0); k < C.k1; ++k) {
        if (t < XM) {
          float b = vec(C, V_Y, k)[t];
          const float* xp = (k == C.k0) ? dL : vec(C, V_DNU, k - 1);
          const float* Lk = &bL(C, k, 0, 0);
#pragma unroll
          for (int l = 0; l < XM; ++l) b -= Lk[l * XM + t] * xp[l];
          W[t] = b;
        }
        __syncwarp();
        if (t < XM) {
          const float* Pk = &bP(C, k, 0, 0);
          float x = 0.f;
#pragma unroll
          for (int l = 0; l < XM; ++l) x += Pk[l * XM + t] * W[l];
          vec(C, V_DNU, k)[t] = x;
        }
        __syncwarp();
      }
      // the last dnu to the next CTA (unless dnu_m went there already)
      if (t < XM && C.rank + 1 < C.csize && C.k1 <= N && !(C.rank == rm && m == C.k1 - 1))
        cg::this_cluster().map_shared_rank(dL, C.rank + 1)[t] = vec(C, V_DNU, C.k1 - 1)[t];
    }
    csync(C);
  }
  // the right neighbour's first dnu is this CTA's halo for the recovery
  if (t < XM && C.rank > 0 && own)
    cg::this_cluster().map_shared_rank(dR, C.rank - 1)[t] = vec(C, V_DNU, C.k0)[t];
  csync(C);
  if (t < XM && C.rank + 1 < C.csize && C.k1 <= N) vec(C, V_DNU, C.k1)[t] = dR[t];
}

// The direct solve as a call of its own (kept out of the kernel body so that
// the PCG's register allocation does not change with it), with the fields it
// reads passed by value rather than through the caller's Ctx in memory.
struct DirectView {
  float *Dm, *Lm, *Pm, *vb, *red, *scal;
  int bk0, vstride, vk0, k0, k1, N, rank, csize;
};

static __device__ __noinline__ void st_direct_call(DirectView v) {
  Ctx C;
  C.Dm = v.Dm;
  C.Lm = v.Lm;
  C.Pm = v.Pm;
  C.vb = v.vb;
  C.red = v.red;
  C.scal = v.scal;
  C.bk0 = v.bk0;
  C.vstride = v.vstride;
  C.vk0 = v.vk0;
  C.k0 = v.k0;
  C.k1 = v.k1;
  C.N = v.N;
  C.rank = v.rank;
  C.csize = v.csize;
  st_direct_body(C);
}

__device__ __forceinline__ void st_direct(const Ctx& C) {
  st_direct_call(DirectView{C.Dm, C.Lm, C.Pm, C.vb, C.red, C.scal, C.bk0, C.vstride, C.vk0, C.k0, C.k1, C.N,
                            C.rank, C.csize});
}

// dx_k = -Q_k^-1 (q_k + nu_k - A_k^T nu_{k+1}), du_k = -R_k^-1 (r_k - B_k^T nu_{k+1})
// (Eq. 4 with Eq. 1's sign convention C dZ = c), evaluated as -G^-1 (d + C^T dnu); then nu += dnu.
__device__ inline void st_recover(const Ctx& C) {
  const int N = C.N;
  const float h = C.h;
  bool bad = false;
  OWN_KNOT(C);
  float bt = 0.f;
  float* wv = act ? vec(C, V_W, k) : nullptr;
  if (act) {
    const float* dn = vec(C, V_DNU, k);
    float at0 = 0.f, at1 = 0.f;
    if (k < N) {
      const float* dn1 = vec(C, V_DNU, k + 1);
      float cf[QM];
      at_factor(dn1, h, cf);
      at_rows(C.Fq + k * FQS, C.Fv + k * FQS, dn1, cf, h, j, at0, at1);
      bt = bt_row(C.Mi + k * FQS, cf, j);
    }
    wv[j] = C.Dx[k * VS + j] + dn[j] - at0;
    wv[j + QM] = C.Dx[k * VS + j + QM] + dn[j + QM] - at1;
  }
  __syncwarp();
  if (act) {
    const float* Qi = C.Qi + k * QIS;
    float a = 0.f;
#pragma unroll
    for (int l = 0; l < QM; ++l) a += Qi[j * QM + l] * wv[l];
    const float dx0 = -a;
    const float dx1 = -Qi[49 + j] * wv[j + QM];
    C.dX[k * VS + j] = dx0;
    C.dX[k * VS + j + QM] = dx1;
    bad = bad || !isfinite(dx0) || !isfinite(dx1);
    if (k < N) {
      const float du = -C.Ri[k * US + j] * (C.Du[k * US + j] - bt);
      C.dU[k * US + j] = du;
      bad = bad || !isfinite(du);
    }
    const float* dn = vec(C, V_DNU, k);
    C.nu[k * VS + j] += dn[j];
    C.nu[k * VS + j + QM] += dn[j + QM];
  }
  if (bad) flag_nonfinite(C);
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


// High-precision trial merits: the trial point (X + Xlo) + alpha dX in
// double-float (dfl); qdd from the FP32 factor refined twice against a
// double-float RNEA residual u - ID(q, qd, qdd_0); defects and costs in
// double-float (sin and cos of q by FP64).  Each per-knot value is stored as
// an (hi, lo) float pair (hi in `hi`, lo in `lo`, [na][K] each).
struct LsView {
  const DevModel* M;
  const float *X, *Xlo, *U, *Ulo, *dX, *dU, *xs, *x_ref, *ee_ref;
  float *hi, *lo;
  float w[6];
  float fx, fy, fz;
  float h, mu, beta;
  int N, dof, cost_kind, k0, k1, na;
  bool base;
};

static __device__ __noinline__ void st_line_search_hp(LsView v) {
  const int N = v.N, K = v.k1 - v.k0;
  const DevModel& M = *v.M;
  const int nx = 2 * v.dof;
  const dfl half(0.5f);
  for (int it = threadIdx.x; it < v.na * K; it += NTHR) {
    const int a = it / K, k = v.k0 + it % K;
    // the step length as the accept stage forms it (a float)
    float alpha = 1.f;
    for (int i = 0; i < a; ++i) alpha /= v.beta;
    if (v.base) alpha = 0.f;
    auto xat = [&](int idx) { return dfl(v.X[idx], v.Xlo[idx]) + dfl(alpha) * dfl(v.dX[idx]); };
    auto uat = [&](int idx) { return dfl(v.U[idx], v.Ulo[idx]) + dfl(alpha) * dfl(v.dU[idx]); };
    const dfl s = (k == N) ? dfl(v.w[3]) : dfl(1);
    dfl x[XM];
#pragma unroll
    for (int i = 0; i < XM; ++i) x[i] = xat(k * VS + i);
    // sin and cos of the trial q, shared by the kinematics and the dynamics
    dfl sq[QM], cq[QM];
    if (v.cost_kind != 0 || k < N) {
#pragma unroll
      for (int i = 0; i < QM; ++i) sincos(x[i], &sq[i], &cq[i]);
    }
    dfl val(0);
    // stage cost
    if (v.cost_kind == 0) {
#pragma unroll
      for (int i = 0; i < XM; ++i) {
        const int ui = i < QM ? i : i - QM + v.dof;  // user layout of x_ref
        const bool used = (i < QM ? i : i - QM) < v.dof;
        const dfl wi(i < QM ? v.w[0] : v.w[1]);
        const dfl d = used ? x[i] - dfl(v.x_ref[k * nx + ui]) : dfl(0);
        val += half * s * wi * d * d;
      }
    } else {
      dfl p[3];
      fk_ee_sc<dfl>(M, sq, cq, p, nullptr);
      const float* pr = v.ee_ref + 3 * k;
      const dfl d0 = p[0] - dfl(pr[0]), d1 = p[1] - dfl(pr[1]), d2 = p[2] - dfl(pr[2]);
      val += half * s * dfl(v.w[4]) * (d0 * d0 + d1 * d1 + d2 * d2);
#pragma unroll
      for (int i = 0; i < QM; ++i) val += half * s * dfl(v.w[1]) * x[QM + i] * x[QM + i];
    }
    if (k < N) {
      dfl u[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        u[i] = uat(k * US + i);
        val += half * dfl(v.w[2]) * u[i] * u[i];
      }
      // FP32 forward dynamics at the rounded point, then refinement
      // against the double-float inverse dynamics at the exact trial point
      float qf[QM], qdf[QM], sqf[QM], cqf[QM], Ml[28], z[QM], b[QM], qdd[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        qf[i] = x[i].hi;
        qdf[i] = x[QM + i].hi;
        sincosf(qf[i], &sqf[i], &cqf[i]);
        z[i] = 0.f;
      }
      mass_matrix_crba(M, sqf, cqf, Ml);
      const V3 fw = v3(v.fx, v.fy, v.fz);
      rnea_value(M, sqf, cqf, qdf, z, M.g, fw, b, nullptr);
#pragma unroll
      for (int i = 0; i < QM; ++i) qdd[i] = u[i].hi - b[i];
      chol7(Ml);
      chol7_solve(Ml, qdd);
      dfl qd[QM], a0[QM], tau[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        qd[i] = x[QM + i];
        a0[i] = dfl(qdd[i]);
      }
      // two refinement steps: each shrinks the error of qdd by ~kappa(M) eps_32
      // (the FP32 CRBA factor is the preconditioner), from ~1e-5 to ~1e-12
      // relative, below the merit decreases the line search must resolve
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        rnea_value<dfl>(M, sq, cq, qd, a0, dfl(M.g), v3t<dfl>(dfl(v.fx), dfl(v.fy), dfl(v.fz)), tau, nullptr);
        float r[QM];
#pragma unroll
        for (int i = 0; i < QM; ++i) r[i] = i < v.dof ? (u[i] - tau[i]).hi : 0.f;
        chol7_solve(Ml, r);
#pragma unroll
        for (int i = 0; i < QM; ++i) a0[i] += dfl(r[i]);
      }
      const dfl h(v.h), h2 = h * h;
      dfl c1(0);
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= v.dof) continue;
        const dfl acc = a0[i];
        const dfl cqd = (x[QM + i] - xat((k + 1) * VS + QM + i)) + h * acc;
        const dfl cq_ = (x[i] - xat((k + 1) * VS + i)) + h * x[QM + i] + h2 * acc;
        c1 += dfl_abs(cq_) + dfl_abs(cqd);
      }
      val += dfl(v.mu) * c1;
    }
    if (k == 0) {
      dfl c0(0);
#pragma unroll
      for (int i = 0; i < XM; ++i) c0 += dfl_abs(dfl(v.xs[i]) - x[i]);
      val += dfl(v.mu) * c0;
    }
    v.hi[a * K + (k - v.k0)] = val.hi;
    v.lo[a * K + (k - v.k0)] = val.lo;
  }
}

// Merit (Eq. 3) of Z + alpha_i dZ for alpha_i = beta^-i (Eq. 7), i < n_alpha:
// one thread per (alpha, own knot); per-alpha sums over the CTA's knots in a
// fixed order, then over the cluster's CTAs in rank order.
__device__ inline void st_line_search(const Ctx& C, float mu, float beta, int n_alpha, int& rbuf,
                                      bool base = false) {
  const int N = C.N, K = C.k1 - C.k0;
  const int na = base ? 1 : n_alpha;
  float* contrib = vec(C, V_Y, C.k0);  // [na][K] (free during the line search)
  float* contrib_lo = vec(C, V_Z, C.k0);  // low parts in the high-precision mode
  if (C.hp) {
    LsView v;
    v.M = C.M;
    v.X = C.X;
    v.Xlo = C.Xlo;
    v.U = C.U;
    v.Ulo = C.Ulo;
    v.dX = C.dX;
    v.dU = C.dU;
    v.xs = C.xs;
    v.x_ref = C.x_ref;
    v.ee_ref = C.ee_ref;
    v.hi = contrib;
    v.lo = contrib_lo;
#pragma unroll
    for (int i = 0; i < 6; ++i) v.w[i] = C.w[i];
    const V3 fw = ee_force(C);
    v.fx = fw.x;
    v.fy = fw.y;
    v.fz = fw.z;
    v.h = C.h;
    v.mu = mu;
    v.beta = beta;
    v.N = N;
    v.dof = C.dof;
    v.cost_kind = C.cost_kind;
    v.k0 = C.k0;
    v.k1 = C.k1;
    v.na = na;
    v.base = base;
    st_line_search_hp(v);
  }
  for (int it = threadIdx.x; it < (C.hp ? 0 : na * K); it += NTHR) {
    const int a = it / K, k = C.k0 + it % K;
    float alpha = 1.f;
    for (int i = 0; i < a; ++i) alpha /= beta;
    // the iterate itself (base) or its trial point Z + alpha dZ
    auto xat = [&](int idx) { return base ? C.X[idx] : C.X[idx] + alpha * C.dX[idx]; };
    auto uat = [&](int idx) { return base ? C.U[idx] : C.U[idx] + alpha * C.dU[idx]; };
    float x[XM], u[QM];
#pragma unroll
    for (int i = 0; i < XM; ++i) x[i] = xat(k * VS + i);
    float v;
    if (k < N) {
#pragma unroll
      for (int i = 0; i < QM; ++i) u[i] = uat(k * US + i);
      float qdd[QM];
      forward_dynamics(*C.M, x, x + QM, u, ee_force(C), qdd);
      float c1 = 0.f;
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        const float qdn = x[QM + i] + C.h * qdd[i];
        const float qn = x[i] + C.h * qdn;
        c1 += fabsf(qn - xat((k + 1) * VS + i));
        c1 += fabsf(qdn - xat((k + 1) * VS + QM + i));
      }
      v = trial_cost(C, k, x, u) + mu * c1;
    } else {
      v = trial_cost(C, k, x, nullptr);
    }
    if (k == 0) {
      float c0 = 0.f;
#pragma unroll
      for (int i = 0; i < XM; ++i) c0 += fabsf(C.xs[i] - xat(i));
      v += mu * c0;
    }
    contrib[a * K + (k - C.k0)] = v;
  }
  __syncthreads();
  // warp a: this CTA's partial of alpha_a (lane-strided over its knots, fixed tree)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* slots = C.red + rbuf * RED_SLOTS * RED_W;  // [rank][alpha] pairs
  for (int a = warp; a < na; a += NWARP) {
    DF s = df_zero();
    for (int kk = lane; kk < K; kk += 32) {
      s = df_add(s, contrib[a * K + kk]);
      if (C.hp) s = df_add(s, contrib_lo[a * K + kk]);
    }
    s = warp_df_sum(s);
    if (lane == 0) {
      const int o = (C.rank * MAX_ALPHA + a) * 2;
      if (C.csize > 1) {
        cg::cluster_group cl = cg::this_cluster();
        for (int r = 0; r < C.csize; ++r) {
          float* dst = cl.map_shared_rank(slots, r);
          dst[o] = s.hi;
          dst[o + 1] = s.lo;
        }
      } else {
        slots[o] = s.hi;
        slots[o + 1] = s.lo;
      }
    }
  }
  csync(C);
  if (threadIdx.x < na) {
    const int a = threadIdx.x;
    DF s = df_zero();
    for (int r = 0; r < C.csize; ++r)
      s = df_addd(s, DF{slots[(r * MAX_ALPHA + a) * 2], slots[(r * MAX_ALPHA + a) * 2 + 1]});
    s = df_norm(s);
    if (!isfinite(s.hi) || !isfinite(s.lo)) s = DF{INFINITY, 0.f};
    const int o = base ? S_MDF : S_MDF + 2 + 2 * a;
    C.scal[o] = s.hi;
    C.scal[o + 1] = s.lo;
    C.scal[base ? S_MERIT0 : S_MERITS + a] = s.hi;
  }
  rbuf ^= 1;
  __syncthreads();
}

// a < b for normalised (hi, lo) merits
__device__ __forceinline__ bool df_less(const float* a, const float* b) {
  return a[0] < b[0] || (a[0] == b[0] && a[1] < b[1]);
}

// Argmin with ties to the smallest index; accept only a strict decrease
// (the paper does not say what happens when no step size lowers the merit).
// The base merit is the accepted trial's (the same evaluation of the same
// point), so trial and base merits always come from the same code.
__device__ inline int st_accept(const Ctx& C, float beta, int n_alpha) {
  const int N = C.N;
  const float* md = C.scal + S_MDF;
  int best = 0;
  for (int a = 1; a < n_alpha; ++a)
    if (df_less(md + 2 + 2 * a, md + 2 + 2 * best)) best = a;
  const int choice = df_less(md + 2 + 2 * best, md) ? best : -1;
  if (choice >= 0) {
    float alpha = 1.f;
    for (int i = 0; i < choice; ++i) alpha /= beta;
    const int ke = C.k1 < N ? C.k1 : N;
    if (C.hp) {  // the double-float iterate: (hi, lo) <- hi + lo + alpha d, rounded to a pair
      for (int i = threadIdx.x; i < (C.k1 - C.k0) * VS; i += NTHR) {
        const int o = C.k0 * VS + i;
        const dfl v = dfl(C.X[o], C.Xlo[o]) + dfl(alpha) * dfl(C.dX[o]);  // the line search's trial point
        C.X[o] = v.hi;
        C.Xlo[o] = v.lo;
      }
      for (int i = threadIdx.x; i < (ke - C.k0) * US; i += NTHR) {
        const int o = C.k0 * US + i;
        const dfl v = dfl(C.U[o], C.Ulo[o]) + dfl(alpha) * dfl(C.dU[o]);
        C.U[o] = v.hi;
        C.Ulo[o] = v.lo;
      }
    } else {
      for (int i = threadIdx.x; i < (C.k1 - C.k0) * VS; i += NTHR) C.X[C.k0 * VS + i] += alpha * C.dX[C.k0 * VS + i];
      for (int i = threadIdx.x; i < (ke - C.k0) * US; i += NTHR) C.U[C.k0 * US + i] += alpha * C.dU[C.k0 * US + i];
    }
  }
  csync(C);  // every thread (and CTA) has read the old base merit
  if (choice >= 0 && threadIdx.x == 0) {
    C.scal[S_MDF] = md[2 + 2 * choice];
    C.scal[S_MDF + 1] = md[3 + 2 * choice];
    C.scal[S_MERIT0] = md[2 + 2 * choice];
  }
  return choice;
}

}  // namespace gato
