// Device-side types, compensated arithmetic and rigid-body dynamics for the
// batched SQP kernels (GATO, arXiv 2510.07625).
//
// Dynamics are written in 3-D Newton-Euler form in link coordinates: a value
// pass of the recursive Newton-Euler algorithm (RNEA) and a tangent pass that
// propagates one directional derivative d/dq_j or d/dqd_j through the same
// recursion using the value pass's stored link quantities.  The paper uses an
// external dynamics library for these (Sec. III-A); this is a from-scratch
// replacement.  Every model is padded to 7 joints: joints past the model's dof
// are massless, sit at the end effector, and get a unit diagonal in M, so the
// padded rows of every matrix and vector stay exactly zero.
#pragma once

#include <type_traits>
#include <cstdint>
#include <cuda_runtime.h>

namespace gato {

constexpr int QM = 7;    // joints (padded)
constexpr int XM = 14;   // state rows [q(7); qd(7)]
constexpr int VS = 16;   // per-knot stride of state-sized vectors
constexpr int US = 8;    // per-knot stride of control-sized vectors
constexpr int BS = 199;  // per-knot stride of a 14x14 column-major block (196 + pad, 199 = 7 mod 32)
constexpr int LVS = 24;  // floats per stored link record
constexpr int MAX_ALPHA = 16;

struct DevModel {
  int dof;
  int axis[QM];
  float L[QM];
  float m[QM];
  float com[3 * QM];
  float Ic[3 * QM];
  float g;
  float pad[3];
};

struct ProbDesc {
  int model, N, cost_kind, dof;
  float dt;
  float w[6];
  float fext[3];  // constant external force on the end effector (base frame)
  const float* x_s;
  const float* x_ref;
  const float* ee_ref;
  float* X;
  float* U;
  float* lam;
};

struct Params {
  float mu, beta;
  int n_alpha;
  float pcg_eps;
  int pcg_max;
  int precond;
  float kkt_tol;
  int max_iter;
  int linsolve;  // 0 PCG, 1 direct block elimination
  int rho_adapt; // 1: rho / 3 after an accepted step, * 2 after a rejected one
  int escalate;  // 1: with kkt_tol > 0, a solve whose FP32 line search finds no
                 // decrease, or whose FP32 KKT test passes, repeats the iteration
                 // in the high-precision mode and stays in it
  int high;      // 1: every iteration in the high-precision mode from the start
};

struct Result {
  int flags, sqp_iters, pcg_iters;
  float kkt, merit;
};

enum : int {
  F_CONVERGED = 1, F_MAXITER = 2, F_LSFAIL = 4, F_PCGMAX = 8, F_NONFINITE = 16
};

// ----------------------------------------------------------------- 3-vectors
// Templated on the scalar: float on the hot path, double for the FP64
// evaluation of the merit's dynamics.  A scalar factor converts to the
// vector's type (the scalar argument does not take part in deduction).

template <typename T>
struct Vec3 {
  T x, y, z;
};
using V3 = Vec3<float>;
template <typename T>
struct Same {
  using type = T;
};
template <typename T>
__device__ __forceinline__ Vec3<T> v3t(T x, T y, T z) { return Vec3<T>{x, y, z}; }
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
template <typename T = float>
__device__ __forceinline__ Vec3<T> vzero() { return Vec3<T>{T(0), T(0), T(0)}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator+(Vec3<T> a, Vec3<T> b) { return Vec3<T>{a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator-(Vec3<T> a, Vec3<T> b) { return Vec3<T>{a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ Vec3<T> operator*(typename Same<T>::type s, Vec3<T> a) {
  return Vec3<T>{s * a.x, s * a.y, s * a.z};
}
template <typename T>
__device__ __forceinline__ Vec3<T> cross(Vec3<T> a, Vec3<T> b) {
  return Vec3<T>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ T dot(Vec3<T> a, Vec3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ Vec3<T> mulI(Vec3<T> I, Vec3<T> v) { return Vec3<T>{I.x * v.x, I.y * v.y, I.z * v.z}; }

// Coordinates of a parent-frame vector in the child frame rotated by q about axis a.
template <typename T>
__device__ __forceinline__ Vec3<T> rotT(int a, T s, T c, Vec3<T> v) {
  if (a == 2) return Vec3<T>{c * v.x + s * v.y, -s * v.x + c * v.y, v.z};
  if (a == 1) return Vec3<T>{c * v.x - s * v.z, v.y, s * v.x + c * v.z};
  return Vec3<T>{v.x, c * v.y + s * v.z, -s * v.y + c * v.z};
}
// Child-frame vector expressed in the parent frame.
template <typename T>
__device__ __forceinline__ Vec3<T> rot(int a, T s, T c, Vec3<T> v) {
  if (a == 2) return Vec3<T>{c * v.x - s * v.y, s * v.x + c * v.y, v.z};
  if (a == 1) return Vec3<T>{c * v.x + s * v.z, v.y, -s * v.x + c * v.z};
  return Vec3<T>{v.x, c * v.y - s * v.z, s * v.y + c * v.z};
}
// e_a x v
template <typename T>
__device__ __forceinline__ Vec3<T> ecross(int a, Vec3<T> v) {
  if (a == 2) return Vec3<T>{-v.y, v.x, T(0)};
  if (a == 1) return Vec3<T>{v.z, T(0), -v.x};
  return Vec3<T>{T(0), -v.z, v.y};
}
template <typename T = float>
__device__ __forceinline__ Vec3<T> unitv(int a) {
  return a == 0 ? Vec3<T>{T(1), T(0), T(0)} : (a == 1 ? Vec3<T>{T(0), T(1), T(0)} : Vec3<T>{T(0), T(0), T(1)});
}
template <typename T>
__device__ __forceinline__ T comp(int a, Vec3<T> v) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// ------------------------------------------------------ compensated sums (Dot2)
// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct) keep a
// running (hi, lo) pair, as in Ogita-Rump-Oishi's Dot2: the result is as
// accurate as a sum carried in twice the working precision.

struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_zero() { return DF{0.f, 0.f}; }
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ DF df_add(DF x, float y) {
  float s, e;
  two_sum(x.hi, y, s, e);
  return DF{s, __fadd_rn(x.lo, e)};
}
__device__ __forceinline__ DF df_fma(DF x, float a, float b) {
  float p = __fmul_rn(a, b);
  float pe = __fmaf_rn(a, b, -p);
  float s, e;
  two_sum(x.hi, p, s, e);
  return DF{s, __fadd_rn(x.lo, __fadd_rn(e, pe))};
}
__device__ __forceinline__ DF df_addd(DF x, DF y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  return DF{s, __fadd_rn(__fadd_rn(x.lo, y.lo), e)};
}
__device__ __forceinline__ float df_val(DF x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ DF df_norm(DF x) {
  float s, e;
  two_sum(x.hi, x.lo, s, e);
  return DF{s, e};
}
__device__ __forceinline__ DF warp_df_sum(DF x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF y;
    y.hi = __shfl_xor_sync(0xffffffffu, x.hi, o);
    y.lo = __shfl_xor_sync(0xffffffffu, x.lo, o);
    x = df_addd(x, y);
  }
  return x;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------ double-float scalar (dfl)
// A value carried as a normalised pair hi + lo of floats (|lo| <= ulp(hi)),
// with the arithmetic of Dekker and Knuth: TwoSum for sums, an FMA-based
// TwoProduct for products, each result renormalised by a fast two-sum.
// About 44-48 bits of significand from FP32 operations; on this part the
// FP32 pipe is some 64 times the FP64 rate, so the templated dynamics run
// much faster on dfl than on double at the accuracy the high-precision mode
// needs.  Products with a float are exact before the renormalisation.
struct dfl {
  float hi, lo;
  __device__ __forceinline__ dfl() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ dfl(float h) : hi(h), lo(0.f) {}
  __device__ __forceinline__ dfl(int h) : hi((float)h), lo(0.f) {}
  __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
};
// (s, e) with |e| small next to |s| as a normalised pair
__device__ __forceinline__ dfl dfl_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfl(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ dfl dfl_of(double d) {
  const float h = (float)d;
  return dfl(h, (float)(d - (double)h));
}
__device__ __forceinline__ double dfl_double(dfl a) { return (double)a.hi + (double)a.lo; }
// a + b of two floats, exactly
__device__ __forceinline__ dfl dfl_sum(float a, float b) {
  float s, e;
  two_sum(a, b, s, e);
  return dfl(s, e);
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dfl_fast(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfl_fast(p, e);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ dfl dfl_abs(dfl a) { return a.hi < 0.f ? -a : a; }
// (the double overload keeps unqualified calls on doubles resolving here)
__device__ __forceinline__ void sincos(double x, double* s, double* c) { ::sincos(x, s, c); }
// sin and cos to double-float accuracy: one FP64 sincos, split
__device__ __forceinline__ void sincos(dfl x, dfl* s, dfl* c) {
  double sd, cd;
  ::sincos(dfl_double(x), &sd, &cd);
  *s = dfl_of(sd);
  *c = dfl_of(cd);
}

// ------------------------------------------------------------------ dynamics

struct LinkRec {  // value-pass quantities of one link (link coordinates)
  float s, c;
  V3 wpT;   // parent angular velocity, in this frame
  V3 wdpT;  // parent angular acceleration, in this frame
  V3 w, wd; // this link's angular velocity / acceleration
  V3 a;     // linear acceleration of this frame's origin (gravity included)
  V3 f, n;  // total force / moment transmitted through this joint
  float pad;
};
static_assert(sizeof(LinkRec) == LVS * sizeof(float), "link record size");

template <typename T = float>
__device__ __forceinline__ Vec3<T> mcom(const DevModel& M, int i) {
  return Vec3<T>{T(M.com[3 * i]), T(M.com[3 * i + 1]), T(M.com[3 * i + 2])};
}
template <typename T = float>
__device__ __forceinline__ Vec3<T> minert(const DevModel& M, int i) {
  return Vec3<T>{T(M.Ic[3 * i]), T(M.Ic[3 * i + 1]), T(M.Ic[3 * i + 2])};
}

// Inverse dynamics tau = ID(q, qd, qdd) by RNEA.  sq/cq are sin/cos of q.
// `grav` is the magnitude of gravity along -z (0 turns it off).  fw is a force
// on the end-effector point (0, 0, L_last) of the last frame, in base
// coordinates: rotated into each frame on the way out like gravity, it is
// taken off the last link's force and moment on the way back, so the result is
// ID - J_p^T fw.  When rec is non-null (float only) the link quantities are
// stored for a tangent pass.
template <typename T>
__device__ __forceinline__ void rnea_value(const DevModel& M, const T* sq, const T* cq, const T* qd,
                                           const T* qdd, T grav, Vec3<T> fw, T* tau, LinkRec* rec) {
  using W = Vec3<T>;
  W F[QM], Nm[QM];
  W wp = vzero<T>(), wdp = vzero<T>(), ap = v3t<T>(T(0), T(0), grav);
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    const int a = M.axis[i];
    const T s = sq[i], c = cq[i];
    const W r = v3t<T>(T(0), T(0), i > 0 ? T(M.L[i - 1]) : T(0));
    const W ao = ap + cross(wdp, r) + cross(wp, cross(wp, r));
    const W wpT = rotT(a, s, c, wp);
    const W wdpT = rotT(a, s, c, wdp);
    const W e = unitv<T>(a);
    const W w = wpT + qd[i] * e;
    const W wd = wdpT + qd[i] * cross(wpT, e) + qdd[i] * e;
    const W acc = rotT(a, s, c, ao);
    const W cm = mcom<T>(M, i), Ii = minert<T>(M, i);
    const W ac = acc + cross(wd, cm) + cross(w, cross(w, cm));
    F[i] = T(M.m[i]) * ac;
    Nm[i] = mulI(Ii, wd) + cross(w, mulI(Ii, w));
    if constexpr (std::is_same<T, float>::value) {
      if (rec) {
        rec[i].s = s;
        rec[i].c = c;
        rec[i].wpT = wpT;
        rec[i].wdpT = wdpT;
        rec[i].w = w;
        rec[i].wd = wd;
        rec[i].a = acc;
      }
    }
    wp = w;
    wdp = wd;
    ap = acc;
  }
  // the force in the last frame's coordinates, taken off the last link
  if (fw.x != T(0) || fw.y != T(0) || fw.z != T(0)) {
#pragma unroll
    for (int i = 0; i < QM; ++i) fw = rotT(M.axis[i], sq[i], cq[i], fw);
    F[QM - 1] = F[QM - 1] - fw;
    Nm[QM - 1] = Nm[QM - 1] - cross(v3t<T>(T(0), T(0), T(M.L[QM - 1])), fw) + cross(mcom<T>(M, QM - 1), fw);
  }
  W fc = vzero<T>(), nc = vzero<T>();
#pragma unroll
  for (int i = QM - 1; i >= 0; --i) {
    W f = F[i];
    W n = Nm[i] + cross(mcom<T>(M, i), F[i]);
    if (i < QM - 1) {
      const int a1 = M.axis[i + 1];
      const W Rf = rot(a1, sq[i + 1], cq[i + 1], fc);
      const W Rn = rot(a1, sq[i + 1], cq[i + 1], nc);
      f = f + Rf;
      n = n + Rn + cross(v3t<T>(T(0), T(0), T(M.L[i])), Rf);
    }
    tau[i] = comp(M.axis[i], n);
    if constexpr (std::is_same<T, float>::value) {
      if (rec) {
        rec[i].f = f;
        rec[i].n = n;
      }
    }
    fc = f;
    nc = n;
  }
}

// Directional derivative of ID at the stored value pass, along q_j
// (wrt_qd = false) or qd_j (wrt_qd = true); qdd is held fixed.  fw is the
// value pass's end-effector force (base frame): its coordinates in frame i
// turn with q, so their tangent follows the same rotation rule as gravity's.
__device__ __forceinline__ void rnea_tangent(const DevModel& M, const LinkRec* R, const float* qd,
                                             bool wrt_qd, int j, V3 fw, float* dtau) {
  V3 Ft[QM], Nt[QM];
  V3 wpt = vzero(), wdpt = vzero(), apt = vzero();
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    const int a = M.axis[i];
    const float s = R[i].s, c = R[i].c;
    const float qt = (!wrt_qd && i == j) ? 1.f : 0.f;
    const float qdt = (wrt_qd && i == j) ? 1.f : 0.f;
    const V3 wp = i > 0 ? R[i - 1].w : vzero();
    const V3 r = v3(0.f, 0.f, i > 0 ? M.L[i - 1] : 0.f);
    const V3 aot = apt + cross(wdpt, r) + cross(wpt, cross(wp, r)) + cross(wp, cross(wpt, r));
    const V3 e = unitv(a);
    const V3 Rwt = rotT(a, s, c, wpt) - qt * ecross(a, R[i].wpT);
    const V3 wt = Rwt + qdt * e;
    const V3 Rwdt = rotT(a, s, c, wdpt) - qt * ecross(a, R[i].wdpT);
    const V3 wdt = Rwdt + qd[i] * cross(Rwt, e) + qdt * cross(R[i].wpT, e);
    const V3 at = rotT(a, s, c, aot) - qt * ecross(a, R[i].a);
    const V3 cm = mcom(M, i), Ii = minert(M, i);
    const V3 w = R[i].w;
    const V3 act = at + cross(wdt, cm) + cross(wt, cross(w, cm)) + cross(w, cross(wt, cm));
    Ft[i] = M.m[i] * act;
    Nt[i] = mulI(Ii, wdt) + cross(wt, mulI(Ii, w)) + cross(w, mulI(Ii, wt));
    wpt = wt;
    wdpt = wdt;
    apt = at;
  }
  // tangent of the force's last-frame coordinates (only q_j turns them)
  if (!wrt_qd && (fw.x != 0.f || fw.y != 0.f || fw.z != 0.f)) {
    V3 fet = vzero();
#pragma unroll
    for (int i = 0; i < QM; ++i) {
      const int a = M.axis[i];
      fw = rotT(a, R[i].s, R[i].c, fw);
      fet = rotT(a, R[i].s, R[i].c, fet) - (i == j ? 1.f : 0.f) * ecross(a, fw);
    }
    Ft[QM - 1] = Ft[QM - 1] - fet;
    Nt[QM - 1] = Nt[QM - 1] - cross(v3(0.f, 0.f, M.L[QM - 1]), fet) + cross(mcom(M, QM - 1), fet);
  }
  V3 fct = vzero(), nct = vzero();
#pragma unroll
  for (int i = QM - 1; i >= 0; --i) {
    V3 ft = Ft[i];
    V3 nt = Nt[i] + cross(mcom(M, i), Ft[i]);
    if (i < QM - 1) {
      const int a1 = M.axis[i + 1];
      const float s1 = R[i + 1].s, c1 = R[i + 1].c;
      const float q1t = (!wrt_qd && i + 1 == j) ? 1.f : 0.f;
      const V3 Rft = rot(a1, s1, c1, fct) + q1t * ecross(a1, rot(a1, s1, c1, R[i + 1].f));
      const V3 Rnt = rot(a1, s1, c1, nct) + q1t * ecross(a1, rot(a1, s1, c1, R[i + 1].n));
      ft = ft + Rft;
      nt = nt + Rnt + cross(v3(0.f, 0.f, M.L[i]), Rft);
    }
    dtau[i] = comp(M.axis[i], nt);
    fct = ft;
    nct = nt;
  }
}

// Lower-triangular mass matrix by composite rigid bodies, for the per-thread
// forward dynamics of the line search.  From the tip, the composite of links
// i..n (rotational inertia J about joint i's origin, first moment h about it,
// mass, all in link-i coordinates) is built from link i and the child
// composite rotated into link i and shifted by (0, 0, L_i).  Unit
// acceleration of joint i moves the composite rigidly: the moment about joint
// i's origin is n = J e_i and the force f = e_i x h; carried down to joint j
// (f rotated, n rotated plus (0, 0, L_j) x f) their e_j component is M_ij.
// About a fifth of the work of seven unit-acceleration RNEA columns, with a
// small live state.  Padded joints get a unit diagonal.
__device__ __forceinline__ void mass_matrix_crba(const DevModel& M, const float* sq, const float* cq,
                                                 float* Ml) {
  float J[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // composite, row-major
  V3 h = vzero();
  float mc = 0.f;
#pragma unroll
  for (int i = QM - 1; i >= 0; --i) {
    const V3 cm = mcom(M, i), Ii = minert(M, i);
    const float m = M.m[i];
    const float c2 = dot(cm, cm);
    float Jn[9] = {Ii.x + m * (c2 - cm.x * cm.x), -m * cm.x * cm.y, -m * cm.x * cm.z,
                   -m * cm.y * cm.x, Ii.y + m * (c2 - cm.y * cm.y), -m * cm.y * cm.z,
                   -m * cm.z * cm.x, -m * cm.z * cm.y, Ii.z + m * (c2 - cm.z * cm.z)};
    V3 hn = m * cm;
    if (i < QM - 1) {
      const int a1 = M.axis[i + 1];
      const float s1 = sq[i + 1], c1 = cq[i + 1];
      V3 col[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) col[c] = rot(a1, s1, c1, V3{J[c], J[3 + c], J[6 + c]});  // R J
#pragma unroll
      for (int r = 0; r < 3; ++r) {  // (R J) R^T
        const V3 row = r == 0 ? V3{col[0].x, col[1].x, col[2].x}
                              : (r == 1 ? V3{col[0].y, col[1].y, col[2].y} : V3{col[0].z, col[1].z, col[2].z});
        const V3 t = rot(a1, s1, c1, row);
        Jn[3 * r] += t.x;
        Jn[3 * r + 1] += t.y;
        Jn[3 * r + 2] += t.z;
      }
      const V3 hp = rot(a1, s1, c1, h);
      const float L = M.L[i];
      // shift to joint i's origin: m_c ([p]x^T [p]x) + 2 (p.h') I - h' p^T - p h'^T, p = (0, 0, L)
      const float ph = L * hp.z;
      Jn[0] += mc * L * L + 2.f * ph;
      Jn[4] += mc * L * L + 2.f * ph;
      Jn[8] += 2.f * ph - 2.f * hp.z * L;
      Jn[2] -= hp.x * L;
      Jn[5] -= hp.y * L;
      Jn[6] -= L * hp.x;
      Jn[7] -= L * hp.y;
      hn = hn + hp + v3(0.f, 0.f, mc * L);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) J[t] = Jn[t];
    h = hn;
    mc += m;
    const int ai = M.axis[i];
    const V3 e = unitv(ai);
    // J e_i, column picked by selects (a runtime index would move J to local memory)
    V3 n = ai == 0 ? V3{J[0], J[3], J[6]} : (ai == 1 ? V3{J[1], J[4], J[7]} : V3{J[2], J[5], J[8]});
    V3 f = cross(e, h);
    Ml[i * (i + 1) / 2 + i] = comp(ai, n);
#pragma unroll
    for (int j = i - 1; j >= 0; --j) {
      const int a = M.axis[j + 1];
      f = rot(a, sq[j + 1], cq[j + 1], f);
      n = rot(a, sq[j + 1], cq[j + 1], n) + cross(v3(0.f, 0.f, M.L[j]), f);
      Ml[i * (i + 1) / 2 + j] = comp(M.axis[j], n);
    }
  }
#pragma unroll
  for (int j = 0; j < QM; ++j)
    if (j >= M.dof) Ml[j * (j + 1) / 2 + j] = 1.f;
}

// In-place Cholesky of a packed lower-triangular 7x7; returns false if not PD.
__device__ __forceinline__ bool chol7(float* Ml) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < QM; ++j) {
    float s = Ml[j * (j + 1) / 2 + j];
#pragma unroll
    for (int l = 0; l < j; ++l) s -= Ml[j * (j + 1) / 2 + l] * Ml[j * (j + 1) / 2 + l];
    ok = ok && (s > 0.f);
    const float d = sqrtf(fmaxf(s, 1e-30f));
    const float inv = 1.f / d;
    Ml[j * (j + 1) / 2 + j] = d;
#pragma unroll
    for (int i = j + 1; i < QM; ++i) {
      float t = Ml[i * (i + 1) / 2 + j];
#pragma unroll
      for (int l = 0; l < j; ++l) t -= Ml[i * (i + 1) / 2 + l] * Ml[j * (j + 1) / 2 + l];
      Ml[i * (i + 1) / 2 + j] = t * inv;
    }
  }
  return ok;
}

// Solves (L L^T) x = b in place with the packed factor.
__device__ __forceinline__ void chol7_solve(const float* Lf, float* b) {
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    float t = b[i];
#pragma unroll
    for (int l = 0; l < i; ++l) t -= Lf[i * (i + 1) / 2 + l] * b[l];
    b[i] = t / Lf[i * (i + 1) / 2 + i];
  }
#pragma unroll
  for (int i = QM - 1; i >= 0; --i) {
    float t = b[i];
#pragma unroll
    for (int l = i + 1; l < QM; ++l) t -= Lf[l * (l + 1) / 2 + i] * b[l];
    b[i] = t / Lf[i * (i + 1) / 2 + i];
  }
}

// Forward dynamics M(q) qdd = u + J_p^T fw - ID(q, qd, 0) of one knot
// (fw: end-effector force, base frame).
__device__ __forceinline__ bool forward_dynamics(const DevModel& M, const float* q, const float* qd,
                                                 const float* u, V3 fw, float* qdd) {
  float sq[QM], cq[QM], Ml[QM * (QM + 1) / 2], z[QM], b[QM];
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    sincosf(q[i], &sq[i], &cq[i]);
    z[i] = 0.f;
  }
  mass_matrix_crba(M, sq, cq, Ml);
  rnea_value(M, sq, cq, qd, z, M.g, fw, b, nullptr);
#pragma unroll
  for (int i = 0; i < QM; ++i) qdd[i] = u[i] - b[i];
  const bool ok = chol7(Ml);
  chol7_solve(Ml, qdd);
  return ok;
}

// End-effector position and (float only, J non-null) its 3x7 Jacobian
// (row-major) in base coordinates.
// fk_ee_sc takes sin and cos of q (sq, cq); fk_ee forms them.
template <typename T>
__device__ __forceinline__ void fk_ee_sc(const DevModel& M, const T* sq, const T* cq, T* p, float* J) {
  T R[9] = {T(1), T(0), T(0), T(0), T(1), T(0), T(0), T(0), T(1)};  // row-major, columns are the frame axes
  Vec3<T> pos = vzero<T>();
  Vec3<T> pj[QM], ej[QM];
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    if (i > 0) pos = pos + T(M.L[i - 1]) * v3t<T>(R[2], R[5], R[8]);
    const T s = sq[i], c = cq[i];
    const int a = M.axis[i];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T c0 = R[3 * r], c1 = R[3 * r + 1], c2 = R[3 * r + 2];
      if (a == 2) {
        R[3 * r] = c * c0 + s * c1;
        R[3 * r + 1] = -s * c0 + c * c1;
      } else if (a == 1) {
        R[3 * r] = c * c0 - s * c2;
        R[3 * r + 2] = s * c0 + c * c2;
      } else {
        R[3 * r + 1] = c * c1 + s * c2;
        R[3 * r + 2] = -s * c1 + c * c2;
      }
    }
    pj[i] = pos;
    ej[i] = v3t<T>(R[a], R[3 + a], R[6 + a]);
  }
  const Vec3<T> pe = pos + T(M.L[QM - 1]) * v3t<T>(R[2], R[5], R[8]);
  p[0] = pe.x;
  p[1] = pe.y;
  p[2] = pe.z;
  if constexpr (std::is_same<T, float>::value) {
    if (J) {
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        const Vec3<T> col = cross(ej[i], pe - pj[i]);
        J[i] = col.x;
        J[QM + i] = col.y;
        J[2 * QM + i] = col.z;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void fk_ee(const DevModel& M, const T* q, T* p, float* J) {
  T sq[QM], cq[QM];
#pragma unroll
  for (int i = 0; i < QM; ++i) {
    if constexpr (std::is_same<T, float>::value)
      sincosf(q[i], &sq[i], &cq[i]);
    else
      sincos(q[i], &sq[i], &cq[i]);
  }
  fk_ee_sc<T>(M, sq, cq, p, J);
}

}  // namespace gato
