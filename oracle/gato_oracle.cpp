/*
 * FP64 CPU oracle for the batched SQP method of "GATO: GPU-Accelerated and
 * Batched Trajectory Optimization" (arXiv 2510.07625).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA path and the product never calls it.
 *
 * It is plain and slow on purpose: dense 6x6 spatial algebra, dense small
 * matrices, dual numbers for derivatives, one scalar loop per formula.
 *
 *   dynamics   RNEA in spatial-vector form (Featherstone); M(q) column j is
 *              ID(q, 0, e_j) without gravity; qdd = M^-1 (tau - ID(q, qd, 0));
 *              semi-implicit Euler (Sec. II-A leaves the integrator open).
 *   gradients  A_k, B_k by forward-mode dual numbers through the whole step.
 *   QP         Eq. 1 (Sec. II-A Step 1), second-order cost, first-order dynamics.
 *   KKT        Eq. 2 with the sign convention of Eq. 1:
 *              [G C^T; C 0][dZ; nu] = [-g; c]   (Eq. 2's sign of c is garbled).
 *   Schur      Eq. 4-5: S = C G^-1 C^T (the SPD sign; the printed minus signs
 *              on S and Phi^-1 cancel), blocks
 *              Q_0^-1, theta_k, phi_k; rhs = -c - C G^-1 g built from zeta_k.
 *   precond    Eq. 6 stair preconditioner assembled block by block from
 *              theta_k^-1 and phi_k; or block-Jacobi (diagonal only).
 *   PCG        Sec. II-B / III-B, standard preconditioned CG warm-started from
 *              the previous multiplier; stops when the preconditioned residual
 *              relative to the warm start's, sqrt(eta/eta_0), is <= eps,
 *              so the correction to the multiplier is accurate relative to its
 *              own size; no iterations when eta_0 < 1e-30.  Optionally (the
 *              direct alternative Sec. II-B sets against iterative methods) the
 *              same system S nu = rhs by block elimination (ora_blocktri_solve).
 *   recovery   dZ = -G^-1 (g + C^T nu)  (Eq. 4, with Eq. 1's sign of c).
 *   merit      Eq. 3: J + mu * ||c||_1 (mu = 10 by default).
 *   line srch  Eq. 7: alpha_i = beta^-i, i = 0..A-1, argmin with ties to the
 *              smallest i; rejected when no alpha lowers the merit (the paper leaves
 *              that case open: the iterate is kept).
 *   KKT resid  max(||c||_inf, ||g + C^T nu||_inf / max(1, ||g||_inf)) (the paper names no
 *              formula).
 *
 * Pinned by the tests against things other than itself: the dynamics (a
 * symbolic Lagrangian, central differences, energy, power balance, a tip
 * point mass for the end-effector force), the KKT system and Schur blocks
 * (dense LU), the preconditioner identity, PCG and block elimination (dense
 * solves), one SQP step of a linear-quadratic special case (Riccati), the
 * merit's closed form, and single SQP iterations on the nonlinear arms (joint
 * and end-effector costs, full and shortened steps) rebuilt from those pinned
 * parts: dense KKT solve, merit and KKT residual restated from their
 * definitions, the first argmin over the step lengths.  The loop repeats that
 * iteration; across iterations only invariants check it (accepted steps lower
 * the merit, full steps near the solution, zero defects at convergence).
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

extern "C" {

typedef struct {
  int32_t dof;
  int32_t axis[7];        /* 0 = x, 1 = y, 2 = z */
  double link_len[7];
  double mass[7];
  double com[21];
  double inertia[21];     /* principal moments about the centre of mass */
  double gravity;         /* along -z */
} ora_model;

typedef struct {
  int32_t N;
  int32_t cost_kind;      /* 0 = joint targets, 1 = end-effector track */
  double dt;
  const double* x_s;      /* [nx] */
  const double* x_ref;    /* [(N+1)*nx] or NULL */
  const double* ee_ref;   /* [(N+1)*3] or NULL */
  double w[6];            /* wq, wqd, wr, terminal scale, wee, rho */
  double f_ext[3];        /* constant external force on the end effector, base
                             frame (Sec. IV-D's disturbance hypotheses); zeros = none */
} ora_problem;

typedef struct {
  double mu;
  double beta;
  int32_t n_alpha;
  double pcg_eps;
  int32_t pcg_max;
  int32_t precond;        /* 0 = stair (Eq. 6), 1 = block Jacobi */
  double kkt_tol;         /* <= 0: run the fixed iteration count */
  int32_t max_iter;
  int32_t linsolve;       /* 0 = PCG (Sec. II-B), 1 = direct block elimination */
  int32_t rho_adapt;      /* 1: rho /= 3 after an accepted step, *= 2 after a rejected
                             one, within [1e-8, 1e1], the range Sec. IV-C samples
                             rho over (Fig. 4); no factors are given there */
} ora_params;

typedef struct {
  int32_t iters;          /* SQP iterations that took a step (or tried to) */
  int32_t flags;          /* 1 converged, 2 max-iter, 4 line-search fail, 8 PCG max-iter, 16 non-finite */
  int32_t pcg_total;
  double kkt;
  double merit;
} ora_result;

}  // extern "C"

namespace {

/* ----------------------------------------------------------------- scalars */

/* FLOP-counting scalar: a double whose arithmetic adds to a per-thread
   counter, 1 per +, -, *, / and 1 per sin, cos or sqrt (a multiply-add counts
   2).  Running the templated code below on it counts the operations of the
   formulas as written (ora_count_flops). */
thread_local long long g_flops = 0;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_flops; return Cnt(a.v / b.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt sin(Cnt a) { ++g_flops; return Cnt(std::sin(a.v)); }
inline Cnt cos(Cnt a) { ++g_flops; return Cnt(std::cos(a.v)); }
inline Cnt sqrt(Cnt a) { ++g_flops; return Cnt(std::sqrt(a.v)); }

/* Forward-mode dual numbers over a scalar S (double for the oracle's
   derivatives, Cnt for counting them). */
template <class S> struct DualT {
  S v, d;
  DualT() : v(0.0), d(0.0) {}
  DualT(double x) : v(x), d(0.0) {}
  DualT(S x, S dx) : v(x), d(dx) {}
};
template <class S> inline DualT<S> operator+(DualT<S> a, DualT<S> b) { return DualT<S>(a.v + b.v, a.d + b.d); }
template <class S> inline DualT<S> operator-(DualT<S> a, DualT<S> b) { return DualT<S>(a.v - b.v, a.d - b.d); }
template <class S> inline DualT<S> operator-(DualT<S> a) { return DualT<S>(-a.v, -a.d); }
template <class S> inline DualT<S> operator*(DualT<S> a, DualT<S> b) {
  return DualT<S>(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <class S> inline DualT<S> operator/(DualT<S> a, DualT<S> b) {
  return DualT<S>(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
template <class S> inline DualT<S>& operator+=(DualT<S>& a, DualT<S> b) { a = a + b; return a; }
template <class S> inline DualT<S>& operator-=(DualT<S>& a, DualT<S> b) { a = a - b; return a; }
template <class S> inline DualT<S> sin(DualT<S> a) {
  using std::sin; using std::cos;
  return DualT<S>(sin(a.v), cos(a.v) * a.d);
}
template <class S> inline DualT<S> cos(DualT<S> a) {
  using std::sin; using std::cos;
  return DualT<S>(cos(a.v), -sin(a.v) * a.d);
}
template <class S> inline DualT<S> sqrt(DualT<S> a) {
  using std::sqrt;
  S r = sqrt(a.v);
  return DualT<S>(r, a.d / (S(2.0) * r));
}
typedef DualT<double> Dual;
inline double val(double a) { return a; }
inline double val(Cnt a) { return a.v; }
template <class S> inline double val(DualT<S> a) { return val(a.v); }

/* --------------------------------------------------- spatial algebra (6D) */
/* Motion vectors are [angular; linear], forces [moment; force]. */

template <class T> struct V3 { T a[3]; };
template <class T> struct V6 { T a[6]; };
template <class T> struct M3 { T a[3][3]; };
template <class T> struct M6 { T a[6][6]; };

template <class T> M3<T> rot_coord(int axis, T q) {
  /* Coordinate transform E from parent to child for a rotation q about the
     joint axis (child axes = parent axes rotated by q). */
  using std::cos; using std::sin;
  T c = cos(q), s = sin(q);
  M3<T> E;
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) E.a[i][j] = T(i == j ? 1.0 : 0.0);
  int i1 = (axis + 1) % 3, i2 = (axis + 2) % 3;
  E.a[i1][i1] = c;  E.a[i1][i2] = s;
  E.a[i2][i1] = -s; E.a[i2][i2] = c;
  return E;
}

template <class T> M3<T> skew(const V3<T>& r) {
  M3<T> S;
  S.a[0][0] = T(0.0);  S.a[0][1] = -r.a[2]; S.a[0][2] = r.a[1];
  S.a[1][0] = r.a[2];  S.a[1][1] = T(0.0);  S.a[1][2] = -r.a[0];
  S.a[2][0] = -r.a[1]; S.a[2][1] = r.a[0];  S.a[2][2] = T(0.0);
  return S;
}

template <class T> M6<T> plucker(const M3<T>& E, const V3<T>& r) {
  /* X = [E 0; -E skew(r) E]: motion transform to a frame rotated by E whose
     origin sits at r (parent coordinates). */
  M6<T> X;
  M3<T> rx = skew(r);
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) X.a[i][j] = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      X.a[i][j] = E.a[i][j];
      X.a[i + 3][j + 3] = E.a[i][j];
      T s = T(0.0);
      for (int l = 0; l < 3; ++l) s = s + E.a[i][l] * rx.a[l][j];
      X.a[i + 3][j] = -s;
    }
  return X;
}

template <class T> V6<T> mul(const M6<T>& X, const V6<T>& v) {
  V6<T> o;
  for (int i = 0; i < 6; ++i) {
    T s = T(0.0);
    for (int j = 0; j < 6; ++j) s = s + X.a[i][j] * v.a[j];
    o.a[i] = s;
  }
  return o;
}

template <class T> V6<T> mul_t(const M6<T>& X, const V6<T>& f) {
  /* X^T f: force transform from child back to parent. */
  V6<T> o;
  for (int i = 0; i < 6; ++i) {
    T s = T(0.0);
    for (int j = 0; j < 6; ++j) s = s + X.a[j][i] * f.a[j];
    o.a[i] = s;
  }
  return o;
}

template <class T> V3<T> cross3(const T* a, const T* b) {
  V3<T> o;
  o.a[0] = a[1] * b[2] - a[2] * b[1];
  o.a[1] = a[2] * b[0] - a[0] * b[2];
  o.a[2] = a[0] * b[1] - a[1] * b[0];
  return o;
}

template <class T> V6<T> crm(const V6<T>& v, const V6<T>& m) {
  /* v x m for motion vectors. */
  V3<T> a = cross3(v.a, m.a);
  V3<T> b = cross3(v.a, m.a + 3);
  V3<T> c = cross3(v.a + 3, m.a);
  V6<T> o;
  for (int i = 0; i < 3; ++i) { o.a[i] = a.a[i]; o.a[i + 3] = b.a[i] + c.a[i]; }
  return o;
}

template <class T> V6<T> crf(const V6<T>& v, const V6<T>& f) {
  /* v x* f for force vectors. */
  V3<T> a = cross3(v.a, f.a);
  V3<T> b = cross3(v.a + 3, f.a + 3);
  V3<T> c = cross3(v.a, f.a + 3);
  V6<T> o;
  for (int i = 0; i < 3; ++i) { o.a[i] = a.a[i] + b.a[i]; o.a[i + 3] = c.a[i]; }
  return o;
}

M6<double> spatial_inertia(const ora_model& m, int i) {
  /* Inertia of link i about its frame origin: [Ic + m cx cx^T, m cx; m cx^T, m 1]. */
  M6<double> I;
  for (int a = 0; a < 6; ++a) for (int b = 0; b < 6; ++b) I.a[a][b] = 0.0;
  V3<double> c;
  for (int a = 0; a < 3; ++a) c.a[a] = m.com[3 * i + a];
  M3<double> cx = skew(c);
  double mass = m.mass[i];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int l = 0; l < 3; ++l) s += cx.a[a][l] * cx.a[b][l];
      I.a[a][b] = mass * s + (a == b ? m.inertia[3 * i + a] : 0.0);
      I.a[a][b + 3] = mass * cx.a[a][b];
      I.a[a + 3][b] = mass * cx.a[b][a];
    }
    I.a[a + 3][a + 3] = mass;
  }
  return I;
}

/* ------------------------------------------------------------- dynamics */

template <class T>
void rnea(const ora_model& m, const T* q, const T* qd, const T* qdd, bool gravity, T* tau) {
  int n = m.dof;
  std::vector<M6<T>> X(n);
  std::vector<V6<T>> v(n), a(n), f(n);
  for (int i = 0; i < n; ++i) {
    V3<T> r;
    r.a[0] = T(0.0); r.a[1] = T(0.0); r.a[2] = T(i == 0 ? 0.0 : m.link_len[i - 1]);
    X[i] = plucker(rot_coord(m.axis[i], q[i]), r);
    V6<T> S;
    for (int l = 0; l < 6; ++l) S.a[l] = T(0.0);
    S.a[m.axis[i]] = T(1.0);
    V6<T> vp, ap;
    if (i == 0) {
      for (int l = 0; l < 6; ++l) { vp.a[l] = T(0.0); ap.a[l] = T(0.0); }
      if (gravity) ap.a[5] = T(m.gravity);  /* base accelerates upward: -a_gravity */
    } else {
      vp = v[i - 1];
      ap = a[i - 1];
    }
    V6<T> xv = mul(X[i], vp), xa = mul(X[i], ap);
    V6<T> vj, aj;
    for (int l = 0; l < 6; ++l) { vj.a[l] = S.a[l] * qd[i]; aj.a[l] = S.a[l] * qdd[i]; }
    for (int l = 0; l < 6; ++l) v[i].a[l] = xv.a[l] + vj.a[l];
    V6<T> cor = crm(v[i], vj);
    for (int l = 0; l < 6; ++l) a[i].a[l] = xa.a[l] + aj.a[l] + cor.a[l];
    M6<double> Id = spatial_inertia(m, i);
    M6<T> I;
    for (int r1 = 0; r1 < 6; ++r1) for (int c1 = 0; c1 < 6; ++c1) I.a[r1][c1] = T(Id.a[r1][c1]);
    V6<T> Ia = mul(I, a[i]), Iv = mul(I, v[i]);
    V6<T> g = crf(v[i], Iv);
    for (int l = 0; l < 6; ++l) f[i].a[l] = Ia.a[l] + g.a[l];
  }
  for (int i = n - 1; i >= 0; --i) {
    tau[i] = f[i].a[m.axis[i]];
    if (i > 0) {
      V6<T> fp = mul_t(X[i], f[i]);
      for (int l = 0; l < 6; ++l) f[i - 1].a[l] = f[i - 1].a[l] + fp.a[l];
    }
  }
}

template <class T>
void mass_matrix(const ora_model& m, const T* q, T* M) {
  /* Column j of M is ID(q, 0, e_j) with gravity off. */
  int n = m.dof;
  std::vector<T> z(n, T(0.0)), e(n), col(n);
  for (int j = 0; j < n; ++j) {
    for (int l = 0; l < n; ++l) e[l] = T(l == j ? 1.0 : 0.0);
    rnea(m, q, z.data(), e.data(), false, col.data());
    for (int i = 0; i < n; ++i) M[i * n + j] = col[i];
  }
}

template <class T>
bool cholesky_solve(int n, std::vector<T> A, T* b) {
  /* Solves A x = b in place for symmetric positive definite A. */
  using std::sqrt;
  for (int j = 0; j < n; ++j) {
    T s = A[j * n + j];
    for (int l = 0; l < j; ++l) s = s - A[j * n + l] * A[j * n + l];
    if (!(val(s) > 0.0)) return false;
    T d = sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      T t = A[i * n + j];
      for (int l = 0; l < j; ++l) t = t - A[i * n + l] * A[j * n + l];
      A[i * n + j] = t / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    T t = b[i];
    for (int l = 0; l < i; ++l) t = t - A[i * n + l] * b[l];
    b[i] = t / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    T t = b[i];
    for (int l = i + 1; l < n; ++l) t = t - A[l * n + i] * b[l];
    b[i] = t / A[i * n + i];
  }
  return true;
}

template <class T>
void ee_joint_torque(const ora_model& m, const T* q, const double* f, T* tau) {
  /* Joint torques of a force f (base frame) acting at the end-effector point:
   * tau = J_p(q)^T f with the geometric Jacobian of a revolute chain, column
   * i = z_i x (p_ee - o_i), z_i and o_i joint i's axis and origin in the base
   * frame (the frames chained as in fk_ee). */
  int n = m.dof;
  T R[3][3], pos[3];
  std::vector<V3<T>> z(n), o(n);
  for (int i = 0; i < 3; ++i) { pos[i] = T(0.0); for (int j = 0; j < 3; ++j) R[i][j] = T(i == j ? 1.0 : 0.0); }
  for (int i = 0; i <= n; ++i) {
    double L = (i == 0) ? 0.0 : m.link_len[i - 1];
    for (int r = 0; r < 3; ++r) pos[r] = pos[r] + R[r][2] * T(L);
    if (i == n) break;
    M3<T> E = rot_coord(m.axis[i], q[i]);
    T Rn[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        T s = T(0.0);
        for (int l = 0; l < 3; ++l) s = s + R[r][l] * E.a[c][l];
        Rn[r][c] = s;
      }
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) R[r][c] = Rn[r][c];
    /* joint i turns about its own frame's axis, which the rotation leaves fixed */
    for (int r = 0; r < 3; ++r) { z[i].a[r] = R[r][m.axis[i]]; o[i].a[r] = pos[r]; }
  }
  for (int i = 0; i < n; ++i) {
    T d[3] = {pos[0] - o[i].a[0], pos[1] - o[i].a[1], pos[2] - o[i].a[2]};
    V3<T> col = cross3(z[i].a, d);
    tau[i] = col.a[0] * T(f[0]) + col.a[1] * T(f[1]) + col.a[2] * T(f[2]);
  }
}

template <class T>
bool forward_dynamics(const ora_model& m, const T* q, const T* qd, const T* tau, T* qdd,
                      const double* f_ext = nullptr) {
  /* M(q) qdd = tau + J_p(q)^T f_ext - ID(q, qd, 0). */
  int n = m.dof;
  std::vector<T> M(n * n), z(n, T(0.0)), bias(n), te(n, T(0.0));
  mass_matrix(m, q, M.data());
  rnea(m, q, qd, z.data(), true, bias.data());
  if (f_ext && (f_ext[0] != 0.0 || f_ext[1] != 0.0 || f_ext[2] != 0.0))
    ee_joint_torque(m, q, f_ext, te.data());
  for (int i = 0; i < n; ++i) qdd[i] = tau[i] + te[i] - bias[i];
  return cholesky_solve(n, M, qdd);
}

template <class T>
bool step(const ora_model& m, const T* x, const T* u, double h, T* xn,
          const double* f_ext = nullptr) {
  /* Semi-implicit Euler: qd+ = qd + h qdd, q+ = q + h qd+. */
  int n = m.dof;
  std::vector<T> qdd(n);
  bool ok = forward_dynamics(m, x, x + n, u, qdd.data(), f_ext);
  for (int i = 0; i < n; ++i) {
    T qdn = x[n + i] + T(h) * qdd[i];
    xn[n + i] = qdn;
    xn[i] = x[i] + T(h) * qdn;
  }
  return ok;
}

void step_jacobians(const ora_model& m, const double* x, const double* u, double h,
                    double* A, double* B, const double* f_ext = nullptr) {
  /* A = d step / d x (nx x nx), B = d step / d u (nx x nu), one dual pass per column. */
  int n = m.dof, nx = 2 * n;
  std::vector<Dual> xd(nx), ud(n), out(nx);
  for (int j = 0; j < nx + n; ++j) {
    for (int l = 0; l < nx; ++l) xd[l] = Dual(x[l], (j == l) ? 1.0 : 0.0);
    for (int l = 0; l < n; ++l) ud[l] = Dual(u[l], (j == nx + l) ? 1.0 : 0.0);
    step(m, xd.data(), ud.data(), h, out.data(), f_ext);
    for (int i = 0; i < nx; ++i) {
      if (j < nx) A[i * nx + j] = out[i].d;
      else B[i * n + (j - nx)] = out[i].d;
    }
  }
}

template <class T>
void fk_ee(const ora_model& m, const T* q, T* p) {
  /* End-effector position in base coordinates by chaining rotations. */
  int n = m.dof;
  T R[3][3], pos[3];
  for (int i = 0; i < 3; ++i) { pos[i] = T(0.0); for (int j = 0; j < 3; ++j) R[i][j] = T(i == j ? 1.0 : 0.0); }
  for (int i = 0; i <= n; ++i) {
    double L = (i == 0) ? 0.0 : m.link_len[i - 1];
    for (int r = 0; r < 3; ++r) pos[r] = pos[r] + R[r][2] * T(L);
    if (i == n) break;
    /* child rotation in parent = E^T */
    M3<T> E = rot_coord(m.axis[i], q[i]);
    T Rn[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        T s = T(0.0);
        for (int l = 0; l < 3; ++l) s = s + R[r][l] * E.a[c][l];
        Rn[r][c] = s;
      }
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) R[r][c] = Rn[r][c];
  }
  for (int r = 0; r < 3; ++r) p[r] = pos[r];
}

void fk_jacobian(const ora_model& m, const double* q, double* p, double* J) {
  int n = m.dof;
  std::vector<Dual> qd(n);
  Dual pd[3];
  for (int j = 0; j < n; ++j) {
    for (int l = 0; l < n; ++l) qd[l] = Dual(q[l], l == j ? 1.0 : 0.0);
    fk_ee(m, qd.data(), pd);
    for (int r = 0; r < 3; ++r) { J[r * n + j] = pd[r].d; p[r] = pd[r].v; }
  }
}

/* ------------------------------------------------------ small dense algebra */

typedef std::vector<double> Vec;

template <class T>
void matmul(int n, int k, int mm, const T* A, const T* B, T* C) {
  /* C (n x mm) = A (n x k) B (k x mm) */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < mm; ++j) {
      T s = T(0.0);
      for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * mm + j];
      C[i * mm + j] = s;
    }
}

bool spd_inverse(int n, const double* A, double* Ainv) {
  /* Inverse of an SPD matrix: solve A x = e_j column by column. */
  std::vector<double> Af(A, A + n * n), col(n);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) col[i] = (i == j) ? 1.0 : 0.0;
    if (!cholesky_solve(n, Af, col.data())) return false;
    for (int i = 0; i < n; ++i) Ainv[i * n + j] = col[i];
  }
  return true;
}

/* ---------------------------------------------------- problem linearisation */

struct Lin {
  int N, nx, nu;
  Vec A, B;      /* [N][nx][nx], [N][nx][nu] */
  Vec Q, R;      /* [N+1][nx][nx], [N][nu][nu] */
  Vec q, r;      /* [N+1][nx], [N][nu] */
  Vec c;         /* [N+1][nx]: x_s - x_0, e_0 .. e_{N-1} */
  double J;
  bool ok;
};

double knot_cost(const ora_model& m, const ora_problem& p, int k, const double* x,
                 const double* u, double* qg, double* Qh, double* rg, double* Rh) {
  /* Cost of knot k and its gradient / (Gauss-Newton) Hessian; u == NULL at k = N. */
  int n = m.dof, nx = 2 * n, N = p.N;
  double wq = p.w[0], wqd = p.w[1], wr = p.w[2], ts = p.w[3], wee = p.w[4], rho = p.w[5];
  double s = (k == N) ? ts : 1.0;
  double J = 0.0;
  if (qg) for (int i = 0; i < nx; ++i) qg[i] = 0.0;
  if (Qh) for (int i = 0; i < nx * nx; ++i) Qh[i] = 0.0;
  if (p.cost_kind == 0) {
    const double* xr = p.x_ref + (size_t)k * nx;
    for (int i = 0; i < nx; ++i) {
      double wi = (i < n) ? wq : wqd;
      double d = x[i] - xr[i];
      J += 0.5 * s * wi * d * d;
      if (qg) qg[i] = s * wi * d;
      if (Qh) Qh[i * nx + i] = s * wi;
    }
  } else {
    double pe[3], Jp[21];
    fk_jacobian(m, x, pe, Jp);
    const double* pr = p.ee_ref + (size_t)k * 3;
    double d[3];
    for (int r = 0; r < 3; ++r) { d[r] = pe[r] - pr[r]; J += 0.5 * s * wee * d[r] * d[r]; }
    for (int i = 0; i < n; ++i) {
      double t = 0.0;
      for (int r = 0; r < 3; ++r) t += Jp[r * n + i] * d[r];
      if (qg) qg[i] = s * wee * t;
      for (int j = 0; j < n; ++j) {
        double h = 0.0;
        for (int r = 0; r < 3; ++r) h += Jp[r * n + i] * Jp[r * n + j];
        if (Qh) Qh[i * nx + j] = s * wee * h;
      }
    }
    for (int i = 0; i < n; ++i) {
      double v = x[n + i];
      J += 0.5 * s * wqd * v * v;
      if (qg) qg[n + i] = s * wqd * v;
      if (Qh) Qh[(n + i) * nx + (n + i)] = s * wqd;
    }
  }
  if (Qh) for (int i = 0; i < nx; ++i) Qh[i * nx + i] += rho;  /* damping rho on diag(Q_k), Sec. IV-C */
  if (u) {
    for (int i = 0; i < n; ++i) {
      J += 0.5 * wr * u[i] * u[i];
      if (rg) rg[i] = wr * u[i];
      if (Rh) for (int j = 0; j < n; ++j) Rh[i * n + j] = (i == j) ? wr : 0.0;
    }
  }
  return J;
}

Lin linearize(const ora_model& m, const ora_problem& p, const double* X, const double* U) {
  Lin L;
  int n = m.dof, nx = 2 * n, N = p.N;
  L.N = N; L.nx = nx; L.nu = n; L.ok = true;
  L.A.assign((size_t)N * nx * nx, 0.0);
  L.B.assign((size_t)N * nx * n, 0.0);
  L.Q.assign((size_t)(N + 1) * nx * nx, 0.0);
  L.R.assign((size_t)N * n * n, 0.0);
  L.q.assign((size_t)(N + 1) * nx, 0.0);
  L.r.assign((size_t)N * n, 0.0);
  L.c.assign((size_t)(N + 1) * nx, 0.0);
  L.J = 0.0;
  for (int i = 0; i < nx; ++i) L.c[i] = p.x_s[i] - X[i];
  std::vector<double> xn(nx);
  for (int k = 0; k < N; ++k) {
    const double* x = X + (size_t)k * nx;
    const double* u = U + (size_t)k * n;
    if (!step(m, x, u, p.dt, xn.data(), p.f_ext)) L.ok = false;
    for (int i = 0; i < nx; ++i) L.c[(size_t)(k + 1) * nx + i] = xn[i] - X[(size_t)(k + 1) * nx + i];
    step_jacobians(m, x, u, p.dt, &L.A[(size_t)k * nx * nx], &L.B[(size_t)k * nx * n], p.f_ext);
    L.J += knot_cost(m, p, k, x, u, &L.q[(size_t)k * nx], &L.Q[(size_t)k * nx * nx],
                     &L.r[(size_t)k * n], &L.R[(size_t)k * n * n]);
  }
  L.J += knot_cost(m, p, N, X + (size_t)N * nx, nullptr, &L.q[(size_t)N * nx],
                   &L.Q[(size_t)N * nx * nx], nullptr, nullptr);
  return L;
}

double merit(const ora_model& m, const ora_problem& p, const double* X, const double* U,
             double mu, bool* ok) {
  /* Eq. 3: M = J + mu * ||c||_1. */
  int n = m.dof, nx = 2 * n, N = p.N;
  double J = 0.0, c1 = 0.0;
  for (int i = 0; i < nx; ++i) c1 += std::fabs(p.x_s[i] - X[i]);
  std::vector<double> xn(nx);
  bool good = true;
  for (int k = 0; k < N; ++k) {
    const double* x = X + (size_t)k * nx;
    const double* u = U + (size_t)k * n;
    if (!step(m, x, u, p.dt, xn.data(), p.f_ext)) good = false;
    for (int i = 0; i < nx; ++i) c1 += std::fabs(xn[i] - X[(size_t)(k + 1) * nx + i]);
    J += knot_cost(m, p, k, x, u, nullptr, nullptr, nullptr, nullptr);
  }
  J += knot_cost(m, p, N, X + (size_t)N * nx, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (ok) *ok = good;
  return J + mu * c1;
}

/* ----------------------------------------------------- Schur complement */

struct Schur {
  int N, nx;
  Vec Sd, Ss;    /* diagonal blocks [N+1][nx][nx]; sub-diagonal S_{k+1,k} = phi_k [N][nx][nx] */
  Vec Pd, Ps;    /* preconditioner, same layout */
  Vec rhs;       /* [N+1][nx] */
  Vec Qinv, Rinv;
  bool ok;
};

Schur form_schur(const Lin& L, int precond) {
  /* Eq. 5-6 blocks with the SPD sign S = C G^-1 C^T. */
  Schur S;
  int N = L.N, nx = L.nx, nu = L.nu;
  S.N = N; S.nx = nx; S.ok = true;
  size_t bb = (size_t)nx * nx;
  S.Sd.assign((N + 1) * bb, 0.0);
  S.Ss.assign(N * bb, 0.0);
  S.Pd.assign((N + 1) * bb, 0.0);
  S.Ps.assign(N * bb, 0.0);
  S.rhs.assign((size_t)(N + 1) * nx, 0.0);
  S.Qinv.assign((N + 1) * bb, 0.0);
  S.Rinv.assign((size_t)N * nu * nu, 0.0);
  for (int k = 0; k <= N; ++k)
    if (!spd_inverse(nx, &L.Q[k * bb], &S.Qinv[k * bb])) S.ok = false;
  for (int k = 0; k < N; ++k)
    if (!spd_inverse(nu, &L.R[(size_t)k * nu * nu], &S.Rinv[(size_t)k * nu * nu])) S.ok = false;

  /* block 0: Q_0^-1 and -c_0 - Q_0^-1 q_0 */
  for (size_t i = 0; i < bb; ++i) S.Sd[i] = S.Qinv[i];
  for (int i = 0; i < nx; ++i) {
    double t = 0.0;
    for (int j = 0; j < nx; ++j) t += S.Qinv[i * nx + j] * L.q[j];
    S.rhs[i] = -L.c[i] - t;
  }
  Vec AQi(bb), BRi((size_t)nx * nu), T1(bb), T2(bb), At(bb), Bt((size_t)nu * nx);
  for (int k = 0; k < N; ++k) {
    const double* A = &L.A[k * bb];
    const double* B = &L.B[(size_t)k * nx * nu];
    const double* Qi = &S.Qinv[k * bb];
    const double* Qi1 = &S.Qinv[(k + 1) * bb];
    const double* Ri = &S.Rinv[(size_t)k * nu * nu];
    for (int i = 0; i < nx; ++i) for (int j = 0; j < nx; ++j) At[j * nx + i] = A[i * nx + j];
    for (int i = 0; i < nx; ++i) for (int j = 0; j < nu; ++j) Bt[j * nx + i] = B[i * nu + j];
    matmul(nx, nx, nx, A, Qi, AQi.data());           /* A Q^-1 */
    matmul(nx, nu, nu, B, Ri, BRi.data());           /* B R^-1 */
    matmul(nx, nx, nx, AQi.data(), At.data(), T1.data());
    matmul(nx, nu, nx, BRi.data(), Bt.data(), T2.data());
    double* theta = &S.Sd[(k + 1) * bb];
    double* phi = &S.Ss[k * bb];
    for (size_t i = 0; i < bb; ++i) {
      theta[i] = T1[i] + T2[i] + Qi1[i];             /* theta_k */
      phi[i] = -AQi[i];                              /* phi_k */
    }
    /* zeta_k = -A Q^-1 q_k - B R^-1 r_k + Q_{k+1}^-1 q_{k+1};  rhs_{k+1} = -e_k - zeta_k */
    for (int i = 0; i < nx; ++i) {
      double z = 0.0;
      for (int j = 0; j < nx; ++j) z -= AQi[i * nx + j] * L.q[(size_t)k * nx + j];
      for (int j = 0; j < nu; ++j) z -= BRi[i * nu + j] * L.r[(size_t)k * nu + j];
      for (int j = 0; j < nx; ++j) z += Qi1[i * nx + j] * L.q[(size_t)(k + 1) * nx + j];
      S.rhs[(size_t)(k + 1) * nx + i] = -L.c[(size_t)(k + 1) * nx + i] - z;
    }
  }
  /* Eq. 6: diagonal Q_0, theta_k^-1; off-diagonal -D_{k+1}^-1 phi_k D_k^-1 */
  for (size_t i = 0; i < bb; ++i) S.Pd[i] = L.Q[i];
  for (int k = 0; k < N; ++k)
    if (!spd_inverse(nx, &S.Sd[(k + 1) * bb], &S.Pd[(k + 1) * bb])) S.ok = false;
  if (precond == 0) {
    for (int k = 0; k < N; ++k) {
      matmul(nx, nx, nx, &S.Pd[(k + 1) * bb], &S.Ss[k * bb], T1.data());
      matmul(nx, nx, nx, T1.data(), &S.Pd[k * bb], T2.data());
      for (size_t i = 0; i < bb; ++i) S.Ps[k * bb + i] = -T2[i];
    }
  }
  return S;
}

template <class T>
void blocktri_mv(int N, int nx, const T* D, const T* Lw, const T* x, T* y) {
  /* y = T x for a symmetric block-tridiagonal T with diagonal D and sub-diagonal Lw. */
  size_t bb = (size_t)nx * nx;
  for (int k = 0; k <= N; ++k)
    for (int i = 0; i < nx; ++i) {
      T s = T(0.0);
      for (int j = 0; j < nx; ++j) s += D[k * bb + i * nx + j] * x[(size_t)k * nx + j];
      if (k > 0)
        for (int j = 0; j < nx; ++j) s += Lw[(k - 1) * bb + i * nx + j] * x[(size_t)(k - 1) * nx + j];
      if (k < N)
        for (int j = 0; j < nx; ++j) s += Lw[k * bb + j * nx + i] * x[(size_t)(k + 1) * nx + j];
      y[(size_t)k * nx + i] = s;
    }
}

int pcg(const Schur& S, double eps, int maxit, double* nu, bool* hit_max) {
  /* Sec. II-B: preconditioned CG on S nu = rhs, warm-started from nu. */
  int N = S.N, nx = S.nx;
  size_t n = (size_t)(N + 1) * nx;
  Vec r(n), z(n), p(n), q(n);
  blocktri_mv(N, nx, S.Sd.data(), S.Ss.data(), nu, q.data());
  for (size_t i = 0; i < n; ++i) r[i] = S.rhs[i] - q[i];
  blocktri_mv(N, nx, S.Pd.data(), S.Ps.data(), r.data(), z.data());
  double eta = 0.0;
  for (size_t i = 0; i < n; ++i) eta += r[i] * z[i];
  double eta0 = eta;
  *hit_max = false;
  if (!(eta0 > 1e-30)) return 0;
  p = z;
  int it = 0;
  while (true) {
    blocktri_mv(N, nx, S.Sd.data(), S.Ss.data(), p.data(), q.data());
    double pq = 0.0;
    for (size_t i = 0; i < n; ++i) pq += p[i] * q[i];
    double alpha = eta / pq;
    for (size_t i = 0; i < n; ++i) { nu[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    blocktri_mv(N, nx, S.Pd.data(), S.Ps.data(), r.data(), z.data());
    double eta_new = 0.0;
    for (size_t i = 0; i < n; ++i) eta_new += r[i] * z[i];
    ++it;
    if (!(eta_new > 0.0) || std::sqrt(eta_new / eta0) <= eps) break;
    if (it >= maxit) { *hit_max = true; break; }
    double beta = eta_new / eta;
    for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    eta = eta_new;
  }
  return it;
}

void recover(const Lin& L, const Schur& S, const double* nu, double* dX, double* dU) {
  /* dZ = -G^-1 (g + C^T nu):
     dx_k = -Q_k^-1 (q_k + nu_k - A_k^T nu_{k+1}), dx_N = -Q_N^-1 (q_N + nu_N),
     du_k = -R_k^-1 (r_k - B_k^T nu_{k+1}). */
  int N = L.N, nx = L.nx, nu_ = L.nu;
  size_t bb = (size_t)nx * nx;
  Vec t(nx), s(nu_);
  for (int k = 0; k <= N; ++k) {
    for (int i = 0; i < nx; ++i) {
      double v = L.q[(size_t)k * nx + i] + nu[(size_t)k * nx + i];
      if (k < N)
        for (int j = 0; j < nx; ++j) v -= L.A[k * bb + j * nx + i] * nu[(size_t)(k + 1) * nx + j];
      t[i] = v;
    }
    for (int i = 0; i < nx; ++i) {
      double v = 0.0;
      for (int j = 0; j < nx; ++j) v -= S.Qinv[k * bb + i * nx + j] * t[j];
      dX[(size_t)k * nx + i] = v;
    }
    if (k < N) {
      for (int i = 0; i < nu_; ++i) {
        double v = L.r[(size_t)k * nu_ + i];
        for (int j = 0; j < nx; ++j) v -= L.B[(size_t)k * nx * nu_ + j * nu_ + i] * nu[(size_t)(k + 1) * nx + j];
        s[i] = v;
      }
      for (int i = 0; i < nu_; ++i) {
        double v = 0.0;
        for (int j = 0; j < nu_; ++j) v -= S.Rinv[(size_t)k * nu_ * nu_ + i * nu_ + j] * s[j];
        dU[(size_t)k * nu_ + i] = v;
      }
    }
  }
}

double kkt_residual(const Lin& L, const double* nu) {
  /* c17: max(||c||_inf, ||g + C^T nu||_inf / max(1, ||g||_inf)). */
  int N = L.N, nx = L.nx, nu_ = L.nu;
  size_t bb = (size_t)nx * nx;
  double cinf = 0.0, ginf = 0.0, dinf = 0.0;
  for (double v : L.c) cinf = std::max(cinf, std::fabs(v));
  for (int k = 0; k <= N; ++k) {
    for (int i = 0; i < nx; ++i) {
      double g = L.q[(size_t)k * nx + i];
      double v = g + nu[(size_t)k * nx + i];
      if (k < N)
        for (int j = 0; j < nx; ++j) v -= L.A[k * bb + j * nx + i] * nu[(size_t)(k + 1) * nx + j];
      ginf = std::max(ginf, std::fabs(g));
      dinf = std::max(dinf, std::fabs(v));
    }
    if (k < N)
      for (int i = 0; i < nu_; ++i) {
        double g = L.r[(size_t)k * nu_ + i];
        double v = g;
        for (int j = 0; j < nx; ++j) v -= L.B[(size_t)k * nx * nu_ + j * nu_ + i] * nu[(size_t)(k + 1) * nx + j];
        ginf = std::max(ginf, std::fabs(g));
        dinf = std::max(dinf, std::fabs(v));
      }
  }
  return std::max(cinf, dinf / std::max(1.0, ginf));
}

bool all_finite(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i) if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

/* =========================================================== C interface */

extern "C" {

void ora_rnea(const ora_model* m, const double* q, const double* qd, const double* qdd,
              int32_t gravity, double* tau) {
  rnea(*m, q, qd, qdd, gravity != 0, tau);
}

void ora_mass_matrix(const ora_model* m, const double* q, double* M) { mass_matrix(*m, q, M); }

/* f_ext: NULL or the 3 components of a force at the end effector (base frame). */
int32_t ora_forward_dynamics(const ora_model* m, const double* q, const double* qd,
                             const double* tau, const double* f_ext, double* qdd) {
  return forward_dynamics(*m, q, qd, tau, qdd, f_ext) ? 0 : -1;
}

int32_t ora_step(const ora_model* m, const double* x, const double* u, double h,
                 const double* f_ext, double* xn) {
  return step(*m, x, u, h, xn, f_ext) ? 0 : -1;
}

void ora_step_jacobians(const ora_model* m, const double* x, const double* u, double h,
                        const double* f_ext, double* A, double* B) {
  step_jacobians(*m, x, u, h, A, B, f_ext);
}

void ora_ee_joint_torque(const ora_model* m, const double* q, const double* f, double* tau) {
  ee_joint_torque(*m, q, f, tau);
}

void ora_fk(const ora_model* m, const double* q, double* p, double* J) {
  if (J) fk_jacobian(*m, q, p, J);
  else fk_ee(*m, q, p);
}

double ora_merit(const ora_model* m, const ora_problem* p, const double* X, const double* U,
                 double mu) {
  return merit(*m, *p, X, U, mu, nullptr);
}

/* Linearisation at (X, U): all arrays caller-allocated, dense row-major. */
double ora_linearize(const ora_model* m, const ora_problem* p, const double* X, const double* U,
                     double* A, double* B, double* Q, double* R, double* q, double* r, double* c) {
  Lin L = linearize(*m, *p, X, U);
  std::memcpy(A, L.A.data(), L.A.size() * sizeof(double));
  std::memcpy(B, L.B.data(), L.B.size() * sizeof(double));
  std::memcpy(Q, L.Q.data(), L.Q.size() * sizeof(double));
  std::memcpy(R, L.R.data(), L.R.size() * sizeof(double));
  std::memcpy(q, L.q.data(), L.q.size() * sizeof(double));
  std::memcpy(r, L.r.data(), L.r.size() * sizeof(double));
  std::memcpy(c, L.c.data(), L.c.size() * sizeof(double));
  return L.J;
}

/* Schur blocks, rhs and preconditioner at (X, U). */
int32_t ora_schur(const ora_model* m, const ora_problem* p, const double* X, const double* U,
                  int32_t precond, double* Sd, double* Ss, double* Pd, double* Ps, double* rhs) {
  Lin L = linearize(*m, *p, X, U);
  Schur S = form_schur(L, precond);
  std::memcpy(Sd, S.Sd.data(), S.Sd.size() * sizeof(double));
  std::memcpy(Ss, S.Ss.data(), S.Ss.size() * sizeof(double));
  std::memcpy(Pd, S.Pd.data(), S.Pd.size() * sizeof(double));
  std::memcpy(Ps, S.Ps.data(), S.Ps.size() * sizeof(double));
  std::memcpy(rhs, S.rhs.data(), S.rhs.size() * sizeof(double));
  return S.ok ? 0 : -1;
}

/* PCG on caller-provided blocks (used by the pins). Returns iterations. */
int32_t ora_pcg(int32_t N, int32_t nx, const double* Sd, const double* Ss, const double* Pd,
                const double* Ps, const double* rhs, double eps, int32_t maxit, double* nu) {
  Schur S;
  size_t bb = (size_t)nx * nx;
  S.N = N; S.nx = nx; S.ok = true;
  S.Sd.assign(Sd, Sd + (N + 1) * bb);
  S.Ss.assign(Ss, Ss + N * bb);
  S.Pd.assign(Pd, Pd + (N + 1) * bb);
  S.Ps.assign(Ps, Ps + N * bb);
  S.rhs.assign(rhs, rhs + (size_t)(N + 1) * nx);
  bool hit = false;
  return pcg(S, eps, maxit, nu, &hit);
}

/* One QP step at (X, U): solves the Schur system by PCG (warm start nu) and
   returns the recovered dX, dU.  Returns PCG iterations, -1 on failure. */
int32_t ora_qp_step(const ora_model* m, const ora_problem* p, const double* X, const double* U,
                    int32_t precond, double eps, int32_t maxit, double* nu, double* dX, double* dU) {
  Lin L = linearize(*m, *p, X, U);
  Schur S = form_schur(L, precond);
  if (!S.ok) return -1;
  bool hit = false;
  int it = pcg(S, eps, maxit, nu, &hit);
  recover(L, S, nu, dX, dU);
  return it;
}

double ora_kkt_residual(const ora_model* m, const ora_problem* p, const double* X,
                        const double* U, const double* nu) {
  Lin L = linearize(*m, *p, X, U);
  return kkt_residual(L, nu);
}

/* Full SQP solve (Sec. II-A Steps 1-3 with the Alg. 1 stages).
   X, U, nu: in = initial guess / warm start, out = final iterate.
   replay: NULL, or [max_iter] line-search indices to force (-1 = reject).
   Per-iteration logs (each [max_iter] or NULL): chosen alpha index (-1 reject),
   PCG iterations, merit before the step, merit after, KKT residual, and the
   margin of the line-search decision relative to the best trial merit (the
   smaller of its gaps to the runner-up trial and to the current merit). */
int32_t ora_blocktri_solve(int32_t N, int32_t nx, const double* Sd, const double* Ss,
                           const double* rhs, double* x);

int32_t ora_solve(const ora_model* m, const ora_problem* p, const ora_params* prm,
                  double* X, double* U, double* nu, const int32_t* replay,
                  int32_t* log_alpha, int32_t* log_pcg, double* log_m0, double* log_m1,
                  double* log_kkt, double* log_gap, ora_result* res) {
  int n = m->dof, nx = 2 * n, N = p->N;
  size_t nX = (size_t)(N + 1) * nx, nU = (size_t)N * n;
  Vec dX(nX), dU(nU), Xt(nX), Ut(nU), mer(std::max(1, (int)prm->n_alpha));
  ora_result R;
  R.iters = 0; R.flags = 0; R.pcg_total = 0; R.kkt = 0.0; R.merit = 0.0;
  ora_problem pr = *p;  /* its rho (w[5]) follows the adaptation when that is on */
  for (int it = 0;; ++it) {
    if (it == prm->max_iter && prm->kkt_tol <= 0.0) break;
    Lin L = linearize(*m, pr, X, U);
    if (!L.ok || !all_finite(L.c.data(), L.c.size())) { R.flags |= 16; break; }
    double rk = kkt_residual(L, nu);
    R.kkt = rk;
    if (log_kkt && it < prm->max_iter) log_kkt[it] = rk;
    double m0 = L.J;
    for (double v : L.c) m0 += prm->mu * std::fabs(v);
    R.merit = m0;
    if (prm->kkt_tol > 0.0 && rk <= prm->kkt_tol) { R.flags |= 1; break; }
    if (it == prm->max_iter) { R.flags |= 2; break; }
    Schur S = form_schur(L, prm->precond);
    if (!S.ok) { R.flags |= 16; break; }
    bool hit = false;
    int pit = 0;
    if (prm->linsolve == 1) {
      if (ora_blocktri_solve(N, nx, S.Sd.data(), S.Ss.data(), S.rhs.data(), nu) != 0) {
        R.flags |= 16;
        break;
      }
    } else {
      pit = pcg(S, prm->pcg_eps, prm->pcg_max, nu, &hit);
    }
    if (hit) R.flags |= 8;
    R.pcg_total += pit;
    recover(L, S, nu, dX.data(), dU.data());
    if (!all_finite(dX.data(), nX) || !all_finite(dU.data(), nU) || !all_finite(nu, nX)) {
      R.flags |= 16; break;
    }
    double alpha = 1.0;
    for (int i = 0; i < prm->n_alpha; ++i) {
      for (size_t l = 0; l < nX; ++l) Xt[l] = X[l] + alpha * dX[l];
      for (size_t l = 0; l < nU; ++l) Ut[l] = U[l] + alpha * dU[l];
      bool ok = true;
      double mi = merit(*m, pr, Xt.data(), Ut.data(), prm->mu, &ok);
      if (!ok || !std::isfinite(mi)) mi = INFINITY;
      mer[i] = mi;
      alpha /= prm->beta;
    }
    int best = 0;                       /* first minimum: ties go to the largest alpha */
    for (int i = 1; i < prm->n_alpha; ++i) if (mer[i] < mer[best]) best = i;
    double bestm = mer[best], second = INFINITY;
    for (int i = 0; i < prm->n_alpha; ++i) if (i != best) second = std::min(second, mer[i]);
    int choice = (bestm < m0) ? best : -1;
    if (replay) choice = replay[it];
    if (log_gap && it < prm->max_iter) {
      /* the margin of the decision of Eq. 7, relative to the best merit: the
         gap to the runner-up trial merit and the gap to the current merit
         (accept versus reject), whichever is smaller */
      const double sc = std::max(1e-300, std::fabs(bestm));
      double g = std::isfinite(second) ? (second - bestm) / sc : INFINITY;
      if (std::isfinite(bestm)) g = std::min(g, std::fabs(m0 - bestm) / sc);
      log_gap[it] = g;
    }
    if (log_m0 && it < prm->max_iter) log_m0[it] = m0;
    if (choice >= 0) {
      double a = std::pow(prm->beta, -choice);
      for (size_t l = 0; l < nX; ++l) X[l] += a * dX[l];
      for (size_t l = 0; l < nU; ++l) U[l] += a * dU[l];
      R.merit = mer[choice];
    } else {
      R.flags |= 4;
    }
    if (prm->rho_adapt)
      pr.w[5] = choice >= 0 ? std::max(pr.w[5] / 3.0, 1e-8) : std::min(pr.w[5] * 2.0, 1e1);
    if (log_alpha && it < prm->max_iter) log_alpha[it] = choice;
    if (log_pcg && it < prm->max_iter) log_pcg[it] = pit;
    if (log_m1 && it < prm->max_iter) log_m1[it] = R.merit;
    R.iters = it + 1;
  }
  if (res) *res = R;
  return 0;
}

/* Operation counts of the method's primitive computations, from the
   templated code above run on the counting scalar Cnt (FMA = 2), for the
   model m at a generic state (nonzero q, qd, qdd; gravity on):
     0  inverse dynamics, one RNEA pass (Sec. II-A's dynamics f; the same code
        gives one column of M with a unit acceleration)
     1  an RNEA pass carrying one forward-mode directional derivative
        (value + tangent; the tangent alone is 1 minus 0)
     2  Cholesky factor and one solve of a dof x dof SPD system
     3  end-effector position (forward kinematics)
     4  end-effector position carrying one directional derivative
     5  product of two 14 x 14 blocks (also the cost of a Gauss-Jordan
        inverse of a 14 x 14 block: n^3 multiply-adds)
     6  one block row (14 rows) of a block-tridiagonal matrix-vector product
     7  forward dynamics as the oracle writes it: M by dof RNEA columns, the
        bias pass and a Cholesky solve
   Returns -1 for an unknown `what`. */
int64_t ora_count_flops(const ora_model* m, int32_t what) {
  const int n = m->dof;
  std::vector<Cnt> q(n), qd(n), qdd(n), tau(n);
  for (int i = 0; i < n; ++i) {
    q[i] = Cnt(0.3 + 0.1 * i);
    qd[i] = Cnt(0.2 - 0.05 * i);
    qdd[i] = Cnt(1.0 + 0.5 * i);
  }
  g_flops = 0;
  switch (what) {
    case 0:
      rnea(*m, q.data(), qd.data(), qdd.data(), true, tau.data());
      break;
    case 1: {
      typedef DualT<Cnt> DC;
      std::vector<DC> a(n), b(n), c(n), t(n);
      for (int i = 0; i < n; ++i) {
        a[i] = DC(q[i], Cnt(i == 0 ? 1.0 : 0.0));
        b[i] = DC(qd[i], Cnt(0.0));
        c[i] = DC(qdd[i], Cnt(0.0));
      }
      g_flops = 0;
      rnea(*m, a.data(), b.data(), c.data(), true, t.data());
      break;
    }
    case 2: {
      std::vector<Cnt> A((size_t)n * n);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = Cnt(i == j ? 4.0 : 0.5);
      g_flops = 0;
      cholesky_solve(n, A, qdd.data());
      break;
    }
    case 3: {
      Cnt p[3];
      fk_ee(*m, q.data(), p);
      break;
    }
    case 4: {
      typedef DualT<Cnt> DC;
      std::vector<DC> a(n);
      for (int i = 0; i < n; ++i) a[i] = DC(q[i], Cnt(i == 0 ? 1.0 : 0.0));
      DC p[3];
      g_flops = 0;
      fk_ee(*m, a.data(), p);
      break;
    }
    case 5: {
      std::vector<Cnt> A(196, Cnt(0.5)), B(196, Cnt(0.25)), C(196);
      g_flops = 0;
      matmul(14, 14, 14, A.data(), B.data(), C.data());
      break;
    }
    case 6: {
      const int N = 3;  /* four block rows; the count is per block row */
      std::vector<Cnt> D((N + 1) * 196, Cnt(0.5)), L(N * 196, Cnt(0.25)), x((N + 1) * 14, Cnt(1.0)),
          y((N + 1) * 14);
      g_flops = 0;
      blocktri_mv(N, 14, D.data(), L.data(), x.data(), y.data());
      return (int64_t)(g_flops / (N + 1));
    }
    case 7:
      forward_dynamics(*m, q.data(), qd.data(), qdd.data(), tau.data());
      break;
    default:
      return -1;
  }
  return (int64_t)g_flops;
}

/* Direct solve of the block-tridiagonal SPD system (block Cholesky), for checks. */
int32_t ora_blocktri_solve(int32_t N, int32_t nx, const double* Sd, const double* Ss,
                           const double* rhs, double* x) {
  size_t bb = (size_t)nx * nx;
  std::vector<Vec> Dk(N + 1, Vec(bb)), Lk(N, Vec(bb));
  /* Eliminate forward: D_0 = S_00, L_k = S_{k+1,k} D_k^-1, D_{k+1} = S_{k+1,k+1} - L_k S_{k+1,k}^T */
  Dk[0].assign(Sd, Sd + bb);
  Vec Dinv(bb), tmp(bb);
  Vec y(rhs, rhs + (size_t)(N + 1) * nx);
  for (int k = 0; k < N; ++k) {
    if (!spd_inverse(nx, Dk[k].data(), Dinv.data())) return -1;
    matmul(nx, nx, nx, &Ss[k * bb], Dinv.data(), Lk[k].data());
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < nx; ++j) {
        double s = 0.0;
        for (int l = 0; l < nx; ++l) s += Lk[k][i * nx + l] * Ss[k * bb + j * nx + l];
        Dk[k + 1][i * nx + j] = Sd[(k + 1) * bb + i * nx + j] - s;
      }
    for (int i = 0; i < nx; ++i) {
      double s = 0.0;
      for (int l = 0; l < nx; ++l) s += Lk[k][i * nx + l] * y[(size_t)k * nx + l];
      y[(size_t)(k + 1) * nx + i] -= s;
    }
  }
  for (int k = N; k >= 0; --k) {
    Vec b(&y[(size_t)k * nx], &y[(size_t)k * nx] + nx);
    if (k < N)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int l = 0; l < nx; ++l) s += Ss[k * bb + l * nx + i] * x[(size_t)(k + 1) * nx + l];
        b[i] -= s;
      }
    if (!cholesky_solve(nx, Dk[k], b.data())) return -1;
    for (int i = 0; i < nx; ++i) x[(size_t)k * nx + i] = b[i];
  }
  return 0;
}

}  // extern "C"
