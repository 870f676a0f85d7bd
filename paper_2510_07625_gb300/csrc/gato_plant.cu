// Plant simulation for closed-loop runs: the simulated robot that the
// controller acts on (Sec. IV-E runs the plant at 1 kHz with RK4 while the
// solver runs at its own rate).  Host code in FP64; nothing here is on the
// solve path, which runs entirely in the CUDA kernels.
//
// Dynamics of the serial revolute chain of gato_model_desc (joint i turns
// about axis[i] of its own frame, its origin at the parent origin plus
// (0, 0, link_len[i-1]) in the parent frame; end effector at (0, 0,
// link_len[dof-1]) of the last frame; gravity along -z), with a constant force
// f on the end-effector point:
//     M(q) qdd = u + J_p(q)^T f - C(q, qd) qd - g(q).
// Newton-Euler with every quantity in base coordinates: rotation matrices
// R_i, joint axes z_i = R_i e_{axis_i}, origins p_i; the outward pass gives
// angular velocity and acceleration and the origins' linear acceleration (the
// base accelerates upward by g in place of gravity), the inward pass the
// force and moment each joint transmits, the force f entering the last link.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "gato.h"

namespace {

struct V { double x, y, z; };
inline V add(V a, V b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V sub(V a, V b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V scl(double s, V a) { return {s * a.x, s * a.y, s * a.z}; }
inline V crs(V a, V b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double dt3(V a, V b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

struct Mat { double a[3][3]; };
inline V mv(const Mat& R, V v) {
  return {R.a[0][0] * v.x + R.a[0][1] * v.y + R.a[0][2] * v.z,
          R.a[1][0] * v.x + R.a[1][1] * v.y + R.a[1][2] * v.z,
          R.a[2][0] * v.x + R.a[2][1] * v.y + R.a[2][2] * v.z};
}
inline V mtv(const Mat& R, V v) {  // R^T v
  return {R.a[0][0] * v.x + R.a[1][0] * v.y + R.a[2][0] * v.z,
          R.a[0][1] * v.x + R.a[1][1] * v.y + R.a[2][1] * v.z,
          R.a[0][2] * v.x + R.a[1][2] * v.y + R.a[2][2] * v.z};
}
inline Mat mm(const Mat& A, const Mat& B) {
  Mat C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[i][0] * B.a[0][j] + A.a[i][1] * B.a[1][j] + A.a[i][2] * B.a[2][j];
  return C;
}
inline Mat axis_rot(int axis, double q) {  // rotation by q about a coordinate axis
  const double c = std::cos(q), s = std::sin(q);
  Mat R;
  std::memset(&R, 0, sizeof(R));
  const int i = (axis + 1) % 3, j = (axis + 2) % 3;
  R.a[axis][axis] = 1.0;
  R.a[i][i] = c;
  R.a[j][j] = c;
  R.a[j][i] = s;
  R.a[i][j] = -s;
  return R;
}
inline V col(const Mat& R, int k) { return {R.a[0][k], R.a[1][k], R.a[2][k]}; }

struct Kin {
  int n;
  Mat R[7];
  V p[7], z[7], ee;
};

bool model_ok(const gato_model_desc* m) {
  if (!m || m->dof < 1 || m->dof > 7 || !(m->gravity >= 0.f) || !std::isfinite(m->gravity)) return false;
  for (int i = 0; i < m->dof; ++i) {
    if (m->axis[i] < 0 || m->axis[i] > 2) return false;
    if (!(m->link_len[i] >= 0.f) || !(m->mass[i] > 0.f) || !std::isfinite(m->link_len[i]) || !std::isfinite(m->mass[i]))
      return false;
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(m->com[3 * i + a]) || !(m->inertia[3 * i + a] >= 0.f)) return false;
  }
  return true;
}

void kinematics(const gato_model_desc& m, const double* q, Kin& k) {
  k.n = m.dof;
  Mat Rp;
  std::memset(&Rp, 0, sizeof(Rp));
  Rp.a[0][0] = Rp.a[1][1] = Rp.a[2][2] = 1.0;
  V pp = {0, 0, 0};
  for (int i = 0; i < k.n; ++i) {
    k.p[i] = i == 0 ? pp : add(k.p[i - 1], scl(m.link_len[i - 1], col(Rp, 2)));
    k.R[i] = mm(Rp, axis_rot(m.axis[i], q[i]));
    k.z[i] = col(k.R[i], m.axis[i]);
    Rp = k.R[i];
  }
  k.ee = add(k.p[k.n - 1], scl(m.link_len[k.n - 1], col(k.R[k.n - 1], 2)));
}

// tau = ID(q, qd, qdd) with gravity g_on and the end-effector force f (may be null).
void inverse_dynamics(const gato_model_desc& m, const Kin& k, const double* qd, const double* qdd,
                      bool g_on, const double* f, double* tau) {
  const int n = k.n;
  V w = {0, 0, 0}, wd = {0, 0, 0}, a = {0, 0, g_on ? (double)m.gravity : 0.0};
  V F[7], Nc[7], c[7];
  for (int i = 0; i < n; ++i) {
    if (i > 0) {
      const V r = sub(k.p[i], k.p[i - 1]);
      a = add(a, add(crs(wd, r), crs(w, crs(w, r))));
    }
    const V wn = add(w, scl(qd[i], k.z[i]));
    wd = add(add(wd, scl(qdd[i], k.z[i])), crs(w, scl(qd[i], k.z[i])));
    w = wn;
    const V rc = mv(k.R[i], {m.com[3 * i], m.com[3 * i + 1], m.com[3 * i + 2]});
    c[i] = rc;
    const V ac = add(a, add(crs(wd, rc), crs(w, crs(w, rc))));
    F[i] = scl(m.mass[i], ac);
    // I_world v = R diag(I) R^T v
    const V Id = {m.inertia[3 * i], m.inertia[3 * i + 1], m.inertia[3 * i + 2]};
    auto Iw = [&](V v) {
      const V b = mtv(k.R[i], v);
      return mv(k.R[i], {Id.x * b.x, Id.y * b.y, Id.z * b.z});
    };
    Nc[i] = add(Iw(wd), crs(w, Iw(w)));
  }
  V fc = {0, 0, 0}, nc = {0, 0, 0};
  if (f) {  // the force acts on the last link at the end-effector point
    const V fe = {f[0], f[1], f[2]};
    fc = scl(-1.0, fe);
    nc = scl(-1.0, crs(sub(k.ee, k.p[n - 1]), fe));
  }
  for (int i = n - 1; i >= 0; --i) {
    // moment about p_i: the link's own, its weight-and-inertia force at c_i,
    // and what the child transmits at p_{i+1} (or the external force)
    V nn = add(Nc[i], crs(c[i], F[i]));
    if (i < n - 1) nn = add(nn, add(nc, crs(sub(k.p[i + 1], k.p[i]), fc)));
    else nn = add(nn, nc);
    const V ff = add(F[i], fc);
    tau[i] = dt3(k.z[i], nn);
    fc = ff;
    nc = nn;
  }
}

// xdot for x = (q, qd); false when the mass matrix is not positive definite.
bool xdot(const gato_model_desc& m, const double* x, const double* u, const double* f, double* out) {
  const int n = m.dof;
  Kin k;
  kinematics(m, x, k);
  double Mm[49], z[7] = {}, e[7], b[7];
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) e[i] = i == j ? 1.0 : 0.0;
    double colv[7];
    inverse_dynamics(m, k, z, e, false, nullptr, colv);
    for (int i = 0; i < n; ++i) Mm[i * n + j] = colv[i];
  }
  inverse_dynamics(m, k, x + n, z, true, f, b);
  double r[7];
  for (int i = 0; i < n; ++i) r[i] = u[i] - b[i];
  // Cholesky M = L L^T in place (lower triangle), then two triangular solves
  for (int j = 0; j < n; ++j) {
    double s = Mm[j * n + j];
    for (int l = 0; l < j; ++l) s -= Mm[j * n + l] * Mm[j * n + l];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    Mm[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = Mm[i * n + j];
      for (int l = 0; l < j; ++l) t -= Mm[i * n + l] * Mm[j * n + l];
      Mm[i * n + j] = t / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double t = r[i];
    for (int l = 0; l < i; ++l) t -= Mm[i * n + l] * r[l];
    r[i] = t / Mm[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = r[i];
    for (int l = i + 1; l < n; ++l) t -= Mm[l * n + i] * r[l];
    r[i] = t / Mm[i * n + i];
  }
  for (int i = 0; i < n; ++i) {
    out[i] = x[n + i];
    out[n + i] = r[i];
  }
  return true;
}

}  // namespace

extern "C" {

gato_status gato_plant_rk4(const gato_model_desc* model, const double* x, const double* u,
                           const double* f_ext, double h, int32_t steps, double* x_out) {
  if (!model_ok(model) || !x || !u || !x_out || !(h > 0.0) || !std::isfinite(h) || steps < 0)
    return GATO_E_INVALID;
  const int nx = 2 * model->dof;
  double y[14], k1[14], k2[14], k3[14], k4[14], t[14];
  for (int i = 0; i < nx; ++i) y[i] = x[i];
  for (int s = 0; s < steps; ++s) {
    bool ok = xdot(*model, y, u, f_ext, k1);
    for (int i = 0; i < nx; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    ok = ok && xdot(*model, t, u, f_ext, k2);
    for (int i = 0; i < nx; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    ok = ok && xdot(*model, t, u, f_ext, k3);
    for (int i = 0; i < nx; ++i) t[i] = y[i] + h * k3[i];
    ok = ok && xdot(*model, t, u, f_ext, k4);
    if (!ok) return GATO_E_INVALID;
    for (int i = 0; i < nx; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
  for (int i = 0; i < nx; ++i) {
    if (!std::isfinite(y[i])) return GATO_E_INVALID;
    x_out[i] = y[i];
  }
  return GATO_OK;
}

gato_status gato_plant_ee(const gato_model_desc* model, const double* q, double* p) {
  if (!model_ok(model) || !q || !p) return GATO_E_INVALID;
  Kin k;
  kinematics(*model, q, k);
  p[0] = k.ee.x;
  p[1] = k.ee.y;
  p[2] = k.ee.z;
  return GATO_OK;
}

}  // extern "C"
