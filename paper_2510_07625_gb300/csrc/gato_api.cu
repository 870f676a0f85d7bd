// C ABI of the batched SQP library (declared in include/gato.h).
//
// Host-side duties only: validation, model conversion, staging of host
// problems through pinned memory, longest-horizon-first ordering, launching
// the kernels in gato_kernels.cu and copying results back.  No arithmetic of
// the method runs here.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gato.h"
#include "gato_internal.h"

using namespace gato;

namespace {

struct HostCopyBack {
  float* X;
  float* U;
  float* lam;
  size_t nX, nU;              // element counts in user layout (lam has nX)
  size_t offX, offU, offL;    // staging offsets (floats)
  size_t end;                 // staging end of this problem
};

}  // namespace

namespace gato {

const char* check_model(const gato_model_desc& d, DevModel& m) {
  if (d.dof < 1 || d.dof > QM) return "model dof must be 1..7";
  if (!(d.gravity >= 0.f) || !std::isfinite(d.gravity)) return "gravity must be finite and >= 0";
  std::memset(&m, 0, sizeof(m));
  m.dof = d.dof;
  m.g = d.gravity;
  for (int i = 0; i < QM; ++i) {
    if (i < d.dof) {
      if (d.axis[i] < 0 || d.axis[i] > 2) return "joint axis must be 0, 1 or 2";
      if (!(d.link_len[i] >= 0.f) || !std::isfinite(d.link_len[i])) return "link lengths must be finite and >= 0";
      if (!(d.mass[i] > 0.f) || !std::isfinite(d.mass[i])) return "link masses must be finite and > 0";
      m.axis[i] = d.axis[i];
      m.L[i] = d.link_len[i];
      m.m[i] = d.mass[i];
      for (int a = 0; a < 3; ++a) {
        const float c = d.com[3 * i + a], I = d.inertia[3 * i + a];
        if (!std::isfinite(c) || !(I >= 0.f) || !std::isfinite(I)) return "com / inertia must be finite, inertia >= 0";
        m.com[3 * i + a] = c;
        m.Ic[3 * i + a] = I;
      }
    } else {
      // massless padding joint at the end effector: exact zero rows downstream
      m.axis[i] = 2;
    }
  }
  return nullptr;
}

const char* check_params(const gato_solver_params& p) {
  if (!(p.mu >= 0.f) || !std::isfinite(p.mu)) return "mu must be finite and >= 0";
  if (!(p.beta > 1.f) || !std::isfinite(p.beta)) return "beta must be > 1";
  if (p.n_alpha < 1 || p.n_alpha > MAX_ALPHA) return "n_alpha must be 1..16";
  if (!(p.pcg_eps > 0.f)) return "pcg_eps must be > 0";
  if (p.pcg_max_iter < 1) return "pcg_max_iter must be >= 1";
  if (p.precond != GATO_PRECOND_STAIR && p.precond != GATO_PRECOND_JACOBI) return "unknown preconditioner";
  if (p.linsolve != GATO_LINSOLVE_PCG && p.linsolve != GATO_LINSOLVE_DIRECT) return "unknown linear solver";
  if (p.rho_adapt != 0 && p.rho_adapt != 1) return "rho_adapt must be 0 or 1";
  if (p.precision != GATO_PRECISION_FP32 && p.precision != GATO_PRECISION_ESCALATE &&
      p.precision != GATO_PRECISION_HIGH)
    return "precision must be GATO_PRECISION_FP32, _ESCALATE or _HIGH";
  if (!std::isfinite(p.kkt_tol)) return "kkt_tol must be finite";
  return nullptr;
}

const char* check_problem(const gato_problem& p, int n_models, int max_horizon) {
  if (p.model < 0 || p.model >= n_models) return "model index out of range";
  if (p.N < 1 || p.N > max_horizon) return "N must be 1..max_horizon";
  if (!(p.dt > 0.f) || !std::isfinite(p.dt)) return "dt must be finite and > 0";
  if (p.mem != GATO_MEM_HOST && p.mem != GATO_MEM_DEVICE) return "mem must be HOST or DEVICE";
  if (!p.x_s || !p.X || !p.U) return "x_s, X and U are required";
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(p.w[i]) || p.w[i] < 0.f) return "weights must be finite and >= 0";
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(p.f_ext[i])) return "f_ext must be finite";
  const float wq = p.w[0], wqd = p.w[1], wr = p.w[2], ts = p.w[3], rho = p.w[5];
  if (!(wr > 0.f)) return "control weight must be > 0";
  if (!(ts > 0.f)) return "terminal scale must be > 0";
  if (p.cost_kind == GATO_COST_JOINT) {
    if (!p.x_ref) return "joint cost needs x_ref";
    if (!(wq + rho > 0.f) || !(wqd + rho > 0.f)) return "joint cost Hessian must be positive definite";
  } else if (p.cost_kind == GATO_COST_EE) {
    if (!p.ee_ref) return "end-effector cost needs ee_ref";
    if (!(rho > 0.f) || !(wqd + rho > 0.f)) return "end-effector cost needs rho > 0";
  } else {
    return "unknown cost kind";
  }
  return nullptr;
}

}  // namespace gato

struct gato_batch {
  int max_batch = 0, max_horizon = 0, n_models = 0;
  DevModel models_h[8];
  int model_dof[8];
  gato_solver_params params;
  cudaStream_t stream = nullptr;
  DevModel* models_d = nullptr;
  ProbDesc* probs_d = nullptr;
  ProbDesc* probs_h = nullptr;
  int* order_d = nullptr;
  int* order_h = nullptr;
  Result* res_d = nullptr;
  Result* res_h = nullptr;
  float* ws_d = nullptr;
  size_t ws_stride = 0;
  WsLayout layout;
  float* plain_ws_d = nullptr;
  WsLayout plain_layout;
  float* stage_d = nullptr;
  float* stage_h = nullptr;
  size_t stage_stride = 0;
  cudaEvent_t done = nullptr;
  int last_n = 0;
  bool pending = false;
  std::vector<HostCopyBack> copy_back;
  std::vector<int> N_h;   // horizon of each solve of the current call
  long long* timing_d = nullptr;  // per-stage cycle counters while profiling is on
  int* itlog_d = nullptr;         // per-iteration records while the log is on
  int itlog_iters = 0;
  // launch plans: one set by gato_set_launch_config, else the autotuner's
  // choice for the call's (batch size, horizon) bucket, else automatic
  bool forced = false;
  LaunchPlan forced_plan;
  struct Tuned { int n_bucket, n_key; LaunchPlan plan; };
  std::vector<Tuned> tuned;
  LaunchPlan cur_plan;            // plan of the call being prepared
  cudaStream_t aux[7] = {};       // fork streams for concurrent cluster-size groups
  cudaEvent_t fork_ev[8] = {};
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  std::string err;
};

namespace {

gato_status fail(gato_batch* b, gato_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

gato_status cuda_fail(gato_batch* b, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(b, GATO_E_CUDA, m);
}

int pow2_bucket(int n) {
  int b = 1;
  while (b < n) b <<= 1;
  return b;
}

int horizon_key(int nmax) { return (nmax + 15) / 16; }

LaunchPlan plan_for(const gato_batch* b, int n, int nmax) {
  LaunchPlan p;
  if (b->forced) {
    p = b->forced_plan;
  } else {
    for (const auto& t : b->tuned)
      if (t.n_bucket == pow2_bucket(n) && t.n_key == horizon_key(nmax)) p = t.plan;
  }
  p.aux = b->aux;
  p.ev = b->fork_ev;
  p.n_aux = b->aux[0] ? 7 : 0;
  return p;
}

bool finite_all(const float* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

size_t stage_floats(int nmax) {
  const size_t K = nmax + 1;
  return align32(16 + K * XM + K * 3 + K * XM + (size_t)nmax * QM + K * XM);
}

bool convert_model(const gato_model_desc& d, DevModel& m, std::string& why) {
  const char* r = check_model(d, m);
  if (r) why = r;
  return r == nullptr;
}

gato_status validate_params(gato_batch* b, const gato_solver_params& p) {
  const char* r = check_params(p);
  return r ? fail(b, GATO_E_INVALID, r) : GATO_OK;
}

gato_status validate_problem(gato_batch* b, const gato_problem& p, int idx) {
  char buf[160];
  auto bad = [&](const char* why) {
    std::snprintf(buf, sizeof(buf), "problem %d: %s", idx, why);
    return fail(b, GATO_E_INVALID, buf);
  };
  if (const char* r = check_problem(p, b->n_models, b->max_horizon)) return bad(r);
  if (p.mem == GATO_MEM_HOST) {
    const int nx = 2 * b->model_dof[p.model], nu = b->model_dof[p.model];
    if (!finite_all(p.x_s, nx)) return bad("x_s is not finite");
    if (!finite_all(p.X, (size_t)(p.N + 1) * nx) || !finite_all(p.U, (size_t)p.N * nu))
      return bad("initial X / U not finite");
    if (p.cost_kind == GATO_COST_JOINT && !finite_all(p.x_ref, (size_t)(p.N + 1) * nx))
      return bad("x_ref not finite");
    if (p.cost_kind == GATO_COST_EE && !finite_all(p.ee_ref, (size_t)(p.N + 1) * 3))
      return bad("ee_ref not finite");
    if (p.lambda && !finite_all(p.lambda, (size_t)(p.N + 1) * nx)) return bad("lambda not finite");
  }
  return GATO_OK;
}

Params to_params(const gato_solver_params& p, int iters) {
  Params o;
  o.mu = p.mu;
  o.beta = p.beta;
  o.n_alpha = p.n_alpha;
  o.pcg_eps = p.pcg_eps;
  o.pcg_max = p.pcg_max_iter;
  o.precond = p.precond;
  o.kkt_tol = p.kkt_tol;
  o.max_iter = iters;
  o.linsolve = p.linsolve;
  o.rho_adapt = p.rho_adapt;
  o.escalate = p.precision == GATO_PRECISION_ESCALATE;
  o.high = p.precision == GATO_PRECISION_HIGH;
  return o;
}

// Builds the device descriptors (staging host problems), returns max N.
gato_status prepare(gato_batch* b, const gato_problem* probs, int n, int* nmax_out) {
  if (!probs || n < 1) return fail(b, GATO_E_INVALID, "need at least one problem");
  if (n > b->max_batch) return fail(b, GATO_E_INVALID, "more problems than max_batch");
  if (b->pending) {
    gato_status s = gato_sync(b, -1);
    if (s != GATO_OK) return s;
  }
  for (int i = 0; i < n; ++i) {
    gato_status s = validate_problem(b, probs[i], i);
    if (s != GATO_OK) return s;
  }
  b->copy_back.clear();
  b->h2d_bytes = b->d2h_bytes = 0;
  int nmax = 1;
  size_t staged = 0;
  for (int i = 0; i < n; ++i) {
    const gato_problem& p = probs[i];
    const int dof = b->model_dof[p.model], nx = 2 * dof, nu = dof, N = p.N;
    ProbDesc& d = b->probs_h[i];
    std::memset(&d, 0, sizeof(d));
    d.model = p.model;
    d.N = N;
    d.cost_kind = p.cost_kind;
    d.dof = dof;
    d.dt = p.dt;
    for (int k = 0; k < 6; ++k) d.w[k] = p.w[k];
    for (int k = 0; k < 3; ++k) d.fext[k] = p.f_ext[k];
    nmax = std::max(nmax, N);
    if (p.mem == GATO_MEM_DEVICE) {
      d.x_s = p.x_s;
      d.x_ref = p.cost_kind == GATO_COST_JOINT ? p.x_ref : nullptr;
      d.ee_ref = p.cost_kind == GATO_COST_EE ? p.ee_ref : nullptr;
      d.X = p.X;
      d.U = p.U;
      d.lam = p.lambda;
    } else {
      const size_t base = (size_t)i * b->stage_stride;
      float* h = b->stage_h + base;
      float* dv = b->stage_d + base;
      const size_t K = N + 1;
      size_t o = 0;
      std::memcpy(h + o, p.x_s, nx * sizeof(float));
      d.x_s = dv + o;
      o += 16;
      if (p.cost_kind == GATO_COST_JOINT) {
        std::memcpy(h + o, p.x_ref, K * nx * sizeof(float));
        d.x_ref = dv + o;
      } else {
        std::memcpy(h + o, p.ee_ref, K * 3 * sizeof(float));
        d.ee_ref = dv + o;
      }
      o += K * XM;
      const size_t oX = o;
      std::memcpy(h + o, p.X, K * nx * sizeof(float));
      d.X = dv + o;
      o += K * XM;
      std::memcpy(h + o, p.U, (size_t)N * nu * sizeof(float));
      d.U = dv + o;
      o += (size_t)N * QM;
      if (p.lambda) {
        std::memcpy(h + o, p.lambda, K * nx * sizeof(float));
        d.lam = dv + o;
      } else {
        d.lam = nullptr;
      }
      o += K * XM;
      HostCopyBack cb{p.X, p.U, p.lambda, K * nx, (size_t)N * nu, base + oX,
                      base + oX + K * XM, base + oX + K * XM + (size_t)N * QM, base + o};
      b->copy_back.push_back(cb);
      staged = std::max(staged, base + o);
      b->h2d_bytes += (int64_t)(nx + (p.cost_kind == GATO_COST_JOINT ? K * nx : K * 3) + K * nx +
                                (size_t)N * nu + (p.lambda ? K * nx : 0)) * 4;
      b->d2h_bytes += (int64_t)(K * nx + (size_t)N * nu + (p.lambda ? K * nx : 0)) * 4;
    }
  }
  // grouped by cluster size, longest horizon first within a group: long solves
  // start in the first wave
  b->N_h.resize(n);
  for (int i = 0; i < n; ++i) b->N_h[i] = probs[i].N;
  b->cur_plan = plan_for(b, n, nmax);
  order_solves(b->N_h.data(), n, b->order_h, b->cur_plan);
  cudaError_t e;
  if (staged > 0) {
    e = cudaMemcpyAsync(b->stage_d, b->stage_h, staged * sizeof(float), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "stage problems");
  }
  e = cudaMemcpyAsync(b->probs_d, b->probs_h, n * sizeof(ProbDesc), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "copy descriptors");
  e = cudaMemcpyAsync(b->order_d, b->order_h, n * sizeof(int), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "copy order");
  *nmax_out = nmax;
  return GATO_OK;
}

gato_status finish_launch(gato_batch* b, int n, gato_result* results) {
  cudaError_t e = cudaMemcpyAsync(b->res_h, b->res_d, n * sizeof(Result), cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "copy results");
  if (!b->copy_back.empty()) {
    size_t hi = 0;
    for (auto& c : b->copy_back) hi = std::max(hi, c.end);
    e = cudaMemcpyAsync(b->stage_h, b->stage_d, hi * sizeof(float), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "copy solutions");
  }
  b->d2h_bytes += (int64_t)n * sizeof(Result);
  e = cudaEventRecord(b->done, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "record completion");
  b->last_n = n;
  b->pending = true;
  if (results) {
    gato_status s = gato_sync(b, -1);
    if (s != GATO_OK) return s;
    return gato_get_results(b, results, n);
  }
  return GATO_OK;
}

// The fused launches of a prepared call (descriptors and order on the device).
cudaError_t launch_solve(gato_batch* b, int n, int nmax, int iters) {
  FusedLaunch a;
  a.probs = b->probs_d;
  a.models = b->models_d;
  a.order = b->order_d;
  a.results = b->res_d;
  a.ws = b->ws_d;
  a.ws_stride = b->ws_stride;
  a.layout = b->layout;
  a.n = n;
  a.nmax = nmax;
  a.csize = 1;
  a.iters = iters;
  a.prm = to_params(b->params, iters);
  a.timing = b->timing_d;
  a.itlog = b->itlog_d;
  a.itlog_iters = b->itlog_iters;
  a.variant = 0;
  return launch_fused_grouped(a, b->order_h, b->order_d, b->N_h.data(), n, b->stream, b->cur_plan);
}

// Copies of the iterates (X, U, lambda) of a call's problems, so that the
// autotuner can start every timed run from the same point.
struct IterateSnapshot {
  std::vector<std::vector<float>> host;
  float* dev = nullptr;
  std::vector<size_t> off;
  ~IterateSnapshot() { cudaFree(dev); }
};

size_t iterate_floats(const gato_batch* b, const gato_problem& p, int part) {
  const size_t nx = 2 * b->model_dof[p.model], K = p.N + 1;
  return part == 1 ? (size_t)p.N * (nx / 2) : K * nx;
}

float* iterate_ptr(const gato_problem& p, int part) {
  return part == 0 ? p.X : part == 1 ? p.U : p.lambda;
}

gato_status snapshot_take(gato_batch* b, const gato_problem* p, int n, IterateSnapshot& s) {
  size_t total = 0;
  s.off.assign((size_t)n * 3, 0);
  s.host.assign((size_t)n * 3, {});
  for (int i = 0; i < n; ++i)
    for (int part = 0; part < 3; ++part) {
      if (!iterate_ptr(p[i], part)) continue;
      const size_t m = iterate_floats(b, p[i], part);
      if (p[i].mem == GATO_MEM_DEVICE) {
        s.off[i * 3 + part] = total;
        total += m;
      } else {
        s.host[i * 3 + part].assign(iterate_ptr(p[i], part), iterate_ptr(p[i], part) + m);
      }
    }
  if (total && cudaMalloc(&s.dev, total * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(b, GATO_E_NOMEM, "autotune snapshot");
  }
  for (int i = 0; i < n; ++i)
    for (int part = 0; part < 3; ++part)
      if (iterate_ptr(p[i], part) && p[i].mem == GATO_MEM_DEVICE &&
          cudaMemcpyAsync(s.dev + s.off[i * 3 + part], iterate_ptr(p[i], part),
                          iterate_floats(b, p[i], part) * sizeof(float), cudaMemcpyDeviceToDevice,
                          b->stream) != cudaSuccess)
        return cuda_fail(b, cudaGetLastError(), "autotune snapshot");
  return GATO_OK;
}

gato_status snapshot_restore(gato_batch* b, const gato_problem* p, int n, const IterateSnapshot& s) {
  if (b->pending) {
    gato_status st = gato_sync(b, -1);
    if (st != GATO_OK) return st;
  }
  for (int i = 0; i < n; ++i)
    for (int part = 0; part < 3; ++part) {
      float* dst = iterate_ptr(p[i], part);
      if (!dst) continue;
      const size_t m = iterate_floats(b, p[i], part);
      if (p[i].mem == GATO_MEM_DEVICE) {
        if (cudaMemcpyAsync(dst, s.dev + s.off[i * 3 + part], m * sizeof(float), cudaMemcpyDeviceToDevice,
                            b->stream) != cudaSuccess)
          return cuda_fail(b, cudaGetLastError(), "autotune restore");
      } else {
        std::memcpy(dst, s.host[i * 3 + part].data(), m * sizeof(float));
      }
    }
  return GATO_OK;
}

}  // namespace

// Helpers for the serving loop (gato_server.cu), which keeps its model table
// and parameters in a one-solve batch.
namespace gato {
gato_status batch_validate_problem(gato_batch* b, const gato_problem& p) { return validate_problem(b, p, 0); }
const DevModel* batch_models_device(const gato_batch* b) { return b->models_d; }
int batch_model_dof(const gato_batch* b, int model) { return b->model_dof[model]; }
int batch_n_models(const gato_batch* b) { return b->n_models; }
Params batch_params(const gato_batch* b, int iters) { return to_params(b->params, iters); }
}  // namespace gato

extern "C" {

void gato_default_params(gato_solver_params* o) {
  if (!o) return;
  o->mu = 10.f;
  o->beta = 2.f;
  o->n_alpha = 8;
  o->pcg_eps = 1e-6f;
  o->pcg_max_iter = 1000;
  o->precond = GATO_PRECOND_STAIR;
  o->kkt_tol = 0.f;
  o->linsolve = GATO_LINSOLVE_PCG;
  o->rho_adapt = 0;
  o->precision = GATO_PRECISION_ESCALATE;
}

const char* gato_status_string(gato_status s) {
  switch (s) {
    case GATO_OK: return "ok";
    case GATO_E_INVALID: return "invalid argument";
    case GATO_E_NOMEM: return "out of memory";
    case GATO_E_CUDA: return "CUDA error";
    case GATO_E_TIMEOUT: return "timeout";
    case GATO_E_BUSY: return "busy";
  }
  return "unknown status";
}

const char* gato_last_error(const gato_batch* b) { return b ? b->err.c_str() : "no batch"; }

gato_status gato_create_batch(const gato_batch_desc* desc, void* cuda_stream, gato_batch** out) {
  if (!out) return GATO_E_INVALID;
  *out = nullptr;
  if (!desc || !desc->models) return GATO_E_INVALID;
  if (desc->max_batch < 1 || desc->max_horizon < 1 || desc->max_horizon > NMAX_LIMIT ||
      desc->n_models < 1 || desc->n_models > 8)
    return GATO_E_INVALID;
  gato_batch* b = new (std::nothrow) gato_batch();
  if (!b) return GATO_E_NOMEM;
  b->max_batch = desc->max_batch;
  b->max_horizon = desc->max_horizon;
  b->n_models = desc->n_models;
  b->params = desc->params;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  std::string why;
  for (int i = 0; i < desc->n_models; ++i) {
    if (!convert_model(desc->models[i], b->models_h[i], why)) {
      delete b;
      return GATO_E_INVALID;
    }
    b->model_dof[i] = desc->models[i].dof;
  }
  if (validate_params(b, desc->params) != GATO_OK) {
    delete b;
    return GATO_E_INVALID;
  }
  const int nmax = desc->max_horizon;
  b->layout = ws_layout(nmax, false, false);
  b->ws_stride = b->layout.total;
  b->plain_layout = ws_layout(nmax, true, true);
  b->stage_stride = stage_floats(nmax);
  const size_t nb = b->max_batch;
  bool ok = true;
  ok = ok && cudaMalloc(&b->models_d, 8 * sizeof(DevModel)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->probs_d, nb * sizeof(ProbDesc)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->order_d, nb * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->res_d, nb * sizeof(Result)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->ws_d, nb * b->ws_stride * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->plain_ws_d, b->plain_layout.total * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->stage_d, nb * b->stage_stride * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->probs_h, nb * sizeof(ProbDesc)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->order_h, nb * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->res_h, nb * sizeof(Result)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->stage_h, nb * b->stage_stride * sizeof(float)) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 7 && ok; ++i)
    ok = cudaStreamCreateWithFlags(&b->aux[i], cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < 8 && ok; ++i)
    ok = cudaEventCreateWithFlags(&b->fork_ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gato_destroy_batch(b);
    return GATO_E_NOMEM;
  }
  if (cudaMemcpy(b->models_d, b->models_h, 8 * sizeof(DevModel), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->ws_d, 0, nb * b->ws_stride * sizeof(float)) != cudaSuccess ||
      cudaMemset(b->plain_ws_d, 0, b->plain_layout.total * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    gato_destroy_batch(b);
    return GATO_E_CUDA;
  }
  *out = b;
  return GATO_OK;
}

void gato_destroy_batch(gato_batch* b) {
  if (!b) return;
  if (b->pending && b->done) cudaEventSynchronize(b->done);
  cudaFree(b->models_d);
  cudaFree(b->probs_d);
  cudaFree(b->order_d);
  cudaFree(b->res_d);
  cudaFree(b->ws_d);
  cudaFree(b->plain_ws_d);
  cudaFree(b->stage_d);
  cudaFree(b->timing_d);
  cudaFree(b->itlog_d);
  cudaFreeHost(b->probs_h);
  cudaFreeHost(b->order_h);
  cudaFreeHost(b->res_h);
  cudaFreeHost(b->stage_h);
  if (b->done) cudaEventDestroy(b->done);
  for (int i = 0; i < 7; ++i)
    if (b->aux[i]) cudaStreamDestroy(b->aux[i]);
  for (int i = 0; i < 8; ++i)
    if (b->fork_ev[i]) cudaEventDestroy(b->fork_ev[i]);
  delete b;
}

gato_status gato_solve(gato_batch* b, const gato_problem* problems, int32_t n,
                       int32_t max_sqp_iters, gato_result* results) {
  if (!b) return GATO_E_INVALID;
  if (max_sqp_iters < 1) return fail(b, GATO_E_INVALID, "max_sqp_iters must be >= 1");
  int nmax = 0;
  gato_status s = prepare(b, problems, n, &nmax);
  if (s != GATO_OK) return s;
  cudaError_t e = launch_solve(b, n, nmax, max_sqp_iters);
  if (e != cudaSuccess) return cuda_fail(b, e, "launch fused kernel");
  return finish_launch(b, n, results);
}

gato_status gato_step(gato_batch* b, const gato_problem* problems, int32_t n, gato_result* results) {
  return gato_solve(b, problems, n, 1, results);
}

gato_status gato_solve_plain(gato_batch* b, const gato_problem* problems, int32_t n,
                             int32_t max_sqp_iters, gato_result* results) {
  if (!b) return GATO_E_INVALID;
  if (max_sqp_iters < 1) return fail(b, GATO_E_INVALID, "max_sqp_iters must be >= 1");
  int nmax = 0;
  gato_status s = prepare(b, problems, n, &nmax);
  if (s != GATO_OK) return s;
  const Params prm = to_params(b->params, max_sqp_iters);
  for (int i = 0; i < n; ++i) {
    cudaError_t e = launch_plain(b->probs_d, b->models_d, b->res_d, i, b->N_h[i], b->plain_ws_d,
                                 b->plain_layout, b->max_horizon, max_sqp_iters, prm, -1, b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "launch plain stages");
  }
  return finish_launch(b, n, results);
}

gato_status gato_sync(gato_batch* b, int64_t timeout_us) {
  if (!b) return GATO_E_INVALID;
  if (!b->pending) return GATO_OK;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      b->pending = false;
      return cuda_fail(b, e, "wait for batch");
    }
    if (timeout_us >= 0) {
      const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                          std::chrono::steady_clock::now() - t0).count();
      if (us >= timeout_us) return fail(b, GATO_E_TIMEOUT, "sync deadline passed");
    }
    std::this_thread::yield();
  }
  b->pending = false;
  // scatter host outputs: X, U, lambda from the staging copy
  for (auto& c : b->copy_back) {
    std::memcpy(c.X, b->stage_h + c.offX, c.nX * sizeof(float));
    std::memcpy(c.U, b->stage_h + c.offU, c.nU * sizeof(float));
    if (c.lam) std::memcpy(c.lam, b->stage_h + c.offL, c.nX * sizeof(float));
  }
  b->copy_back.clear();
  return GATO_OK;
}

gato_status gato_get_results(gato_batch* b, gato_result* out, int32_t n) {
  if (!b || !out) return GATO_E_INVALID;
  if (b->pending) return fail(b, GATO_E_BUSY, "call gato_sync first");
  if (n > b->last_n) return fail(b, GATO_E_INVALID, "more results requested than solves");
  for (int i = 0; i < n; ++i) {
    out[i].flags = b->res_h[i].flags;
    out[i].sqp_iters = b->res_h[i].sqp_iters;
    out[i].pcg_iters = b->res_h[i].pcg_iters;
    out[i].kkt_residual = b->res_h[i].kkt;
    out[i].merit = b->res_h[i].merit;
  }
  return GATO_OK;
}

gato_status gato_last_transfer_bytes(const gato_batch* b, int64_t* h2d, int64_t* d2h) {
  if (!b) return GATO_E_INVALID;
  if (h2d) *h2d = b->h2d_bytes;
  if (d2h) *d2h = b->d2h_bytes;
  return GATO_OK;
}

int64_t gato_debug_layout(const gato_batch* b, int64_t* o) {
  if (!b || !o) return -1;
  const WsLayout& L = b->plain_layout;
  const size_t K = b->max_horizon + 1;
  const size_t v[25] = {L.X,  L.U,  L.dX, L.dU, L.Fq, L.Fv, L.Mi, L.qdd, L.dT, L.Qi, L.Ri, L.qg, L.rg,
                        L.cv, L.Jk, L.Li, L.LV, L.Dm, L.Lm, L.Pm, L.vec, L.vec + NVEC * (K + 2) * VW,
                        L.Dx, L.Du, L.nu};
  for (int i = 0; i < 25; ++i) o[i] = (int64_t)v[i];
  return (int64_t)L.total;
}

gato_status gato_debug_plain_stage(gato_batch* b, const gato_problem* problems, int32_t stop_stage,
                                   float* ws_out, int64_t ws_floats) {
  if (!b || !ws_out) return GATO_E_INVALID;
  if (stop_stage < PS_MASS || stop_stage > PS_ACCEPT) return fail(b, GATO_E_INVALID, "bad stage");
  if (ws_floats < (int64_t)b->plain_layout.total) return fail(b, GATO_E_INVALID, "ws_out too small");
  int nmax = 0;
  gato_status s = prepare(b, problems, 1, &nmax);
  if (s != GATO_OK) return s;
  const Params prm = to_params(b->params, 1);
  cudaError_t e = launch_plain(b->probs_d, b->models_d, b->res_d, 0, b->N_h[0], b->plain_ws_d,
                               b->plain_layout, b->max_horizon, 1, prm, stop_stage, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "launch plain stages");
  e = cudaMemcpyAsync(ws_out, b->plain_ws_d, b->plain_layout.total * sizeof(float),
                      cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "copy workspace");
  e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "stage run");
  b->copy_back.clear();
  return GATO_OK;
}

gato_status gato_debug_stage_cycles(gato_batch* b, int32_t enable, int64_t* cycles, int32_t n) {
  if (!b) return GATO_E_INVALID;
  if (b->pending) {
    gato_status s = gato_sync(b, -1);
    if (s != GATO_OK) return s;
  }
  const size_t bytes = (size_t)b->max_batch * T_COUNT * sizeof(long long);
  if (enable) {
    if (!b->timing_d && cudaMalloc(&b->timing_d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(b, GATO_E_NOMEM, "timing buffer");
    }
    if (cudaMemsetAsync(b->timing_d, 0, bytes, b->stream) != cudaSuccess) return GATO_E_CUDA;
    return GATO_OK;
  }
  if (!b->timing_d) return fail(b, GATO_E_INVALID, "stage timing was not enabled");
  if (cycles) {
    if (n < 1 || n > b->max_batch) return fail(b, GATO_E_INVALID, "bad solve count");
    std::vector<long long> h((size_t)n * T_COUNT);
    if (cudaMemcpy(h.data(), b->timing_d, h.size() * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
      return GATO_E_CUDA;
    for (size_t i = 0; i < h.size(); ++i) cycles[i] = h[i];
  }
  cudaFree(b->timing_d);
  b->timing_d = nullptr;
  return GATO_OK;
}

gato_status gato_debug_iteration_log(gato_batch* b, int32_t enable, int32_t max_iters, int32_t* log,
                                     int32_t n) {
  if (!b) return GATO_E_INVALID;
  if (b->pending) {
    gato_status s = gato_sync(b, -1);
    if (s != GATO_OK) return s;
  }
  if (enable) {
    if (max_iters < 1) return fail(b, GATO_E_INVALID, "max_iters must be >= 1");
    cudaFree(b->itlog_d);
    b->itlog_d = nullptr;
    b->itlog_iters = 0;
    const size_t bytes = (size_t)b->max_batch * max_iters * ITLOG_W * sizeof(int);
    if (cudaMalloc(&b->itlog_d, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(b, GATO_E_NOMEM, "iteration log");
    }
    if (cudaMemsetAsync(b->itlog_d, 0, bytes, b->stream) != cudaSuccess) return GATO_E_CUDA;
    b->itlog_iters = max_iters;
    return GATO_OK;
  }
  if (!b->itlog_d) return fail(b, GATO_E_INVALID, "the iteration log was not enabled");
  if (log) {
    if (n < 1 || n > b->max_batch) return fail(b, GATO_E_INVALID, "bad solve count");
    if (max_iters != b->itlog_iters) return fail(b, GATO_E_INVALID, "max_iters differs from the enabled log");
    if (cudaMemcpy(log, b->itlog_d, (size_t)n * max_iters * ITLOG_W * sizeof(int), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return GATO_E_CUDA;
  }
  cudaFree(b->itlog_d);
  b->itlog_d = nullptr;
  b->itlog_iters = 0;
  return GATO_OK;
}

struct gato_graph {
  gato_batch* b = nullptr;
  int n = 0;
  ProbDesc* probs_d = nullptr;
  int* order_d = nullptr;
  Result* res_d = nullptr;
  Result* res_h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool pending = false;
};

void gato_graph_destroy(gato_graph* g) {
  if (!g) return;
  if (g->pending && g->out) cudaEventSynchronize(g->out);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->in) cudaEventDestroy(g->in);
  if (g->out) cudaEventDestroy(g->out);
  if (g->stream) cudaStreamDestroy(g->stream);
  cudaFree(g->probs_d);
  cudaFree(g->order_d);
  cudaFree(g->res_d);
  cudaFreeHost(g->res_h);
  delete g;
}

gato_status gato_graph_create(gato_batch* b, const gato_problem* problems, int32_t n,
                              int32_t max_sqp_iters, gato_graph** out) {
  if (!out) return GATO_E_INVALID;
  *out = nullptr;
  if (!b) return GATO_E_INVALID;
  if (max_sqp_iters < 1) return fail(b, GATO_E_INVALID, "max_sqp_iters must be >= 1");
  if (!problems || n < 1 || n > b->max_batch) return fail(b, GATO_E_INVALID, "bad problem count");
  for (int i = 0; i < n; ++i)
    if (problems[i].mem != GATO_MEM_DEVICE)
      return fail(b, GATO_E_INVALID, "a captured solve needs device problems");
  int nmax = 0;
  gato_status s = prepare(b, problems, n, &nmax);
  if (s != GATO_OK) return s;
  gato_graph* g = new (std::nothrow) gato_graph();
  if (!g) return GATO_E_NOMEM;
  g->b = b;
  g->n = n;
  bool ok = cudaMalloc(&g->probs_d, n * sizeof(ProbDesc)) == cudaSuccess &&
            cudaMalloc(&g->order_d, n * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&g->res_d, n * sizeof(Result)) == cudaSuccess &&
            cudaMallocHost(&g->res_h, n * sizeof(Result)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->out, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gato_graph_destroy(g);
    return fail(b, GATO_E_NOMEM, "graph buffers");
  }
  // the graph owns its descriptors: later calls on the batch rewrite the batch's
  cudaError_t e = cudaMemcpyAsync(g->probs_d, b->probs_h, n * sizeof(ProbDesc), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->order_d, b->order_h, n * sizeof(int), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  size_t smem = 0;
  for (int i = 0; i < n; ++i)
    smem = std::max(smem, fused_smem_bytes(problems[i].N, cluster_size(problems[i].N, b->cur_plan.knots_per_cta,
                                                                        b->cur_plan.cluster)));
  if (e == cudaSuccess) e = configure_fused(smem);
  if (e != cudaSuccess) {
    gato_graph_destroy(g);
    return cuda_fail(b, e, "graph set-up");
  }
  b->copy_back.clear();
  FusedLaunch a;
  a.probs = g->probs_d;
  a.models = b->models_d;
  a.order = g->order_d;
  a.results = g->res_d;
  a.ws = b->ws_d;
  a.ws_stride = b->ws_stride;
  a.layout = b->layout;
  a.n = n;
  a.nmax = nmax;
  a.csize = 1;
  a.iters = max_sqp_iters;
  a.prm = to_params(b->params, max_sqp_iters);
  a.timing = nullptr;
  a.variant = 0;
  e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = launch_fused_grouped(a, b->order_h, g->order_d, b->N_h.data(), n, g->stream, b->cur_plan);
    if (le == cudaSuccess)
      le = cudaMemcpyAsync(g->res_h, g->res_d, n * sizeof(Result), cudaMemcpyDeviceToHost, g->stream);
    e = cudaStreamEndCapture(g->stream, &g->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gato_graph_destroy(g);
    return cuda_fail(b, e, "graph capture");
  }
  *out = g;
  return GATO_OK;
}

gato_status gato_graph_wait(gato_graph* g, gato_result* results) {
  if (!g) return GATO_E_INVALID;
  if (g->pending) {
    cudaError_t e = cudaEventSynchronize(g->out);
    g->pending = false;
    if (e != cudaSuccess) return cuda_fail(g->b, e, "graph replay");
  }
  if (results)
    for (int i = 0; i < g->n; ++i) {
      results[i].flags = g->res_h[i].flags;
      results[i].sqp_iters = g->res_h[i].sqp_iters;
      results[i].pcg_iters = g->res_h[i].pcg_iters;
      results[i].kkt_residual = g->res_h[i].kkt;
      results[i].merit = g->res_h[i].merit;
    }
  return GATO_OK;
}

gato_status gato_graph_launch(gato_graph* g, gato_result* results) {
  if (!g) return GATO_E_INVALID;
  gato_batch* b = g->b;
  if (g->pending) {
    gato_status s = gato_graph_wait(g, nullptr);
    if (s != GATO_OK) return s;
  }
  if (b->pending) {
    gato_status s = gato_sync(b, -1);
    if (s != GATO_OK) return s;
  }
  // ordered after earlier work on the batch's stream, and later work after it
  cudaError_t e = cudaEventRecord(g->in, b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, g->stream);
  if (e == cudaSuccess) e = cudaEventRecord(g->out, g->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, g->out, 0);
  if (e != cudaSuccess) return cuda_fail(b, e, "graph launch");
  g->pending = true;
  return results ? gato_graph_wait(g, results) : GATO_OK;
}

gato_status gato_set_launch_config(gato_batch* b, const gato_launch_config* cfg) {
  if (!b) return GATO_E_INVALID;
  if (!cfg) {
    b->forced = false;
    return GATO_OK;
  }
  if (cfg->variant < 0 || cfg->variant > 2 || cfg->knots_per_cta == 1 || cfg->knots_per_cta < 0 ||
      cfg->knots_per_cta > KPC_MAX || cfg->cluster < 0 || cfg->cluster > 8)
    return fail(b, GATO_E_INVALID, "launch config out of range");
  b->forced = true;
  b->forced_plan = LaunchPlan();
  b->forced_plan.variant = cfg->variant;
  b->forced_plan.knots_per_cta = cfg->knots_per_cta;
  b->forced_plan.cluster = cfg->cluster;
  return GATO_OK;
}

gato_status gato_query_launch(int32_t N, int32_t n_solves, const gato_launch_config* cfg,
                              gato_launch_info* out) {
  if (!out || N < 1 || N > NMAX_LIMIT || n_solves < 1) return GATO_E_INVALID;
  LaunchPlan p;
  if (cfg) {
    if (cfg->variant < 0 || cfg->variant > 2 || cfg->knots_per_cta == 1 || cfg->knots_per_cta < 0 ||
        cfg->knots_per_cta > KPC_MAX || cfg->cluster < 0 || cfg->cluster > 8)
      return GATO_E_INVALID;
    p.variant = cfg->variant;
    p.knots_per_cta = cfg->knots_per_cta;
    p.cluster = cfg->cluster;
  }
  const int c = cluster_size(N, p.knots_per_cta, p.cluster);
  const size_t smem = fused_smem_bytes(N, c);
  if (smem > SMEM_LIMIT_BYTES) return GATO_E_INVALID;
  const bool reg = !use_throughput_variant(n_solves, c, p.variant, smem);
  int active = 0;
  const cudaError_t e = fused_active_clusters(N, c, reg, &active);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GATO_E_CUDA;
  }
  out->ctas_per_solve = c;
  out->variant = reg ? 1 : 2;
  out->smem_bytes = (int32_t)smem;
  out->max_resident_solves = active;
  return GATO_OK;
}

gato_status gato_autotune(gato_batch* b, const gato_problem* problems, int32_t n, int32_t max_sqp_iters,
                          int32_t reps, gato_launch_config* best, float* best_ms) {
  if (!b) return GATO_E_INVALID;
  if (max_sqp_iters < 1 || reps < 1) return fail(b, GATO_E_INVALID, "max_sqp_iters and reps must be >= 1");
  if (!problems || n < 1 || n > b->max_batch) return fail(b, GATO_E_INVALID, "bad problem count");
  for (int i = 0; i < n; ++i) {
    gato_status s = validate_problem(b, problems[i], i);
    if (s != GATO_OK) return s;
  }
  if (b->pending) {
    gato_status s = gato_sync(b, -1);
    if (s != GATO_OK) return s;
  }
  int nmax = 1;
  for (int i = 0; i < n; ++i) nmax = std::max(nmax, (int)problems[i].N);
  IterateSnapshot snap;
  gato_status s = snapshot_take(b, problems, n, snap);
  if (s != GATO_OK) return s;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
    if (t0) cudaEventDestroy(t0);
    cudaGetLastError();
    return fail(b, GATO_E_NOMEM, "autotune events");
  }
  const bool was_forced = b->forced;
  const LaunchPlan was_plan = b->forced_plan;
  // candidates: both kernel forms x knots per CTA; configurations that give
  // every solve the same cluster sizes as an earlier one are skipped
  const int kpcs[] = {0, 24, 17, 12, 9, 6};
  int cmax = 1;
  for (int i = 0; i < n; ++i) cmax = std::max(cmax, cluster_for(problems[i].N));
  struct Cand { int kpc, cluster; };
  std::vector<Cand> cands;
  for (int k : kpcs) cands.push_back({k, 0});
  for (int c = cmax; c <= 8; c *= 2) cands.push_back({0, c});  // one launch for the whole batch
  std::vector<std::vector<int>> seen;
  float best_t = -1.f;
  LaunchPlan best_p;
  gato_status st = GATO_OK;
  for (int variant = 1; variant <= 2 && st == GATO_OK; ++variant) {
    seen.clear();
    for (const Cand& cd : cands) {
      std::vector<int> sizes(n);
      size_t smem_max = 0;
      for (int i = 0; i < n; ++i) {
        sizes[i] = cluster_size(problems[i].N, cd.kpc, cd.cluster);
        smem_max = std::max(smem_max, fused_smem_bytes(problems[i].N, sizes[i]));
      }
      if (std::find(seen.begin(), seen.end(), sizes) != seen.end()) continue;
      seen.push_back(sizes);
      // the throughput form only pays when two CTAs fit an SM
      if (variant == 2 && 2 * (smem_max + 1024) > 233472) continue;
      b->forced = true;
      b->forced_plan = LaunchPlan();
      b->forced_plan.variant = variant;
      b->forced_plan.knots_per_cta = cd.kpc;
      b->forced_plan.cluster = cd.cluster;
      std::vector<float> ts;
      for (int r = 0; r <= reps && st == GATO_OK; ++r) {  // r = 0 warms up
        st = snapshot_restore(b, problems, n, snap);
        if (st != GATO_OK) break;
        int nm = 0;
        st = prepare(b, problems, n, &nm);
        if (st != GATO_OK) break;
        cudaError_t e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = launch_solve(b, n, nm, max_sqp_iters);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) {
          st = cuda_fail(b, e, "autotune run");
          break;
        }
        b->copy_back.clear();
        if (r > 0) ts.push_back(ms);
      }
      if (st != GATO_OK) break;
      std::sort(ts.begin(), ts.end());
      const float med = ts[ts.size() / 2];
      if (best_t < 0.f || med < best_t) {
        best_t = med;
        best_p = b->forced_plan;
      }
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  b->forced = was_forced;
  b->forced_plan = was_plan;
  gato_status rs = snapshot_restore(b, problems, n, snap);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess && rs == GATO_OK)
    rs = cuda_fail(b, cudaGetLastError(), "autotune restore");
  if (st != GATO_OK) return st;
  if (rs != GATO_OK) return rs;
  const int nb = pow2_bucket(n), nk = horizon_key(nmax);
  b->tuned.erase(std::remove_if(b->tuned.begin(), b->tuned.end(),
                                [&](const gato_batch::Tuned& t) { return t.n_bucket == nb && t.n_key == nk; }),
                 b->tuned.end());
  best_p.aux = nullptr;
  best_p.ev = nullptr;
  best_p.n_aux = 0;
  b->tuned.push_back({nb, nk, best_p});
  if (best) {
    best->variant = best_p.variant;
    best->knots_per_cta = best_p.knots_per_cta;
    best->cluster = best_p.cluster;
  }
  if (best_ms) *best_ms = best_t;
  return GATO_OK;
}

}  // extern "C"
