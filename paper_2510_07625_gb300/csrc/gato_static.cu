// gato_solve_noalloc: the batched SQP solve for callers that must not allocate
// device memory (declared in include/gato.h).
//
// It runs the same persistent fused kernel as gato_solve, but that kernel's
// scratch (the per-solve workspace), the solve descriptors, the models and the
// launch order live in file-scope __device__ arrays of fixed size, so the call
// performs no cudaMalloc/cudaFree and needs no gato_batch.  The arrays exist on
// every GPU that loads the library, for the life of the process, and every call
// shares them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gato.h"
#include "gato_internal.h"

using namespace gato;

namespace {

constexpr int kMaxSolves = 16;   // most solves per call
constexpr int kMaxHorizon = 64;  // largest N per solve
constexpr int kMaxModels = 8;
constexpr int kMaxDevices = 64;
// Floats of one solve's workspace at N = 64 (Schur blocks in shared memory);
// checked against ws_layout() at set-up.
constexpr size_t kWsStride = 40960;

static __device__ __align__(256) float g_scratch[kMaxSolves * kWsStride];
static __device__ __align__(256) ProbDesc g_probs[kMaxSolves];
static __device__ __align__(256) DevModel g_models[kMaxModels];
static __device__ __align__(256) int g_order[kMaxSolves];

struct DevicePtrs {
  bool ready = false;
  float* scratch = nullptr;
  ProbDesc* probs = nullptr;
  DevModel* models = nullptr;
  int* order = nullptr;
};
DevicePtrs g_ptrs[kMaxDevices];
std::mutex g_setup_mutex;

static_assert(sizeof(gato_result) == sizeof(Result), "result layout");

// Device addresses of the file-scope arrays, looked up once per device with
// that device current (a host-side use of the array names would not be a
// device address).
gato_status setup_device(DevicePtrs** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GATO_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DevicePtrs& p = g_ptrs[dev];
  if (!p.ready) {
    if (ws_layout(kMaxHorizon, false, false).total > kWsStride) return GATO_E_INVALID;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p.scratch), g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&p.probs), g_probs) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&p.models), g_models) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&p.order), g_order) != cudaSuccess) {
      cudaGetLastError();
      return GATO_E_CUDA;
    }
    p.ready = true;
  }
  *out = &p;
  return GATO_OK;
}

bool model_ok(const gato_model_desc& d, DevModel& m) {
  if (d.dof < 1 || d.dof > QM || !(d.gravity >= 0.f) || !std::isfinite(d.gravity)) return false;
  std::memset(&m, 0, sizeof(m));
  m.dof = d.dof;
  m.g = d.gravity;
  for (int i = 0; i < QM; ++i) {
    if (i >= d.dof) {
      m.axis[i] = 2;  // massless padding joint at the end effector
      continue;
    }
    if (d.axis[i] < 0 || d.axis[i] > 2 || !(d.link_len[i] >= 0.f) || !std::isfinite(d.link_len[i]) ||
        !(d.mass[i] > 0.f) || !std::isfinite(d.mass[i]))
      return false;
    m.axis[i] = d.axis[i];
    m.L[i] = d.link_len[i];
    m.m[i] = d.mass[i];
    for (int a = 0; a < 3; ++a) {
      const float c = d.com[3 * i + a], I = d.inertia[3 * i + a];
      if (!std::isfinite(c) || !(I >= 0.f) || !std::isfinite(I)) return false;
      m.com[3 * i + a] = c;
      m.Ic[3 * i + a] = I;
    }
  }
  return true;
}

bool problem_ok(const gato_problem& p, int n_models) {
  if (p.mem != GATO_MEM_DEVICE) return false;
  if (p.model < 0 || p.model >= n_models || p.N < 1 || p.N > kMaxHorizon) return false;
  if (!(p.dt > 0.f) || !std::isfinite(p.dt) || !p.x_s || !p.X || !p.U) return false;
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(p.w[i]) || p.w[i] < 0.f) return false;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(p.f_ext[i])) return false;
  const float wq = p.w[0], wqd = p.w[1], wr = p.w[2], ts = p.w[3], rho = p.w[5];
  if (!(wr > 0.f) || !(ts > 0.f)) return false;
  if (p.cost_kind == GATO_COST_JOINT) return p.x_ref && wq + rho > 0.f && wqd + rho > 0.f;
  if (p.cost_kind == GATO_COST_EE) return p.ee_ref && rho > 0.f && wqd + rho > 0.f;
  return false;
}

}  // namespace

extern "C" gato_status gato_solve_noalloc(const gato_model_desc* models, int32_t n_models,
                                          const gato_solver_params* params,
                                          const gato_problem* problems, int32_t n,
                                          int32_t max_sqp_iters, gato_result* results,
                                          void* cuda_stream) {
  if (!models || !params || !problems || !results) return GATO_E_INVALID;
  if (n < 1 || n > kMaxSolves || n_models < 1 || n_models > kMaxModels || max_sqp_iters < 1)
    return GATO_E_INVALID;
  const gato_solver_params& sp = *params;
  if (!(sp.mu >= 0.f) || !std::isfinite(sp.mu) || !(sp.beta > 1.f) || !std::isfinite(sp.beta) ||
      sp.n_alpha < 1 || sp.n_alpha > MAX_ALPHA || !(sp.pcg_eps > 0.f) || sp.pcg_max_iter < 1 ||
      (sp.precond != GATO_PRECOND_STAIR && sp.precond != GATO_PRECOND_JACOBI) ||
      (sp.linsolve != GATO_LINSOLVE_PCG && sp.linsolve != GATO_LINSOLVE_DIRECT) ||
      (sp.rho_adapt != 0 && sp.rho_adapt != 1) ||
      !std::isfinite(sp.kkt_tol))
    return GATO_E_INVALID;
  DevModel dm[kMaxModels];
  int dofs[kMaxModels];
  for (int i = 0; i < n_models; ++i) {
    if (!model_ok(models[i], dm[i])) return GATO_E_INVALID;
    dofs[i] = models[i].dof;
  }
  ProbDesc pd[kMaxSolves];
  int order[kMaxSolves];
  int Ns[kMaxSolves];
  for (int i = 0; i < n; ++i) {
    const gato_problem& p = problems[i];
    if (!problem_ok(p, n_models)) return GATO_E_INVALID;
    ProbDesc& d = pd[i];
    std::memset(&d, 0, sizeof(d));
    d.model = p.model;
    d.N = p.N;
    d.cost_kind = p.cost_kind;
    d.dof = dofs[p.model];
    d.dt = p.dt;
    for (int k = 0; k < 6; ++k) d.w[k] = p.w[k];
    for (int k = 0; k < 3; ++k) d.fext[k] = p.f_ext[k];
    d.x_s = p.x_s;
    d.x_ref = p.cost_kind == GATO_COST_JOINT ? p.x_ref : nullptr;
    d.ee_ref = p.cost_kind == GATO_COST_EE ? p.ee_ref : nullptr;
    d.X = p.X;
    d.U = p.U;
    d.lam = p.lambda;
    Ns[i] = p.N;
  }
  // grouped by cluster size, longest horizon first within a group
  order_solves(Ns, n, order, LaunchPlan());
  DevicePtrs* P = nullptr;
  gato_status s = setup_device(&P);
  if (s != GATO_OK) return s;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // pageable sources: each copy has consumed its host buffer when it returns
  if (cudaMemcpyAsync(P->models, dm, n_models * sizeof(DevModel), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(P->probs, pd, n * sizeof(ProbDesc), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(P->order, order, n * sizeof(int), cudaMemcpyHostToDevice, stream) != cudaSuccess) {
    cudaGetLastError();
    return GATO_E_CUDA;
  }
  FusedLaunch a;
  a.probs = P->probs;
  a.models = P->models;
  a.order = P->order;
  a.results = reinterpret_cast<Result*>(results);
  a.ws = P->scratch;
  a.ws_stride = kWsStride;
  a.layout = ws_layout(kMaxHorizon, false, false);
  a.n = n;
  a.nmax = 1;
  a.csize = 1;
  a.iters = max_sqp_iters;
  a.prm.mu = sp.mu;
  a.prm.beta = sp.beta;
  a.prm.n_alpha = sp.n_alpha;
  a.prm.pcg_eps = sp.pcg_eps;
  a.prm.pcg_max = sp.pcg_max_iter;
  a.prm.precond = sp.precond;
  a.prm.kkt_tol = sp.kkt_tol;
  a.prm.max_iter = max_sqp_iters;
  a.prm.linsolve = sp.linsolve;
  a.prm.rho_adapt = sp.rho_adapt;
  a.timing = nullptr;
  a.variant = 0;
  if (launch_fused_grouped(a, order, P->order, Ns, n, stream, LaunchPlan()) != cudaSuccess) {
    cudaGetLastError();
    return GATO_E_CUDA;
  }
  return GATO_OK;
}
