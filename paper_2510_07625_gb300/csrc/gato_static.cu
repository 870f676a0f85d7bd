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
constexpr size_t kWsStride = 43008;

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

// The call's descriptors, passed to a one-block kernel by value (kernel
// parameters travel with the launch itself), which stores them into the
// file-scope arrays ahead of the solve on the same stream: no host-to-device
// copy from pageable memory.
struct NoallocDescs {
  DevModel models[kMaxModels];
  ProbDesc probs[kMaxSolves];
  int order[kMaxSolves];
  int n_models, n;
};
static_assert(sizeof(NoallocDescs) <= 4096, "descriptors must fit the classic kernel-parameter limit");

__global__ void noalloc_store_descs(const NoallocDescs d) {
  const int t = threadIdx.x;
  if (t < d.n_models) g_models[t] = d.models[t];
  if (t < d.n) {
    g_probs[t] = d.probs[t];
    g_order[t] = d.order[t];
  }
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
  if (check_params(sp)) return GATO_E_INVALID;
  NoallocDescs D;
  std::memset(&D, 0, sizeof(D));
  D.n_models = n_models;
  D.n = n;
  int dofs[kMaxModels];
  for (int i = 0; i < n_models; ++i) {
    if (check_model(models[i], D.models[i])) return GATO_E_INVALID;
    dofs[i] = models[i].dof;
  }
  int Ns[kMaxSolves];
  for (int i = 0; i < n; ++i) {
    const gato_problem& p = problems[i];
    if (p.mem != GATO_MEM_DEVICE || check_problem(p, n_models, kMaxHorizon)) return GATO_E_INVALID;
    ProbDesc& d = D.probs[i];
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
  order_solves(Ns, n, D.order, LaunchPlan());
  DevicePtrs* P = nullptr;
  gato_status s = setup_device(&P);
  if (s != GATO_OK) return s;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  noalloc_store_descs<<<1, 32, 0, stream>>>(D);
  if (cudaGetLastError() != cudaSuccess) return GATO_E_CUDA;
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
  a.prm.escalate = sp.precision == GATO_PRECISION_ESCALATE;
  a.prm.high = sp.precision == GATO_PRECISION_HIGH;
  a.timing = nullptr;
  a.variant = 0;
  if (launch_fused_grouped(a, D.order, P->order, Ns, n, stream, LaunchPlan()) != cudaSuccess) {
    cudaGetLastError();
    return GATO_E_CUDA;
  }
  return GATO_OK;
}
