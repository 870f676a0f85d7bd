// Internal launch interface between the C ABI (gato_api.cu, gato_static.cu)
// and the kernels (gato_kernels.cu).  Not part of the public header.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/gato.h"
#include "gato_device.cuh"
#include "gato_phases.cuh"

namespace gato {

// Opt-in shared memory per CTA on sm_103a (227 KB).
constexpr size_t SMEM_LIMIT_BYTES = 232448;
// Largest horizon the library accepts (8 CTAs of KPC_MAX knots).
constexpr int NMAX_LIMIT = 256;

struct FusedLaunch {
  const ProbDesc* probs;   // device [n_total]
  const DevModel* models;  // device
  const int* order;        // device: solve index of each cluster
  Result* results;         // device [n_total]
  float* ws;               // device workspace base
  size_t ws_stride;        // floats per solve
  WsLayout layout;         // layout of one solve's workspace
  int n;                   // clusters (solves) in this launch
  int nmax;                // largest N in this launch (sets the shared-memory layout)
  int csize;               // CTAs per cluster
  int iters;
  Params prm;
  long long* timing;       // device [n_total][T_COUNT] cycle counters, or null
  int* itlog = nullptr;    // device [n_total][itlog_iters][ITLOG_W] iteration records, or null
  int itlog_iters = 0;
  int variant;             // 0 = automatic, 1 = register rows (1 CTA/SM), 2 = 2 CTAs/SM
  int resume = 0;          // high-precision kernel: resume the FP32 launch's hand-over records
};

// How solves map onto the GPU: the space the autotuner searches.
struct LaunchPlan {
  int variant = 0;        // 0 automatic, 1 block rows in registers (1 CTA/SM), 2 two CTAs/SM
  int knots_per_cta = 0;  // 0 = KPC_MAX; smaller values spread a solve over more CTAs
  int cluster = 0;        // > 0: every solve uses this many CTAs where it can (one launch)
  // optional fork streams: cluster-size groups run concurrently on these
  // (joined back into the caller's stream with the events)
  const cudaStream_t* aux = nullptr;
  const cudaEvent_t* ev = nullptr;  // [n_aux + 1]
  int n_aux = 0;
};

int num_sms();
bool use_throughput_variant(int n, int csize, int variant, size_t smem);

// CTAs per cluster for horizon N under a knots-per-CTA target (0 = KPC_MAX):
// at least cluster_for(N), at most 8, and never a CTA without knots.
int cluster_size(int N, int knots_per_cta, int cluster = 0);

// Sets the shared-memory attribute of both kernel forms for launches of up to
// `smem` bytes (done by the launcher on demand; call it before stream capture).
cudaError_t configure_fused(size_t smem);

// One persistent fused launch: n clusters of csize CTAs, one solve each.
// FP32 kernel, followed on the same stream by the high-precision kernel that
// resumes the escalated solves when the parameters allow escalation; the
// high-precision kernel alone in the high-precision mode.
cudaError_t launch_fused(const FusedLaunch& a, cudaStream_t s);

// The high-precision instantiations (gato_kernels_hp.cu): one launch, and the
// shared-memory attribute of both forms.
cudaError_t launch_fused_hp(const FusedLaunch& a, size_t smem, cudaStream_t s, bool reg);
cudaError_t configure_fused_hp(size_t smem);

// Launches the solves in `order_host` (sorted by cluster size, then horizon,
// both descending; order_dev is its device copy) as one launch per cluster
// size.  N_of[i] is the horizon of solve i.
cudaError_t launch_fused_grouped(FusedLaunch base, const int* order_host, const int* order_dev,
                                 const int* N_of, int n, cudaStream_t s, const LaunchPlan& plan);

// Sorts solve indices by (cluster size, horizon), both descending, stable.
void order_solves(const int* N_of, int n, int* order, const LaunchPlan& plan);

// Plain form: every stage of every SQP iteration of solve `b` is its own launch.
// `ws` must have the layout ws_layout(nmax, true, true).
cudaError_t launch_plain(const ProbDesc* probs, const DevModel* models, Result* results, int b,
                         int N_b, float* ws, const WsLayout& L, int nmax, int iters, const Params& prm,
                         int stop_stage, cudaStream_t s);

size_t fused_smem_bytes(int nmax, int csize);

// Clusters of csize CTAs of the fused kernel (latency form if reg) that the
// current device holds at once for a launch whose largest horizon is nmax.
cudaError_t fused_active_clusters(int nmax, int csize, bool reg, int* out);

// Host-side input checks shared by every entry point.  Each returns nullptr
// when its input is valid, else a short reason.  check_model also fills the
// device form of the model (padded to QM joints).  check_problem looks at the
// fields of one problem, not at the contents of its arrays.
const char* check_model(const gato_model_desc& d, DevModel& m);
const char* check_params(const gato_solver_params& p);
const char* check_problem(const gato_problem& p, int n_models, int max_horizon);

enum PlainStage : int {
  PS_LOAD = 0, PS_MASS, PS_FD, PS_VALUE, PS_TANGENT, PS_JAC, PS_KKT, PS_SCHUR, PS_BINV, PS_PCG,
  PS_RECOVER, PS_LS, PS_ACCEPT, PS_STORE, PS_COUNT
};

}  // namespace gato
