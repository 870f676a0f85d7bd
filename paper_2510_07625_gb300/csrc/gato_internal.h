// Internal launch interface between the C ABI (gato_api.cu) and the kernels
// (gato_kernels.cu).  Not part of the public header.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "gato_device.cuh"
#include "gato_phases.cuh"

namespace gato {

// Largest horizon whose Schur/preconditioner blocks fit in one CTA's shared memory.
constexpr int SMEM_BLOCKS_NMAX = 75;
// Opt-in shared memory per CTA on sm_103a (227 KB).
constexpr size_t SMEM_LIMIT_BYTES = 232448;
// Largest horizon the library accepts.
constexpr int NMAX_LIMIT = 256;

struct FusedLaunch {
  const ProbDesc* probs;   // device [n]
  const DevModel* models;  // device
  const int* order;        // device [n] or null
  Result* results;         // device [n]
  float* ws;               // device workspace base
  size_t ws_stride;        // floats per solve
  WsLayout layout;         // layout of one solve's workspace
  int n;                   // solves
  int nmax;                // largest N in this launch (sets shared-memory layout)
  int iters;
  Params prm;
  int threads;             // 0 = automatic
};

// One persistent fused launch: grid = n CTAs, one solve per CTA.
cudaError_t launch_fused(const FusedLaunch& a, cudaStream_t s);

// Plain form: every stage of every SQP iteration of solve `b` is its own launch.
// `ws` must have the layout ws_layout(nmax, true, true).
cudaError_t launch_plain(const ProbDesc* probs, const DevModel* models, Result* results, int b,
                         float* ws, const WsLayout& L, int nmax, int iters, const Params& prm,
                         int stop_stage, cudaStream_t s);

int fused_threads_for(int nmax);
size_t fused_smem_bytes(int nmax);

enum PlainStage : int {
  PS_LOAD = 0, PS_MASS, PS_FD, PS_VALUE, PS_TANGENT, PS_JAC, PS_KKT, PS_SCHUR, PS_BINV, PS_PCG,
  PS_RECOVER, PS_LS, PS_ACCEPT, PS_STORE, PS_COUNT
};

}  // namespace gato
