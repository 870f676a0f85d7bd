/*
 * gato.h -- C ABI of the batched SQP trajectory-optimisation library.
 *
 * Method: GATO, "GPU-Accelerated and Batched Trajectory Optimization for
 * Scalable Edge Model Predictive Control" (arXiv 2510.07625).  Each solve is
 * the direct multiple-shooting problem of Sec. II-A: states x_0..x_N, controls
 * u_0..u_{N-1}, dynamics x_{k+1} = f(x_k, u_k, h), x_0 = x_s, additive cost J.
 * One SQP iteration (Sec. II-A Steps 1-3, Alg. 1):
 *   1. linearise: defects e_k, A_k, B_k, cost gradient/Hessian (Eq. 1),
 *   2. reduce the KKT system (Eq. 2) to its Schur complement (Eq. 4-5) and
 *      solve it by PCG with the stair or block-Jacobi preconditioner (Eq. 6),
 *   3. recover dZ (Eq. 4) and take the parallel line search on the L1 merit
 *      (Eq. 3, Eq. 7).
 *
 * All compute runs in the library's own sm_103a CUDA kernels.  No call aborts,
 * traps or throws across this boundary: every entry point returns a
 * gato_status and the text of the last error is kept per batch.
 *
 * Layouts (all row-major, float32, sizes in the solve's own model sizes):
 *   nq = dof (1..7), nx = 2*nq (state [q; qd]), nu = nq (joint torques).
 *   x_s     [nx]             initial state
 *   x_ref   [(N+1)*nx]       joint-space target per knot   (cost_kind JOINT)
 *   ee_ref  [(N+1)*3]        end-effector target per knot  (cost_kind EE)
 *   X       [(N+1)*nx]       in: initial guess, out: final states
 *   U       [N*nu]           in: initial guess, out: final controls
 *   lambda  [(N+1)*nx]       in: multiplier warm start, out: last multiplier
 * Pointers in a gato_problem are all host or all device memory, as its
 * `mem` field says; the caller owns them and keeps them valid until the call
 * has completed (gato_sync, or a non-NULL results argument).
 */
#ifndef GATO_H_
#define GATO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GATO_OK = 0,
  GATO_E_INVALID = -1,   /* bad argument; nothing was launched */
  GATO_E_NOMEM = -2,     /* device or pinned allocation failed */
  GATO_E_CUDA = -3,      /* a CUDA call failed (message via gato_last_error) */
  GATO_E_TIMEOUT = -4,   /* gato_sync deadline passed; work still in flight */
  GATO_E_BUSY = -5       /* serving queue full / no free slot */
} gato_status;

/* Per-solve outcome flags (gato_result.flags). */
enum {
  GATO_SOLVE_CONVERGED = 1,  /* KKT residual reached the tolerance */
  GATO_SOLVE_MAXITER = 2,    /* tolerance set and not reached */
  GATO_SOLVE_LSFAIL = 4,     /* some line search found no merit decrease (step rejected) */
  GATO_SOLVE_PCG_MAXIT = 8,  /* some PCG solve stopped at its iteration cap */
  GATO_SOLVE_NONFINITE = 16  /* a non-finite value appeared; the solve stopped */
};

enum { GATO_COST_JOINT = 0, GATO_COST_EE = 1 };
enum { GATO_PRECOND_STAIR = 0, GATO_PRECOND_JACOBI = 1 };
enum { GATO_MEM_HOST = 0, GATO_MEM_DEVICE = 1 };

/* Serial revolute chain (Sec. II-A "discrete-time dynamical system"; the
 * paper's robots are modelled the same way by its dynamics library).  Joint i
 * rotates about axis[i] of its own frame; its origin sits at the parent origin
 * plus (0, 0, link_len[i-1]) in the parent frame (joint 0 at the base origin);
 * link i has its centre of mass at com[3i..3i+2] (link frame) and principal
 * moments inertia[3i..3i+2] about it; the end effector is at
 * (0, 0, link_len[dof-1]) of the last frame; gravity acts along -z. */
typedef struct {
  int32_t dof;             /* 1..7 */
  int32_t axis[7];         /* 0 = x, 1 = y, 2 = z */
  float link_len[7];
  float mass[7];
  float com[21];
  float inertia[21];
  float gravity;           /* m/s^2, > 0 */
} gato_model_desc;

/* Solver hyperparameters (the paper defers their values to its code; the
 * defaults from gato_default_params are this library's readings). */
typedef struct {
  float mu;                /* L1 merit penalty (Eq. 3), default 10 */
  float beta;              /* line-search ratio, alpha_i = beta^-i (Eq. 7), default 2 */
  int32_t n_alpha;         /* number of trial step lengths A, 1..16, default 8 */
  float pcg_eps;           /* PCG relative preconditioned residual, default 1e-6 */
  int32_t pcg_max_iter;    /* PCG iteration cap, default 1000 */
  int32_t precond;         /* GATO_PRECOND_STAIR (Eq. 6) or GATO_PRECOND_JACOBI */
  float kkt_tol;           /* > 0: a solve stops once its KKT residual <= kkt_tol */
} gato_solver_params;

typedef struct {
  int32_t max_batch;       /* most solves per call */
  int32_t max_horizon;     /* largest N of any solve, 1..256 */
  int32_t n_models;        /* 1..8 */
  const gato_model_desc* models;   /* host array, copied at create */
  gato_solver_params params;
} gato_batch_desc;

/* One solve (Sec. II-A problem statement; Alg. 1 arguments X_init, U_init, N). */
typedef struct {
  int32_t model;           /* index into the batch's models */
  int32_t N;               /* horizon, 1..max_horizon */
  float dt;                /* time step h > 0 */
  int32_t cost_kind;       /* GATO_COST_JOINT or GATO_COST_EE */
  float w[6];              /* weights: q, qd, u, terminal scale, ee, rho (diag damping) */
  int32_t mem;             /* GATO_MEM_HOST or GATO_MEM_DEVICE for every pointer below */
  const float* x_s;
  const float* x_ref;      /* used when cost_kind == JOINT, else may be NULL */
  const float* ee_ref;     /* used when cost_kind == EE, else may be NULL */
  float* X;
  float* U;
  float* lambda;           /* may be NULL: zero warm start, not written back */
} gato_problem;

typedef struct {
  int32_t flags;           /* GATO_SOLVE_* bits */
  int32_t sqp_iters;       /* SQP iterations that computed a step */
  int32_t pcg_iters;       /* PCG iterations summed over those steps */
  float kkt_residual;      /* max(||c||_inf, ||g + C^T lambda||_inf / max(1, ||g||_inf)) at the
                              last linearisation */
  float merit;             /* merit (Eq. 3) of the returned iterate */
} gato_result;

typedef struct gato_batch gato_batch;

/* Fills the library defaults (mu 10, beta 2, A 8, eps 1e-6, cap 1000, stair, no tolerance). */
void gato_default_params(gato_solver_params* out);

/* Creates a batch: validates and copies the models, allocates device scratch
 * for max_batch solves of up to max_horizon knots, binds cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream).  *out is NULL on failure. */
gato_status gato_create_batch(const gato_batch_desc* desc, void* cuda_stream, gato_batch** out);

/* Runs up to max_sqp_iters SQP iterations (Alg. 1, repeated) for n solves in one
 * persistent fused launch (one CTA per solve, longest horizon first).  Host
 * problems are staged through pinned memory; device problems are used in place.
 * Asynchronous on the batch stream; if `results` is non-NULL the call waits and
 * fills results[0..n-1], otherwise call gato_sync then gato_get_results. */
gato_status gato_solve(gato_batch* b, const gato_problem* problems, int32_t n,
                       int32_t max_sqp_iters, gato_result* results);

/* One SQP iteration ("real-time iteration", Sec. IV-A) = gato_solve with 1. */
gato_status gato_step(gato_batch* b, const gato_problem* problems, int32_t n,
                      gato_result* results);

/* The plain GPU form used as the comparison baseline: the same arithmetic, but
 * each solve runs alone and every stage of every SQP iteration (setup, Schur,
 * PCG, recovery, merit, line search) is its own kernel launch. */
gato_status gato_solve_plain(gato_batch* b, const gato_problem* problems, int32_t n,
                             int32_t max_sqp_iters, gato_result* results);

/* gato_solve for callers that cannot allocate device memory: a real-time
 * control loop that must not pay allocation latency or implicit device
 * synchronisation once it runs, a controller with a fixed memory budget, or
 * code hosted inside an application that owns every device allocation.  (The
 * paper has no counterpart; this is a deployment variant of gato_solve.)
 *
 * Same solver and kernel as gato_solve, but it needs no gato_batch: its
 * scratch (per-solve workspace, descriptors, models, launch order) is a set of
 * fixed-size arrays compiled into the library, about 3.2 MiB held on every GPU
 * that loads it until the process exits.  Limits: n <= 16 solves, N <= 64,
 * n_models <= 8, and every problem must use GATO_MEM_DEVICE pointers; larger
 * or host problems return GATO_E_INVALID and launch nothing.  `results` is a
 * DEVICE array of n gato_result that the kernel writes.  The call is
 * asynchronous on cuda_stream (a cudaStream_t, NULL = legacy default stream);
 * synchronise the stream before reading X, U, lambda or results.  It calls no
 * cudaMalloc or cudaFree.  The first call on each device looks up the device
 * addresses of the arrays (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the same
 * arrays, so calls whose kernels overlap on the GPU (another stream, another
 * host thread) race: serialise them.  Nothing in the arrays has to start at
 * zero (every call writes its scratch before reading it). */
gato_status gato_solve_noalloc(const gato_model_desc* models, int32_t n_models,
                               const gato_solver_params* params,
                               const gato_problem* problems, int32_t n, int32_t max_sqp_iters,
                               gato_result* results, void* cuda_stream);

/* Waits for the batch stream, at most timeout_us microseconds (< 0 = forever);
 * GATO_E_TIMEOUT leaves the work running.  Uses a polling host wait, never a
 * device-side spin. */
gato_status gato_sync(gato_batch* b, int64_t timeout_us);

/* Copies the results of the last completed call (n entries). */
gato_status gato_get_results(gato_batch* b, gato_result* out, int32_t n);

void gato_destroy_batch(gato_batch* b);

/* Bytes copied host->device and device->host by the last solve call (host
 * problems are staged through pinned memory; device problems copy only the
 * descriptors and results).  Descriptor/result traffic is included. */
gato_status gato_last_transfer_bytes(const gato_batch* b, int64_t* h2d, int64_t* d2h);

/* ---- introspection for stage-level checks (not needed by solvers) ----
 * Runs the plain form on problems[0] for its first SQP iteration, stopping
 * after stage `stop_stage` (1 dynamics columns, 2 forward dynamics, 3 value
 * pass + costs, 4 tangents, 5 dynamics Jacobians, 6 KKT residual, 7 Schur
 * blocks, 8 preconditioner blocks, 9 PCG, 10 step recovery, 11 line search,
 * 12 accept), then copies that solve's whole workspace (floats, layout given
 * by gato_debug_layout) to ws_out[0..ws_floats).  Synchronous. */
gato_status gato_debug_plain_stage(gato_batch* b, const gato_problem* problems, int32_t stop_stage,
                                   float* ws_out, int64_t ws_floats);

/* Fills offsets[0..23] (floats) of the workspace arrays in the order
 * X U dX dU Fq Fv Minv qdd dTau Qinv Rinv q r c Jk Linv links D L P vec scal
 * dres_x dres_u,
 * and returns the workspace size in floats (or -1). */
int64_t gato_debug_layout(const gato_batch* b, int64_t* offsets);

const char* gato_status_string(gato_status s);
const char* gato_last_error(const gato_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* GATO_H_ */
