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
/* Linear solver of the Schur system (gato_solver_params.linsolve). */
enum { GATO_LINSOLVE_PCG = 0, GATO_LINSOLVE_DIRECT = 1 };
enum { GATO_MEM_HOST = 0, GATO_MEM_DEVICE = 1 };
/* Arithmetic of a solve (gato_solver_params.precision). */
enum { GATO_PRECISION_FP32 = 0, GATO_PRECISION_ESCALATE = 1, GATO_PRECISION_HIGH = 2 };

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
  int32_t linsolve;        /* GATO_LINSOLVE_PCG (the method, default) or
                              GATO_LINSOLVE_DIRECT: S dnu = rhs by block elimination
                              from both ends of the horizon towards knot (N+1)/2
                              (sequential over knots; the same result for any split
                              of a solve over CTAs; precond, pcg_eps and
                              pcg_max_iter unused; pcg_iters reads 0) */
  int32_t rho_adapt;       /* 1: each solve's rho (w[5]) is adjusted after every SQP
                              iteration from its line search (Sec. IV-C): / 3 after an
                              accepted step, * 2 after a rejected one, within
                              [1e-8, 1e1]; it starts from w[5] at every call.
                              0 (default): rho fixed */
  int32_t precision;       /* GATO_PRECISION_ESCALATE (default): the bulk runs in FP32;
                              when a KKT tolerance is set (kkt_tol > 0), a solve whose
                              FP32 line search finds no merit decrease (near a
                              solution, where FP32 rounding of the dynamics and of the
                              iterate exceeds the decrease), or whose FP32 KKT test
                              passes, repeats that SQP iteration in a high-precision
                              mode and stays in it for the rest of the call: mass
                              matrix and bias in double-float (FP32 pairs; sin and cos
                              of q in FP64), each dynamics solve refined against them,
                              the iterate kept as double-float pairs, trial merits in
                              double-float.
                              The repeated iteration counts once.  Without a tolerance
                              (fixed iteration counts, real-time ticks) nothing
                              escalates.  GATO_PRECISION_FP32: never escalate (the step
                              is then rejected with GATO_SOLVE_LSFAIL).
                              GATO_PRECISION_HIGH: every iteration in the
                              high-precision mode from the start */
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
  float f_ext[3];          /* constant external force on the end-effector point, base
                              frame (N): the dynamics become M qdd = u + J_p^T f_ext -
                              ID(q, qd, 0); zeros = none.  Sec. IV-D's disturbance
                              hypotheses are solves differing only in it */
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

/* Fills the library defaults (mu 10, beta 2, A 8, eps 1e-6, cap 1000, stair, no tolerance,
 * PCG, rho fixed, precision escalation on). */
void gato_default_params(gato_solver_params* out);

/* Creates a batch: validates and copies the models, allocates device scratch
 * for max_batch solves of up to max_horizon knots, binds cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream).  *out is NULL on failure. */
gato_status gato_create_batch(const gato_batch_desc* desc, void* cuda_stream, gato_batch** out);

/* Runs up to max_sqp_iters SQP iterations (Alg. 1, repeated) for n solves in
 * persistent fused launches: each solve is one thread-block cluster of
 * ceil((N+1)/33) CTAs or more (gato_launch_config), one launch per cluster
 * size, the launches running concurrently, longest horizon first.  Host
 * problems are staged through pinned memory; device problems are used in place.
 * Asynchronous on the batch stream; if `results` is non-NULL the call waits and
 * fills results[0..n-1], otherwise call gato_sync then gato_get_results. */
gato_status gato_solve(gato_batch* b, const gato_problem* problems, int32_t n,
                       int32_t max_sqp_iters, gato_result* results);

/* One SQP iteration ("real-time iteration", Sec. IV-B) = gato_solve with 1. */
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
 * fixed-size arrays compiled into the library, about 2.7 MiB held on every GPU
 * that loads it until the process exits.  Limits: n <= 16 solves, N <= 64,
 * n_models <= 8, and every problem must use GATO_MEM_DEVICE pointers; larger
 * or host problems return GATO_E_INVALID and launch nothing.  `results` is a
 * DEVICE array of n gato_result that the kernel writes.  The call is
 * asynchronous on cuda_stream (a cudaStream_t, NULL = legacy default stream);
 * synchronise the stream before reading X, U, lambda or results.  It calls no
 * cudaMalloc or cudaFree, and it makes no host-to-device copy: the call's
 * descriptors travel as the by-value argument of a one-block kernel launched
 * on cuda_stream ahead of the solve, which stores them into the arrays.  The first call on each device looks up the device
 * addresses of the arrays (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the same
 * arrays, so calls whose kernels overlap on the GPU (another stream, another
 * host thread) race: serialise them.  Nothing in the arrays has to start at
 * zero (every call writes its scratch before reading it). */
gato_status gato_solve_noalloc(const gato_model_desc* models, int32_t n_models,
                               const gato_solver_params* params,
                               const gato_problem* problems, int32_t n, int32_t max_sqp_iters,
                               gato_result* results, void* cuda_stream);

/* ---- launch configuration and autotuning (Sec. III's M-block mapping made tunable) ----
 * How solves map onto the GPU.  variant: 0 automatic (the latency form), 1 the
 * latency form (the PCG's block rows held in registers, one CTA per SM), 2 the
 * throughput form (off-diagonal rows read from shared memory, two CTAs per SM
 * when the shared memory fits).
 * knots_per_cta: 0 = 33 (the most one CTA holds), 2..33 spreads each solve
 * over more CTAs.  cluster: 0 = per solve, 1..8 = every solve uses this many
 * CTAs where its horizon allows (a uniform batch is then a single launch).
 * A cluster never exceeds 8 CTAs nor holds a CTA with fewer than 2 knots
 * (except the last). */
typedef struct {
  int32_t variant;
  int32_t knots_per_cta;
  int32_t cluster;
} gato_launch_config;

/* Forces a launch configuration for later calls; cfg = NULL returns to the
 * autotuned / automatic choice.  GATO_E_INVALID for out-of-range fields. */
gato_status gato_set_launch_config(gato_batch* b, const gato_launch_config* cfg);

/* What a launch of n_solves solves of horizon N looks like on the current
 * device under cfg (NULL = the automatic choice): the CTAs per solve, the
 * kernel form (1 latency, 2 throughput), the dynamic shared memory per CTA,
 * and how many solves (thread-block clusters) the device holds at once
 * (cudaOccupancyMaxActiveClusters; clusters are placed within one GPC, so this
 * can be below SMs / CTAs per solve).  Solves beyond that count wait for a
 * free cluster slot.  GATO_E_INVALID for N outside 1..256, n_solves < 1 or an
 * out-of-range cfg; GATO_E_CUDA if the query fails.  No device memory is
 * allocated. */
typedef struct {
  int32_t ctas_per_solve;
  int32_t variant;
  int32_t smem_bytes;
  int32_t max_resident_solves;
} gato_launch_info;
gato_status gato_query_launch(int32_t N, int32_t n_solves, const gato_launch_config* cfg,
                              gato_launch_info* out);

/* Times every candidate configuration (both variants x knots per CTA
 * {33, 24, 17, 12, 9, 6} x uniform clusters, skipping duplicates and
 * throughput forms whose shared memory does not fit two CTAs per SM) on these
 * problems for max_sqp_iters iterations, `reps` timed runs each after one
 * warm-up, every run from the problems' current iterate (X, U, lambda are
 * restored afterwards: the call leaves them unchanged).  The fastest median
 * becomes the batch's choice for calls with the same batch-size bucket (next
 * power of two) and horizon bucket (max N / 16, rounded up), unless a
 * configuration is forced.  Writes the winner to *best and its median
 * milliseconds to *best_ms (either may be NULL).  Synchronous. */
gato_status gato_autotune(gato_batch* b, const gato_problem* problems, int32_t n, int32_t max_sqp_iters,
                          int32_t reps, gato_launch_config* best, float* best_ms);

/* ---- CUDA graph capture of a solve ----
 * Captures gato_solve(problems, n, max_sqp_iters) into a CUDA graph (all
 * cluster-size launches, forked and joined, plus the copy of the results to
 * pinned memory).  Every problem must use device pointers; the graph keeps the
 * pointers, so refill X, U, x_s, references in place between replays.  The
 * graph uses the batch's workspace: its replays are ordered with the batch's
 * stream (the replay waits for earlier work there, later work waits for it),
 * and it must not run concurrently with other calls on the batch.  The
 * configuration in force at capture time is baked in. */
typedef struct gato_graph gato_graph;
gato_status gato_graph_create(gato_batch* b, const gato_problem* problems, int32_t n,
                              int32_t max_sqp_iters, gato_graph** out);
/* Replays the graph.  results non-NULL: waits and fills results[0..n-1];
 * NULL: returns at once, gato_graph_wait(g, results) waits later. */
gato_status gato_graph_launch(gato_graph* g, gato_result* results);
gato_status gato_graph_wait(gato_graph* g, gato_result* results);
void gato_graph_destroy(gato_graph* g);

/* ---- serving loop: continuous batching of MPC control ticks ----
 * A server keeps each session's trajectory (X, U, lambda, x_s, reference)
 * resident on the device.  A request is one control tick of a session: a new
 * measured state x_s, optionally a one-knot warm-start shift (X_k <- X_{k+1},
 * U_k <- U_{k+1}, lambda_k <- lambda_{k+1}; the last knot keeps its value),
 * then sqp_iters SQP iterations.  A worker thread launches every pending
 * request together whenever one of max_inflight launch contexts is free, so
 * requests that arrive while others run join the next launch and their work
 * overlaps on the GPU.  A request's arithmetic depends only on its own
 * session (cluster size fixed by its horizon), so its result is the same
 * alone and in any mix.  Thread-safe: any host thread may submit and poll. */
typedef struct gato_server gato_server;

typedef struct {
  int32_t max_sessions;      /* resident trajectories wanted (slots) */
  int32_t max_horizon;       /* largest N of a session (<= 256) */
  int32_t max_batch;         /* requests per launch (halved until memory allows) */
  int32_t max_inflight;      /* launch contexts on the GPU at once, 1..8 */
  int32_t sqp_iters;         /* SQP iterations per request */
  int64_t mem_budget_bytes;  /* device memory the server may reserve; 0 = 90% of free */
} gato_server_desc;

typedef struct {
  gato_result result;
  float u0[7];               /* first control of the new solution (dof entries used) */
  float x1[14];              /* its predicted state at knot 1 (2*dof entries used) */
  int64_t submit_ns, done_ns;/* steady-clock times of submission and completion */
} gato_reply;

typedef struct {
  int32_t capacity;          /* session slots admitted by memory */
  int32_t sessions_open;
  int32_t max_batch, max_inflight;
  int64_t submitted, completed, launches, pending;
  int64_t reserved_bytes;    /* device memory held by the server */
} gato_server_stats;

/* Creates a server over the models and solver parameters of models_desc
 * (its max_batch / max_horizon are ignored).  Device memory is reserved here:
 * max_inflight launch contexts of max_batch solves each (max_batch halves
 * until they fit half the budget), then as many session slots as the rest of
 * the budget holds, at most max_sessions (see gato_server_stats).  Uses the
 * current CUDA device.  GATO_E_NOMEM if not even one slot fits. */
gato_status gato_server_create(const gato_batch_desc* models_desc, const gato_server_desc* d,
                               gato_server** out);

/* Admits a session from a host problem (mem = GATO_MEM_HOST; X, U, lambda
 * may be NULL for the cold start).  GATO_E_BUSY when every slot is taken:
 * retry after a gato_server_close.  Synchronous (copies the slot image). */
gato_status gato_server_open(gato_server* s, const gato_problem* p, int32_t* session);

/* Queues one control tick: x_s is a host array of 2*dof floats, shift != 0
 * shifts the warm start by one knot first.  GATO_E_BUSY if the session still
 * has a request pending or on the GPU (ticks of a session are sequential). */
gato_status gato_server_submit(gato_server* s, int32_t session, const float* x_s, int32_t shift,
                               int64_t* ticket);

/* Waits up to timeout_us (0 = just check, < 0 = forever) for a ticket and
 * consumes it: GATO_OK with *out filled (out may be NULL), GATO_E_TIMEOUT if
 * it is not done yet, GATO_E_INVALID for an unknown or consumed ticket. */
gato_status gato_server_poll(gato_server* s, int64_t ticket, int64_t timeout_us, gato_reply* out);

/* Copies a session's resident X [(N+1)*2dof], U [N*dof], lambda [(N+1)*2dof]
 * to host arrays (any may be NULL).  GATO_E_BUSY while it has a request. */
gato_status gato_server_read(gato_server* s, int32_t session, float* X, float* U, float* lambda);

/* Frees a session's slot (GATO_E_BUSY while it has a request). */
gato_status gato_server_close(gato_server* s, int32_t session);

gato_status gato_server_get_stats(gato_server* s, gato_server_stats* out);

/* Load driver for measuring the loop (config: Poisson arrivals of MPC ticks).
 * Replays an arrival schedule on the calling thread: arrival i, due at
 * t_arrival[i] seconds after the call starts (sorted), is a tick of client
 * client[i] (an index into sessions[0..n_sessions)), whose new state is the
 * client's last predicted state x1 (x_init[c*14..] before its first reply)
 * plus noise[i*14..] (2*dof entries used), submitted with a one-knot shift.
 * A client's ticks are sequential: an arrival for a busy client waits for
 * its previous reply.  latency_ms[i] = completion time - scheduled arrival
 * (host steady clock), so waiting of any kind is included.  Every session
 * must be open and idle; one drive at a time. */
typedef struct {
  int64_t completed;
  double elapsed_s;
  int64_t launches;      /* kernel batches launched during the drive */
  int64_t max_backlog;   /* most arrivals waiting for a busy client at once */
} gato_drive_stats;
gato_status gato_server_drive(gato_server* s, const int32_t* sessions, int32_t n_sessions,
                              const float* x_init, const double* t_arrival, const int32_t* client,
                              const float* noise, int64_t n, float* latency_ms, gato_drive_stats* out);
const char* gato_server_last_error(const gato_server* s);

/* Stops the worker, waits for launches in flight, frees everything. */
void gato_server_destroy(gato_server* s);

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

/* Per-stage cycle counters of the fused kernel (clock64 deltas taken by the
 * first thread of each solve's first CTA at stage boundaries).  enable = 1
 * allocates and zeroes the counters; the following gato_solve calls add to
 * them; enable = 0 copies n x 16 counters (cycles) to `cycles` if non-NULL and
 * frees them.  Order: load, mass matrix, forward dynamics, value pass + cost,
 * tangents, Jacobians, KKT, Schur, block inverse, PCG start, PCG S-phase,
 * PCG y-phase, PCG w/z-phase, recovery, line search, accept. */
gato_status gato_debug_stage_cycles(gato_batch* b, int32_t enable, int64_t* cycles, int32_t n);

/* Per-iteration log of the fused kernel (the parity tests compare the
 * line-search choices with the FP64 oracle's, Sec. II-A Step 3 / Eq. 7).
 * enable = 1 allocates a log of max_iters records per solve (device memory);
 * every following gato_solve / gato_step call of the batch rewrites it from
 * iteration 0.  enable = 0 copies n x max_iters records to `log` (if non-NULL;
 * max_iters must equal the enabled value) and frees it.  A record is 8 int32:
 * the line search's choice (alpha index i of alpha = beta^-i, -1 = step
 * rejected, -2 = iteration not reached), the PCG iterations of that SQP
 * iteration, the KKT residual at its linearisation (the bits of a float),
 * 1 if the iteration ran in the high-precision mode, the merit (Eq. 3) of the
 * iterate and the merit of the full step's trial point (alpha = 1), each as
 * the bits of a (hi, lo) float pair whose sum is the value.  Synchronous.
 * GATO_E_INVALID for bad arguments, GATO_E_NOMEM if the log cannot be
 * allocated. */
gato_status gato_debug_iteration_log(gato_batch* b, int32_t enable, int32_t max_iters, int32_t* log,
                                     int32_t n);

/* Fills offsets[0..24] (floats) of the workspace arrays in the order
 * X U dX dU Fq Fv Minv qdd dTau Qinv Rinv q r c Jk Linv links D L P vec scal
 * dres_x dres_u nu,
 * and returns the workspace size in floats (or -1).  Linv is empty (its offset
 * equals that of links): the block inverse keeps its rows in registers. */
int64_t gato_debug_layout(const gato_batch* b, int64_t* offsets);

const char* gato_status_string(gato_status s);
const char* gato_last_error(const gato_batch* b);

/* ------------------------------------------------------------------ plant
 * The simulated robot of closed-loop runs (Sec. IV-E simulates its plant with
 * RK4 at 1 kHz while the solver runs at its own rate).  Host code in double;
 * no GPU call and not part of the solve path. */

/* Advances x = (q, qd) (2*dof doubles) by `steps` classic RK4 steps of size h
 * under a control u (dof) held constant and the constant end-effector force
 * f_ext (3, base frame; NULL = none):
 *     qdd = M(q)^-1 (u + J_p(q)^T f_ext - ID(q, qd, 0)).
 * x_out (2*dof) may alias x.  GATO_E_INVALID for a bad model or argument, a
 * mass matrix that is not positive definite or a non-finite result (x_out
 * then unchanged). */
gato_status gato_plant_rk4(const gato_model_desc* model, const double* x, const double* u,
                           const double* f_ext, double h, int32_t steps, double* x_out);

/* End-effector position p (3, base frame) at configuration q (dof). */
gato_status gato_plant_ee(const gato_model_desc* model, const double* q, double* p);

#ifdef __cplusplus
}
#endif
#endif /* GATO_H_ */
