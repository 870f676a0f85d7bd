// Serving loop: continuous batching of MPC control ticks (declared in
// include/gato.h, gato_server_*).
//
// A server keeps every session's trajectory (X, U, lambda, x_s, reference)
// resident in device memory.  A request is one control tick of one session:
// a new measured state, an optional one-knot warm-start shift, and a fixed
// number of SQP iterations.  A worker thread takes the requests that are
// pending whenever one of `max_inflight` launch contexts is free and launches
// them together (the fused kernel, grouped by cluster size), so requests that
// arrive while others run on the GPU join the next launch and their work
// overlaps on the device.  Completion is signalled by a host function on the
// context's stream; nothing polls the GPU.  Sessions are admitted while slots
// are free; the number of slots and the per-launch batch follow from the
// device memory the server may take.
//
// Each solve's arithmetic depends only on its own data and cluster size (fixed
// per horizon here), so a request's result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gato.h"
#include "gato_internal.h"

using namespace gato;

namespace {

constexpr int kMaxCtx = 8;

// What the preparation kernel needs for one request.
struct PrepRec {
  float* x_s;
  float* X;
  float* U;
  float* lam;
  int N, nx, nu, shift;
  float xs_new[16];
};

// Reply of one request as the gather kernel writes it (32 words).
struct ReplyRec {
  int flags, sqp_iters, pcg_iters;
  float kkt, merit;
  float u0[7];
  float x1[14];
  int pad[6];
};
static_assert(sizeof(ReplyRec) == 128, "reply record");

// Moves rows 1..rows-1 of a row-major [rows][w] array up by one row; the last
// row keeps its value (the warm start's terminal guess).
__device__ void shift_rows(float* a, int rows, int w, float* buf) {
  const int m = (rows - 1) * w;
  for (int i = threadIdx.x; i < m; i += blockDim.x) buf[i] = a[i + w];
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) a[i] = buf[i];
  __syncthreads();
}

// One CTA per request: write the measured state and shift the warm start.
__global__ void tick_prepare(const PrepRec* recs) {
  extern __shared__ float buf[];
  const PrepRec r = recs[blockIdx.x];
  if (r.shift) {
    shift_rows(r.X, r.N + 1, r.nx, buf);
    shift_rows(r.U, r.N, r.nu, buf);
    if (r.lam) shift_rows(r.lam, r.N + 1, r.nx, buf);
  }
  for (int i = threadIdx.x; i < r.nx; i += blockDim.x) r.x_s[i] = r.xs_new[i];
}

// One warp per request: results, first control and the predicted next state.
__global__ void tick_reply(const ProbDesc* probs, const Result* res, ReplyRec* out) {
  const int i = blockIdx.x, t = threadIdx.x;
  const ProbDesc& p = probs[i];
  ReplyRec& o = out[i];
  const int nu = p.dof, nx = 2 * p.dof;
  if (t == 0) {
    o.flags = res[i].flags;
    o.sqp_iters = res[i].sqp_iters;
    o.pcg_iters = res[i].pcg_iters;
    o.kkt = res[i].kkt;
    o.merit = res[i].merit;
  }
  if (t < 7) o.u0[t] = t < nu ? p.U[t] : 0.f;
  if (t < 14) o.x1[t] = t < nx ? p.X[nx + t] : 0.f;
  if (t < 6) o.pad[t] = 0;
}

struct Request {
  int64_t ticket;
  int session;
  int shift;
  float x_s[16];
  int64_t t_submit;
};

struct Done {
  bool done = false;
  gato_status status = GATO_OK;
  ReplyRec reply;
  int64_t t_submit = 0, t_done = 0;
};

struct Session {
  bool open = false;
  bool busy = false;  // a request is pending or on the GPU
  int model = 0, N = 0, cost_kind = 0, dof = 0;
  float dt = 0.f, w[6] = {}, fext[3] = {};
  float *x_s = nullptr, *ref = nullptr, *X = nullptr, *U = nullptr, *lam = nullptr;
};

struct LaunchCtx {
  gato_server* srv = nullptr;
  int id = 0;
  bool busy = false;
  cudaStream_t s = nullptr;
  cudaStream_t aux[7] = {};
  cudaEvent_t ev[8] = {};
  float* ws = nullptr;
  ProbDesc *probs_d = nullptr, *probs_h = nullptr;
  int *order_d = nullptr, *order_h = nullptr;
  PrepRec *prep_d = nullptr, *prep_h = nullptr;
  Result* res_d = nullptr;
  ReplyRec *reply_d = nullptr, *reply_h = nullptr;
  std::vector<Request> reqs;
  std::vector<int> N_h;
};

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

struct gato_server {
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  gato_status failed = GATO_OK;
  std::string err;
  // configuration
  gato_batch* models = nullptr;  // model table, parameters and validation
  int max_horizon = 0, max_batch = 0, n_ctx = 0, sqp_iters = 0, capacity = 0;
  Params prm;
  DevModel* models_d = nullptr;
  WsLayout layout;
  size_t ws_stride = 0, slot_floats = 0;
  int64_t reserved = 0;
  // state
  float* slab = nullptr;  // resident trajectories, slot_floats per session
  std::vector<Session> sessions;
  std::deque<Request> pending;
  std::unordered_map<int64_t, Done> done;
  LaunchCtx ctx[kMaxCtx];
  int64_t next_ticket = 1, submitted = 0, completed = 0, launches = 0;
  bool driving = false;                 // gato_server_drive is collecting completions
  std::deque<int64_t> completed_order;  // tickets completed while driving
  cudaStream_t admin = nullptr;
  float* admin_h = nullptr;  // pinned staging for open/read
};

// exported by gato_api.cu for the server (validation and model table)
namespace gato {
gato_status batch_validate_problem(gato_batch* b, const gato_problem& p);
const DevModel* batch_models_device(const gato_batch* b);
int batch_model_dof(const gato_batch* b, int model);
int batch_n_models(const gato_batch* b);
Params batch_params(const gato_batch* b, int iters);
}  // namespace gato

namespace {

void CUDART_CB on_done(void* p) {
  LaunchCtx* c = static_cast<LaunchCtx*>(p);
  gato_server* s = c->srv;
  const int64_t t = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < c->reqs.size(); ++i) {
      const Request& r = c->reqs[i];
      Done& d = s->done[r.ticket];
      d.done = true;
      d.status = GATO_OK;
      d.reply = c->reply_h[i];
      d.t_submit = r.t_submit;
      d.t_done = t;
      s->sessions[r.session].busy = false;
      if (s->driving) s->completed_order.push_back(r.ticket);
    }
    s->completed += (int64_t)c->reqs.size();
    c->reqs.clear();
    c->busy = false;
  }
  s->cv.notify_all();
}

// Launches the requests in c->reqs (called by the worker without the lock;
// the sessions of these requests are busy, so nobody else touches them).
cudaError_t dispatch(gato_server* s, LaunchCtx* c) {
  const int n = (int)c->reqs.size();
  c->N_h.resize(n);
  int nmax = 1;
  for (int i = 0; i < n; ++i) {
    const Request& r = c->reqs[i];
    const Session& ss = s->sessions[r.session];
    ProbDesc& d = c->probs_h[i];
    std::memset(&d, 0, sizeof(d));
    d.model = ss.model;
    d.N = ss.N;
    d.cost_kind = ss.cost_kind;
    d.dof = ss.dof;
    d.dt = ss.dt;
    for (int k = 0; k < 6; ++k) d.w[k] = ss.w[k];
    for (int k = 0; k < 3; ++k) d.fext[k] = ss.fext[k];
    d.x_s = ss.x_s;
    d.x_ref = ss.cost_kind == GATO_COST_JOINT ? ss.ref : nullptr;
    d.ee_ref = ss.cost_kind == GATO_COST_EE ? ss.ref : nullptr;
    d.X = ss.X;
    d.U = ss.U;
    d.lam = ss.lam;
    PrepRec& pr = c->prep_h[i];
    pr.x_s = ss.x_s;
    pr.X = ss.X;
    pr.U = ss.U;
    pr.lam = ss.lam;
    pr.N = ss.N;
    pr.nx = 2 * ss.dof;
    pr.nu = ss.dof;
    pr.shift = r.shift;
    std::memcpy(pr.xs_new, r.x_s, sizeof(pr.xs_new));
    c->N_h[i] = ss.N;
    nmax = std::max(nmax, ss.N);
  }
  LaunchPlan plan;
  plan.aux = c->aux;
  plan.ev = c->ev;
  plan.n_aux = 7;
  order_solves(c->N_h.data(), n, c->order_h, plan);
  cudaError_t e = cudaMemcpyAsync(c->prep_d, c->prep_h, n * sizeof(PrepRec), cudaMemcpyHostToDevice, c->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->probs_d, c->probs_h, n * sizeof(ProbDesc), cudaMemcpyHostToDevice, c->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->order_d, c->order_h, n * sizeof(int), cudaMemcpyHostToDevice, c->s);
  if (e != cudaSuccess) return e;
  tick_prepare<<<n, 128, (size_t)s->max_horizon * XM * sizeof(float), c->s>>>(c->prep_d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  FusedLaunch a;
  a.probs = c->probs_d;
  a.models = s->models_d;
  a.order = c->order_d;
  a.results = c->res_d;
  a.ws = c->ws;
  a.ws_stride = s->ws_stride;
  a.layout = s->layout;
  a.n = n;
  a.nmax = nmax;
  a.csize = 1;
  a.iters = s->sqp_iters;
  a.prm = s->prm;
  a.timing = nullptr;
  a.variant = 0;
  e = launch_fused_grouped(a, c->order_h, c->order_d, c->N_h.data(), n, c->s, plan);
  if (e != cudaSuccess) return e;
  tick_reply<<<n, 32, 0, c->s>>>(c->probs_d, c->res_d, c->reply_d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaMemcpyAsync(c->reply_h, c->reply_d, n * sizeof(ReplyRec), cudaMemcpyDeviceToHost, c->s);
  if (e != cudaSuccess) return e;
  return cudaLaunchHostFunc(c->s, on_done, c);
}

void worker_main(gato_server* s, int device) {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    LaunchCtx* c = nullptr;
    s->cv.wait(lk, [&] {
      if (s->stop) return true;
      if (s->pending.empty() || s->failed != GATO_OK) return false;
      for (int i = 0; i < s->n_ctx; ++i)
        if (!s->ctx[i].busy) return true;
      return false;
    });
    if (s->stop) break;
    for (int i = 0; i < s->n_ctx && !c; ++i)
      if (!s->ctx[i].busy) c = &s->ctx[i];
    // every pending request joins this launch, up to the context's batch
    while (!s->pending.empty() && (int)c->reqs.size() < s->max_batch) {
      c->reqs.push_back(s->pending.front());
      s->pending.pop_front();
    }
    c->busy = true;
    ++s->launches;
    lk.unlock();
    const cudaError_t e = dispatch(s, c);
    lk.lock();
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->failed = GATO_E_CUDA;
      s->err = std::string("server launch: ") + cudaGetErrorString(e);
      const int64_t t = now_ns();
      for (const Request& r : c->reqs) {
        Done& d = s->done[r.ticket];
        d.done = true;
        d.status = GATO_E_CUDA;
        d.t_submit = r.t_submit;
        d.t_done = t;
        s->sessions[r.session].busy = false;
      }
      c->reqs.clear();
      c->busy = false;
      s->cv.notify_all();
    }
  }
}

void free_ctx(LaunchCtx& c) {
  if (c.s) cudaStreamSynchronize(c.s);
  for (auto& a : c.aux)
    if (a) cudaStreamDestroy(a);
  for (auto& e : c.ev)
    if (e) cudaEventDestroy(e);
  if (c.s) cudaStreamDestroy(c.s);
  cudaFree(c.ws);
  cudaFree(c.probs_d);
  cudaFree(c.order_d);
  cudaFree(c.prep_d);
  cudaFree(c.res_d);
  cudaFree(c.reply_d);
  cudaFreeHost(c.probs_h);
  cudaFreeHost(c.order_h);
  cudaFreeHost(c.prep_h);
  cudaFreeHost(c.reply_h);
}

gato_status server_fail(gato_server* s, gato_status st, const std::string& m) {
  s->err = m;
  return st;
}

}  // namespace

extern "C" {

void gato_server_destroy(gato_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (int i = 0; i < kMaxCtx; ++i) free_ctx(s->ctx[i]);
  if (s->admin) {
    cudaStreamSynchronize(s->admin);
    cudaStreamDestroy(s->admin);
  }
  cudaFreeHost(s->admin_h);
  cudaFree(s->slab);
  gato_destroy_batch(s->models);
  delete s;
}

gato_status gato_server_create(const gato_batch_desc* models_desc, const gato_server_desc* d,
                               gato_server** out) {
  if (!out) return GATO_E_INVALID;
  *out = nullptr;
  if (!models_desc || !d) return GATO_E_INVALID;
  if (d->max_sessions < 1 || d->max_horizon < 1 || d->max_horizon > NMAX_LIMIT || d->max_batch < 1 ||
      d->max_inflight < 1 || d->max_inflight > kMaxCtx || d->sqp_iters < 1 || d->mem_budget_bytes < 0)
    return GATO_E_INVALID;
  gato_server* s = new (std::nothrow) gato_server();
  if (!s) return GATO_E_NOMEM;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    delete s;
    return GATO_E_CUDA;
  }
  // the model table and parameters live in a one-solve batch (validation, models)
  gato_batch_desc md = *models_desc;
  md.max_batch = 1;
  md.max_horizon = d->max_horizon;
  gato_status st = gato_create_batch(&md, nullptr, &s->models);
  if (st != GATO_OK) {
    delete s;
    return st;
  }
  s->max_horizon = d->max_horizon;
  s->sqp_iters = d->sqp_iters;
  s->n_ctx = d->max_inflight;
  s->prm = batch_params(s->models, d->sqp_iters);
  s->models_d = const_cast<DevModel*>(batch_models_device(s->models));
  s->layout = ws_layout(d->max_horizon, false, false);
  s->ws_stride = s->layout.total;
  const size_t K = d->max_horizon + 1;
  s->slot_floats = align32(16 + 3 * K * XM + (size_t)d->max_horizon * QM);
  // admission by device memory: launch contexts first, then session slots
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    gato_server_destroy(s);
    return GATO_E_CUDA;
  }
  size_t budget = (size_t)(0.9 * (double)free_b);
  if (d->mem_budget_bytes > 0) budget = std::min(budget, (size_t)d->mem_budget_bytes);
  const size_t per_solve = s->ws_stride * sizeof(float) + sizeof(ProbDesc) + sizeof(int) + sizeof(PrepRec) +
                           sizeof(Result) + sizeof(ReplyRec);
  const size_t slot_bytes = s->slot_floats * sizeof(float);
  int mb = d->max_batch;
  while (mb > 1 && (size_t)s->n_ctx * mb * per_solve > budget / 2) mb /= 2;
  const size_t ctx_bytes = (size_t)s->n_ctx * mb * per_solve;
  if (ctx_bytes + slot_bytes > budget) {
    gato_server_destroy(s);
    return GATO_E_NOMEM;
  }
  s->max_batch = mb;
  s->capacity = (int)std::min<size_t>((size_t)d->max_sessions, (budget - ctx_bytes) / slot_bytes);
  s->reserved = (int64_t)(ctx_bytes + (size_t)s->capacity * slot_bytes);
  bool ok = cudaMalloc(&s->slab, (size_t)s->capacity * slot_bytes) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMallocHost(&s->admin_h, slot_bytes) == cudaSuccess;
  for (int i = 0; i < s->n_ctx && ok; ++i) {
    LaunchCtx& c = s->ctx[i];
    c.srv = s;
    c.id = i;
    ok = cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaMalloc(&c.ws, (size_t)mb * s->ws_stride * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c.probs_d, mb * sizeof(ProbDesc)) == cudaSuccess &&
         cudaMalloc(&c.order_d, mb * sizeof(int)) == cudaSuccess &&
         cudaMalloc(&c.prep_d, mb * sizeof(PrepRec)) == cudaSuccess &&
         cudaMalloc(&c.res_d, mb * sizeof(Result)) == cudaSuccess &&
         cudaMalloc(&c.reply_d, mb * sizeof(ReplyRec)) == cudaSuccess &&
         cudaMallocHost(&c.probs_h, mb * sizeof(ProbDesc)) == cudaSuccess &&
         cudaMallocHost(&c.order_h, mb * sizeof(int)) == cudaSuccess &&
         cudaMallocHost(&c.prep_h, mb * sizeof(PrepRec)) == cudaSuccess &&
         cudaMallocHost(&c.reply_h, mb * sizeof(ReplyRec)) == cudaSuccess;
    for (int k = 0; k < 7 && ok; ++k) ok = cudaStreamCreateWithFlags(&c.aux[k], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 8 && ok; ++k) ok = cudaEventCreateWithFlags(&c.ev[k], cudaEventDisableTiming) == cudaSuccess;
  }
  // shared-memory attributes are set here, not by the worker's first launch
  if (ok) ok = configure_fused(fused_smem_bytes(d->max_horizon, cluster_size(d->max_horizon, 0))) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gato_server_destroy(s);
    return GATO_E_NOMEM;
  }
  s->sessions.resize(s->capacity);
  for (int i = 0; i < s->capacity; ++i) {
    Session& ss = s->sessions[i];
    float* base = s->slab + (size_t)i * s->slot_floats;
    ss.x_s = base;
    ss.ref = base + 16;
    ss.X = ss.ref + K * XM;
    ss.lam = ss.X + K * XM;
    ss.U = ss.lam + K * XM;
  }
  try {
    s->worker = std::thread(worker_main, s, device);
  } catch (...) {
    gato_server_destroy(s);
    return GATO_E_NOMEM;
  }
  *out = s;
  return GATO_OK;
}

const char* gato_server_last_error(const gato_server* s) { return s ? s->err.c_str() : "no server"; }

gato_status gato_server_open(gato_server* s, const gato_problem* p, int32_t* session) {
  if (!s || !p || !session) return GATO_E_INVALID;
  *session = -1;
  if (p->mem != GATO_MEM_HOST) return server_fail(s, GATO_E_INVALID, "sessions open from host problems");
  if (p->N > s->max_horizon) return server_fail(s, GATO_E_INVALID, "N above the server's max_horizon");
  if (p->N < 1 || p->model < 0 || p->model >= batch_n_models(s->models) || !p->x_s)
    return server_fail(s, GATO_E_INVALID, "bad horizon, model or x_s");
  // validation wants a warm start: the cold start where the problem has none
  gato_problem q = *p;
  std::vector<float> Xc, Uc;
  const int dof0 = batch_model_dof(s->models, p->model);
  if (!q.X) {
    Xc.resize((size_t)(p->N + 1) * 2 * dof0);
    for (int k = 0; k <= p->N; ++k) std::memcpy(Xc.data() + (size_t)k * 2 * dof0, p->x_s, 2 * dof0 * sizeof(float));
    q.X = Xc.data();
  }
  if (!q.U) {
    Uc.assign((size_t)p->N * dof0, 0.f);
    q.U = Uc.data();
  }
  gato_status st = batch_validate_problem(s->models, q);
  if (st != GATO_OK) return server_fail(s, st, gato_last_error(s->models));
  std::unique_lock<std::mutex> lk(s->mu);
  int slot = -1;
  for (int i = 0; i < s->capacity && slot < 0; ++i)
    if (!s->sessions[i].open) slot = i;
  if (slot < 0) return server_fail(s, GATO_E_BUSY, "no free session slot");
  Session& ss = s->sessions[slot];
  ss.open = true;
  ss.busy = true;  // until its data is on the device
  lk.unlock();
  ss.model = p->model;
  ss.N = p->N;
  ss.cost_kind = p->cost_kind;
  ss.dof = batch_model_dof(s->models, p->model);
  ss.dt = p->dt;
  for (int k = 0; k < 6; ++k) ss.w[k] = p->w[k];
  for (int k = 0; k < 3; ++k) ss.fext[k] = p->f_ext[k];
  const int nx = 2 * ss.dof, nu = ss.dof, N = ss.N;
  const size_t K = N + 1;
  // the slot image in pinned memory: x_s | ref | X | lambda | U (cold start
  // X_k = x_s, U = 0, lambda = 0 where the problem gives none)
  float* h = s->admin_h;
  std::memset(h, 0, s->slot_floats * sizeof(float));
  const size_t oref = 16, oX = oref + (size_t)(s->max_horizon + 1) * XM;
  const size_t oL = oX + (size_t)(s->max_horizon + 1) * XM, oU = oL + (size_t)(s->max_horizon + 1) * XM;
  std::memcpy(h, p->x_s, nx * sizeof(float));
  if (p->cost_kind == GATO_COST_JOINT)
    std::memcpy(h + oref, p->x_ref, K * nx * sizeof(float));
  else
    std::memcpy(h + oref, p->ee_ref, K * 3 * sizeof(float));
  for (size_t k = 0; k < K; ++k)
    std::memcpy(h + oX + k * nx, p->X ? p->X + k * nx : p->x_s, nx * sizeof(float));
  if (p->U) std::memcpy(h + oU, p->U, (size_t)N * nu * sizeof(float));
  if (p->lambda) std::memcpy(h + oL, p->lambda, K * nx * sizeof(float));
  cudaError_t e = cudaMemcpyAsync(ss.x_s, h, s->slot_floats * sizeof(float), cudaMemcpyHostToDevice, s->admin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->admin);
  lk.lock();
  ss.busy = false;
  if (e != cudaSuccess) {
    ss.open = false;
    cudaGetLastError();
    return server_fail(s, GATO_E_CUDA, std::string("open: ") + cudaGetErrorString(e));
  }
  *session = slot;
  return GATO_OK;
}

gato_status gato_server_close(gato_server* s, int32_t session) {
  if (!s) return GATO_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (session < 0 || session >= s->capacity || !s->sessions[session].open)
    return server_fail(s, GATO_E_INVALID, "no such session");
  if (s->sessions[session].busy) return server_fail(s, GATO_E_BUSY, "session has a request in flight");
  s->sessions[session].open = false;
  return GATO_OK;
}

gato_status gato_server_submit(gato_server* s, int32_t session, const float* x_s, int32_t shift,
                               int64_t* ticket) {
  if (!s || !x_s || !ticket) return GATO_E_INVALID;
  Request r;
  std::memset(&r, 0, sizeof(r));
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed != GATO_OK) return s->failed;
    if (session < 0 || session >= s->capacity || !s->sessions[session].open)
      return server_fail(s, GATO_E_INVALID, "no such session");
    Session& ss = s->sessions[session];
    if (ss.busy) return server_fail(s, GATO_E_BUSY, "session has a request in flight");
    const int nx = 2 * ss.dof;
    for (int i = 0; i < nx; ++i)
      if (!std::isfinite(x_s[i])) return server_fail(s, GATO_E_INVALID, "non-finite state");
    std::memcpy(r.x_s, x_s, nx * sizeof(float));
    r.session = session;
    r.shift = shift ? 1 : 0;
    r.ticket = s->next_ticket++;
    r.t_submit = now_ns();
    ss.busy = true;
    s->done[r.ticket] = Done();
    s->pending.push_back(r);
    ++s->submitted;
    *ticket = r.ticket;
  }
  s->cv.notify_all();
  return GATO_OK;
}

gato_status gato_server_poll(gato_server* s, int64_t ticket, int64_t timeout_us, gato_reply* out) {
  if (!s) return GATO_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return server_fail(s, GATO_E_INVALID, "unknown ticket");
  if (!it->second.done && timeout_us != 0) {
    auto ready = [&] { return s->done[ticket].done || s->failed != GATO_OK; };
    if (timeout_us < 0)
      s->cv.wait(lk, ready);
    else
      s->cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    it = s->done.find(ticket);
  }
  if (!it->second.done) return s->failed != GATO_OK ? s->failed : GATO_E_TIMEOUT;
  const Done d = it->second;
  s->done.erase(it);
  if (d.status != GATO_OK) return d.status;
  if (out) {
    out->result.flags = d.reply.flags;
    out->result.sqp_iters = d.reply.sqp_iters;
    out->result.pcg_iters = d.reply.pcg_iters;
    out->result.kkt_residual = d.reply.kkt;
    out->result.merit = d.reply.merit;
    std::memcpy(out->u0, d.reply.u0, sizeof(out->u0));
    std::memcpy(out->x1, d.reply.x1, sizeof(out->x1));
    out->submit_ns = d.t_submit;
    out->done_ns = d.t_done;
  }
  return GATO_OK;
}

gato_status gato_server_read(gato_server* s, int32_t session, float* X, float* U, float* lambda) {
  if (!s) return GATO_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (session < 0 || session >= s->capacity || !s->sessions[session].open)
    return server_fail(s, GATO_E_INVALID, "no such session");
  Session& ss = s->sessions[session];
  if (ss.busy) return server_fail(s, GATO_E_BUSY, "session has a request in flight");
  ss.busy = true;
  lk.unlock();
  const size_t K = ss.N + 1, nx = 2 * ss.dof, nu = ss.dof;
  cudaError_t e = cudaSuccess;
  if (X) e = cudaMemcpyAsync(X, ss.X, K * nx * sizeof(float), cudaMemcpyDeviceToHost, s->admin);
  if (U && e == cudaSuccess) e = cudaMemcpyAsync(U, ss.U, ss.N * nu * sizeof(float), cudaMemcpyDeviceToHost, s->admin);
  if (lambda && e == cudaSuccess)
    e = cudaMemcpyAsync(lambda, ss.lam, K * nx * sizeof(float), cudaMemcpyDeviceToHost, s->admin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->admin);
  lk.lock();
  ss.busy = false;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return server_fail(s, GATO_E_CUDA, std::string("read: ") + cudaGetErrorString(e));
  }
  return GATO_OK;
}

gato_status gato_server_drive(gato_server* s, const int32_t* sessions, int32_t n_sessions,
                              const float* x_init, const double* t_arrival, const int32_t* client,
                              const float* noise, int64_t n, float* latency_ms, gato_drive_stats* out) {
  if (!s || !sessions || n_sessions < 1 || !x_init || (n > 0 && (!t_arrival || !client || !noise || !latency_ms)) ||
      n < 0)
    return GATO_E_INVALID;
  for (int64_t i = 0; i < n; ++i) {
    if (client[i] < 0 || client[i] >= n_sessions) return server_fail(s, GATO_E_INVALID, "client out of range");
    if (i > 0 && t_arrival[i] < t_arrival[i - 1]) return server_fail(s, GATO_E_INVALID, "arrivals not sorted");
  }
  std::vector<int> nx(n_sessions);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->driving) return server_fail(s, GATO_E_BUSY, "another drive is running");
    for (int c = 0; c < n_sessions; ++c) {
      const int sid = sessions[c];
      if (sid < 0 || sid >= s->capacity || !s->sessions[sid].open)
        return server_fail(s, GATO_E_INVALID, "no such session");
      if (s->sessions[sid].busy) return server_fail(s, GATO_E_BUSY, "session has a request in flight");
      nx[c] = 2 * s->sessions[sid].dof;
    }
    s->driving = true;
    s->completed_order.clear();
  }
  std::vector<float> last(x_init, x_init + (size_t)n_sessions * 14);
  std::vector<std::deque<int64_t>> waiting(n_sessions);
  std::vector<char> busy(n_sessions, 0);
  std::unordered_map<int64_t, int64_t> in_flight;
  const int64_t launches0 = s->launches;
  const int64_t t0 = now_ns();
  int64_t next = 0, done = 0, backlog = 0, max_backlog = 0;
  gato_status st = GATO_OK;
  auto submit = [&](int64_t i) -> gato_status {
    const int c = client[i];
    float x[16] = {0.f};
    for (int k = 0; k < nx[c]; ++k) x[k] = last[(size_t)c * 14 + k] + noise[(size_t)i * 14 + k];
    int64_t t = 0;
    gato_status r = gato_server_submit(s, sessions[c], x, 1, &t);
    if (r != GATO_OK) return r;
    in_flight[t] = i;
    busy[c] = 1;
    return GATO_OK;
  };
  while (done < n && st == GATO_OK) {
    const double now = (now_ns() - t0) * 1e-9;
    while (next < n && t_arrival[next] <= now && st == GATO_OK) {
      const int c = client[next];
      if (busy[c]) {
        waiting[c].push_back(next);
        max_backlog = std::max(max_backlog, ++backlog);
      } else {
        st = submit(next);
      }
      ++next;
    }
    if (st != GATO_OK) break;
    std::vector<int64_t> fin;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto have = [&] { return !s->completed_order.empty() || s->failed != GATO_OK; };
      if (next < n) {
        const auto until = std::chrono::steady_clock::time_point(std::chrono::nanoseconds(
            t0 + (int64_t)(t_arrival[next] * 1e9)));
        s->cv.wait_until(lk, until, have);
      } else {
        s->cv.wait_for(lk, std::chrono::milliseconds(100), have);
      }
      if (s->failed != GATO_OK) st = s->failed;
      fin.assign(s->completed_order.begin(), s->completed_order.end());
      s->completed_order.clear();
    }
    for (int64_t t : fin) {
      auto it = in_flight.find(t);
      if (it == in_flight.end()) continue;
      const int64_t i = it->second;
      in_flight.erase(it);
      gato_reply r;
      gato_status ps = gato_server_poll(s, t, 0, &r);
      if (ps != GATO_OK) {
        st = ps;
        break;
      }
      const int c = client[i];
      latency_ms[i] = (float)(((double)(r.done_ns - t0) * 1e-9 - t_arrival[i]) * 1e3);
      for (int k = 0; k < 14; ++k) last[(size_t)c * 14 + k] = r.x1[k];
      busy[c] = 0;
      ++done;
      if (!waiting[c].empty()) {
        const int64_t w = waiting[c].front();
        waiting[c].pop_front();
        --backlog;
        st = submit(w);
        if (st != GATO_OK) break;
      }
    }
  }
  const double elapsed = (now_ns() - t0) * 1e-9;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->driving = false;
    s->completed_order.clear();
  }
  // requests still on the GPU after an error are waited for (their tickets consumed)
  for (auto& kv : in_flight) gato_server_poll(s, kv.first, -1, nullptr);
  if (out) {
    out->completed = done;
    out->elapsed_s = elapsed;
    out->launches = s->launches - launches0;
    out->max_backlog = max_backlog;
  }
  return st;
}

gato_status gato_server_get_stats(gato_server* s, gato_server_stats* out) {
  if (!s || !out) return GATO_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  out->capacity = s->capacity;
  int open = 0;
  for (const auto& ss : s->sessions) open += ss.open ? 1 : 0;
  out->sessions_open = open;
  out->max_batch = s->max_batch;
  out->max_inflight = s->n_ctx;
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->launches = s->launches;
  out->pending = (int64_t)s->pending.size();
  out->reserved_bytes = s->reserved;
  return GATO_OK;
}

}  // extern "C"
