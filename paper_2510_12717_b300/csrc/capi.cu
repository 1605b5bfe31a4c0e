// C ABI of the batched MPC solver: context, device arenas, tickets.
// Declarations and argument conventions: include/mpcgpu.h.
#include <cuda_runtime.h>
#include <math.h>
#include <cmath>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "mpcgpu.h"
#include "solver.h"
#include "policy.h"

using mpc::Arena;

namespace {

constexpr int kMaxTickets = 64;

struct Ticket {
  uint64_t id = 0;
  int state = 0;   // 0 free, 1 submitted, 2 solved
  mpc::Batch b{};
  cudaStream_t stream = nullptr;   // stream the ticket was solved on
  // the slot's work-queue buffers are in use until this event (recorded after
  // the gather) has completed: a free slot is reused only then
  cudaEvent_t done = nullptr;
  bool pending = false;
};

// a captured solve (graph mode): replayed while the batch buffers and the
// stream are the same.  Each entry owns its work-queue buffers (replays of
// one entry are ordered on its stream).
struct GraphEntry {
  int n = -1;
  const void* ptrs[5] = {};
  cudaStream_t stream = nullptr;
  int variant = 0, check_every = 0, trees = 0, grid = 0;
  int flags = 0;                    // mpc_solve_ex flags of the captured solve
  int kernels = 0;                  // kernels the captured graph launches
  float early_polish = 0.f;
  cudaGraphExec_t exec = nullptr;
};
constexpr int kMaxGraphs = 16;

// A tuned launch configuration, kept per (factor precision, batch-size bin
// = floor(log2 n)): kernel variant (register cap, resident warps), resident
// grid of the persistent kernel in blocks per SM (agents in flight; 0 = all
// that fit), ADMM residual-check interval and early-polish threshold.
// mean_horizon records the tuned batch's horizon mix.
struct TuneEntry {
  int precision = 0, size_bin = 0;
  int variant = 1, check_every = 10, grid_per_sm = 0;
  float early_polish = 100.f, ms = 0.f, mean_horizon = 0.f;
};
int size_bin(int n) { int b = 0; while ((2 << b) <= n) ++b; return b; }

}  // namespace

struct mpc_ctx {
  mpc_config cfg{};
  cudaStream_t stream = nullptr;
  Arena ar{};
  // non-const views of the model arenas
  float* model = nullptr;
  double* sched = nullptr;
  int* horizon = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  std::vector<int> live;            // host copy: horizon of live slots, 0 = free
  Ticket tickets[kMaxTickets];
  uint64_t next_ticket = 1;
  // staging for the host-buffer path and model uploads
  int* d_ids = nullptr;
  float *d_x0 = nullptr, *d_qd = nullptr, *d_cmd = nullptr, *d_phase = nullptr;
  float *d_tau = nullptr, *d_qset = nullptr, *d_qdset = nullptr, *d_val = nullptr;
  int* d_status = nullptr;
  float* d_mstage = nullptr;
  double* d_sstage = nullptr;
  int* d_hstage = nullptr;
  // pinned host staging of mpc_set_models_async (allocated by its first call)
  int* h_ids = nullptr;
  float* h_mstage = nullptr;
  double* h_sstage = nullptr;
  int* h_hstage = nullptr;
  int* qorder = nullptr;             // per-ticket work-queue buffers [kMaxTickets][A]
  int* qcount = nullptr;             // per-ticket queue counters [kMaxTickets][8]
  GraphEntry graphs[kMaxGraphs];
  int graph_next = 0;
  int* gorder = nullptr;             // per-graph work-queue buffers [kMaxGraphs][A]
  int* gcount = nullptr;             // per-graph queue counters [kMaxGraphs][8]
  long long launches = 0;
  long long solves = 0;
  long long graph_replays = 0;
  std::vector<TuneEntry> tuned;      // mpc_autotune's choices, used by every later solve of their key
  int nsm = 0;                       // SMs of the context's device
  // residual policy (mpc_set_policy): bfloat16 weights, FP32 biases
  mpc::PolicyDev pol{};
  bool has_policy = false;
  bool has_trees = false;            // some agent was given a kinematic tree (mpc_set_trees)
  std::string err = "ok";
};

static mpc_status fail(mpc_ctx* c, mpc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

static mpc_status cuda_fail(mpc_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, MPC_ERR_CUDA, m);
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

template <class T>
static cudaError_t alloc(mpc_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back(q);
  ctx->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return cudaMemset(q, 0, count * sizeof(T));
}

// bytes of all arenas for A agents of horizon up to n
static size_t arena_bytes(size_t A, size_t n) {
  using namespace mpc;
  size_t f = 0;
  f += A * MODEL_F;                                  // model
  f += A * SCHED_D * 2;                              // sched (doubles)
  f += A;                                            // horizon
  f += A * ((n + 1) * VS + n * VS + 2 * n * RS + 1); // xs us ws ys rho
  f += A;                                            // warm
  f += A * (OUT_F + ST_I);                           // out, stat
  f += A * IN_F;
  f += A * ((n + 1) * VS + n * VS + 3 * n * RS);     // xref uref rlo rhi rcls
  f += A * lin_floats((int)n);
  f += A * (2 * n * BLK + n * 64 + n * 128 + n * VS); // cK cH cE cEl cD
  f += A * ((n + 1) * VS + 2 * n * VS + n * RS + 1); // xt ut dv act order
  f += A * (1 + 30 + 18 + 4 + 1 + 18 * 3 + 2);       // host-path staging
  f += A * (MODEL_F + 2 * SCHED_D + 1);              // model upload staging
  f += A * (kMaxTickets + kMaxGraphs) + (kMaxTickets + kMaxGraphs) * 8;   // work queues
  f += F_COUNT;                                      // device event counters
  return f * 4;
}

// bytes of the literal form's extra arenas (block LDL^T factors, forward
// vectors, dynamics multipliers)
static size_t ldl_bytes(size_t A, size_t n) {
  using namespace mpc;
  return A * n * (size_t)(LDL_REC + LDL_W + VS + LDL_S) * 4 + A * 4;
}

extern "C" {

mpc_status mpc_default_config(mpc_config* cfg) {
  if (!cfg) return MPC_ERR_INVALID;
  memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->max_agents = 16384;
  cfg->max_horizon = 20;
  cfg->hbm_budget_bytes = 0;
  cfg->precision = MPC_FP32;
  cfg->form = MPC_FORM_FUSED;
  cfg->rho0 = 0.1f;
  cfg->sigma = 1e-6f;
  cfg->alpha = 1.6f;
  cfg->eps_abs = 1e-5f;
  cfg->eps_rel = 1e-5f;
  cfg->max_iter = 4000;
  cfg->fixed_iters = 0;
  cfg->check_every = 10;
  cfg->adaptive_rho = 1;
  cfg->polish = 1;
  cfg->warm_start = 1;
  cfg->variant = 1;
  cfg->early_polish = 100.f;
  cfg->graph = 0;
  cfg->warm_polish = 1;
  cfg->refine_steps = -1;
  cfg->spin_limit = mpc::kSpinLimit;
  cfg->wait_test_agent = -1;
  cfg->ruiz_iters = 0;
  cfg->kin_rows = 0;
  cfg->swing_height = 0.075f;
  cfg->v_takeoff = 0.1f;
  cfg->v_touchdown = -0.1f;
  return MPC_OK;
}

mpc_status mpc_create(const mpc_config* cfg, mpc_ctx** out) {
  if (!out) return MPC_ERR_INVALID;
  *out = nullptr;
  if (!cfg) return MPC_ERR_INVALID;
  if (cfg->max_agents <= 0 || cfg->max_horizon < 2 || cfg->max_horizon > MPC_MAX_HORIZON)
    return MPC_ERR_INVALID;
  if (cfg->precision < MPC_FP32 || cfg->precision > MPC_TF32X3) return MPC_ERR_INVALID;
  if (cfg->refine_steps < -1 || cfg->refine_steps > 4) return MPC_ERR_INVALID;
  if (cfg->spin_limit <= 0 || cfg->wait_test_agent < -1 || cfg->wait_test_agent >= cfg->max_agents)
    return MPC_ERR_INVALID;
  if (cfg->form != MPC_FORM_PLAIN && cfg->form != MPC_FORM_FUSED && cfg->form != MPC_FORM_LDL)
    return MPC_ERR_INVALID;
  if (cfg->ruiz_iters < 0 || cfg->ruiz_iters > 50) return MPC_ERR_INVALID;
  // the kinematic rows exist in the literal form only, and not with its scaling
  if (cfg->kin_rows < 0 || cfg->kin_rows > 1 ||
      (cfg->kin_rows && (cfg->form != MPC_FORM_LDL || cfg->ruiz_iters != 0)) ||
      !std::isfinite(cfg->swing_height) || !std::isfinite(cfg->v_takeoff) || !std::isfinite(cfg->v_touchdown))
    return MPC_ERR_INVALID;
  if (!(cfg->rho0 > 0.f) || !(cfg->sigma > 0.f) || !(cfg->alpha > 0.f && cfg->alpha < 2.f) ||
      !(cfg->eps_abs >= 0.f) || !(cfg->eps_rel >= 0.f) || cfg->max_iter <= 0 || cfg->fixed_iters < 0 ||
      cfg->graph < 0 || cfg->graph > 1 ||
      cfg->check_every <= 0 || cfg->variant < 1 || cfg->variant > 2 || !(cfg->early_polish >= 0.f))
    return MPC_ERR_INVALID;
  const size_t A = (size_t)cfg->max_agents, n = (size_t)cfg->max_horizon;
  const size_t extra = cfg->form == MPC_FORM_LDL ? ldl_bytes(A, n) : 0;
  if (cfg->hbm_budget_bytes && arena_bytes(A, n) + extra > cfg->hbm_budget_bytes) return MPC_ERR_BUDGET;

  mpc_ctx* ctx = new mpc_ctx();
  ctx->cfg = *cfg;
  ctx->stream = static_cast<cudaStream_t>(cfg->stream);
  ctx->live.assign(A, 0);
  auto bail = [&](mpc_status s) {
    for (void* p : ctx->allocs) cudaFree(p);
    delete ctx;
    return s;
  };
  if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(MPC_ERR_CUDA);
  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, cfg->device);
  Arena& a = ctx->ar;
  a.max_agents = (int)A;
  a.maxN = (int)n;
  using namespace mpc;
  cudaError_t e = cudaSuccess;
#define AL(ptr, cnt) if (e == cudaSuccess) e = alloc(ctx, &(ptr), (cnt))
  AL(ctx->model, A * MODEL_F);
  AL(ctx->sched, A * SCHED_D);
  AL(ctx->horizon, A);
  AL(a.xs, A * (n + 1) * VS);
  AL(a.us, A * n * VS);
  AL(a.ws, A * n * RS);
  AL(a.ys, A * n * RS);
  AL(a.rho, A);
  AL(a.warm_valid, A);
  AL(a.out, A * OUT_F);
  AL(a.stat, A * ST_I);
  AL(a.inp, A * IN_F);
  AL(a.xref, A * (n + 1) * VS);
  AL(a.uref, A * n * VS);
  AL(a.rlo, A * n * RS);
  AL(a.rhi, A * n * RS);
  AL(a.rcls, A * n * RS);
  AL(a.lin, A * (size_t)lin_floats((int)n));
  AL(a.cK, A * n * BLK);
  AL(a.cH, A * n * BLK);
  AL(a.cE, A * n * 64);
  AL(a.cEl, A * n * 128);
  AL(a.cD, A * n * VS);
  AL(a.xt, A * (n + 1) * VS);
  AL(a.ut, A * n * VS);
  AL(a.dv, A * n * VS);
  AL(a.act, A * n * RS);
  AL(a.order, A);
  AL(a.counter, 4);
  AL(a.fault, mpc::F_COUNT);
  AL(ctx->d_ids, A);
  AL(ctx->d_x0, A * 30);
  AL(ctx->d_qd, A * 18);
  AL(ctx->d_cmd, A * 4);
  AL(ctx->d_phase, A);
  AL(ctx->d_tau, A * 18);
  AL(ctx->d_qset, A * 18);
  AL(ctx->d_qdset, A * 18);
  AL(ctx->d_val, A);
  AL(ctx->d_status, A);
  AL(ctx->d_mstage, A * MODEL_F);
  AL(ctx->d_sstage, A * SCHED_D);
  AL(ctx->d_hstage, A);
  AL(ctx->qorder, (size_t)kMaxTickets * A);
  AL(ctx->qcount, (size_t)kMaxTickets * 8);
  AL(ctx->gorder, (size_t)kMaxGraphs * A);
  AL(ctx->gcount, (size_t)kMaxGraphs * 8);
  if (cfg->form == MPC_FORM_LDL) {
    AL(a.lL, A * n * LDL_REC);
    AL(a.lw, A * n * LDL_W);
    AL(a.ly, A * n * VS);
    AL(a.lS, A * n * LDL_S);
    AL(a.lc, A);
  }
#undef AL
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(e == cudaErrorMemoryAllocation ? MPC_ERR_BUDGET : MPC_ERR_CUDA);
  }
  if (cfg->hbm_budget_bytes && ctx->bytes > cfg->hbm_budget_bytes) return bail(MPC_ERR_BUDGET);
  a.model = ctx->model;
  a.sched = ctx->sched;
  a.horizon = ctx->horizon;
  *out = ctx;
  return MPC_OK;
}

mpc_status mpc_destroy(mpc_ctx* ctx) {
  if (!ctx) return MPC_ERR_INVALID;
  cudaSetDevice(ctx->cfg.device);
  cudaStreamSynchronize(ctx->stream);
  cudaDeviceSynchronize();
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& t : ctx->tickets)
    if (t.done) cudaEventDestroy(t.done);
  for (void* p : ctx->allocs) cudaFree(p);
  cudaFreeHost(ctx->h_ids);
  cudaFreeHost(ctx->h_mstage);
  cudaFreeHost(ctx->h_sstage);
  cudaFreeHost(ctx->h_hstage);
  delete ctx;
  return MPC_OK;
}

static bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return false;
  return true;
}

static const char* check_model(const mpc_agent_model& m, int maxN) {
  if (m.N < 2 || m.N > maxN) return "horizon N outside [2, max_horizon]";
  if (!(m.dt > 0) || !(m.period > 0) || !isfinite(m.dt) || !isfinite(m.period)) return "dt and period must be > 0";
  if (!(m.mass > 0)) return "mass must be > 0";
  for (int i = 0; i < 3; ++i) if (!(m.inertia[i] > 0)) return "inertia must be > 0";
  for (int i = 0; i < 30; ++i) {
    if (!(m.R[i] > 0) || !isfinite(m.R[i])) return "R must be > 0 (strictly convex QP)";
    if (!(m.Q[i] >= 0) || !isfinite(m.Q[i])) return "Q must be >= 0";
  }
  if (!(m.mu > 0) || !(m.fz_max > 0) || !(m.qd_max > 0) || !(m.q_lim > 0)) return "bounds must be > 0";
  if (!finite_all(&m.lever[0][0], 6) || !finite_all(&m.J_leg[0][0][0], 60) || !finite_all(m.M_j, 18) ||
      !finite_all(m.h_j, 18) || !finite_all(m.Kp, 18) || !finite_all(m.Kd, 18) || !finite_all(m.q_nom, 18) ||
      !finite_all(m.duty, 2) || !finite_all(m.offset, 2))
    return "non-finite model entry";
  return nullptr;
}

static void pack_model(const mpc_agent_model& m, float* f, double* s) {
  using namespace mpc;
  memset(f, 0, sizeof(float) * MODEL_F);
  f[M_MASS] = (float)m.mass;
  f[M_INVM] = (float)(1.0 / m.mass);
  for (int i = 0; i < 3; ++i) f[M_INERTIA + i] = (float)m.inertia[i];
  for (int i = 0; i < 2; ++i)
    for (int c = 0; c < 3; ++c) f[M_LEVER + 3 * i + c] = (float)m.lever[i][c];
  for (int i = 0; i < 2; ++i)
    for (int r = 0; r < 6; ++r)
      for (int j = 0; j < 5; ++j) f[M_JLEG + 30 * i + 5 * r + j] = (float)m.J_leg[i][r][j];
  for (int j = 0; j < 18; ++j) {
    f[M_MJ + j] = (float)m.M_j[j];
    f[M_HJ + j] = (float)m.h_j[j];
    f[M_KP + j] = (float)m.Kp[j];
    f[M_KD + j] = (float)m.Kd[j];
    f[M_QNOM + j] = (float)m.q_nom[j];
  }
  for (int i = 0; i < 30; ++i) {
    f[M_Q + i] = (float)m.Q[i];
    f[M_R + i] = (float)m.R[i];
  }
  f[M_MU] = (float)m.mu;
  f[M_FZMAX] = (float)m.fz_max;
  f[M_QDMAX] = (float)m.qd_max;
  f[M_QLIM] = (float)m.q_lim;
  f[M_DT] = (float)m.dt;
  memset(s, 0, sizeof(double) * SCHED_D);
  s[S_DT] = m.dt;
  s[S_PERIOD] = m.period;
  s[S_DUTY] = m.duty[0];
  s[S_DUTY + 1] = m.duty[1];
  s[S_OFF] = m.offset[0];
  s[S_OFF + 1] = m.offset[1];
}

}  // extern "C"

// scatter packed kinematic trees into their agents' model records and mark them
__global__ void mpc_k_scatter_trees(int n, const int* ids, const float* tf, float* model) {
  const int row = blockIdx.x;
  if (row >= n) return;
  float* rec = model + (size_t)ids[row] * mpc::MODEL_F;
  for (int t = threadIdx.x; t < mpc::TREE_F; t += blockDim.x) rec[mpc::M_TREE + t] = tf[(size_t)row * mpc::TREE_F + t];
  if (threadIdx.x == 0) rec[mpc::M_TREE_ON] = 1.f;
}

// scatter packed models into their slots, clear warm starts
__global__ void mpc_k_scatter_models(int n, const int* ids, const float* mf, const double* ms, const int* hz,
                                     float* model, double* sched, int* horizon, int* warm) {
  const int row = blockIdx.x;
  if (row >= n) return;
  const int s = ids[row];
  for (int t = threadIdx.x; t < mpc::MODEL_F; t += blockDim.x)
    model[(size_t)s * mpc::MODEL_F + t] = mf[(size_t)row * mpc::MODEL_F + t];
  for (int t = threadIdx.x; t < mpc::SCHED_D; t += blockDim.x)
    sched[(size_t)s * mpc::SCHED_D + t] = ms[(size_t)row * mpc::SCHED_D + t];
  if (threadIdx.x == 0) {
    horizon[s] = hz[row];
    warm[s] = 0;
  }
}

extern "C" {

mpc_status mpc_set_models(mpc_ctx* ctx, int32_t n, const int32_t* ids, const mpc_agent_model* models) {
  if (!ctx) return MPC_ERR_INVALID;
  if (n < 0 || n > ctx->cfg.max_agents || (n > 0 && (!ids || !models)))
    return fail(ctx, MPC_ERR_INVALID, "set_models: bad count or NULL buffer");
  if (n == 0) return MPC_OK;
  std::vector<float> mf((size_t)n * mpc::MODEL_F);
  std::vector<double> ms((size_t)n * mpc::SCHED_D);
  std::vector<int> hz(n);
  for (int i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= ctx->cfg.max_agents)
      return fail(ctx, MPC_ERR_INVALID, "set_models: agent id out of range");
    const char* why = check_model(models[i], ctx->cfg.max_horizon);
    if (why) return fail(ctx, MPC_ERR_INVALID, std::string("set_models: ") + why);
    pack_model(models[i], &mf[(size_t)i * mpc::MODEL_F], &ms[(size_t)i * mpc::SCHED_D]);
    hz[i] = models[i].N;
  }
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaMemcpyAsync(ctx->d_ids, ids, sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_mstage, mf.data(), sizeof(float) * mf.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_sstage, ms.data(), sizeof(double) * ms.size(), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_hstage, hz.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  mpc_k_scatter_models<<<n, 128, 0, ctx->stream>>>(n, ctx->d_ids, ctx->d_mstage, ctx->d_sstage, ctx->d_hstage,
                                                    ctx->model, ctx->sched, ctx->horizon, ctx->ar.warm_valid);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < n; ++i) ctx->live[ids[i]] = hz[i];
  return MPC_OK;
}

mpc_status mpc_set_models_async(mpc_ctx* ctx, int32_t n, const int32_t* ids, const mpc_agent_model* models,
                                void* stream) {
  if (!ctx) return MPC_ERR_INVALID;
  if (n < 0 || n > ctx->cfg.max_agents || (n > 0 && (!ids || !models)))
    return fail(ctx, MPC_ERR_INVALID, "set_models_async: bad count or NULL buffer");
  for (int i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= ctx->cfg.max_agents)
      return fail(ctx, MPC_ERR_INVALID, "set_models_async: agent id out of range");
    const char* why = check_model(models[i], ctx->cfg.max_horizon);
    if (why) return fail(ctx, MPC_ERR_INVALID, std::string("set_models_async: ") + why);
  }
  CK(cudaSetDevice(ctx->cfg.device));
  if (!ctx->h_mstage) {
    const size_t A = (size_t)ctx->cfg.max_agents;
    CK(cudaMallocHost(&ctx->h_ids, sizeof(int) * A));
    CK(cudaMallocHost(&ctx->h_mstage, sizeof(float) * A * mpc::MODEL_F));
    CK(cudaMallocHost(&ctx->h_sstage, sizeof(double) * A * mpc::SCHED_D));
    CK(cudaMallocHost(&ctx->h_hstage, sizeof(int) * A));
  }
  if (n == 0) return MPC_OK;
  for (int i = 0; i < n; ++i) {
    pack_model(models[i], ctx->h_mstage + (size_t)i * mpc::MODEL_F, ctx->h_sstage + (size_t)i * mpc::SCHED_D);
    ctx->h_hstage[i] = models[i].N;
    ctx->h_ids[i] = ids[i];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(ctx->d_ids, ctx->h_ids, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_mstage, ctx->h_mstage, sizeof(float) * (size_t)n * mpc::MODEL_F,
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_sstage, ctx->h_sstage, sizeof(double) * (size_t)n * mpc::SCHED_D,
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_hstage, ctx->h_hstage, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  mpc_k_scatter_models<<<n, 128, 0, st>>>(n, ctx->d_ids, ctx->d_mstage, ctx->d_sstage, ctx->d_hstage,
                                          ctx->model, ctx->sched, ctx->horizon, ctx->ar.warm_valid);
  CK(cudaGetLastError());
  for (int i = 0; i < n; ++i) ctx->live[ids[i]] = models[i].N;
  return MPC_OK;
}

static const char* check_tree(const mpc_tree_model& t) {
  for (int j = 0; j < 18; ++j) {
    double nn = 0.0;
    for (int c = 0; c < 3; ++c) {
      if (!std::isfinite(t.axis[j][c]) || !std::isfinite(t.offset[j][c]) || !std::isfinite(t.com[j][c]) ||
          !std::isfinite(t.inertia[j][c]))
        return "non-finite tree value";
      if (t.inertia[j][c] < 0.0) return "negative link inertia";
      nn += t.axis[j][c] * t.axis[j][c];
    }
    if (std::fabs(std::sqrt(nn) - 1.0) > 1e-6) return "joint axis is not a unit vector";
    if (!std::isfinite(t.mass[j]) || t.mass[j] < 0.0) return "bad link mass";
  }
  return nullptr;
}

mpc_status mpc_set_trees(mpc_ctx* ctx, int32_t n, const int32_t* ids, const mpc_tree_model* trees) {
  if (!ctx) return MPC_ERR_INVALID;
  if (n < 0 || n > ctx->cfg.max_agents || (n > 0 && (!ids || !trees)))
    return fail(ctx, MPC_ERR_INVALID, "set_trees: bad count or NULL buffer");
  if (n == 0) return MPC_OK;
  using namespace mpc;
  std::vector<float> tf((size_t)n * TREE_F);
  for (int i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= ctx->cfg.max_agents) return fail(ctx, MPC_ERR_INVALID, "set_trees: agent id out of range");
    const char* why = check_tree(trees[i]);
    if (why) return fail(ctx, MPC_ERR_INVALID, std::string("set_trees: ") + why);
    float* f = &tf[(size_t)i * TREE_F];
    for (int j = 0; j < 18; ++j) {
      float* J = f + j * TREE_J;
      for (int c = 0; c < 3; ++c) {
        J[TA_AXIS + c] = (float)trees[i].axis[j][c];
        J[TA_OFF + c] = (float)trees[i].offset[j][c];
        J[TA_COM + c] = (float)trees[i].com[j][c];
        J[TA_INER + c] = (float)trees[i].inertia[j][c];
      }
      J[TA_MASS] = (float)trees[i].mass[j];
    }
  }
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaMemcpyAsync(ctx->d_ids, ids, sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_mstage, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice, ctx->stream));
  mpc_k_scatter_trees<<<n, 128, 0, ctx->stream>>>(n, ctx->d_ids, ctx->d_mstage, ctx->model);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_trees = true;
  return MPC_OK;
}

mpc_status mpc_set_model(mpc_ctx* ctx, int32_t agent_id, const mpc_agent_model* model) {
  return mpc_set_models(ctx, 1, &agent_id, model);
}

mpc_status mpc_release_agent(mpc_ctx* ctx, int32_t agent_id) {
  if (!ctx) return MPC_ERR_INVALID;
  if (agent_id < 0 || agent_id >= ctx->cfg.max_agents || !ctx->live[agent_id])
    return fail(ctx, MPC_ERR_INVALID, "release: unknown agent");
  ctx->live[agent_id] = 0;
  int zero = 0;
  CK(cudaMemcpyAsync(ctx->ar.warm_valid + agent_id, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->horizon + agent_id, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MPC_OK;
}

mpc_status mpc_submit(mpc_ctx* ctx, int32_t n, const int32_t* ids, const float* x0, const float* qd,
                      const float* cmd, const float* phase, uint64_t* ticket) {
  if (!ctx) return MPC_ERR_INVALID;
  if (!ticket) return fail(ctx, MPC_ERR_INVALID, "submit: NULL ticket");
  if (n < 0 || n > ctx->cfg.max_agents) return fail(ctx, MPC_ERR_INVALID, "submit: n outside [0, max_agents]");
  if (n > 0 && (!ids || !x0 || !qd || !cmd || !phase)) return fail(ctx, MPC_ERR_INVALID, "submit: NULL buffer");
  for (int t = 0; t < kMaxTickets; ++t) {
    Ticket& tk = ctx->tickets[t];
    if (tk.state == 0 && tk.pending) {
      const cudaError_t q = cudaEventQuery(tk.done);
      if (q == cudaErrorNotReady) continue;        // its kernels may still read the slot
      if (q != cudaSuccess) return cuda_fail(ctx, q, "submit: ticket event");
      tk.pending = false;
    }
    if (tk.state == 0) {
      tk.id = ctx->next_ticket++;
      tk.state = 1;
      tk.b = mpc::Batch{n, ids, x0, qd, cmd, phase, ctx->qorder + (size_t)t * ctx->cfg.max_agents,
                        ctx->qcount + (size_t)t * 8};
      *ticket = tk.id;
      return MPC_OK;
    }
  }
  return fail(ctx, MPC_ERR_STATE, "submit: too many pending tickets (64)");
}

static Ticket* find_ticket(mpc_ctx* ctx, uint64_t id) {
  for (int t = 0; t < kMaxTickets; ++t)
    if (ctx->tickets[t].state && ctx->tickets[t].id == id) return &ctx->tickets[t];
  return nullptr;
}

static mpc::SolverParams params_of(const mpc_config& c) {
  mpc::SolverParams p;
  p.rho0 = c.rho0; p.sigma = c.sigma; p.alpha = c.alpha; p.eps_abs = c.eps_abs; p.eps_rel = c.eps_rel;
  p.early_polish = c.early_polish;
  p.max_iter = c.max_iter; p.fixed_iters = c.fixed_iters; p.check_every = c.check_every;
  p.adaptive_rho = c.adaptive_rho; p.polish = c.polish; p.warm_start = c.warm_start;
  p.warm_polish = c.warm_polish;
  p.precision = c.precision;
  // automatic: where the stage products are TF32 / BF16, the steps that win
  // back the products' rounding (measured against the FP64 oracle: TF32 needs
  // 2, BF16 3); otherwise (FP32, split TF32, FP64) one on every polish: the FP32 factor's rounding
  // (stage Schur complements whose weights span 10^4) leaves the joint rates
  // of about one agent in 400 a few 1e-4 off, which the torque map's
  // qddot = (qdot_1 - qdot_0)/dt turns into torque errors of several times
  // the tolerance; one step removes them
  const int low = c.precision == MPC_TF32 ? 2 : c.precision == MPC_BF16 ? 3 : 1;
  p.refine = c.refine_steps >= 0 ? c.refine_steps : low;
  p.refine_admm = c.refine_steps >= 0 ? c.refine_steps : low;
  p.trees = 0;
  p.split = 1;
  // the literal form starts every solve from f_init: the set-up kernel's cold start
  if (c.form == MPC_FORM_LDL) p.warm_start = 0;
  p.spin_limit = c.spin_limit;
  p.wait_test_slot = c.wait_test_agent;
  p.defer = 0;
  p.ruiz = c.ruiz_iters;
  // the swing curve's control points: B(0) = B(1) = 0, dB/dt(0) = 5 (b1 - b0)
  // = v_to, dB/dt(1) = 5 (b5 - b4) = v_td; then b2 + b3 from B(0.5) = z_swing
  // (32 B(0.5) = b0 + 5 b1 + 10 (b2 + b3) + 5 b4 + b5) and b3 - b2 from
  // dB/dt(0.5) = 0 (16/5 dB/dt(0.5) = 3 (b4 - b1) + 2 (b3 - b2) + b5 - b0)
  p.kin = c.kin_rows;
  {
    const double b1 = c.v_takeoff / 5.0, b4 = -c.v_touchdown / 5.0;
    const double sum23 = (32.0 * c.swing_height - 5.0 * (b1 + b4)) / 10.0;
    const double dif32 = 1.5 * (b1 - b4);
    const double bz[6] = {0.0, b1, 0.5 * (sum23 - dif32), 0.5 * (sum23 + dif32), b4, 0.0};
    for (int j = 0; j < 6; ++j) p.kin_b[j] = (float)bz[j];
  }
  return p;
}

// the launch configuration of a batch: the tuned entry of its key if there
// is one, else the context's options
static const TuneEntry* tuned_for(const mpc_ctx* ctx, int n) {
  const int bin = size_bin(n);
  for (const auto& t : ctx->tuned)
    if (t.precision == ctx->cfg.precision && t.size_bin == bin) return &t;
  return nullptr;
}

static cudaError_t enqueue_solve(mpc_ctx* ctx, Ticket* tk, cudaStream_t st, int flags) {
  int launches = 0;
  mpc_config cfg = ctx->cfg;
  int grid = 0;
  if (const TuneEntry* t = tuned_for(ctx, tk->b.n)) {
    cfg.variant = t->variant; cfg.check_every = t->check_every; cfg.early_polish = t->early_polish;
    grid = t->grid_per_sm * ctx->nsm;
  }
  mpc::SolverParams prm = params_of(cfg);
  prm.trees = ctx->has_trees ? 1 : 0;
  prm.defer = (flags & MPC_SOLVE_DEFER_COLD) ? 3 : (flags & MPC_SOLVE_DEFER_SLOW) ? 2
                                                : (flags & MPC_SOLVE_DEFER_ADMM) ? 1 : 0;
  if (flags & MPC_SOLVE_ADMM_ONLY) prm.warm_polish = 0;
  const int form = ctx->cfg.form;
  // graph capture needs a non-default stream; on the legacy stream the
  // solve is launched directly
  if (!ctx->cfg.graph || form != MPC_FORM_FUSED || st == nullptr || st == cudaStreamLegacy) {
    cudaError_t e = mpc::launch_solve(ctx->ar, tk->b, prm, form, grid, st, &launches, cfg.variant);
    ctx->launches += launches;
    return e;
  }
  const void* ptrs[5] = {tk->b.ids, tk->b.x0, tk->b.qd, tk->b.cmd, tk->b.phase};
  for (int gi = 0; gi < kMaxGraphs; ++gi) {
    GraphEntry& g = ctx->graphs[gi];
    if (g.exec && g.n == tk->b.n && g.stream == st && g.variant == cfg.variant &&
        g.check_every == cfg.check_every && g.early_polish == cfg.early_polish && g.grid == grid &&
        g.trees == prm.trees && g.flags == flags && !memcmp(g.ptrs, ptrs, sizeof(ptrs))) {
      ctx->graph_replays += 1;
      ctx->launches += g.kernels;       // the kernels recorded in the graph
      return cudaGraphLaunch(g.exec, st);
    }
  }
  // first time: one-time set-up outside the capture, then capture the solve
  // with this entry's own queue buffers
  cudaError_t e = mpc::launch_solve(ctx->ar, mpc::Batch{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                        nullptr},
                                    prm, form, 0, st, nullptr, cfg.variant);
  if (e != cudaSuccess) return e;
  const int gi = ctx->graph_next;
  ctx->graph_next = (ctx->graph_next + 1) % kMaxGraphs;
  GraphEntry& g = ctx->graphs[gi];
  if (g.exec) {
    // the evicted entry's queue buffers may still be read by a replay in flight
    cudaStreamSynchronize(g.stream);
    cudaGraphExecDestroy(g.exec);
  }
  g = GraphEntry{};
  mpc::Batch b = tk->b;
  b.order = ctx->gorder + (size_t)gi * ctx->cfg.max_agents;
  b.counter = ctx->gcount + (size_t)gi * 8;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  e = mpc::launch_solve(ctx->ar, b, prm, form, grid, st, &launches, cfg.variant);
  cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { g.exec = nullptr; return e; }
  g.n = tk->b.n;
  memcpy(g.ptrs, ptrs, sizeof(ptrs));
  g.stream = st;
  g.variant = cfg.variant;
  g.check_every = cfg.check_every;
  g.early_polish = cfg.early_polish;
  g.grid = grid;
  g.trees = prm.trees;
  g.flags = flags;
  g.kernels = launches;
  ctx->launches += launches;
  return cudaGraphLaunch(g.exec, st);
}

mpc_status mpc_solve_ex(mpc_ctx* ctx, uint64_t ticket, void* stream, int32_t flags) {
  if (!ctx) return MPC_ERR_INVALID;
  Ticket* tk = find_ticket(ctx, ticket);
  if (!tk) return fail(ctx, MPC_ERR_NOT_READY, "solve: unknown ticket");
  if (tk->state != 1) return fail(ctx, MPC_ERR_STATE, "solve: ticket already solved");
  if (flags & ~(MPC_SOLVE_DEFER_ADMM | MPC_SOLVE_ADMM_ONLY | MPC_SOLVE_DEFER_SLOW | MPC_SOLVE_DEFER_COLD))
    return fail(ctx, MPC_ERR_INVALID, "solve: unknown flag");
  if ((flags & (MPC_SOLVE_DEFER_SLOW | MPC_SOLVE_DEFER_COLD)) && (flags & ~(MPC_SOLVE_DEFER_SLOW | MPC_SOLVE_DEFER_COLD)))
    return fail(ctx, MPC_ERR_INVALID, "solve: DEFER_SLOW / DEFER_COLD combine with no other flag");
  if ((flags & MPC_SOLVE_DEFER_SLOW) && (flags & MPC_SOLVE_DEFER_COLD))
    return fail(ctx, MPC_ERR_INVALID, "solve: DEFER_SLOW and DEFER_COLD exclude each other");
  if (flags && ctx->cfg.form != MPC_FORM_FUSED)
    return fail(ctx, MPC_ERR_INVALID, "solve: flags need the fused form");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = enqueue_solve(ctx, tk, st, flags);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "solve: kernel launch");
  ctx->solves += 1;
  tk->state = 2;
  tk->stream = st;
  return MPC_OK;
}

mpc_status mpc_solve_on(mpc_ctx* ctx, uint64_t ticket, void* stream) { return mpc_solve_ex(ctx, ticket, stream, 0); }

mpc_status mpc_solve(mpc_ctx* ctx, uint64_t ticket) { return mpc_solve_ex(ctx, ticket, ctx ? ctx->stream : nullptr, 0); }

mpc_status mpc_get_torques(mpc_ctx* ctx, uint64_t ticket, float* tau, float* q_set, float* qd_set, float* value,
                           int32_t* agent_status) {
  if (!ctx) return MPC_ERR_INVALID;
  Ticket* tk = find_ticket(ctx, ticket);
  if (!tk) return fail(ctx, MPC_ERR_NOT_READY, "get_torques: unknown ticket");
  if (tk->state != 2) return fail(ctx, MPC_ERR_NOT_READY, "get_torques: ticket not solved");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaError_t e = mpc::launch_gather(ctx->ar, tk->b.n, tk->b.ids, tau, q_set, qd_set, value, agent_status,
                                     tk->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "get_torques: gather");
  ctx->launches += 1;
  if (!tk->done) CK(cudaEventCreateWithFlags(&tk->done, cudaEventDisableTiming));
  CK(cudaEventRecord(tk->done, tk->stream));
  tk->pending = true;
  tk->state = 0;
  return MPC_OK;
}

mpc_status mpc_solve_host(mpc_ctx* ctx, int32_t n, const int32_t* ids, const float* x0, const float* qd,
                          const float* cmd, const float* phase, float* tau, float* q_set, float* qd_set,
                          float* value, int32_t* agent_status) {
  if (!ctx) return MPC_ERR_INVALID;
  if (n < 0 || n > ctx->cfg.max_agents) return fail(ctx, MPC_ERR_INVALID, "solve_host: bad n");
  if (n > 0 && (!ids || !x0 || !qd || !cmd || !phase)) return fail(ctx, MPC_ERR_INVALID, "solve_host: NULL input");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->d_ids, ids, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_x0, x0, sizeof(float) * 30 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_qd, qd, sizeof(float) * 18 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_cmd, cmd, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_phase, phase, sizeof(float) * n, cudaMemcpyHostToDevice, st));
  uint64_t t = 0;
  mpc_status s = mpc_submit(ctx, n, ctx->d_ids, ctx->d_x0, ctx->d_qd, ctx->d_cmd, ctx->d_phase, &t);
  if (s != MPC_OK) return s;
  s = mpc_solve(ctx, t);
  if (s != MPC_OK) return s;
  s = mpc_get_torques(ctx, t, ctx->d_tau, ctx->d_qset, ctx->d_qdset, ctx->d_val, ctx->d_status);
  if (s != MPC_OK) return s;
  if (tau) CK(cudaMemcpyAsync(tau, ctx->d_tau, sizeof(float) * 18 * n, cudaMemcpyDeviceToHost, st));
  if (q_set) CK(cudaMemcpyAsync(q_set, ctx->d_qset, sizeof(float) * 18 * n, cudaMemcpyDeviceToHost, st));
  if (qd_set) CK(cudaMemcpyAsync(qd_set, ctx->d_qdset, sizeof(float) * 18 * n, cudaMemcpyDeviceToHost, st));
  if (value) CK(cudaMemcpyAsync(value, ctx->d_val, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
  if (agent_status) CK(cudaMemcpyAsync(agent_status, ctx->d_status, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return MPC_OK;
}

mpc_status mpc_get_agent_stats(mpc_ctx* ctx, int32_t n, const int32_t* ids, int32_t* iters, int32_t* refactors,
                               int32_t* polished, float* prim, float* dual, float* prim_n, float* dual_n) {
  if (!ctx) return MPC_ERR_INVALID;
  if (n < 0 || (n > 0 && !ids)) return fail(ctx, MPC_ERR_INVALID, "get_agent_stats: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t A = ctx->cfg.max_agents;
  std::vector<int> st(A * mpc::ST_I);
  std::vector<float> out(A * mpc::OUT_F);
  CK(cudaMemcpy(st.data(), ctx->ar.stat, sizeof(int) * st.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(out.data(), ctx->ar.out, sizeof(float) * out.size(), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= (int)A) return fail(ctx, MPC_ERR_INVALID, "get_agent_stats: id out of range");
    const int* s = &st[(size_t)ids[i] * mpc::ST_I];
    const float* o = &out[(size_t)ids[i] * mpc::OUT_F];
    if (iters) iters[i] = s[mpc::T_ITERS];
    if (refactors) refactors[i] = s[mpc::T_REFAC];
    if (polished) polished[i] = s[mpc::T_POLISHED] ? (s[mpc::T_FIRST] ? 2 : 1) : 0;
    if (prim) prim[i] = o[mpc::O_PRIM];
    if (dual) dual[i] = o[mpc::O_DUAL];
    if (prim_n) prim_n[i] = o[mpc::O_PRIM_N];
    if (dual_n) dual_n[i] = o[mpc::O_DUAL_N];
  }
  return MPC_OK;
}

mpc_status mpc_export_state(mpc_ctx* ctx, int32_t id, float* x, float* u, float* w, float* y, float* rho) {
  if (!ctx) return MPC_ERR_INVALID;
  if (id < 0 || id >= ctx->cfg.max_agents || !ctx->live[id]) return fail(ctx, MPC_ERR_INVALID, "export: unknown agent");
  using namespace mpc;
  const int N = ctx->live[id], n = ctx->cfg.max_horizon;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<float> bx((N + 1) * VS), bu(N * VS), bw(N * RS), by(N * RS);
  CK(cudaMemcpy(bx.data(), ctx->ar.xs + (size_t)id * (n + 1) * VS, sizeof(float) * bx.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bu.data(), ctx->ar.us + (size_t)id * n * VS, sizeof(float) * bu.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bw.data(), ctx->ar.ws + (size_t)id * n * RS, sizeof(float) * bw.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(by.data(), ctx->ar.ys + (size_t)id * n * RS, sizeof(float) * by.size(), cudaMemcpyDeviceToHost));
  for (int k = 0; k <= N; ++k)
    for (int i = 0; i < 30; ++i)
      if (x) x[k * 30 + i] = bx[k * VS + i];
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < 30; ++i)
      if (u) u[k * 30 + i] = bu[k * VS + i];
    for (int r = 0; r < 56; ++r) {
      if (w) w[k * 56 + r] = bw[k * RS + r];
      if (y) y[k * 56 + r] = by[k * RS + r];
    }
  }
  if (rho) CK(cudaMemcpy(rho, ctx->ar.rho + id, sizeof(float), cudaMemcpyDeviceToHost));
  return MPC_OK;
}

mpc_status mpc_export_qp(mpc_ctx* ctx, int32_t id, float* xref, float* uref, float* lo, float* hi, float* A,
                         float* B, float* c) {
  if (!ctx) return MPC_ERR_INVALID;
  if (id < 0 || id >= ctx->cfg.max_agents || !ctx->live[id]) return fail(ctx, MPC_ERR_INVALID, "export_qp: unknown agent");
  using namespace mpc;
  const int N = ctx->live[id], n = ctx->cfg.max_horizon;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<float> bxr((N + 1) * VS), bur(N * VS), blo(N * RS), bhi(N * RS), lin(lin_floats(n));
  std::vector<float> mdl(MODEL_F);
  CK(cudaMemcpy(bxr.data(), ctx->ar.xref + (size_t)id * (n + 1) * VS, sizeof(float) * bxr.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bur.data(), ctx->ar.uref + (size_t)id * n * VS, sizeof(float) * bur.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(blo.data(), ctx->ar.rlo + (size_t)id * n * RS, sizeof(float) * blo.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(bhi.data(), ctx->ar.rhi + (size_t)id * n * RS, sizeof(float) * bhi.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(lin.data(), ctx->ar.lin + (size_t)id * lin_floats(n), sizeof(float) * lin.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(mdl.data(), ctx->model + (size_t)id * MODEL_F, sizeof(float) * MODEL_F, cudaMemcpyDeviceToHost));
  const float dt = mdl[M_DT];
  for (int k = 0; k <= N; ++k)
    for (int i = 0; i < 30; ++i)
      if (xref) xref[k * 30 + i] = bxr[k * VS + i];
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < 30; ++i)
      if (uref) uref[k * 30 + i] = bur[k * VS + i];
    for (int r = 0; r < 56; ++r) {
      if (lo) lo[k * 56 + r] = blo[k * RS + r];
      if (hi) hi[k * 56 + r] = bhi[k * RS + r];
    }
    // the device keeps the coupled 22 x 22 blocks dense (A_base, B) plus the
    // stage's leg-coupling block dA_k and affine term c_k; the arm joints are
    // q+ = q + dt qdot
    const float* st = lin.data() + L_STAGE + k * 64;
    float* Ak = A ? A + (size_t)k * 900 : nullptr;
    float* Bk = B ? B + (size_t)k * 900 : nullptr;
    for (int i = 0; i < 30; ++i)
      for (int j = 0; j < 30; ++j) {
        float a = 0.f, b = 0.f;
        if (i < NC && j < NC) {
          a = lin[L_ABASE + j * LDD_HOST + i];
          b = lin[L_B + j * LDD_HOST + i];
          if (i >= 9 && i < 12 && j >= 12) a += st[(i - 9) * 10 + (j - 12)];
        } else if (i == j) {
          a = 1.f;
          b = dt;
        }
        if (Ak) Ak[i * 30 + j] = a;
        if (Bk) Bk[i * 30 + j] = b;
      }
    for (int i = 0; i < 30; ++i)
      if (c) c[k * 30 + i] = i < NC ? st[32 + i] : 0.f;
  }
  return MPC_OK;
}

mpc_status mpc_import_state(mpc_ctx* ctx, int32_t id, const float* x, const float* u, const float* w,
                            const float* y, float rho) {
  if (!ctx) return MPC_ERR_INVALID;
  if (id < 0 || id >= ctx->cfg.max_agents || !ctx->live[id]) return fail(ctx, MPC_ERR_INVALID, "import: unknown agent");
  if (!x || !u || !w || !y || !(rho > 0.f)) return fail(ctx, MPC_ERR_INVALID, "import: bad state");
  using namespace mpc;
  const int N = ctx->live[id], n = ctx->cfg.max_horizon;
  std::vector<float> bx((N + 1) * VS, 0.f), bu(N * VS, 0.f), bw(N * RS, 0.f), by(N * RS, 0.f);
  for (int k = 0; k <= N; ++k)
    for (int i = 0; i < 30; ++i) bx[k * VS + i] = x[k * 30 + i];
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < 30; ++i) bu[k * VS + i] = u[k * 30 + i];
    for (int r = 0; r < 56; ++r) {
      bw[k * RS + r] = w[k * 56 + r];
      by[k * RS + r] = y[k * 56 + r];
    }
  }
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(ctx->ar.xs + (size_t)id * (n + 1) * VS, bx.data(), sizeof(float) * bx.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ar.us + (size_t)id * n * VS, bu.data(), sizeof(float) * bu.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ar.ws + (size_t)id * n * RS, bw.data(), sizeof(float) * bw.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ar.ys + (size_t)id * n * RS, by.data(), sizeof(float) * by.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ar.rho + id, &rho, sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->ar.warm_valid + id, &N, sizeof(int), cudaMemcpyHostToDevice));
  return MPC_OK;
}

mpc_status mpc_autotune(mpc_ctx* ctx, uint64_t ticket, int32_t repeats, char* report, size_t cap) {
  if (!ctx) return MPC_ERR_INVALID;
  Ticket* tk = find_ticket(ctx, ticket);
  if (!tk) return fail(ctx, MPC_ERR_NOT_READY, "autotune: unknown ticket");
  if (tk->state != 1) return fail(ctx, MPC_ERR_STATE, "autotune: ticket already solved");
  if (ctx->cfg.form == MPC_FORM_LDL) return fail(ctx, MPC_ERR_INVALID, "autotune: not for the literal form");
  if (repeats < 1) repeats = 1;
  CK(cudaSetDevice(ctx->cfg.device));
  // the batch's horizon mix (host copy of its ids; recorded with the choice)
  std::vector<int> ids(tk->b.n);
  if (tk->b.n) CK(cudaMemcpy(ids.data(), tk->b.ids, sizeof(int) * tk->b.n, cudaMemcpyDeviceToHost));
  double hsum = 0.0;
  for (int id : ids) hsum += (id >= 0 && id < ctx->cfg.max_agents) ? ctx->live[id] : 0;
  const float mean_h = tk->b.n ? (float)(hsum / tk->b.n) : 0.f;
  struct Cand { int variant, grid_per_sm, check_every; float early; float ms; float solved; };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<int> st(tk->b.n);
  int* d_st = ctx->d_status;
  auto run = [&](Cand& c) -> cudaError_t {
    mpc_config cfg = ctx->cfg;
    cfg.variant = c.variant; cfg.check_every = c.check_every; cfg.early_polish = c.early;
    mpc::SolverParams prm = params_of(cfg);
    prm.trees = ctx->has_trees ? 1 : 0;
    const int grid = c.grid_per_sm * ctx->nsm;
    int launches = 0;
    // one untimed pass (warm starts from this candidate), then timed passes
    cudaError_t e = mpc::launch_solve(ctx->ar, tk->b, prm, cfg.form, grid, ctx->stream, &launches, cfg.variant);
    if (e != cudaSuccess) return e;
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < repeats && e == cudaSuccess; ++r)
      e = mpc::launch_solve(ctx->ar, tk->b, prm, cfg.form, grid, ctx->stream, &launches, cfg.variant);
    if (e != cudaSuccess) return e;
    cudaEventRecord(e1, ctx->stream);
    e = mpc::launch_gather(ctx->ar, tk->b.n, tk->b.ids, nullptr, nullptr, nullptr, nullptr, d_st, ctx->stream);
    if (e != cudaSuccess) return e;
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(st.data(), d_st, sizeof(int) * tk->b.n, cudaMemcpyDeviceToHost);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int ok = 0;
    for (int v : st) ok += (v == MPC_AGENT_SOLVED);
    c.ms = ms / repeats;
    c.solved = tk->b.n ? (float)ok / tk->b.n : 1.f;
    ctx->launches += launches;
    return e;
  };
  // fastest among the candidates that solve as many agents as the best one
  auto pick = [](const std::vector<Cand>& cs) {
    float best_solved = 0.f;
    for (auto& c : cs) best_solved = c.solved > best_solved ? c.solved : best_solved;
    int best = 0;
    for (size_t i = 0; i < cs.size(); ++i)
      if (cs[i].solved >= best_solved && (cs[best].solved < best_solved || cs[i].ms < cs[best].ms)) best = (int)i;
    return best;
  };
  // stage 1: register cap (resident warps) x agents in flight (resident
  // blocks per SM: all that fit, or fewer, which keeps more of the in-flight
  // agents' stage blocks in L2); stage 2: the ADMM schedule on the best shape
  std::vector<Cand> all;
  std::vector<Cand> shape;
  for (int v = 1; v <= 2; ++v)
    for (int g = 0; g <= v; ++g)      // g = 0: all that fit (v + 1 blocks per SM)
      shape.push_back(Cand{v, g, ctx->cfg.check_every, ctx->cfg.early_polish, 0.f, 0.f});
  for (auto& c : shape) CK(run(c));
  const Cand s1 = shape[pick(shape)];
  std::vector<Cand> sched;
  for (int c : {5, 10})
    for (float ep : {30.f, 100.f, 1000.f}) sched.push_back(Cand{s1.variant, s1.grid_per_sm, c, ep, 0.f, 0.f});
  for (auto& c : sched) CK(run(c));
  const Cand best = sched[pick(sched)];
  all = shape;
  all.insert(all.end(), sched.begin(), sched.end());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the choice: the context's options (as before) and the entry of this key
  ctx->cfg.variant = best.variant;
  ctx->cfg.check_every = best.check_every;
  ctx->cfg.early_polish = best.early;
  TuneEntry te;
  te.precision = ctx->cfg.precision; te.size_bin = size_bin(tk->b.n);
  te.variant = best.variant; te.check_every = best.check_every; te.grid_per_sm = best.grid_per_sm;
  te.early_polish = best.early; te.ms = best.ms; te.mean_horizon = mean_h;
  bool found = false;
  for (auto& t : ctx->tuned)
    if (t.precision == te.precision && t.size_bin == te.size_bin) { t = te; found = true; }
  if (!found) ctx->tuned.push_back(te);
  if (report && cap) {
    char b[256];
    snprintf(b, sizeof(b), "{\"chosen\": {\"variant\": %d, \"grid_per_sm\": %d, \"check_every\": %d, \"early_polish\": %g}, "
             "\"key\": {\"precision\": %d, \"size_bin\": %d, \"mean_horizon\": %.2f}, \"candidates\": [",
             best.variant, best.grid_per_sm, best.check_every, best.early, te.precision, te.size_bin, mean_h);
    std::string js = b;
    for (size_t i = 0; i < all.size(); ++i) {
      snprintf(b, sizeof(b), "%s{\"variant\": %d, \"grid_per_sm\": %d, \"check_every\": %d, \"early_polish\": %g, "
               "\"ms\": %.4f, \"solved\": %.5f}", i ? ", " : "", all[i].variant, all[i].grid_per_sm,
               all[i].check_every, all[i].early, all[i].ms, all[i].solved);
      js += b;
    }
    js += "], \"table\": [";
    for (size_t i = 0; i < ctx->tuned.size(); ++i) {
      const auto& t = ctx->tuned[i];
      snprintf(b, sizeof(b), "%s{\"precision\": %d, \"size_bin\": %d, \"variant\": %d, \"grid_per_sm\": %d, "
               "\"check_every\": %d, \"early_polish\": %g, \"ms\": %.4f, \"mean_horizon\": %.2f}", i ? ", " : "",
               t.precision, t.size_bin, t.variant, t.grid_per_sm, t.check_every, t.early_polish, t.ms, t.mean_horizon);
      js += b;
    }
    js += "]}";
    snprintf(report, cap, "%s", js.c_str());
  }
  return MPC_OK;
}

mpc_status mpc_get_stats(mpc_ctx* ctx, char* buf, size_t cap) {
  if (!ctx || !buf || cap == 0) return MPC_ERR_INVALID;
  int live = 0;
  for (int h : ctx->live) live += h != 0;
  // polish attempts of the live agents' last solves: [0] none accepted, [a] a solves
  long long hist[9] = {0};
  int fault[mpc::F_COUNT] = {0};
  {
    std::vector<int> st((size_t)ctx->cfg.max_agents * mpc::ST_I);
    CK(cudaSetDevice(ctx->cfg.device));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(st.data(), ctx->ar.stat, sizeof(int) * st.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(fault, ctx->ar.fault, sizeof(fault), cudaMemcpyDeviceToHost));
    for (int a = 0; a < ctx->cfg.max_agents; ++a) {
      if (!ctx->live[a]) continue;
      const int t = st[(size_t)a * mpc::ST_I + mpc::T_ATTEMPTS];
      hist[t >= 0 && t <= 8 ? t : 0] += 1;
    }
  }
  snprintf(buf, cap,
           "{\"max_agents\": %d, \"max_horizon\": %d, \"live_agents\": %d, \"arena_bytes\": %zu, "
           "\"form\": \"%s\", \"kernel_launches\": %lld, \"solves\": %lld, \"graph_replays\": %lld, "
           "\"smem_per_block\": %zu, \"warps_per_block\": %d, \"variant\": %d, \"check_every\": %d, "
           "\"early_polish\": %g, \"graph\": %d, \"wait_timeouts\": %d, "
           "\"polish_attempts\": [%lld, %lld, %lld, %lld, %lld, %lld, %lld, %lld, %lld]}",
           ctx->cfg.max_agents, ctx->cfg.max_horizon, live, ctx->bytes,
           ctx->cfg.form == MPC_FORM_FUSED ? "fused" : ctx->cfg.form == MPC_FORM_LDL ? "ldl" : "plain", ctx->launches, ctx->solves, ctx->graph_replays,
           mpc::smem_bytes_per_block(), mpc::WARPS_PER_BLOCK, ctx->cfg.variant, ctx->cfg.check_every,
           (double)ctx->cfg.early_polish, ctx->cfg.graph, fault[mpc::F_WAIT_TIMEOUTS], hist[0], hist[1], hist[2], hist[3], hist[4], hist[5],
           hist[6], hist[7], hist[8]);
  return MPC_OK;
}

const char* mpc_last_error(mpc_ctx* ctx) {
  if (!ctx) return "NULL context";
  return ctx->err.c_str();
}

}  // extern "C"

// ------------------------------------------------------------ residual policy
// round to the nearest bfloat16, ties to even (the bit pattern of a float32)
static uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);   // inf / nan pass through
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// W [in][out] (host, FP32) -> [out_pad][in_pad] bfloat16, zero padding
static std::vector<uint16_t> transpose_bf16(const float* W, int in, int out, int in_pad, int out_pad) {
  std::vector<uint16_t> t((size_t)in_pad * out_pad, 0);
  for (int i = 0; i < in; ++i)
    for (int o = 0; o < out; ++o) t[(size_t)o * in_pad + i] = bf16_bits(W[(size_t)i * out + o]);
  return t;
}

mpc_status mpc_set_policy(mpc_ctx* ctx, const float* W1, const float* b1, const float* W2, const float* b2,
                          const float* W3, const float* b3, const float* W4, const float* b4, float blend_lambda) {
  using namespace mpc;
  if (!ctx) return MPC_ERR_INVALID;
  if (!W1 || !b1 || !W2 || !b2 || !W3 || !b3 || !W4 || !b4) return fail(ctx, MPC_ERR_INVALID, "set_policy: NULL");
  if (!isfinite(blend_lambda)) return fail(ctx, MPC_ERR_INVALID, "set_policy: lambda not finite");
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  const std::vector<uint16_t> w[4] = {transpose_bf16(W1, POL_OBS, POL_HID, POL_K1, POL_HID),
                                      transpose_bf16(W2, POL_HID, POL_HID, POL_HID, POL_HID),
                                      transpose_bf16(W3, POL_HID, POL_HID, POL_HID, POL_HID),
                                      transpose_bf16(W4, POL_HID, POL_ACT, POL_HID, POL_N4)};
  std::vector<float> b4p(POL_N4, 0.f);
  for (int i = 0; i < POL_ACT; ++i) b4p[i] = b4[i];
  const float* b[4] = {b1, b2, b3, b4p.data()};
  const int bn[4] = {POL_HID, POL_HID, POL_HID, POL_N4};
  if (!ctx->has_policy) {
    void* p = nullptr;
    size_t total = 0;
    for (int l = 0; l < 4; ++l) total += w[l].size() * 2 + (size_t)bn[l] * 4;
    CK(cudaMalloc(&p, total));
    ctx->allocs.push_back(p);
    ctx->bytes += total;
    uint8_t* q = static_cast<uint8_t*>(p);
    const __nv_bfloat16** W[4] = {&ctx->pol.W1, &ctx->pol.W2, &ctx->pol.W3, &ctx->pol.W4};
    const float** B[4] = {&ctx->pol.b1, &ctx->pol.b2, &ctx->pol.b3, &ctx->pol.b4};
    for (int l = 0; l < 4; ++l) { *W[l] = reinterpret_cast<const __nv_bfloat16*>(q); q += w[l].size() * 2; }
    for (int l = 0; l < 4; ++l) { *B[l] = reinterpret_cast<const float*>(q); q += (size_t)bn[l] * 4; }
  }
  const void* Wd[4] = {ctx->pol.W1, ctx->pol.W2, ctx->pol.W3, ctx->pol.W4};
  const void* Bd[4] = {ctx->pol.b1, ctx->pol.b2, ctx->pol.b3, ctx->pol.b4};
  for (int l = 0; l < 4; ++l) {
    CK(cudaMemcpy(const_cast<void*>(Wd[l]), w[l].data(), w[l].size() * 2, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(const_cast<void*>(Bd[l]), b[l], (size_t)bn[l] * 4, cudaMemcpyHostToDevice));
  }
  ctx->pol.lambda = blend_lambda;
  ctx->has_policy = true;
  return MPC_OK;
}

mpc_status mpc_policy_torques(mpc_ctx* ctx, uint64_t ticket, float* tau, float* action) {
  if (!ctx) return MPC_ERR_INVALID;
  if (!ctx->has_policy) return fail(ctx, MPC_ERR_STATE, "policy_torques: no policy set");
  Ticket* tk = find_ticket(ctx, ticket);
  if (!tk) return fail(ctx, MPC_ERR_NOT_READY, "policy_torques: unknown ticket");
  if (tk->state != 2) return fail(ctx, MPC_ERR_NOT_READY, "policy_torques: ticket not solved");
  CK(cudaSetDevice(ctx->cfg.device));
  cudaError_t e = mpc::launch_policy(ctx->ar, tk->b.n, tk->b.ids, ctx->pol, tau, action, tk->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "policy_torques");
  ctx->launches += 1;
  return MPC_OK;
}
