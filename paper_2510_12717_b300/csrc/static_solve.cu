// Allocation-free solve entry point (mpc_solve_static).
//
// Some callers cannot allocate device memory at the moment they need a
// solve: simulators and plugins that hand over only their own device buffers
// and forbid allocation on their hot path, real-time control loops that must
// not enter the device allocator once running, or processes whose device
// allocator is owned by another framework.  For them this file keeps all of
// the solver's workspace in one file-scope static device array, sized for at
// most kStaticMaxAgents agents of horizon up to kStaticMaxHorizon; every GPU
// that loads the library holds it until the process exits.  The packed models
// pass through process-wide host staging arrays on their way there, so two
// calls that overlap in time race on the host as well as on the GPU, whatever
// their devices or streams.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "mpcgpu.h"
#include "solver.h"

namespace {

constexpr int kStaticMaxAgents = 64;
constexpr int kStaticMaxHorizon = 20;
constexpr int kMaxDevices = 64;

// 256-byte aligned carve-up of the static array (in bytes)
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

struct Layout {
  size_t model, sched, horizon, ids, xs, us, ws, ys, rho, warm, out, stat, inp, xref, uref, rlo, rhi,
      rcls, lin, cK, cH, cE, cEl, cD, xt, ut, dv, act, order, counter, fault, total;
};

constexpr Layout make_layout(size_t A, size_t n) {
  using namespace mpc;
  Layout L{};
  size_t o = 0;
  auto take = [&o](size_t bytes) { size_t at = o; o += align256(bytes); return at; };
  L.model = take(A * MODEL_F * 4);
  L.sched = take(A * SCHED_D * 8);
  L.horizon = take(A * 4);
  L.ids = take(A * 4);
  L.xs = take(A * (n + 1) * VS * 4);
  L.us = take(A * n * VS * 4);
  L.ws = take(A * n * RS * 4);
  L.ys = take(A * n * RS * 4);
  L.rho = take(A * 4);
  L.warm = take(A * 4);
  L.out = take(A * OUT_F * 4);
  L.stat = take(A * ST_I * 4);
  L.inp = take(A * IN_F * 4);
  L.xref = take(A * (n + 1) * VS * 4);
  L.uref = take(A * n * VS * 4);
  L.rlo = take(A * n * RS * 4);
  L.rhi = take(A * n * RS * 4);
  L.rcls = take(A * n * RS * 4);
  L.lin = take(A * (size_t)lin_floats((int)n) * 4);
  L.cK = take(A * n * BLK * 4);
  L.cH = take(A * n * BLK * 4);
  L.cE = take(A * n * 64 * 4);
  L.cEl = take(A * n * 128 * 4);
  L.cD = take(A * n * VS * 4);
  L.xt = take(A * (n + 1) * VS * 4);
  L.ut = take(A * n * VS * 4);
  L.dv = take(A * n * VS * 4);
  L.act = take(A * n * RS * 4);
  L.order = take(A * 4);
  L.counter = take(16);
  L.fault = take(mpc::F_COUNT * 4);
  L.total = o;
  return L;
}

constexpr Layout kL = make_layout(kStaticMaxAgents, kStaticMaxHorizon);

// The workspace.  In host code this name is only a host-side stand-in for the
// device object: its device address must come from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kL.total];

unsigned char* g_base[kMaxDevices] = {};   // device address of g_static_scratch, per device

// host staging of one call's packed models (no allocation: fixed size);
// process-wide, shared by every device and thread
float g_host_model[kStaticMaxAgents * mpc::MODEL_F];
double g_host_sched[kStaticMaxAgents * mpc::SCHED_D];
int g_host_horizon[kStaticMaxAgents];
int g_host_ids[kStaticMaxAgents];

bool finite_n(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return false;
  return true;
}

bool model_ok(const mpc_agent_model& m) {
  if (m.N < 2 || m.N > kStaticMaxHorizon) return false;
  if (!(m.dt > 0) || !(m.period > 0) || !(m.mass > 0) || !(m.mu > 0) || !(m.fz_max > 0) ||
      !(m.qd_max > 0) || !(m.q_lim > 0))
    return false;
  for (int i = 0; i < 3; ++i)
    if (!(m.inertia[i] > 0)) return false;
  for (int i = 0; i < 30; ++i)
    if (!(m.R[i] > 0) || !(m.Q[i] >= 0) || !isfinite(m.R[i]) || !isfinite(m.Q[i])) return false;
  return finite_n(&m.lever[0][0], 6) && finite_n(&m.J_leg[0][0][0], 60) && finite_n(m.M_j, 18) &&
         finite_n(m.h_j, 18) && finite_n(m.Kp, 18) && finite_n(m.Kd, 18) && finite_n(m.q_nom, 18) &&
         finite_n(m.duty, 2) && finite_n(m.offset, 2);
}

void pack(const mpc_agent_model& m, float* f, double* s) {
  using namespace mpc;
  for (int t = 0; t < MODEL_F; ++t) f[t] = 0.f;
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
  for (int t = 0; t < SCHED_D; ++t) s[t] = 0.0;
  s[S_DT] = m.dt;
  s[S_PERIOD] = m.period;
  s[S_DUTY] = m.duty[0];
  s[S_DUTY + 1] = m.duty[1];
  s[S_OFF] = m.offset[0];
  s[S_OFF + 1] = m.offset[1];
}

template <class T>
T* at(unsigned char* base, size_t off) { return reinterpret_cast<T*>(base + off); }

}  // namespace

extern "C" mpc_status mpc_solve_static(int32_t n, const mpc_agent_model* models_host, const float* x0,
                                       const float* qd_meas, const float* cmd, const float* phase,
                                       float* tau, float* q_set, float* qd_set, float* value,
                                       int32_t* agent_status, void* stream) {
  if (n < 0 || n > kStaticMaxAgents) return MPC_ERR_INVALID;   // beyond the static workspace
  if (n == 0) return MPC_OK;
  if (!models_host || !x0 || !qd_meas || !cmd || !phase) return MPC_ERR_INVALID;
  for (int i = 0; i < n; ++i)
    if (!model_ok(models_host[i])) return MPC_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPC_ERR_CUDA;
  // one-time set-up on this device (with it current): the workspace address
  if (!g_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return MPC_ERR_CUDA;
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* b = g_base[dev];
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  for (int i = 0; i < n; ++i) {
    pack(models_host[i], g_host_model + (size_t)i * mpc::MODEL_F, g_host_sched + (size_t)i * mpc::SCHED_D);
    g_host_horizon[i] = models_host[i].N;
    g_host_ids[i] = i;
  }
  mpc::Arena a{};
  a.max_agents = kStaticMaxAgents;
  a.maxN = kStaticMaxHorizon;
  a.model = at<float>(b, kL.model);
  a.sched = at<double>(b, kL.sched);
  a.horizon = at<int>(b, kL.horizon);
  a.xs = at<float>(b, kL.xs);
  a.us = at<float>(b, kL.us);
  a.ws = at<float>(b, kL.ws);
  a.ys = at<float>(b, kL.ys);
  a.rho = at<float>(b, kL.rho);
  a.warm_valid = at<int>(b, kL.warm);
  a.out = at<float>(b, kL.out);
  a.stat = at<int>(b, kL.stat);
  a.inp = at<float>(b, kL.inp);
  a.xref = at<float>(b, kL.xref);
  a.uref = at<float>(b, kL.uref);
  a.rlo = at<float>(b, kL.rlo);
  a.rhi = at<float>(b, kL.rhi);
  a.rcls = at<float>(b, kL.rcls);
  a.lin = at<float>(b, kL.lin);
  a.cK = at<float>(b, kL.cK);
  a.cH = at<float>(b, kL.cH);
  a.cE = at<float>(b, kL.cE);
  a.cEl = at<float>(b, kL.cEl);
  a.cD = at<float>(b, kL.cD);
  a.xt = at<float>(b, kL.xt);
  a.ut = at<float>(b, kL.ut);
  a.dv = at<float>(b, kL.dv);
  a.act = at<int>(b, kL.act);
  a.order = at<int>(b, kL.order);
  a.counter = at<int>(b, kL.counter);
  a.fault = at<int>(b, kL.fault);
  int* d_ids = at<int>(b, kL.ids);

  // models, horizons and the slot list; the whole horizon array is rewritten
  // so that slots of an earlier, larger call are not live
  static int zeros[kStaticMaxAgents] = {};
  if (cudaMemcpyAsync((void*)a.horizon, zeros, sizeof(zeros), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)a.model, g_host_model, sizeof(float) * mpc::MODEL_F * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)a.sched, g_host_sched, sizeof(double) * mpc::SCHED_D * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)a.horizon, g_host_horizon, sizeof(int) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_ids, g_host_ids, sizeof(int) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MPC_ERR_CUDA;
  // every call is a cold start: the warm-start markers must read zero
  if (cudaMemsetAsync(a.warm_valid, 0, sizeof(int) * kStaticMaxAgents, st) != cudaSuccess) return MPC_ERR_CUDA;

  mpc_config c;
  mpc_default_config(&c);
  mpc::SolverParams prm;
  prm.rho0 = c.rho0; prm.sigma = c.sigma; prm.alpha = c.alpha; prm.eps_abs = c.eps_abs;
  prm.eps_rel = c.eps_rel; prm.early_polish = c.early_polish; prm.max_iter = c.max_iter; prm.fixed_iters = c.fixed_iters;
  prm.check_every = c.check_every; prm.adaptive_rho = c.adaptive_rho; prm.polish = c.polish;
  prm.warm_start = 0;
  prm.warm_polish = 0;
  prm.precision = c.precision;
  prm.refine = 0;
  prm.refine_admm = 1;
  prm.trees = 0;
  prm.split = 0;          // no kinematic trees here: the diagonal joint model
  prm.spin_limit = c.spin_limit;
  prm.wait_test_slot = -1;
  prm.defer = 0;
  prm.ruiz = 0;
  prm.kin = 0;
  mpc::Batch bt{n, d_ids, x0, qd_meas, cmd, phase, nullptr, nullptr};
  if (mpc::launch_solve(a, bt, prm, MPC_FORM_FUSED, 0, st, nullptr, c.variant) != cudaSuccess) return MPC_ERR_CUDA;
  if (mpc::launch_gather(a, n, d_ids, tau, q_set, qd_set, value, agent_status, st) != cudaSuccess)
    return MPC_ERR_CUDA;
  return MPC_OK;
}
