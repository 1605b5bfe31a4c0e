// Synthetic request source for the serving form (C ABI in include/mpcgpu.h,
// mpc_load_*): replays a trace of request arrival times and agent slots in
// real time on the server's clock, from a thread of its own, through
// mpc_server_push.  Each request is one 10 ms environment step of its
// agent: gait phase += phase_step and one step of a mean-reverting walk of
// the state around the agent's initial state,
//   x <- x_init + a (x - x_init) + sigma xi,   xi ~ N(0, I),
// measured joint velocities 0.1 xi', commanded height = current height.
// The normal draws come from a pool generated once (Box-Muller on a
// splitmix64 stream, small enough to stay in cache) and read as windows at
// pseudo-random offsets.  The trace is split by slot over kThreads threads
// (each walk state has one writer), and each pushes in chunks of at most
// kChunk requests so that the server's table is never held for long.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "mpcgpu.h"

namespace {
constexpr int kThreads = 2;
constexpr int kChunk = 1024;
}  // namespace

struct mpc_load {
  mpc_server* srv = nullptr;
  int pool = 0;
  std::vector<double> t[kThreads];      // per thread: its requests' arrival times and slots
  std::vector<int32_t> slot[kThreads];
  std::vector<float> X, XI, CMD, PH;   // per slot walk state
  float a = 0.95f, sigma = 0.02f, phase_step = 0.02f;
  std::vector<float> noise;
  uint64_t seed = 0;
  std::mutex mu[kThreads];             // per thread: guards its slots' walk state against resets
  std::thread th[kThreads];
  std::atomic<bool> stop{false};
  std::atomic<int> running{0};
  std::atomic<int> error{MPC_OK};
  std::vector<double> lag[kThreads];   // per pushed chunk: push time minus its oldest arrival
  double base = 0.0;                   // the trace's origin on the server's clock
};

namespace {

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
double unit(uint64_t& s) { return ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

void run(mpc_load* L, int w) {
  const std::vector<double>& T = L->t[w];
  const std::vector<int32_t>& S = L->slot[w];
  const int64_t n = (int64_t)T.size();
  std::vector<int32_t> cs(kChunk);
  std::vector<float> cx((size_t)kChunk * 30), cq((size_t)kChunk * 18), cc((size_t)kChunk * 4), cp(kChunk);
  std::vector<double> ct(kChunk);
  uint64_t rng = L->seed + 0x1234567ull * (uint64_t)(w + 1);
  const uint64_t span = (uint64_t)(L->noise.size() - 48);
  int64_t i = 0;
  while (i < n && !L->stop.load(std::memory_order_relaxed)) {
    const double now = mpc_server_clock(L->srv);
    if (T[i] + L->base > now) {
      const double wait = std::min(T[i] + L->base - now, 1e-4);
      std::this_thread::sleep_for(std::chrono::duration<double>(wait));
      continue;
    }
    int64_t j = i;
    while (j < n && j - i < kChunk && T[j] + L->base <= now) ++j;
    const int m = (int)(j - i);
    {
      std::lock_guard<std::mutex> g(L->mu[w]);
      for (int k = 0; k < m; ++k) {
        const int s = S[i + k];
        cs[k] = s;
        ct[k] = T[i + k] + L->base;
        const float* xi = &L->noise[splitmix64(rng) % span];
        float* x = &L->X[(size_t)s * 30];
        const float* x0 = &L->XI[(size_t)s * 30];
        for (int c = 0; c < 30; ++c) x[c] = x0[c] + L->a * (x[c] - x0[c]) + L->sigma * xi[c];
        float ph = L->PH[s] + L->phase_step;
        ph -= std::floor(ph);
        L->PH[s] = ph;
        std::memcpy(&cx[(size_t)k * 30], x, sizeof(float) * 30);
        for (int c = 0; c < 18; ++c) cq[(size_t)k * 18 + c] = 0.1f * xi[30 + c];
        std::memcpy(&cc[(size_t)k * 4], &L->CMD[(size_t)s * 4], sizeof(float) * 4);
        cc[(size_t)k * 4] = x[2];
        cp[k] = ph;
      }
    }
    const mpc_status r = mpc_server_push(L->srv, m, cs.data(), cx.data(), cq.data(), cc.data(), cp.data(), ct.data());
    if (r != MPC_OK) { L->error = r; break; }
    L->lag[w].push_back(mpc_server_clock(L->srv) - ct[0]);
    i = j;
  }
  L->running.fetch_sub(1);
}

}  // namespace

extern "C" {

mpc_status mpc_load_start(mpc_server* srv, int64_t n, const double* t_arrive, const int32_t* slots, int32_t pool,
                          const float* x_init, const float* cmd, const float* phase, float revert, float sigma,
                          float phase_step, uint64_t seed, mpc_load** out) {
  if (!srv || !out || n < 0 || pool <= 0 || (n > 0 && (!t_arrive || !slots)) || !x_init || !cmd || !phase)
    return MPC_ERR_INVALID;
  for (int64_t k = 0; k < n; ++k) {
    if (slots[k] < 0 || slots[k] >= pool) return MPC_ERR_INVALID;
    if (k && t_arrive[k] < t_arrive[k - 1]) return MPC_ERR_INVALID;
  }
  auto* L = new mpc_load();
  L->srv = srv;
  L->pool = pool;
  for (int64_t k = 0; k < n; ++k) {
    const int w = slots[k] % kThreads;
    L->t[w].push_back(t_arrive[k]);
    L->slot[w].push_back(slots[k]);
  }
  L->X.assign(x_init, x_init + (size_t)pool * 30);
  L->XI = L->X;
  L->CMD.assign(cmd, cmd + (size_t)pool * 4);
  L->PH.assign(phase, phase + pool);
  L->a = revert; L->sigma = sigma; L->phase_step = phase_step;
  L->seed = seed;
  uint64_t rng = seed;
  L->noise.resize(1 << 16);
  for (size_t k = 0; k + 1 < L->noise.size(); k += 2) {
    const double u1 = unit(rng), u2 = unit(rng);
    const double r = std::sqrt(-2.0 * std::log(u1));
    L->noise[k] = (float)(r * std::cos(6.283185307179586 * u2));
    L->noise[k + 1] = (float)(r * std::sin(6.283185307179586 * u2));
  }
  // the trace's times count from the threads' start (the set-up above does
  // not delay the first requests)
  L->base = mpc_server_clock(srv);
  L->running = kThreads;
  for (int w = 0; w < kThreads; ++w) {
    L->lag[w].reserve(1 << 18);
    L->th[w] = std::thread(run, L, w);
  }
  *out = L;
  return MPC_OK;
}

mpc_status mpc_load_reset(mpc_load* L, int32_t n, const int32_t* slots, const float* x_init, const float* cmd,
                          const float* phase) {
  if (!L || n < 0 || (n > 0 && (!slots || !x_init || !cmd || !phase))) return MPC_ERR_INVALID;
  for (int i = 0; i < n; ++i) {
    const int s = slots[i];
    if (s < 0 || s >= L->pool) return MPC_ERR_INVALID;
    std::lock_guard<std::mutex> g(L->mu[s % kThreads]);
    std::memcpy(&L->X[(size_t)s * 30], x_init + (size_t)i * 30, sizeof(float) * 30);
    std::memcpy(&L->XI[(size_t)s * 30], x_init + (size_t)i * 30, sizeof(float) * 30);
    std::memcpy(&L->CMD[(size_t)s * 4], cmd + (size_t)i * 4, sizeof(float) * 4);
    L->PH[s] = phase[i];
  }
  return MPC_OK;
}

mpc_status mpc_load_wait(mpc_load* L, double timeout_s, double* lag_stats) {
  if (!L) return MPC_ERR_INVALID;
  const auto end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (L->running.load() > 0) {
    if (std::chrono::steady_clock::now() > end) return MPC_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(500));
  }
  for (auto& th : L->th)
    if (th.joinable()) th.join();
  if (lag_stats) {
    std::vector<double> v;
    for (auto& l : L->lag) v.insert(v.end(), l.begin(), l.end());
    if (v.empty()) v.push_back(0.0);
    std::sort(v.begin(), v.end());
    lag_stats[0] = v[v.size() / 2];
    lag_stats[1] = v[std::min(v.size() - 1, (size_t)(0.99 * (double)v.size()))];
    lag_stats[2] = v.back();
  }
  return (mpc_status)L->error.load();
}

mpc_status mpc_load_destroy(mpc_load* L) {
  if (!L) return MPC_ERR_INVALID;
  L->stop = true;
  for (auto& th : L->th)
    if (th.joinable()) th.join();
  delete L;
  return MPC_OK;
}

}  // extern "C"
