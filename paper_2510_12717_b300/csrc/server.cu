// Continuous-batching request server over one solver context (C ABI in
// include/mpcgpu.h, mpc_server_*).
//
// Requests (agent slot, state, arrival time) are pushed from any host thread
// into a per-slot pending table: a later request of a slot replaces the
// state of an earlier one that has not been batched yet (coalescing, newest
// state wins) and adds its arrival time to the slot's list.  One worker
// thread owns the context while the server runs.  Whenever fewer than
// max_inflight batches are on the GPU, it forms the next batch from every
// slot that has pending requests and no batch in flight (oldest first, up to
// max_batch), packs their newest states into pinned host buffers, copies them
// to the device and enqueues set-up, solve and gather on one of its streams
// (mpc_submit, mpc_solve_on, mpc_get_torques) followed by the copy of the
// results back and an event.  When that event has completed, every request
// the batch covered is answered: its latency is the completion time minus its
// arrival time, on one steady clock started by mpc_server_start.  Model swaps
// (agents leaving and joining) are queued and applied by the worker to slots
// with no batch in flight: their upload runs on a stream of its own
// (mpc_set_models_async) while batches continue, and the slots join batches
// again once it has completed.  With deferral on, batches are
// solved with a DEFER flag of mpc_solve_ex: an agent whose polish first fails
// (DEFER_ADMM), or that two reduced KKT solves of it do not settle
// (DEFER_SLOW), comes back MPC_AGENT_DEFERRED, keeps its requests and state in
// a queue, stays in flight, and is finished (ADMM from the saved start, or the
// polish continued) in a batch of deferred agents on an extra lane of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "mpcgpu.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kInF = 30 + 18 + 4 + 1;   // x0, qd_meas, cmd, phase per request
constexpr int kOutF = 18;               // tau per answered slot

struct Lane {                            // one stream and its batch buffers
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  bool deferred_batch = false;              // a batch of deferred agents
  int n = 0;
  double t_launch = 0.0;
  int32_t* h_ids = nullptr;  float* h_in = nullptr;  float* h_tau = nullptr;  int32_t* h_st = nullptr;
  int32_t* d_ids = nullptr;  float* d_in = nullptr;  float* d_tau = nullptr;  int32_t* d_st = nullptr;
  std::vector<int32_t> slots;
  std::vector<std::vector<double>> arrivals;   // per batch row: arrival times it answers
};

struct Deferred {                      // an agent whose solve was deferred
  int32_t slot;
  std::vector<double> arrivals;
  float state[kInF];
};

}  // namespace

struct mpc_server {
  mpc_ctx* ctx = nullptr;
  int device = 0;                                 // the creating thread's device (the context's)
  int pool = 0, max_batch = 0, max_inflight = 1;
  std::vector<Lane> lanes;
  // pending table (guarded by mu)
  std::mutex mu;
  std::condition_variable cv;
  std::vector<float> state;                       // [pool][kInF] newest state per slot
  std::vector<std::vector<double>> pending;       // arrival times per slot
  std::vector<uint8_t> inflight;
  std::vector<int32_t> ready_order;               // scratch of the worker
  std::vector<std::pair<int32_t, mpc_agent_model>> swaps;
  int defer = 0;                                   // 0 off, 1 DEFER_ADMM, 2 DEFER_SLOW, 3 DEFER_COLD
  std::vector<Deferred> deferred_q;                // deferred agents awaiting their ADMM batch
  double swaps_since = -1.0;                      // queue time of the oldest pending swap
  std::vector<int32_t> swapping;                  // slots whose new model is being uploaded
  bool swap_busy = false;                         // an upload is in flight (worker only)
  cudaStream_t swap_stream = nullptr;
  cudaEvent_t swap_done = nullptr;
  // results (guarded by mu)
  std::vector<double> latency;
  std::vector<double> batch_log;                   // per batch: launch time, completion time, agents
  std::vector<float> tau;                          // [pool][18] last answer per slot
  std::vector<int32_t> status;                     // [pool]
  long long pushed = 0, answered = 0, batches = 0, solves = 0, not_solved = 0, swapped = 0, deferred = 0;
  // worker
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<int> error{MPC_OK};
  Clock::time_point t0 = Clock::now();
  char msg[256] = {0};
};

namespace {

double now_s(const mpc_server* s) {
  return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

void set_error(mpc_server* s, int code, const char* what) {
  int expect = MPC_OK;
  if (s->error.compare_exchange_strong(expect, code)) snprintf(s->msg, sizeof(s->msg), "%s", what);
}

// completion of a lane's batch: answer its requests, keep its results
void complete(mpc_server* s, Lane& L) {
  const double t = now_s(s);
  std::lock_guard<std::mutex> g(s->mu);
  const int mb = s->max_batch;
  int kept = 0;
  for (int i = 0; i < L.n; ++i) {
    const int slot = L.slots[i];
    if (!L.deferred_batch && L.h_st[i] == MPC_AGENT_DEFERRED) {
      // its requests wait for the agent's ADMM batch; the slot stays in flight
      Deferred d;
      d.slot = slot;
      d.arrivals.swap(L.arrivals[i]);
      std::memcpy(d.state, L.h_in + (size_t)i * 30, sizeof(float) * 30);
      std::memcpy(d.state + 30, L.h_in + (size_t)mb * 30 + (size_t)i * 18, sizeof(float) * 18);
      std::memcpy(d.state + 48, L.h_in + (size_t)mb * 48 + (size_t)i * 4, sizeof(float) * 4);
      d.state[52] = L.h_in[(size_t)mb * 52 + i];
      s->deferred_q.push_back(std::move(d));
      s->deferred += 1;
      ++kept;
      continue;
    }
    for (double ta : L.arrivals[i]) s->latency.push_back(t - ta);
    s->answered += (long long)L.arrivals[i].size();
    std::memcpy(&s->tau[(size_t)slot * kOutF], L.h_tau + (size_t)i * kOutF, sizeof(float) * kOutF);
    s->status[slot] = L.h_st[i];
    if (L.h_st[i] != 0) s->not_solved += 1;
    s->inflight[slot] = 0;
  }
  s->solves += L.n - kept;
  s->batch_log.push_back(L.t_launch);
  s->batch_log.push_back(t);
  s->batch_log.push_back((double)L.n);
  L.busy = false;
  L.n = 0;
}

// form and enqueue one batch on lane L; false when nothing is ready.
// deferred: a batch of deferred agents (the extra lane), else a regular one
bool launch(mpc_server* s, Lane& L, bool deferred) {
  int n = 0;
  if (deferred) {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->deferred_q.empty()) return false;
    {
      const int mb = s->max_batch;
      n = std::min((int)s->deferred_q.size(), mb);
      L.slots.resize(n);
      L.arrivals.resize(n);
      float* hx = L.h_in;
      float* hq = hx + (size_t)mb * 30;
      float* hc = hq + (size_t)mb * 18;
      float* hp = hc + (size_t)mb * 4;
      for (int i = 0; i < n; ++i) {
        Deferred& d = s->deferred_q[i];
        L.slots[i] = d.slot;
        L.arrivals[i].swap(d.arrivals);
        L.h_ids[i] = d.slot;
        std::memcpy(hx + (size_t)i * 30, d.state, sizeof(float) * 30);
        std::memcpy(hq + (size_t)i * 18, d.state + 30, sizeof(float) * 18);
        std::memcpy(hc + (size_t)i * 4, d.state + 48, sizeof(float) * 4);
        hp[i] = d.state[52];
      }
      s->deferred_q.erase(s->deferred_q.begin(), s->deferred_q.begin() + n);
      L.deferred_batch = true;
    }
  } else {
    std::lock_guard<std::mutex> g(s->mu);
    L.deferred_batch = false;
    // oldest pending request first
    s->ready_order.clear();
    for (int slot = 0; slot < s->pool; ++slot)
      if (!s->pending[slot].empty() && !s->inflight[slot]) s->ready_order.push_back(slot);
    if (s->ready_order.empty()) return false;
    if ((int)s->ready_order.size() > s->max_batch) {
      std::nth_element(s->ready_order.begin(), s->ready_order.begin() + s->max_batch, s->ready_order.end(),
                       [&](int a, int b) { return s->pending[a].front() < s->pending[b].front(); });
      s->ready_order.resize(s->max_batch);
    }
    n = (int)s->ready_order.size();
    L.slots.assign(s->ready_order.begin(), s->ready_order.end());
    L.arrivals.resize(n);
    // the newest states, packed into the blocks the C ABI takes:
    // x0 [n][30], qd_meas [n][18], cmd [n][4], phase [n]
    float* hx = L.h_in;
    float* hq = hx + (size_t)s->max_batch * 30;
    float* hc = hq + (size_t)s->max_batch * 18;
    float* hp = hc + (size_t)s->max_batch * 4;
    for (int i = 0; i < n; ++i) {
      const int slot = L.slots[i];
      L.arrivals[i].swap(s->pending[slot]);
      s->pending[slot].clear();
      s->inflight[slot] = 1;
      L.h_ids[i] = slot;
      const float* r = &s->state[(size_t)slot * kInF];
      std::memcpy(hx + (size_t)i * 30, r, sizeof(float) * 30);
      std::memcpy(hq + (size_t)i * 18, r + 30, sizeof(float) * 18);
      std::memcpy(hc + (size_t)i * 4, r + 48, sizeof(float) * 4);
      hp[i] = r[52];
    }
  }
  const int mb = s->max_batch;
  float* hx = L.h_in;
  float* hq = hx + (size_t)mb * 30;
  float* hc = hq + (size_t)mb * 18;
  float* hp = hc + (size_t)mb * 4;
  float* x0 = L.d_in;
  float* qd = x0 + (size_t)mb * 30;
  float* cmd = qd + (size_t)mb * 18;
  float* ph = cmd + (size_t)mb * 4;
  cudaStream_t st = L.stream;
  L.t_launch = now_s(s);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_ids, L.h_ids, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x0, hx, sizeof(float) * 30 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(qd, hq, sizeof(float) * 18 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cmd, hc, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ph, hp, sizeof(float) * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { set_error(s, MPC_ERR_CUDA, cudaGetErrorString(e)); return false; }
  uint64_t tk = 0;
  mpc_status r = mpc_submit(s->ctx, n, L.d_ids, x0, qd, cmd, ph, &tk);
  // regular batches defer their slow agents; a batch of deferred agents runs
  // ADMM from the saved start (DEFER_ADMM) or continues the capped polish
  // (DEFER_SLOW, no flag)
  int flags = 0;
  if (s->defer == 1) flags = L.deferred_batch ? MPC_SOLVE_ADMM_ONLY : MPC_SOLVE_DEFER_ADMM;
  else if (s->defer == 2) flags = L.deferred_batch ? 0 : MPC_SOLVE_DEFER_SLOW;
  else if (s->defer == 3) flags = L.deferred_batch ? 0 : MPC_SOLVE_DEFER_COLD;
  if (r == MPC_OK) r = mpc_solve_ex(s->ctx, tk, st, flags);
  if (r == MPC_OK) r = mpc_get_torques(s->ctx, tk, L.d_tau, nullptr, nullptr, nullptr, L.d_st);
  if (r != MPC_OK) { set_error(s, r, mpc_last_error(s->ctx)); return false; }
  e = cudaMemcpyAsync(L.h_tau, L.d_tau, sizeof(float) * kOutF * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.h_st, L.d_st, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(L.done, st);
  if (e != cudaSuccess) { set_error(s, MPC_ERR_CUDA, cudaGetErrorString(e)); return false; }
  L.n = n;
  L.busy = true;
  std::lock_guard<std::mutex> g(s->mu);
  s->batches += 1;
  return true;
}

// queued model swaps whose slots have no batch in flight: uploaded without
// waiting (mpc_set_models_async on the swap stream); the slots stay in
// flight, so that no batch takes them, until the upload's event completes
void apply_swaps(mpc_server* s) {
  if (s->swap_busy) return;
  std::vector<int32_t> ids;
  std::vector<mpc_agent_model> models;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->swaps.empty()) return;
    std::vector<std::pair<int32_t, mpc_agent_model>> keep;
    for (auto& sw : s->swaps) {
      if (s->inflight[sw.first]) keep.push_back(sw);
      else { ids.push_back(sw.first); models.push_back(sw.second); s->inflight[sw.first] = 1; }
    }
    s->swaps.swap(keep);
    s->swaps_since = keep.empty() ? -1.0 : now_s(s);
    s->swapping.assign(ids.begin(), ids.end());
  }
  if (ids.empty()) return;
  mpc_status r = mpc_set_models_async(s->ctx, (int32_t)ids.size(), ids.data(), models.data(), s->swap_stream);
  if (r != MPC_OK) { set_error(s, r, mpc_last_error(s->ctx)); return; }
  const cudaError_t e = cudaEventRecord(s->swap_done, s->swap_stream);
  if (e != cudaSuccess) { set_error(s, MPC_ERR_CUDA, cudaGetErrorString(e)); return; }
  s->swap_busy = true;
}

// the upload of the last swap has completed: its slots are free again
bool finish_swap(mpc_server* s) {
  if (!s->swap_busy) return false;
  const cudaError_t q = cudaEventQuery(s->swap_done);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) { set_error(s, MPC_ERR_CUDA, cudaGetErrorString(q)); return false; }
  std::lock_guard<std::mutex> g(s->mu);
  for (int32_t slot : s->swapping) s->inflight[slot] = 0;
  s->swapped += (long long)s->swapping.size();
  s->swapping.clear();
  s->swap_busy = false;
  return true;
}

void run_worker(mpc_server* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load(std::memory_order_relaxed) && s->error.load() == MPC_OK) {
    bool work = false;
    int busy = 0;          // regular lanes with a batch on the GPU
    bool busy_def = false; // the deferred agents' lane
    for (int li = 0; li <= s->max_inflight; ++li) {
      Lane& L = s->lanes[li];
      if (!L.busy) continue;
      const cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaSuccess) { complete(s, L); work = true; }
      else if (q != cudaErrorNotReady) { set_error(s, MPC_ERR_CUDA, cudaGetErrorString(q)); return; }
      else if (li < s->max_inflight) ++busy;
      else busy_def = true;
    }
    // regular batches on the first max_inflight lanes; deferred agents on the
    // last lane, so that their ADMM solves never hold a regular lane
    for (int li = 0; li < s->max_inflight; ++li) {
      Lane& L = s->lanes[li];
      if (busy >= s->max_inflight) break;
      if (L.busy) continue;
      if (!launch(s, L, false)) break;
      ++busy;
      work = true;
    }
    {
      Lane& L = s->lanes[s->max_inflight];
      if (!L.busy && launch(s, L, true)) { work = true; busy_def = true; }
    }
    // model swaps: a finished upload frees its slots; pending swaps start
    // their upload at once (it runs on its own stream and the worker does not
    // wait for it)
    if (finish_swap(s)) work = true;
    bool due = false;
    {
      std::lock_guard<std::mutex> g(s->mu);
      due = !s->swaps.empty();
    }
    if (due && !s->swap_busy) apply_swaps(s);
    if (!work) {
      // nothing completed or launched: wait briefly for a push or a completion
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::microseconds(busy || busy_def ? 20 : 200));
    }
  }
}

}  // namespace

extern "C" {

mpc_status mpc_server_create(mpc_ctx* ctx, int32_t pool, int32_t max_batch, int32_t max_inflight,
                             mpc_server** out) {
  if (!ctx || !out || pool <= 0 || max_batch <= 0 || max_inflight < 1 || max_inflight > 4) return MPC_ERR_INVALID;
  auto* s = new mpc_server();
  s->ctx = ctx;
  cudaGetDevice(&s->device);
  s->pool = pool;
  s->max_batch = std::min(max_batch, pool);
  s->max_inflight = max_inflight;
  s->state.assign((size_t)pool * kInF, 0.f);
  s->pending.resize(pool);
  s->inflight.assign(pool, 0);
  s->tau.assign((size_t)pool * kOutF, 0.f);
  s->latency.reserve(1 << 23);     // no reallocation (a copy under the lock) in a run of a few seconds
  s->batch_log.reserve(3 << 16);
  s->status.assign(pool, -1);
  s->lanes.resize(max_inflight + 1);   // + the lane of the deferred agents' batches
  const int mb = s->max_batch;
  for (auto& L : s->lanes) {
    cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_ids, sizeof(int32_t) * mb);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_in, sizeof(float) * (size_t)mb * kInF);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_tau, sizeof(float) * (size_t)mb * kOutF);
    if (e == cudaSuccess) e = cudaMallocHost(&L.h_st, sizeof(int32_t) * mb);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_ids, sizeof(int32_t) * mb);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_in, sizeof(float) * (size_t)mb * kInF);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_tau, sizeof(float) * (size_t)mb * kOutF);
    if (e == cudaSuccess) e = cudaMalloc(&L.d_st, sizeof(int32_t) * mb);
    if (e != cudaSuccess) { mpc_server_destroy(s); return MPC_ERR_CUDA; }
  }
  // the context's pinned staging of model uploads, allocated now rather than
  // on the worker's first swap
  if (cudaStreamCreateWithFlags(&s->swap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->swap_done, cudaEventDisableTiming) != cudaSuccess ||
      mpc_set_models_async(ctx, 0, nullptr, nullptr, s->swap_stream) != MPC_OK) {
    mpc_server_destroy(s);
    return MPC_ERR_CUDA;
  }
  *out = s;
  return MPC_OK;
}

mpc_status mpc_server_set_defer(mpc_server* s, int32_t mode) {
  if (!s || mode < 0 || mode > 3) return MPC_ERR_INVALID;
  if (s->worker.joinable()) return MPC_ERR_STATE;
  s->defer = mode;
  return MPC_OK;
}

int64_t mpc_server_deferred(mpc_server* s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> g(s->mu);
  return s->deferred;
}

mpc_status mpc_server_start(mpc_server* s) {
  if (!s) return MPC_ERR_INVALID;
  if (s->worker.joinable()) return MPC_ERR_STATE;
  s->t0 = Clock::now();
  s->stop = false;
  s->worker = std::thread(run_worker, s);
  return MPC_OK;
}

mpc_status mpc_server_push(mpc_server* s, int32_t n, const int32_t* slots, const float* x0, const float* qd_meas,
                           const float* cmd, const float* phase, const double* t_arrive) {
  if (!s || n < 0 || (n > 0 && (!slots || !x0 || !qd_meas || !cmd || !phase || !t_arrive))) return MPC_ERR_INVALID;
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (int i = 0; i < n; ++i)
      if (slots[i] < 0 || slots[i] >= s->pool) return MPC_ERR_INVALID;
    for (int i = 0; i < n; ++i) {
      float* r = &s->state[(size_t)slots[i] * kInF];
      std::memcpy(r, x0 + (size_t)i * 30, sizeof(float) * 30);
      std::memcpy(r + 30, qd_meas + (size_t)i * 18, sizeof(float) * 18);
      std::memcpy(r + 48, cmd + (size_t)i * 4, sizeof(float) * 4);
      r[52] = phase[i];
      s->pending[slots[i]].push_back(t_arrive[i]);
    }
    s->pushed += n;
  }
  s->cv.notify_one();
  return MPC_OK;
}

mpc_status mpc_server_set_models(mpc_server* s, int32_t n, const int32_t* slots, const mpc_agent_model* models) {
  if (!s || n < 0 || (n > 0 && (!slots || !models))) return MPC_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  for (int i = 0; i < n; ++i)
    if (slots[i] < 0 || slots[i] >= s->pool) return MPC_ERR_INVALID;
  if (s->swaps.empty() && n > 0) s->swaps_since = now_s(s);
  for (int i = 0; i < n; ++i) s->swaps.emplace_back(slots[i], models[i]);
  return MPC_OK;
}

mpc_status mpc_server_drain(mpc_server* s, double timeout_s) {
  if (!s) return MPC_ERR_INVALID;
  const auto end = Clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    if (s->error.load() != MPC_OK) return (mpc_status)s->error.load();
    {
      std::lock_guard<std::mutex> g(s->mu);
      if (s->answered == s->pushed && s->swaps.empty() && s->swapping.empty()) return MPC_OK;
    }
    if (Clock::now() > end) return MPC_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

mpc_status mpc_server_stop(mpc_server* s) {
  if (!s) return MPC_ERR_INVALID;
  s->stop = true;
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& L : s->lanes)
    if (L.busy) {
      cudaEventSynchronize(L.done);
      complete(s, L);
    }
  if (s->swap_busy) {
    cudaEventSynchronize(s->swap_done);
    finish_swap(s);
  }
  return (mpc_status)s->error.load();
}

double mpc_server_clock(mpc_server* s) { return s ? now_s(s) : 0.0; }

mpc_status mpc_server_results(mpc_server* s, double* latency, int64_t cap, int64_t* n_latency, float* tau,
                              int32_t* status, int64_t* counters) {
  if (!s || !n_latency) return MPC_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  *n_latency = (int64_t)s->latency.size();
  if (latency) std::memcpy(latency, s->latency.data(), sizeof(double) * std::min<int64_t>(cap, *n_latency));
  if (tau) std::memcpy(tau, s->tau.data(), sizeof(float) * s->tau.size());
  if (status) std::memcpy(status, s->status.data(), sizeof(int32_t) * s->status.size());
  if (counters) {
    counters[0] = s->pushed; counters[1] = s->answered; counters[2] = s->batches;
    counters[3] = s->solves; counters[4] = s->not_solved; counters[5] = s->swapped;
  }
  return MPC_OK;
}

mpc_status mpc_server_batches(mpc_server* s, double* log, int64_t cap, int64_t* n_batches) {
  if (!s || !n_batches) return MPC_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  *n_batches = (int64_t)(s->batch_log.size() / 3);
  if (log) std::memcpy(log, s->batch_log.data(), sizeof(double) * 3 * std::min<int64_t>(cap, *n_batches));
  return MPC_OK;
}

const char* mpc_server_last_error(mpc_server* s) { return s ? s->msg : "NULL server"; }

mpc_status mpc_server_destroy(mpc_server* s) {
  if (!s) return MPC_ERR_INVALID;
  mpc_server_stop(s);
  for (auto& L : s->lanes) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    cudaFreeHost(L.h_ids); cudaFreeHost(L.h_in); cudaFreeHost(L.h_tau); cudaFreeHost(L.h_st);
    cudaFree(L.d_ids); cudaFree(L.d_in); cudaFree(L.d_tau); cudaFree(L.d_st);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  if (s->swap_stream) cudaStreamSynchronize(s->swap_stream);
  if (s->swap_done) cudaEventDestroy(s->swap_done);
  if (s->swap_stream) cudaStreamDestroy(s->swap_stream);
  delete s;
  return MPC_OK;
}

}  // extern "C"
