// Request queue with continuous batching.
//
// A queue owns one scheduler thread and one CUDA stream.  Submitted requests
// wait in a FIFO until a slot is free and their device footprint fits the HBM
// budget: the optimiser state (q and loss) plus the object's grid and
// min-pyramid, counted once per object however many admitted requests use it.
// Each round launches one fused kernel over the candidates of every admitted
// request (the kernel finds each candidate's request in a slot table), for up
// to steps_per_launch optimisation steps per request.  After the round,
// finished requests are copied to host memory and release their slot and
// bytes; pending requests are admitted before the next round.  Every
// candidate's arithmetic is independent of the other candidates of a round, so
// a request's result does not depend on what it is batched with.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "fg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Request {
  uint64_t id = 0;
  const fg_hand* hand = nullptr;
  const fg_sdf* sdf = nullptr;
  int B = 0, D = 0, steps = 0, step_done = 0;
  fg_params params{};
  std::vector<float> q0, q_out, loss_out;
  ReqState state = kPending;
  fg_status fail = FG_OK;
  std::string fail_msg;
  float* d_q = nullptr;
  float* d_loss = nullptr;
  size_t state_bytes = 0;
  Clock::time_point t_submit, t_done;
};

size_t sdf_bytes(const fg_sdf* s) { return s->bytes + s->pyr_bytes; }

}  // namespace

struct fg_queue {
  size_t budget = 0, used = 0;
  fg_queue_opts opts{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;         // wakes the scheduler (submissions, stop)
  std::condition_variable done_cv;    // wakes waiters (completions)
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<uint64_t, Request*> all;
  std::map<const fg_sdf*, int> sdf_refs;
  uint64_t next_id = 1;
  uint64_t rounds = 0, cand_steps = 0;
  bool stop = false;
  bool joined = false;                // fg_queue_destroy has stopped the scheduler
  bool broken = false;                // a round failed or timed out: no further rounds
  std::string broken_msg;
  std::vector<float*> orphans;        // device state of the requests of a failed round
  cudaStream_t stream = nullptr;
  cudaEvent_t event = nullptr;
  fg::QueueSlotDev* h_slots = nullptr;   // pinned
  fg::QueueSlotDev* d_slots = nullptr;
  std::thread worker;
};

namespace {

void fail_request(fg_queue* Q, Request* r, fg_status st, const std::string& msg) {
  r->state = kFailed;
  r->fail = st;
  r->fail_msg = msg;
  r->t_done = Clock::now();
}

// Frees a request's device state and budget (lock held).
void release(fg_queue* Q, Request* r) {
  if (r->d_q) cudaFreeAsync(r->d_q, Q->stream);
  if (r->d_loss) cudaFreeAsync(r->d_loss, Q->stream);
  r->d_q = r->d_loss = nullptr;
  Q->used -= r->state_bytes;
  int& refs = Q->sdf_refs[r->sdf];
  if (--refs == 0) {
    Q->used -= sdf_bytes(r->sdf);
    Q->sdf_refs.erase(r->sdf);
  }
}

// Admits pending requests in FIFO order while a slot and the budget allow (lock held).
void admit(fg_queue* Q) {
  while (!Q->pending.empty() && !Q->broken) {
    Request* r = Q->pending.front();
    const bool obj_in_use = Q->sdf_refs.count(r->sdf) > 0;
    const size_t need = r->state_bytes + (obj_in_use ? 0 : sdf_bytes(r->sdf));
    if ((int)Q->active.size() >= Q->opts.max_slots || Q->used + need > Q->budget) break;
    Q->pending.pop_front();
    cudaError_t e = cudaMallocAsync(&r->d_q, sizeof(float) * (size_t)r->B * r->D, Q->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&r->d_loss, sizeof(float) * (size_t)r->B, Q->stream);
    if (e == cudaSuccess && fg::alloc_fault()) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->d_q, r->q0.data(), sizeof(float) * (size_t)r->B * r->D, cudaMemcpyHostToDevice,
                          Q->stream);
    Q->used += need;
    Q->sdf_refs[r->sdf] += 1;
    if (e != cudaSuccess) {
      release(Q, r);
      fail_request(Q, r, e == cudaErrorMemoryAllocation ? FG_ERR_OOM : FG_ERR_CUDA,
                   std::string("admission: ") + cudaGetErrorString(e));
      Q->done_cv.notify_all();
      continue;
    }
    r->state = kActive;
    Q->active.push_back(r);
  }
}

// Waits for the round's event with a time limit; returns false on timeout.
bool wait_event(fg_queue* Q, cudaError_t* err) {
  const auto t0 = Clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(Q->event);
    if (e == cudaSuccess) return true;
    if (e != cudaErrorNotReady) {
      *err = e;
      return true;
    }
    if (Clock::now() - t0 > std::chrono::milliseconds(Q->opts.timeout_ms)) return false;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

void scheduler(fg_queue* Q) {
  cudaSetDevice(Q->device);
  std::unique_lock<std::mutex> lock(Q->mu);
  for (;;) {
    if (Q->stop) break;                 // after the round in flight; what is left is discarded below
    admit(Q);
    if (Q->active.empty()) {
      Q->cv.wait_for(lock, std::chrono::milliseconds(5));
      continue;
    }
    // slot table of this round (pinned staging, copied on the stream)
    const int n = (int)Q->active.size();
    int total = 0;
    for (int i = 0; i < n; ++i) {
      Request* r = Q->active[i];
      fg::QueueSlotDev& s = Q->h_slots[i];
      s.hand = r->hand->dev;
      s.q = r->d_q;
      s.loss = r->d_loss;
      s.obj = r->sdf->host;
      s.P = fg::params_from(&r->params);
      s.cand_start = total;
      s.B = r->B;
      s.step0 = r->step_done;
      s.total_steps = r->steps;
      const int left = r->steps - r->step_done;
      s.nsteps = left < Q->opts.steps_per_launch ? left : Q->opts.steps_per_launch;
      total += r->B;
    }
    cudaError_t e = cudaMemcpyAsync(Q->d_slots, Q->h_slots, sizeof(fg::QueueSlotDev) * n, cudaMemcpyHostToDevice,
                                    Q->stream);
    fg::FusedArgs a{};
    a.B = total;
    a.slots = Q->d_slots;
    a.nslots = n;
    for (int i = 0; i < n; ++i) a.any_mesh |= Q->h_slots[i].obj.kind == fg::kObjMesh;
    if (e == cudaSuccess) e = fg::launch_queue_round(a, Q->stream);
    if (e == cudaSuccess) e = cudaEventRecord(Q->event, Q->stream);
    lock.unlock();
    bool in_time = true;
    if (e == cudaSuccess) in_time = wait_event(Q, &e);
    lock.lock();
    if (!in_time || e != cudaSuccess) {
      // the round did not finish: its requests fail and the queue takes no more work
      Q->broken = true;
      Q->broken_msg = !in_time ? "a round exceeded timeout_ms" : std::string(cudaGetErrorString(e));
      for (Request* r : Q->active) {
        fail_request(Q, r, !in_time ? FG_ERR_TIMEOUT : FG_ERR_CUDA, Q->broken_msg);
        // the round may still be running on them: freed by fg_queue_destroy once the stream drains
        Q->orphans.push_back(r->d_q);
        Q->orphans.push_back(r->d_loss);
        r->d_q = r->d_loss = nullptr;
      }
      Q->active.clear();
      for (Request* r : Q->pending) fail_request(Q, r, FG_ERR_CUDA, "queue stopped: " + Q->broken_msg);
      Q->pending.clear();
      Q->done_cv.notify_all();
      break;
    }
    Q->rounds += 1;
    std::vector<Request*> still;
    for (int i = 0; i < n; ++i) {
      Request* r = Q->active[i];
      const int done_now = Q->h_slots[i].nsteps;
      r->step_done += done_now;
      Q->cand_steps += (uint64_t)done_now * r->B;
      if (r->step_done < r->steps) {
        still.push_back(r);
        continue;
      }
      r->q_out.resize((size_t)r->B * r->D);
      r->loss_out.resize((size_t)r->B);
      e = cudaMemcpyAsync(r->q_out.data(), r->d_q, sizeof(float) * r->q_out.size(), cudaMemcpyDeviceToHost,
                          Q->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->loss_out.data(), r->d_loss, sizeof(float) * r->loss_out.size(),
                            cudaMemcpyDeviceToHost, Q->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(Q->stream);
      release(Q, r);
      if (e != cudaSuccess) {
        fail_request(Q, r, FG_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
      } else {
        r->state = kDone;
        r->t_done = Clock::now();
      }
    }
    Q->active.swap(still);
    Q->done_cv.notify_all();
  }
  // stopping: discard what is left
  for (Request* r : Q->active) {
    release(Q, r);
    fail_request(Q, r, FG_ERR_CUDA, "queue destroyed");
  }
  Q->active.clear();
  for (Request* r : Q->pending) fail_request(Q, r, FG_ERR_CUDA, "queue destroyed");
  Q->pending.clear();
  Q->done_cv.notify_all();
}

fg_status qinvalid(const std::string& m) {
  fg::set_error(m);
  return FG_ERR_INVALID;
}

}  // namespace

extern "C" {

fg_status fg_queue_create(size_t budget, const fg_queue_opts* opts, fg_queue** out) {
  if (!out) return qinvalid("fg_queue_create: NULL out");
  *out = nullptr;
  if (budget == 0) return qinvalid("fg_queue_create: budget must be > 0");
  fg_queue_opts o{};
  if (opts) o = *opts;
  if (o.max_slots <= 0) o.max_slots = 32;
  if (o.max_slots > FG_QUEUE_MAX_SLOTS) return qinvalid("fg_queue_create: max_slots > FG_QUEUE_MAX_SLOTS");
  if (o.max_requests <= 0) o.max_requests = 4096;
  if (o.steps_per_launch <= 0) o.steps_per_launch = 10;
  if (o.timeout_ms <= 0) o.timeout_ms = 60000;
  fg_queue* Q = new (std::nothrow) fg_queue;
  if (!Q) return FG_ERR_OOM;
  Q->budget = budget;
  Q->opts = o;
  cudaError_t e = cudaGetDevice(&Q->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&Q->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&Q->event, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc(&Q->h_slots, sizeof(fg::QueueSlotDev) * o.max_slots, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc(&Q->d_slots, sizeof(fg::QueueSlotDev) * o.max_slots);
  if (e != cudaSuccess) {
    if (Q->d_slots) cudaFree(Q->d_slots);
    if (Q->h_slots) cudaFreeHost(Q->h_slots);
    if (Q->event) cudaEventDestroy(Q->event);
    if (Q->stream) cudaStreamDestroy(Q->stream);
    delete Q;
    return fg::cuda_status(e, "fg_queue_create");
  }
  Q->worker = std::thread(scheduler, Q);
  *out = Q;
  return FG_OK;
}

fg_status fg_queue_submit(fg_queue* Q, const fg_request* r, uint64_t* id) {
  if (!Q || !r || !id) return qinvalid("fg_queue_submit: NULL argument");
  if (!r->hand || !r->sdf || !r->host_q0) return qinvalid("fg_queue_submit: request needs hand, sdf and host_q0");
  if (r->B < 1 || r->steps < 1) return qinvalid("fg_queue_submit: need B >= 1 and steps >= 1");
  const fg_params& p = r->params;
  if (!(p.dt > 0.0f) || !(p.v_test >= 0.0f) || !(p.mu >= 0.0f) || !(p.alpha_leak >= 0.0f && p.alpha_leak <= 1.0f) ||
      !(p.r0 >= 0.0f) || (p.schedule != 0 && p.schedule != 1))
    return qinvalid("fg_queue_submit: invalid params");
  if (p.sim_steps != 0) return qinvalid("fg_queue_submit: params.sim_steps must be 0 (one-step metric)");
  if (p.gauss_seidel != 0) return qinvalid("fg_queue_submit: params.gauss_seidel must be 0 (Jacobi form)");
  const int D = r->hand->host.D;
  const size_t state = sizeof(float) * (size_t)r->B * (D + 1);
  if (state + sdf_bytes(r->sdf) > Q->budget) {
    fg::set_error("fg_queue_submit: request needs " + std::to_string(state + sdf_bytes(r->sdf)) +
                  " bytes, more than the queue's budget of " + std::to_string(Q->budget));
    return FG_ERR_BUDGET;
  }
  Request* req = fg::alloc_fault() ? nullptr : new (std::nothrow) Request;
  if (!req) {
    fg::set_error("fg_queue_submit: out of host memory");
    return FG_ERR_OOM;
  }
  req->hand = r->hand;
  req->sdf = r->sdf;
  req->B = r->B;
  req->D = D;
  req->steps = r->steps;
  req->params = p;
  req->state_bytes = state;
  try {
    req->q0.assign(r->host_q0, r->host_q0 + (size_t)r->B * D);
  } catch (...) {
    delete req;
    return FG_ERR_OOM;
  }
  std::lock_guard<std::mutex> lock(Q->mu);
  if (Q->stop || Q->broken) {
    delete req;
    fg::set_error("fg_queue_submit: queue is stopping or failed: " + Q->broken_msg);
    return FG_ERR_CUDA;
  }
  if ((int)Q->all.size() >= Q->opts.max_requests) {
    delete req;
    fg::set_error("fg_queue_submit: max_requests outstanding; collect results first");
    return FG_ERR_BUSY;
  }
  req->id = Q->next_id++;
  req->t_submit = Clock::now();
  Q->all[req->id] = req;
  Q->pending.push_back(req);
  *id = req->id;
  Q->cv.notify_all();
  return FG_OK;
}

fg_status fg_queue_poll(fg_queue* Q, uint64_t id, int* done) {
  if (!Q || !done) return qinvalid("fg_queue_poll: NULL argument");
  std::lock_guard<std::mutex> lock(Q->mu);
  auto it = Q->all.find(id);
  if (it == Q->all.end()) {
    fg::set_error("fg_queue_poll: unknown request id");
    return FG_ERR_NOT_FOUND;
  }
  *done = it->second->state >= kDone ? 1 : 0;
  return FG_OK;
}

fg_status fg_queue_wait(fg_queue* Q, uint64_t id, int timeout_ms) {
  if (!Q) return qinvalid("fg_queue_wait: NULL queue");
  std::unique_lock<std::mutex> lock(Q->mu);
  auto it = Q->all.find(id);
  if (it == Q->all.end()) {
    fg::set_error("fg_queue_wait: unknown request id");
    return FG_ERR_NOT_FOUND;
  }
  Request* r = it->second;
  const bool ok = Q->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                      [r] { return r->state >= kDone; });
  if (!ok) {
    fg::set_error("fg_queue_wait: request not finished within timeout_ms");
    return FG_ERR_TIMEOUT;
  }
  return FG_OK;
}

fg_status fg_queue_result(fg_queue* Q, uint64_t id, float* host_q, float* host_loss, double* latency_s) {
  if (!Q) return qinvalid("fg_queue_result: NULL queue");
  std::lock_guard<std::mutex> lock(Q->mu);
  auto it = Q->all.find(id);
  if (it == Q->all.end()) {
    fg::set_error("fg_queue_result: unknown request id");
    return FG_ERR_NOT_FOUND;
  }
  Request* r = it->second;
  if (r->state < kDone) {
    fg::set_error("fg_queue_result: request not finished");
    return FG_ERR_BUSY;
  }
  fg_status st = FG_OK;
  if (r->state == kFailed) {
    fg::set_error("fg_queue_result: request failed: " + r->fail_msg);
    st = r->fail;
  } else {
    if (host_q) std::memcpy(host_q, r->q_out.data(), sizeof(float) * r->q_out.size());
    if (host_loss) std::memcpy(host_loss, r->loss_out.data(), sizeof(float) * r->loss_out.size());
  }
  if (latency_s) latency_s[0] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  Q->all.erase(it);
  delete r;
  return st;
}

fg_status fg_queue_stats(fg_queue* Q, fg_queue_stat* out) {
  if (!Q || !out) return qinvalid("fg_queue_stats: NULL argument");
  std::lock_guard<std::mutex> lock(Q->mu);
  int done = 0;
  for (auto& kv : Q->all) done += kv.second->state >= kDone ? 1 : 0;
  out->pending = (int)Q->pending.size();
  out->active = (int)Q->active.size();
  out->finished = done;
  out->failed = Q->broken ? 1 : 0;
  out->bytes_in_use = Q->used;
  out->budget = Q->budget;
  out->rounds = Q->rounds;
  out->candidate_steps = Q->cand_steps;
  return FG_OK;
}

fg_status fg_queue_destroy(fg_queue* Q) {
  if (!Q) return FG_OK;
  if (!Q->joined) {
    {
      std::lock_guard<std::mutex> lock(Q->mu);
      Q->stop = true;
      // requests still waiting are dropped; the scheduler finishes the round in flight
      for (Request* r : Q->pending) fail_request(Q, r, FG_ERR_CUDA, "queue destroyed");
      Q->pending.clear();
      Q->cv.notify_all();
    }
    if (Q->worker.joinable()) Q->worker.join();
    Q->joined = true;
  }
  // a round that exceeded timeout_ms may still run: wait for the stream, again at most timeout_ms
  const auto t0 = Clock::now();
  cudaError_t e;
  while ((e = cudaStreamQuery(Q->stream)) == cudaErrorNotReady) {
    if (Clock::now() - t0 > std::chrono::milliseconds(Q->opts.timeout_ms)) {
      fg::set_error("fg_queue_destroy: the queue's stream did not drain within timeout_ms; the handle stays "
                    "valid, call fg_queue_destroy again");
      return FG_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  for (float* p : Q->orphans) cudaFreeAsync(p, Q->stream);
  Q->orphans.clear();
  cudaStreamSynchronize(Q->stream);
  for (auto& kv : Q->all) delete kv.second;
  Q->all.clear();
  cudaFree(Q->d_slots);
  cudaFreeHost(Q->h_slots);
  cudaEventDestroy(Q->event);
  cudaStreamDestroy(Q->stream);
  delete Q;
  return FG_OK;
}

}  // extern "C"
