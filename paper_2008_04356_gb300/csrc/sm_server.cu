// Serving loop (sm_server_*): continuous batching of many sliding-mesh solves on one GPU.
//
// A worker thread owns the device work.  Requests wait in arrival order; a request is
// admitted when a slot is free and its device memory fits in the budget next to the
// resident solves.  Every iteration advances the batchable solves (FP32 Euler plane
// interface) together by the same number of RK steps through one batch with shared launches,
// as many as fit in about 20 ms (one to eight) so that new arrivals join quickly; every other
// solve runs on a stream of its own, one chunk of steps at a time, and is only polled between
// iterations, so that a slow solve (FP64, Navier-Stokes, curvilinear, split form, two
// interfaces) never holds the batch back (except at a retirement: freeing device memory waits
// for the whole device).  Finished solves are retired and their memory freed.  A solve's time
// to solution ends at a CUDA event recorded right after its last step, mapped onto the host
// clock through an anchor event recorded when the worker starts.  Built on the library's own
// C-ABI.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/slidemesh.h"

int sm_batch_autotune_missing(sm_batch* b, void* stream);   // sm_host.cu

namespace {

struct Job {
  uint64_t id = 0;
  sm_request req;
  sm_result res;
  sm_solver* solver = nullptr;
  size_t bytes = 0;
  int remaining = 0;
  cudaEvent_t done_ev = nullptr;   // recorded after the solve's last step
  bool done_recorded = false;
  // solves outside the batch: their own stream, the chunk in flight and its end event
  cudaStream_t stream = nullptr;
  cudaEvent_t chunk_ev = nullptr;
  int in_flight = 0;
  int failed = SM_OK;
  std::vector<unsigned char> state;
};

size_t request_bytes(const sm_mesh_desc& d) {
  const size_t np = d.N + 1, nn = np * np * np, sb = d.precision == SM_FP64 ? 8 : 4;
  const size_t E = (size_t)(d.nel_static[0] + d.nel_moving[0]) * d.nel_static[1] * d.nel_static[2];
  const size_t faces = (size_t)d.nel_static[1] * d.nel_static[2];
  size_t b = 3 * E * nn * 5 * sb + 2 * faces * 5 * np * np * sb + 32 * E + (64 << 10);
  if (d.physics == SM_NAVIER_STOKES) b += E * nn * 15 * sb + 2 * faces * 5 * np * np * sb;   // gradients, lifting
  if (d.geom != SM_GEOM_PLANE) b += E * nn * 13 * sb;                                          // curvilinear geometry
  if (d.physics == SM_EULER && d.geom == SM_GEOM_PLANE && !d.interface_conforming)             // traces (and a second
    b += (d.periodic_x ? 6 : 2) * faces * 5 * np * np * sb;                                    // interface's arrays)
  return b;
}

// FP32 Euler solves on the plane interface share the batched kernels; the others step alone
bool batchable(const sm_mesh_desc& d) {
  return d.precision == SM_FP32 && d.physics == SM_EULER && d.geom == SM_GEOM_PLANE && d.volume == SM_VOLUME_WEAK &&
         !d.periodic_x;
}

}  // namespace

struct sm_server {
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::unordered_map<uint64_t, Job*> jobs;
  size_t budget = 0, used = 0, peak = 0;
  int max_slots = 0;
  int device = 0;
  uint64_t next_id = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  sm_server_stats_out stats;
  sm_batch* batch = nullptr;
  bool batch_dirty = true;
  cudaEvent_t anchor = nullptr;    // recorded (and waited for) when the worker starts
  double anchor_host = 0.0;        // host-clock time of the anchor event
  // seconds per batched step of the current batch (the last iteration's), which sets the
  // steps per iteration: new arrivals wait at most about kIterTarget for the next admission
  double step_s = 0.0;
  static constexpr double kIterTarget = 0.02;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
  void finish(Job* j, int status, cudaStream_t st);
};

void sm_server::finish(Job* j, int status, cudaStream_t batch_stream) {
  const cudaStream_t st = j->stream ? j->stream : batch_stream;
  // time to solution: the event after the last step on the device clock, else the host clock
  float ms = 0.0f;
  if (status == SM_OK && j->done_recorded && anchor && cudaEventElapsedTime(&ms, anchor, j->done_ev) == cudaSuccess)
    j->res.t_done = anchor_host + 1e-3 * (double)ms;
  else
    j->res.t_done = now();
  if (j->done_ev) cudaEventDestroy(j->done_ev);
  j->done_ev = nullptr;
  if (status == SM_OK && j->solver) {
    sm_diag_out d;
    int rc = sm_diag(j->solver, &d, (void*)st);
    if (rc == SM_OK || rc == SM_ERR_NONFINITE) {
      for (int v = 0; v < 5; ++v) j->res.totals[v] = d.totals[v];
      j->res.sim_time = d.t;
      if (rc != SM_OK) status = rc;
    } else {
      status = rc;
    }
    if (status == SM_OK && j->req.keep_state) {
      j->state.resize((size_t)sm_state_size(j->solver) * sm_scalar_bytes(j->solver));
      double t = 0.0;
      status = sm_get_state(j->solver, j->state.data(), 0, &t, (void*)st);
      j->res.state = j->state.data();
      j->res.state_bytes = (long long)j->state.size();
    }
  }
  if (j->solver) sm_destroy(j->solver);
  j->solver = nullptr;
  if (j->chunk_ev) cudaEventDestroy(j->chunk_ev);
  j->chunk_ev = nullptr;
  if (j->stream) cudaStreamDestroy(j->stream);
  j->stream = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  j->res.status = status;
  used -= j->bytes;
  if (status == SM_OK) {
    stats.completed++;
    stats.dof_updates += j->res.dof * 5LL * j->res.steps;
  } else {
    stats.failed++;
  }
  stats.running--;
  done_cv.notify_all();
}

void sm_server::run() {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (cudaEventCreate(&anchor) == cudaSuccess && cudaEventRecord(anchor, st) == cudaSuccess &&
      cudaEventSynchronize(anchor) == cudaSuccess) {
    anchor_host = now();
  } else {
    if (anchor) cudaEventDestroy(anchor);
    anchor = nullptr;
  }
  double busy_since = -1.0;
  while (!stop.load()) {
    std::vector<Job*> admit;
    {
      std::unique_lock<std::mutex> lk(mu);
      while (!queue.empty() && (int)active.size() + (int)admit.size() < max_slots &&
             used + queue.front()->bytes <= budget) {
        Job* j = queue.front();
        queue.pop_front();
        used += j->bytes;
        peak = std::max(peak, used);
        stats.queued--;
        stats.running++;
        admit.push_back(j);
      }
      if (active.empty() && admit.empty()) {
        if (busy_since >= 0.0) { stats.busy_seconds += now() - busy_since; busy_since = -1.0; }
        cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    if (busy_since < 0.0) busy_since = now();
    for (Job* j : admit) {
      j->res.t_admit = now();
      const bool solo = !batchable(j->req.desc);
      int rc = SM_OK;
      if (solo && (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
                   cudaEventCreateWithFlags(&j->chunk_ev, cudaEventDisableTiming) != cudaSuccess))
        rc = SM_ERR_CUDA;
      if (rc == SM_OK) rc = sm_init_mesh(&j->req.desc, &j->solver);
      if (rc == SM_OK) rc = sm_set_motion(j->solver, &j->req.motion);
      if (rc == SM_OK) rc = sm_init_state(j->solver, (void*)(solo ? j->stream : st));
      if (rc == SM_OK && cudaEventCreate(&j->done_ev) != cudaSuccess) { j->done_ev = nullptr; rc = SM_ERR_CUDA; }
      if (rc != SM_OK) { finish(j, rc, st); continue; }
      active.push_back(j);
      if (!solo) batch_dirty = true;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      stats.max_concurrent = std::max(stats.max_concurrent, (int)active.size());
    }
    if (active.empty()) continue;
    if (batch_dirty) {
      if (batch) sm_batch_destroy(batch);
      batch = nullptr;
      std::vector<sm_solver*> sol;
      std::vector<double> dts;
      for (Job* j : active)
        if (batchable(j->req.desc)) {
          sol.push_back(j->solver);
          dts.push_back(j->req.dt);
        }
      if (!sol.empty()) {
        int rc = sm_batch_create(sol.data(), dts.data(), (int)sol.size(), &batch);
        if (rc == SM_OK) rc = sm_batch_autotune_missing(batch, (void*)st);
        if (rc != SM_OK) {
          if (batch) sm_batch_destroy(batch);
          batch = nullptr;
          std::vector<Job*> solo;
          for (Job* j : active) {
            if (batchable(j->req.desc)) finish(j, rc, st);
            else solo.push_back(j);
          }
          active.swap(solo);
          batch_dirty = false;
          continue;
        }
      }
      batch_dirty = false;
    }
    // batched solves: one chunk of k steps through the batch, waited for; k keeps an
    // iteration near kIterTarget (at most 8 steps, at least one)
    int k = step_s > 0.0 ? std::max(1, std::min(8, (int)(kIterTarget / step_s))) : 1;
    bool any_batched = false;
    for (Job* j : active)
      if (batchable(j->req.desc) && j->remaining > 0) {
        k = std::min(k, j->remaining);
        any_batched = true;
      }
    if (!any_batched) k = 0;
    int rc = SM_OK;
    const double t_iter = now();
    if (k > 0) {
      if (batch) rc = sm_batch_step(batch, k, (void*)st);
      // the batched solves that take their last step here end with this launch sequence
      for (Job* j : active)
        if (rc == SM_OK && batchable(j->req.desc) && j->remaining == k)
          j->done_recorded = cudaEventRecord(j->done_ev, st) == cudaSuccess;
    }
    // the other solves: on their own streams, at most one chunk in flight each, polled
    bool solo_waiting = false;
    for (Job* j : active) {
      if (batchable(j->req.desc) || j->failed != SM_OK) continue;
      if (j->in_flight) {
        const cudaError_t q = cudaEventQuery(j->chunk_ev);
        if (q == cudaSuccess) {
          j->remaining -= j->in_flight;
          j->res.steps += j->in_flight;
          j->in_flight = 0;
        } else if (q != cudaErrorNotReady) {
          j->failed = SM_ERR_CUDA;
          continue;
        }
      }
      if (!j->in_flight && j->remaining > 0) {
        const int kj = std::min(8, j->remaining);
        int r2 = sm_step(j->solver, j->req.dt, kj, (void*)j->stream);
        if (r2 == SM_OK && j->remaining == kj) j->done_recorded = cudaEventRecord(j->done_ev, j->stream) == cudaSuccess;
        if (r2 == SM_OK && cudaEventRecord(j->chunk_ev, j->stream) != cudaSuccess) r2 = SM_ERR_CUDA;
        if (r2 != SM_OK) j->failed = r2;
        else j->in_flight = kj;
      }
      if (j->in_flight) solo_waiting = true;
    }
    if (k > 0) {
      if (rc == SM_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SM_ERR_CUDA;
      step_s = (now() - t_iter) / k;
      std::lock_guard<std::mutex> lk(mu);
      stats.batched_steps += k;
    } else if (solo_waiting) {
      // nothing batched to wait for: let the solo chunks run, admit arrivals meanwhile
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::microseconds(200));
    }
    std::vector<Job*> still;
    for (Job* j : active) {
      if (batchable(j->req.desc)) {
        j->remaining -= k;
        j->res.steps += k;
        if (rc != SM_OK || j->remaining <= 0) {
          finish(j, rc, st);
          batch_dirty = true;
          continue;
        }
      } else if (j->failed != SM_OK || (j->remaining <= 0 && !j->in_flight)) {
        if (j->failed != SM_OK && j->stream) cudaStreamSynchronize(j->stream);
        finish(j, j->failed, st);
        continue;
      }
      still.push_back(j);
    }
    active.swap(still);
  }
  if (batch) sm_batch_destroy(batch);
  batch = nullptr;
  for (Job* j : active) {
    if (j->stream) cudaStreamSynchronize(j->stream);
    if (j->solver) sm_destroy(j->solver);
    j->solver = nullptr;
    if (j->done_ev) cudaEventDestroy(j->done_ev);
    j->done_ev = nullptr;
    if (j->chunk_ev) cudaEventDestroy(j->chunk_ev);
    j->chunk_ev = nullptr;
    if (j->stream) cudaStreamDestroy(j->stream);
    j->stream = nullptr;
  }
  active.clear();
  if (anchor) cudaEventDestroy(anchor);
  anchor = nullptr;
  if (st) cudaStreamDestroy(st);
}

extern "C" {

int sm_server_create(size_t hbm_budget_bytes, int max_slots, sm_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) return SM_ERR_ARG;
  sm_server* s = new (std::nothrow) sm_server();
  if (!s) return SM_ERR_OOM;
  s->budget = hbm_budget_bytes;
  s->max_slots = std::min(max_slots, 1024);
  memset(&s->stats, 0, sizeof(s->stats));
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return SM_ERR_CUDA; }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return SM_OK;
}

int sm_submit(sm_server* s, const sm_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return SM_ERR_ARG;
  const sm_mesh_desc& d = req->desc;
  if (d.N < 1 || d.N > 7 || req->nsteps < 0 || !(req->dt > 0.0)) return SM_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (d.nel_static[k] < 1 || d.nel_moving[k] < 1) return SM_ERR_ARG;
  Job* j = new (std::nothrow) Job();
  if (!j) return SM_ERR_OOM;
  j->req = *req;
  memset(&j->res, 0, sizeof(j->res));
  j->res.status = SM_PENDING;
  j->bytes = request_bytes(d);
  j->remaining = req->nsteps;
  j->res.dof = (long long)(d.nel_static[0] + d.nel_moving[0]) * d.nel_static[1] * d.nel_static[2] *
               (d.N + 1) * (d.N + 1) * (d.N + 1);
  if (j->bytes > s->budget) { delete j; return SM_ERR_OOM; }
  std::lock_guard<std::mutex> lk(s->mu);
  j->id = s->next_id++;
  j->res.t_submit = s->now();
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  s->stats.submitted++;
  s->stats.queued++;
  *ticket = j->id;
  s->cv.notify_one();
  return SM_OK;
}

int sm_poll(sm_server* s, uint64_t ticket, sm_result* out) {
  if (!s || !out) return SM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return SM_ERR_ARG;
  *out = it->second->res;
  return out->status;
}

int sm_server_wait(sm_server* s, double timeout_s) {
  if (!s) return SM_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (s->stats.completed + s->stats.failed < s->stats.submitted) {
    if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        s->stats.completed + s->stats.failed < s->stats.submitted)
      return SM_ERR_TIMEOUT;
  }
  return SM_OK;
}

int sm_server_stats(sm_server* s, sm_server_stats_out* out) {
  if (!s || !out) return SM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->bytes_in_use = s->used;
  out->peak_bytes = s->peak;
  return SM_OK;
}

void sm_server_destroy(sm_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->jobs) {
    if (kv.second->solver) sm_destroy(kv.second->solver);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
