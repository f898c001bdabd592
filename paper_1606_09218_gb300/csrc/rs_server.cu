// Serving loop: continuous batching of RS solves of different N and n.
//
// Requests are queued by rs_submit (their inputs copied), and a worker thread admits them to
// slots.  A slot is a context with its own CUDA stream, pinned staging buffers and a completion
// event; it is kept for later requests of the same configuration.  A request is admitted when an
// idle slot of its configuration exists, or when a new slot fits the HBM budget (the sum of the
// slots' workspace bytes), possibly after releasing idle slots of other configurations.  Admitted
// requests run concurrently on their streams; the worker polls the events, reads the results and
// wakes the waiters.  The queue is scanned in arrival order, and a request that cannot be
// admitted yet does not block later requests that can.
//
// Locking: the mutex guards the shared queue, the ticket table, the results and the counters
// that rs_server_info reads.  The slots belong to the worker thread alone, so the worker creates
// contexts (device allocations), runs the host-side checks of rs_solve and enqueues work without
// the mutex: rs_submit and rs_wait never wait behind those calls.
#include "rs_internal.cuh"

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

// a request whose configuration has no slot waits at most this long before an idle slot of
// another configuration is released for it
constexpr double kStarveMs = 10.0;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
  unsigned long long ticket = 0;
  rs_config cfg{};
  int N = 0;
  std::vector<double> xyz, Z;
  int flags = 0;
  void* pot = nullptr;
  Clock::time_point t_sub, t_launch;
  rs_result res{};
  bool done = false;
};

struct Slot {
  rs_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  rs_config cfg{};
  size_t bytes = 0;
  double* hx = nullptr;     // pinned staging, 3 * max_particles
  double* hz = nullptr;     // pinned staging, max_particles
  std::shared_ptr<Job> job;
};

// field by field: a caller's rs_config may carry uninitialised padding bytes
bool same_config(const rs_config& a, const rs_config& b) {
  return a.b == b.b && a.n == b.n && a.R == b.R && a.R_s == b.R_s && a.h_q == b.h_q && a.u0 == b.u0 &&
         a.eps == b.eps && a.rank_cap == b.rank_cap && a.max_rank == b.max_rank && a.delta_rel == b.delta_rel &&
         a.precision == b.precision && a.snap == b.snap && a.max_particles == b.max_particles;
}

}  // namespace

struct rs_server {
  size_t budget = 0;
  int max_slots = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> pending;       // submitted, not yet seen by the worker (mu)
  std::unordered_map<unsigned long long, std::shared_ptr<Job>> jobs;   // (mu)
  std::deque<std::shared_ptr<Job>> waiting;       // seen by the worker, not admitted (worker only)
  std::vector<std::unique_ptr<Slot>> slots;       // (worker only)
  size_t used = 0;                                // (worker only)
  int info_slots = 0, info_waiting = 0;           // published copies for rs_server_info (mu)
  size_t info_used = 0;
  unsigned long long next_ticket = 1;
  bool stop = false;
  std::thread worker;

  void release_slot(size_t i) {
    Slot& s = *slots[i];
    rs_destroy(s.ctx);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.hx) cudaFreeHost(s.hx);
    if (s.hz) cudaFreeHost(s.hz);
    used -= s.bytes;
    slots.erase(slots.begin() + (long)i);
  }

  // create a slot for cfg; nullptr if a CUDA or library call fails
  Slot* make_slot(const rs_config& cfg, size_t bytes) {
    std::unique_ptr<Slot> s(new Slot());
    s->cfg = cfg;
    s->bytes = bytes;
    const size_t cap = (size_t)(cfg.max_particles > 0 ? cfg.max_particles : 1);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&s->hx, sizeof(double) * 3 * cap) != cudaSuccess ||
        cudaMallocHost((void**)&s->hz, sizeof(double) * cap) != cudaSuccess ||
        rs_create(&cfg, s->stream, &s->ctx) != RS_OK) {
      cudaGetLastError();
      if (s->ctx) rs_destroy(s->ctx);
      if (s->ev) cudaEventDestroy(s->ev);
      if (s->stream) cudaStreamDestroy(s->stream);
      if (s->hx) cudaFreeHost(s->hx);
      if (s->hz) cudaFreeHost(s->hz);
      return nullptr;
    }
    used += bytes;
    slots.push_back(std::move(s));
    return slots.back().get();
  }

  // publish a result (takes the mutex: rs_wait reads it)
  void finish(const std::shared_ptr<Job>& job, rs_status st, Slot* s) {
    const auto now = Clock::now();
    char msg[sizeof(job->res.message)] = {0};
    if (st < 0) {
      const char* m = rs_last_error(s ? s->ctx : nullptr);
      std::snprintf(msg, sizeof(msg), "%s", (m && *m) ? m : "error");
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      job->res.status = st;
      if (st < 0) std::memcpy(job->res.message, msg, sizeof(msg));
      job->res.latency_ms = ms_between(job->t_sub, now);
      job->res.queue_ms = ms_between(job->t_sub, job->t_launch);
      job->done = true;
    }
    cv_done.notify_all();
  }

  void launch(Slot* s, const std::shared_ptr<Job>& job) {
    job->t_launch = Clock::now();
    for (size_t i = 0; i < slots.size(); ++i)
      if (slots[i].get() == s) job->res.slot = (int)i;
    if (job->N > 0) {
      std::memcpy(s->hx, job->xyz.data(), sizeof(double) * 3 * (size_t)job->N);
      std::memcpy(s->hz, job->Z.data(), sizeof(double) * (size_t)job->N);
    }
    const int flags = (job->flags & (RS_ENERGY | RS_POTENTIAL)) | RS_INPUT_HOST;
    rs_status st = rs_solve(s->ctx, job->N, s->hx, s->hz, flags, 0.0, job->pot);
    if (st != RS_OK) {
      finish(job, st, s);
      return;
    }
    cudaEventRecord(s->ev, s->stream);
    s->job = job;
  }

  void complete(Slot* s) {
    std::shared_ptr<Job> job = s->job;
    s->job.reset();
    rs_stats stt;
    std::memset(&stt, 0, sizeof(stt));
    rs_status st = rs_report(s->ctx, &stt);
    for (int l = 0; l < 3; ++l) job->res.ranks[l] = stt.ranks[l];
    if (st >= 0 && (job->flags & RS_ENERGY)) {
      double E = 0.0;
      rs_status se = rs_energy(s->ctx, &E);
      job->res.energy = E;
      if (se != RS_OK) st = se;
    }
    finish(job, st, s);
  }

  // one pass of admissions (worker thread, without the mutex); returns true if anything was
  // launched.  First every idle slot takes the earliest waiting request of its configuration;
  // then the remaining requests, in arrival order, get new slots while the HBM budget and the
  // slot limit allow.  To make room, only idle slots of configurations that no waiting request
  // asks for are released (the one of the configuration with the most idle slots first): a
  // slot that a later request of the queue can reuse is kept, so a full queue of mixed sizes
  // does not create and free contexts (device allocations) over and over.
  bool admit() {
    bool any = false;
    // fairness: the earliest waiting request whose configuration has no slot at all, once it
    // has waited kStarveMs, takes the place of an idle slot of another configuration (the one
    // with the most idle slots) even if later requests could reuse that slot
    for (auto it = waiting.begin(); it != waiting.end(); ++it) {
      bool has_slot = false;
      for (auto& s : slots) has_slot = has_slot || same_config(s->cfg, (*it)->cfg);
      if (has_slot) continue;
      if (ms_between((*it)->t_sub, Clock::now()) < kStarveMs) break;
      const size_t need = rs_workspace_bytes(&(*it)->cfg);
      if (need == 0 || (used + need <= budget && (int)slots.size() < max_slots)) break;   // fits anyway
      size_t victim = slots.size();
      int best = 0;
      for (size_t i = 0; i < slots.size(); ++i) {
        if (slots[i]->job) continue;
        int idle_same = 0;
        for (auto& t : slots)
          if (!t->job && same_config(t->cfg, slots[i]->cfg)) ++idle_same;
        if (idle_same > best) { best = idle_same; victim = i; }
      }
      if (victim == slots.size()) break;
      release_slot(victim);
      if (used + need <= budget && (int)slots.size() < max_slots) {
        if (Slot* ns = make_slot((*it)->cfg, need)) {
          std::shared_ptr<Job> job = *it;
          waiting.erase(it);
          launch(ns, job);
          any = true;
        }
      }
      break;
    }
    for (auto& s : slots) {
      if (s->job) continue;
      for (auto it = waiting.begin(); it != waiting.end(); ++it) {
        if (same_config(s->cfg, (*it)->cfg)) {
          std::shared_ptr<Job> job = *it;
          waiting.erase(it);
          launch(s.get(), job);
          any = true;
          break;
        }
      }
    }
    auto wanted = [&](const rs_config& cfg) {
      for (auto& j : waiting)
        if (same_config(j->cfg, cfg)) return true;
      return false;
    };
    for (auto it = waiting.begin(); it != waiting.end();) {
      std::shared_ptr<Job> job = *it;
      const size_t need = rs_workspace_bytes(&job->cfg);
      if (need == 0) {                                   // invalid configuration
        it = waiting.erase(it);
        job->t_launch = Clock::now();
        finish(job, RS_ERR_INVALID_ARG, nullptr);
        continue;
      }
      // release idle slots that no waiting request can use while the new slot does not fit
      while (used + need > budget || (int)slots.size() >= max_slots) {
        size_t victim = slots.size();
        int best = 0;
        for (size_t i = 0; i < slots.size(); ++i) {
          if (slots[i]->job || wanted(slots[i]->cfg)) continue;
          int idle_same = 0;
          for (auto& t : slots)
            if (!t->job && same_config(t->cfg, slots[i]->cfg)) ++idle_same;
          if (idle_same > best) { best = idle_same; victim = i; }
        }
        if (victim == slots.size()) break;
        release_slot(victim);
      }
      Slot* chosen = nullptr;
      if (used + need <= budget && (int)slots.size() < max_slots) {
        chosen = make_slot(job->cfg, need);
        if (!chosen) {                                   // device memory short: free idle slots, retry once
          for (size_t i = slots.size(); i-- > 0;)
            if (!slots[i]->job) release_slot(i);
          chosen = make_slot(job->cfg, need);
        }
      }
      if (!chosen && slots.empty()) {                    // cannot run even alone
        it = waiting.erase(it);
        job->t_launch = Clock::now();
        finish(job, RS_ERR_OOM, nullptr);
        continue;
      }
      if (!chosen) { ++it; continue; }
      it = waiting.erase(it);
      launch(chosen, job);
      any = true;
    }
    return any;
  }

  void publish_info() {
    std::lock_guard<std::mutex> lk(mu);
    info_slots = (int)slots.size();
    info_used = used;
    info_waiting = (int)waiting.size();
  }

  void run() {
    cudaSetDevice(device);
    while (true) {
      bool busy = false;
      for (auto& s : slots)
        if (s->job) {
          busy = true;
          if (cudaEventQuery(s->ev) == cudaSuccess) complete(s.get());
        }
      cudaGetLastError();                                  // cudaErrorNotReady from the polls
      bool stopping = false;
      {
        std::lock_guard<std::mutex> lk(mu);
        while (!pending.empty()) {
          waiting.push_back(pending.front());
          pending.pop_front();
        }
        stopping = stop;
      }
      const bool launched = admit();
      publish_info();
      bool running = false;
      for (auto& s : slots) running = running || (s->job != nullptr);
      if (stopping && waiting.empty() && !running) {
        std::lock_guard<std::mutex> lk(mu);
        if (pending.empty()) break;
        continue;
      }
      if (!launched) {
        std::unique_lock<std::mutex> lk(mu);
        if (pending.empty() && !stop)
          cv_work.wait_for(lk, (running || busy) ? std::chrono::microseconds(50) : std::chrono::microseconds(5000));
      }
    }
    while (!slots.empty()) release_slot(slots.size() - 1);
    publish_info();
  }
};

extern "C" rs_status rs_server_create(size_t hbm_budget, int max_slots, rs_server** out) {
  if (!out || max_slots < 1 || hbm_budget == 0) return RS_ERR_INVALID_ARG;
  *out = nullptr;
  rs_server* s = new (std::nothrow) rs_server();
  if (!s) return RS_ERR_OOM;
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return RS_ERR_CUDA;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return RS_OK;
}

extern "C" rs_status rs_submit(rs_server* s, const rs_request* req, unsigned long long* ticket) {
  if (!s || !req || !ticket || req->N < 0 || (req->N > 0 && (!req->xyz || !req->Z))) return RS_ERR_INVALID_ARG;
  if (req->N > req->cfg.max_particles) return RS_ERR_CAPACITY;
  if ((req->flags & RS_POTENTIAL) && !req->potential_out) return RS_ERR_INVALID_ARG;
  std::shared_ptr<Job> job(new Job());
  job->cfg = req->cfg;
  job->N = req->N;
  job->xyz.assign(req->xyz, req->xyz + 3 * (size_t)req->N);
  job->Z.assign(req->Z, req->Z + (size_t)req->N);
  job->flags = req->flags;
  job->pot = req->potential_out;
  job->t_sub = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    job->ticket = s->next_ticket++;
    s->jobs[job->ticket] = job;
    s->pending.push_back(job);
  }
  s->cv_work.notify_one();
  *ticket = job->ticket;
  return RS_OK;
}

extern "C" rs_status rs_wait(rs_server* s, unsigned long long ticket, int timeout_ms, rs_result* out) {
  if (!s || !out) return RS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return RS_ERR_INVALID_ARG;
  std::shared_ptr<Job> job = it->second;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (!job->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !job->done) return RS_ERR_TIMEOUT;
  }
  *out = job->res;
  s->jobs.erase(ticket);
  return RS_OK;
}

extern "C" void rs_server_destroy(rs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

extern "C" rs_status rs_server_info(rs_server* s, int* slots, size_t* bytes_in_use, int* queued) {
  if (!s) return RS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (slots) *slots = s->info_slots;
  if (bytes_in_use) *bytes_in_use = s->info_used;
  if (queued) *queued = (int)s->pending.size() + s->info_waiting;
  return RS_OK;
}
