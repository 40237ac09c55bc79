// Request server over resident replicas (host code; the device work is that of the
// okmc_grid calls it makes).  The paper runs one simulation at a time and has no
// counterpart; this is the serving loop of the library: continuous batching of
// solve and step requests for many independent replicas on one GPU.
//
//   lanes      worker threads, each with its own non-blocking CUDA stream; a lane
//              takes the oldest runnable request, runs it on its stream and waits
//              for it, so requests for different replicas overlap on the device.
//   replicas   registered with a description and defects; resident (a live
//              okmc_grid) from the first request that needs them.  Requests for
//              one replica run in submission order, never two at a time.
//   admission  a replica becomes resident only when the device bytes of all
//              resident replicas plus its estimate stay within the budget; idle
//              replicas are evicted least recently used first to make room, with
//              their defects and kinetic state saved on the host and restored on
//              re-admission (the trajectory continues exactly).  While the oldest
//              waiting request cannot be admitted, no other replica is admitted
//              ahead of it, so large replicas are not starved.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "okmc.h"

namespace {

struct Replica {
  okmc_grid_desc desc{};
  std::vector<okmc_defect> defs;
  okmc_step_stats saved{};
  bool has_saved = false;
  okmc_grid* g = nullptr;
  bool busy = false;       // a lane is running a request on it, or it is being admitted/evicted
  size_t bytes = 0;        // device bytes when resident (estimate while being admitted)
  size_t estimate = 0;
  unsigned long long last_use = 0;
};

struct Job {
  unsigned long long ticket;
  okmc_request req;
  double t_submit;
};

}  // namespace

struct okmc_server {
  okmc_server_desc desc{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Replica> reps;  // element references stay valid while replicas are added
  std::deque<Job> queue;
  std::map<unsigned long long, okmc_result> done;
  size_t used = 0;  // bytes of resident replicas and reservations
  unsigned long long next_ticket = 1, tick = 0;
  okmc_server_stats stats{};
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::chrono::steady_clock::time_point t0;
  std::string err;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  void worker(int lane);
  // with mu held: index of the queue entry to run next (or -1); may reserve memory
  // and mark eviction victims, returned in `victims`
  int pick(std::vector<int>& victims);
};

namespace {

// Device bytes a replica will hold: the handle's fields (exact) plus a bound on the
// defect tables and stencils.
size_t estimate_bytes(const okmc_grid_desc& d, const std::vector<okmc_defect>& defs) {
  size_t b = okmc_estimate_field_bytes(&d);
  const double h = d.voxel_nm;
  for (const okmc_defect& r : defs) {
    double cells;
    if (r.type == OKMC_SIA_CLUSTER) {
      const double q = 3.0 * r.size / (8.0 * 3.141592653589793);
      const double rv = std::cbrt(q > 1.0 ? q : 1.0) + 2.0;
      cells = 4.19 * rv * rv * rv;
    } else {
      const double rv = r.radius_nm / h + 2.0;
      cells = 3.1416 * rv * rv * 4.0;
    }
    b += (size_t)(2.0 * cells * 5.0) + 512;
  }
  return b + (1u << 20);
}

}  // namespace

int okmc_server::pick(std::vector<int>& victims) {
  bool memory_blocked = false;
  for (size_t q = 0; q < queue.size(); ++q) {
    Replica& r = reps[queue[q].req.replica];
    if (r.busy) continue;
    bool earlier = false;  // an earlier request for the same replica waits: keep order
    for (size_t k = 0; k < q && !earlier; ++k) earlier = queue[k].req.replica == queue[q].req.replica;
    if (earlier) continue;
    if (r.g) return (int)q;
    if (memory_blocked) continue;
    // admission
    const size_t need = r.estimate;
    const size_t budget = desc.hbm_budget;
    if (!budget || used + need <= budget) {
      used += need;
      r.bytes = need;
      return (int)q;
    }
    // evict idle resident replicas, least recently used first, if that makes room
    std::vector<int> idle;
    for (size_t i = 0; i < reps.size(); ++i)
      if (reps[i].g && !reps[i].busy) idle.push_back((int)i);
    std::sort(idle.begin(), idle.end(), [&](int a, int b) { return reps[a].last_use < reps[b].last_use; });
    size_t freed = 0;
    std::vector<int> take;
    for (int i : idle) {
      if (used - freed + need <= budget) break;
      bool wanted = false;  // keep replicas with queued requests ahead in line if possible
      for (size_t k = 0; k < q && !wanted; ++k) wanted = queue[k].req.replica == i;
      if (wanted) continue;
      take.push_back(i);
      freed += reps[i].bytes;
    }
    if (used - freed + need <= budget && need <= budget) {
      for (int i : take) {
        reps[i].busy = true;
        victims.push_back(i);
      }
      used += need;  // the victims' bytes are released once they are gone
      r.bytes = need;
      return (int)q;
    }
    memory_blocked = true;  // the oldest request that needs memory waits; nobody jumps ahead of it
  }
  return -1;
}

void okmc_server::worker(int lane) {
  cudaSetDevice(device);
  cudaStream_t st = streams[lane];
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    std::vector<int> victims;
    int q = -1;
    while (!stop && (q = pick(victims)) < 0) cv_work.wait(lk);
    if (stop) return;
    Job job = queue[q];
    queue.erase(queue.begin() + q);
    Replica& r = reps[job.req.replica];
    r.busy = true;
    const bool admit = (r.g == nullptr);
    lk.unlock();
    okmc_result res{};
    res.t_submit = job.t_submit;
    res.admitted = admit ? 1 : 0;
    int rc = OKMC_OK;
    // eviction: save defects and kinetic state, free the handle
    for (int v : victims) {
      Replica& e = reps[v];
      int erc = okmc_get_defects(e.g, e.defs.data(), (int32_t)e.defs.size());
      if (erc == OKMC_OK) erc = okmc_get_stats(e.g, &e.saved);
      e.has_saved = (erc == OKMC_OK);
      okmc_grid_destroy(e.g);
      e.g = nullptr;
      std::lock_guard<std::mutex> g2(mu);
      used -= e.bytes;
      e.bytes = 0;
      e.busy = false;
      stats.evictions += 1;
    }
    if (admit) {
      okmc_grid_desc d = r.desc;
      d.stream = st;
      d.hbm_budget = 0;
      rc = okmc_grid_create(&d, &r.g);
      if (rc == OKMC_OK) rc = okmc_set_defects(r.g, r.defs.data(), (int32_t)r.defs.size());
      if (rc == OKMC_OK && r.has_saved) rc = okmc_set_kinetic_state(r.g, &r.saved);
      if (rc != OKMC_OK && r.g) {
        okmc_grid_destroy(r.g);
        r.g = nullptr;
      }
      std::lock_guard<std::mutex> g2(mu);
      used -= r.bytes;
      r.bytes = r.g ? okmc_device_bytes(r.g) : 0;
      used += r.bytes;
      stats.admissions += 1;
    } else {
      rc = okmc_set_stream(r.g, st);
    }
    res.t_start = now();
    if (rc == OKMC_OK) {
      if (job.req.kind == OKMC_REQ_SOLVE) {
        rc = okmc_interaction_energies(r.g, job.req.energies, 0);
        if (rc == OKMC_OK) rc = okmc_get_stats(r.g, &res.stats);
      } else {
        rc = okmc_step(r.g, &job.req.params, job.req.n_events, &res.stats);
        if (rc == OKMC_OK && job.req.positions) rc = okmc_get_positions(r.g, job.req.positions, (int32_t)r.defs.size(), 0);
      }
      if (rc == OKMC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = OKMC_ECUDA;
    }
    res.t_end = now();
    res.status = rc;
    lk.lock();
    r.busy = false;
    r.last_use = ++tick;
    stats.completed += 1;
    if (rc != OKMC_OK) stats.failed += 1;
    done[job.ticket] = res;
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

int okmc_server_create(const okmc_server_desc* d, okmc_server** out) {
  if (!d || !out || d->lanes < 1 || d->lanes > 64 || d->reserved != 0) return OKMC_EINVAL;
  *out = nullptr;
  okmc_server* s = new (std::nothrow) okmc_server();
  if (!s) return OKMC_ENOMEM;
  s->desc = *d;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return OKMC_ECUDA;
  }
  for (int i = 0; i < d->lanes; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return OKMC_ECUDA;
    }
    s->streams.push_back(st);
  }
  try {
    for (int i = 0; i < d->lanes; ++i) s->workers.emplace_back(&okmc_server::worker, s, i);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto x : s->streams) cudaStreamDestroy(x);
    delete s;
    return OKMC_ENOMEM;
  }
  *out = s;
  return OKMC_OK;
}

int okmc_server_add_replica(okmc_server* s, const okmc_grid_desc* d, const okmc_defect* defs, int32_t nd, int32_t* id) {
  if (!s || !d || !id || nd < 0 || (nd > 0 && !defs)) return OKMC_EINVAL;
  Replica r;
  r.desc = *d;
  r.defs.assign(defs, defs + nd);
  r.estimate = estimate_bytes(r.desc, r.defs);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->desc.hbm_budget && r.estimate > s->desc.hbm_budget) {
    s->err = "replica larger than the server's budget";
    return OKMC_ENOMEM;
  }
  *id = (int32_t)s->reps.size();
  s->reps.push_back(std::move(r));
  return OKMC_OK;
}

int okmc_server_submit(okmc_server* s, const okmc_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return OKMC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->replica < 0 || r->replica >= (int32_t)s->reps.size()) {
    s->err = "unknown replica";
    return OKMC_EINVAL;
  }
  if (r->kind != OKMC_REQ_SOLVE && r->kind != OKMC_REQ_STEP) {
    s->err = "unknown request kind";
    return OKMC_EINVAL;
  }
  if (r->kind == OKMC_REQ_STEP && r->n_events < 0) {
    s->err = "negative step count";
    return OKMC_EINVAL;
  }
  Job j{s->next_ticket++, *r, s->now()};
  *ticket = j.ticket;
  s->queue.push_back(j);
  s->stats.submitted += 1;
  s->cv_work.notify_one();
  return OKMC_OK;
}

int okmc_server_wait(okmc_server* s, uint64_t ticket, int32_t timeout_ms, okmc_result* out) {
  if (!s || !out) return OKMC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket >= s->next_ticket) return OKMC_EINVAL;
  auto ready = [&] { return s->done.count(ticket) > 0; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return OKMC_ETIMEOUT;
  }
  *out = s->done[ticket];
  s->done.erase(ticket);
  return OKMC_OK;
}

int okmc_server_get_stats(okmc_server* s, okmc_server_stats* out) {
  if (!s || !out) return OKMC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->resident = 0;
  for (const Replica& r : s->reps) out->resident += r.g != nullptr;
  out->device_bytes = s->used;
  out->queued = (int64_t)s->queue.size();
  return OKMC_OK;
}

const char* okmc_server_last_error(const okmc_server* s) { return s ? s->err.c_str() : "null server"; }

int okmc_server_destroy(okmc_server* s) {
  if (!s) return OKMC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (Replica& r : s->reps)
    if (r.g) okmc_grid_destroy(r.g);
  for (auto x : s->streams) cudaStreamDestroy(x);
  delete s;
  return OKMC_OK;
}

}  // extern "C"
