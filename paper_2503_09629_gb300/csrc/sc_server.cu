// sc_server.cu -- continuous batching of independent subcycled evolutions.
//
// A request is one complete hierarchy (wave or Z4c) with analytic initial data
// and a number of coarse steps.  The server keeps a FIFO queue and a set of
// slots, one CUDA stream each.  Every tick it
//   1. retires requests whose last coarse step has completed on the device
//      (their state stays resident until the client releases it),
//   2. admits queued requests, in arrival order, while a slot is free and the
//      request's exact device footprint fits the memory budget left,
//   3. launches the next coarse step (one CUDA graph) of every active request
//      that has fewer than `depth` steps in flight, on the request's stream.
// Requests of different sizes therefore run concurrently and their kernels
// overlap on the GPU; each request's arithmetic is exactly what it would be
// alone (same kernels, same order), so its result does not depend on the mix.
// Device memory of requests comes from a stream-ordered pool
// (cudaMallocAsync on the request's stream), so admission and release never
// synchronise the whole device.
//
// Merged form (sc_server_set_merge; off by default, because one graph per
// request on its own stream measured faster on GB300): wave requests run in
// the persistent coarse-step form, and each tick launches the next coarse
// step of all of them together as one cooperative kernel on the server's
// batch stream (phase i of every request between the same two grid
// barriers), instead of one graph per request.  Z4c requests keep their
// graphs on their own streams and overlap with the merged launches.  The
// arithmetic of every request is unchanged (same device-function bodies), so
// results stay bitwise those of the request running alone.
#include <algorithm>
#include <chrono>
#include <deque>
#include <thread>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "sc_internal.h"
#include "sc_persist.h"

namespace {

using Clock = std::chrono::steady_clock;

struct PoolUser {
  cudaStream_t stream;
  long* fail_countdown;  // server-wide fault injection: the allocation that takes it to 0 fails
};

void* pool_alloc(size_t bytes, void* user) {
  PoolUser* u = static_cast<PoolUser*>(user);
  if (*u->fail_countdown > 0 && --*u->fail_countdown == 0) return nullptr;
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, u->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pool_free(void* p, void* user) { cudaFreeAsync(p, static_cast<PoolUser*>(user)->stream); }

struct Request {
  unsigned long long ticket = 0;
  // deep copy of the descriptor
  sc_desc desc{};
  std::vector<int> nboxes;
  std::vector<sc_box> boxes;
  int id_kind = 0;
  std::vector<double> id_params;
  int steps = 0;
  size_t footprint = 0;
  // state
  int slot = -1;
  sc_ctx* ctx = nullptr;
  std::unique_ptr<PoolUser> pool;
  sc_allocator alloc{};
  int launched = 0;
  int completed = 0;
  std::deque<cudaEvent_t> inflight;
  bool done = false;
  sc_status status = SC_OK;  // SC_ENOMEM when admission could never allocate the request
  Clock::time_point t_submit, t_admit, t_done;
  double zu_finest = 0, zu_actual = 0;
};

sc_status err(sc_status code, const char* msg) { return sc::set_last_error(code, msg); }

}  // namespace

struct sc_server {
  size_t budget = 0;
  size_t in_use = 0;
  int depth = 2;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::deque<Request*> queue;
  std::map<unsigned long long, std::unique_ptr<Request>> all;
  unsigned long long next_ticket = 1;
  long launches = 0;
  double zu_finest_done = 0, zu_actual_done = 0;
  long fail_countdown = 0;  // sc_server_inject_alloc_failure
  int merge = 0;            // merge scalar-wave requests into one persistent launch per tick
  cudaStream_t batch_stream = nullptr;
  sc::GridBarrier* bar = nullptr;
};

namespace {

sc_status admit(sc_server* S, Request* r, int slot) {
  r->slot = slot;
  r->pool.reset(new PoolUser{S->streams[slot], &S->fail_countdown});
  r->alloc.alloc = pool_alloc;
  r->alloc.free = pool_free;
  r->alloc.user = r->pool.get();
  r->desc.nboxes = r->nboxes.data();
  r->desc.boxes = r->boxes.data();
  r->desc.cuda_stream = S->streams[slot];
  r->desc.allocator = &r->alloc;
  if (S->merge && r->desc.system == SC_WAVE) r->desc.exec_mode = SC_EXEC_PERSISTENT;
  sc_status st = sc_create(&r->desc, &r->ctx);
  if (st != SC_OK) return st;
  st = sc_set_initial_data(r->ctx, r->id_kind, r->id_params.empty() ? nullptr : r->id_params.data(),
                           (int)r->id_params.size());
  if (st != SC_OK) {
    sc_destroy(r->ctx);
    r->ctx = nullptr;
    return st;
  }
  S->slot_busy[slot] = true;
  S->in_use += r->footprint;
  r->t_admit = Clock::now();
  return SC_OK;
}

void finish(sc_server* S, Request* r) {
  r->done = true;
  r->t_done = Clock::now();
  S->slot_busy[r->slot] = false;  // the slot's stream is idle; the state stays resident until release
  double f = 0, a = 0;
  sc_zone_updates(r->ctx, &f, &a);
  r->zu_finest = f;
  r->zu_actual = a;
  S->zu_finest_done += f;
  S->zu_actual_done += a;
}

}  // namespace

extern "C" {

sc_status sc_server_create(size_t hbm_budget_bytes, int max_active, int depth, sc_server** out) {
  if (!out || max_active < 1 || max_active > 256 || depth < 1) return err(SC_EINVAL, "bad server arguments");
  std::unique_ptr<sc_server> S(new sc_server());
  S->budget = hbm_budget_bytes;
  S->depth = depth;
  S->streams.resize(max_active);
  S->slot_busy.assign(max_active, false);
  for (auto& s : S->streams) {
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamCreateWithFlags(&S->batch_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&S->bar, sizeof(sc::GridBarrier));
  if (e == cudaSuccess) e = cudaMemset(S->bar, 0, sizeof(sc::GridBarrier));
  if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
  *out = S.release();
  return SC_OK;
}

sc_status sc_server_submit(sc_server* S, const sc_desc* d, int id_kind, const double* id_params, int nparams,
                           int n_coarse_steps, unsigned long long* ticket) {
  if (!S || !d || !ticket || n_coarse_steps < 0 || nparams < 0 || nparams > 8) return err(SC_EINVAL, "bad submit arguments");
  size_t fp = 0;
  sc_status st = sc_footprint_estimate(d, &fp);
  if (st != SC_OK) return st;
  if (fp > S->budget) return err(SC_EBUSY, "request footprint exceeds the server's memory budget");
  std::unique_ptr<Request> r(new Request());
  r->ticket = S->next_ticket++;
  r->desc = *d;
  r->nboxes.assign(d->nboxes, d->nboxes + d->nlevels);
  int nb = 0;
  for (int l = 0; l < d->nlevels; ++l) nb += d->nboxes[l];
  r->boxes.assign(d->boxes, d->boxes + nb);
  r->id_kind = id_kind;
  if (nparams) r->id_params.assign(id_params, id_params + nparams);
  r->steps = n_coarse_steps;
  r->footprint = fp;
  r->t_submit = Clock::now();
  *ticket = r->ticket;
  S->queue.push_back(r.get());
  S->all[r->ticket] = std::move(r);
  return SC_OK;
}

sc_status sc_server_tick(sc_server* S, int* n_active, int* n_queued, int* n_launched) {
  if (!S) return err(SC_EINVAL, "null server");
  int launched = 0;
  // 1. retire completed steps / requests
  for (auto& kv : S->all) {
    Request* r = kv.second.get();
    if (!r->ctx || r->done) continue;
    while (!r->inflight.empty()) {
      cudaError_t e = cudaEventQuery(r->inflight.front());
      if (e == cudaErrorNotReady) break;
      if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
      cudaEventDestroy(r->inflight.front());
      r->inflight.pop_front();
      ++r->completed;
    }
    if (r->completed == r->steps) finish(S, r);
  }
  // 2. admit in arrival order while a slot is free and the footprint fits
  while (!S->queue.empty()) {
    Request* r = S->queue.front();
    if (S->in_use + r->footprint > S->budget) break;
    int slot = -1;
    for (size_t q = 0; q < S->slot_busy.size(); ++q)
      if (!S->slot_busy[q]) {
        slot = (int)q;
        break;
      }
    if (slot < 0) break;
    S->queue.pop_front();
    sc_status st = admit(S, r, slot);
    if (st == SC_ENOMEM) {
      // sc_create released what it had allocated.  Retry once running
      // requests have freed memory; with nothing running, no memory will
      // come free, so the request fails (sc_server_poll reports SC_ENOMEM).
      r->ctx = nullptr;
      r->slot = -1;
      bool any_active = false;
      for (auto& kv : S->all)
        if (kv.second->ctx && !kv.second->done) any_active = true;
      if (any_active) {
        S->queue.push_front(r);
        break;
      }
      r->done = true;
      r->status = SC_ENOMEM;
      r->t_done = Clock::now();
      continue;
    }
    if (st != SC_OK) return st;
    if (r->steps == 0) finish(S, r);
  }
  // 3. launch the next coarse step of every active request: one graph per
  // graph-form request on its stream, one merged launch for the
  // persistent-form requests on the batch stream
  int active = 0;
  std::vector<Request*> merged;
  for (auto& kv : S->all) {
    Request* r = kv.second.get();
    if (!r->ctx || r->done) continue;
    ++active;
    if (r->launched >= r->steps || (int)r->inflight.size() >= S->depth) continue;
    if (r->desc.exec_mode == SC_EXEC_PERSISTENT) {
      merged.push_back(r);
      continue;
    }
    sc_status st = sc_advance(r->ctx, 1);
    if (st != SC_OK) return st;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
    e = cudaEventRecord(ev, S->streams[r->slot]);
    if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
    r->inflight.push_back(ev);
    ++r->launched;
    long per = 0;
    sc_launches_per_step(r->ctx, &per);
    S->launches += per;
    ++launched;
  }
  for (size_t first = 0; first < merged.size(); first += sc::kMaxBatch) {
    const size_t n = std::min(merged.size() - first, (size_t)sc::kMaxBatch);
    sc::PBatch b{};
    b.n = (int)n;
    b.bar = S->bar;
    std::vector<long> work;
    for (size_t q = 0; q < n; ++q) {
      Request* r = merged[first + q];
      sc::PersistView v{};
      sc_status st = sc::persistent_view(r->ctx, &v);
      if (st != SC_OK) return st;
      b.ops[q] = v.ops;
      b.status[q] = v.status;
      b.w = v.w;
      b.nops_r[q] = (int)v.host->size();
      b.nops = std::max(b.nops, b.nops_r[q]);
      if (work.size() < v.host->size()) work.resize(v.host->size(), 0);
      for (size_t i = 0; i < v.host->size(); ++i) work[i] += sc::phase_work_blocks((*v.host)[i]);
    }
    long need = 1;
    for (long w : work) need = std::max(need, w);
    int maxb = 0;
    cudaError_t e = sc::persistent_max_blocks(&maxb);
    if (e == cudaSuccess) e = sc::launch_persistent_step(b, (int)std::min<long>(need, maxb), S->batch_stream);
    if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
    S->launches += 1;
    for (size_t q = 0; q < n; ++q) {
      Request* r = merged[first + q];
      sc::persistent_step_done(r->ctx);
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(ev, S->batch_stream);
      if (e != cudaSuccess) return err(SC_ECUDA, cudaGetErrorString(e));
      r->inflight.push_back(ev);
      ++r->launched;
      ++launched;
    }
  }
  if (n_active) *n_active = active;
  if (n_queued) *n_queued = (int)S->queue.size();
  if (n_launched) *n_launched = launched;
  return SC_OK;
}

sc_status sc_server_poll(sc_server* S, unsigned long long ticket, int* done, double* latency_s) {
  if (!S || !done) return err(SC_EINVAL, "bad poll arguments");
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return err(SC_EINVAL, "unknown ticket");
  Request* r = it->second.get();
  *done = r->done ? 1 : 0;
  if (latency_s) *latency_s = r->done ? std::chrono::duration<double>(r->t_done - r->t_submit).count() : -1.0;
  return r->status;
}

sc_status sc_server_wait(sc_server* S, unsigned long long ticket, double timeout_s, double* latency_s) {
  if (!S || !(timeout_s >= 0)) return err(SC_EINVAL, "bad wait arguments");
  const auto t0 = Clock::now();
  for (;;) {
    sc_status st = sc_server_tick(S, nullptr, nullptr, nullptr);
    if (st != SC_OK) return st;
    int done = 0;
    st = sc_server_poll(S, ticket, &done, latency_s);
    if (done || st != SC_OK) return st;
    if (std::chrono::duration<double>(Clock::now() - t0).count() >= timeout_s)
      return err(SC_ETIMEOUT, "request not finished within the wait's time limit");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

sc_status sc_server_set_merge(sc_server* S, int on) {
  if (!S || (on != 0 && on != 1)) return err(SC_EINVAL, "bad merge argument");
  S->merge = on;
  return SC_OK;
}

sc_status sc_server_inject_alloc_failure(sc_server* S, long k) {
  if (!S || k < 0) return err(SC_EINVAL, "bad fault-injection arguments");
  S->fail_countdown = k;
  return SC_OK;
}

sc_status sc_server_read(sc_server* S, unsigned long long ticket, int level, int box, int field, double* host_dst) {
  if (!S) return err(SC_EINVAL, "null server");
  auto it = S->all.find(ticket);
  if (it == S->all.end() || !it->second->done) return err(SC_EINVAL, "unknown or unfinished ticket");
  return sc_get_field(it->second->ctx, level, box, field, host_dst);
}

sc_status sc_server_release(sc_server* S, unsigned long long ticket) {
  if (!S) return err(SC_EINVAL, "null server");
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return err(SC_EINVAL, "unknown ticket");
  Request* r = it->second.get();
  if (r->ctx && !r->done) return err(SC_EINVAL, "request still running");
  if (r->status != SC_OK) {
    // failed at admission: neither queued nor holding memory
  } else if (r->ctx) {
    sc_destroy(r->ctx);
    S->in_use -= r->footprint;
  } else {
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
      if (*q == r) {
        S->queue.erase(q);
        break;
      }
  }
  S->all.erase(it);
  return SC_OK;
}

sc_status sc_server_stats(sc_server* S, double* zu_finest_done, double* zu_actual_done, long* launches,
                          size_t* bytes_in_use) {
  if (!S) return err(SC_EINVAL, "null server");
  if (zu_finest_done) *zu_finest_done = S->zu_finest_done;
  if (zu_actual_done) *zu_actual_done = S->zu_actual_done;
  if (launches) *launches = S->launches;
  if (bytes_in_use) *bytes_in_use = S->in_use;
  return SC_OK;
}

sc_status sc_server_destroy(sc_server* S) {
  if (!S) return SC_OK;
  for (auto& s : S->streams) cudaStreamSynchronize(s);
  if (S->batch_stream) cudaStreamSynchronize(S->batch_stream);
  for (auto& kv : S->all) {
    Request* r = kv.second.get();
    for (auto ev : r->inflight) cudaEventDestroy(ev);
    if (r->ctx) sc_destroy(r->ctx);
  }
  S->all.clear();
  for (auto& s : S->streams) cudaStreamDestroy(s);
  if (S->batch_stream) cudaStreamDestroy(S->batch_stream);
  if (S->bar) cudaFree(S->bar);
  delete S;
  return SC_OK;
}

}  // extern "C"
