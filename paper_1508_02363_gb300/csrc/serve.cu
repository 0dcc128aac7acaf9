// Serving runtime: continuous batching of CGO solves (dbar_serve_*).
//
// The paper needs CGO solutions for many values of k (Sec. 1; Sec. 7 outlook:
// parallelise over k).  A server takes requests (N, L, Q, k) from any host
// thread and solves them on one GPU.  Requests of one grid class (N, L) share
// a "lane": a plan whose slots each hold one request with its own potential.
// A single worker thread advances the lanes one GMRES cycle at a time (each cycle
// launched in parts, the remaining Krylov chunks skipped once no slot iterates); at
// every cycle boundary a lane retires its finished slots and admits waiting
// requests into the free ones, so new work joins while older work is still
// iterating.  Every slot's arithmetic is independent of the other slots
// (per-slot masks, fixed reduction order), so a result does not depend on
// what it was batched with.
//
// Device memory is admitted by a budget: a lane gets as many slots as the
// budget leaves room for; idle lanes are dropped when another grid class
// needs the memory.  Host copies of potentials and results live in
// page-locked buffers recycled through a pool (no page faults, and the
// copies to and from the GPU run at the host link's rate).  A lane whose GPU work fails has its in-flight requests
// re-queued once (then failed with the error) and is rebuilt on demand.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dbar.h"
#include "plan_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Page-locked host buffers of 2 N^2 doubles, recycled by size.
class HostPool {
 public:
  double* get(size_t n) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      std::vector<double*>& f = free_[n];
      if (!f.empty()) {
        double* p = f.back();
        f.pop_back();
        pooled_ -= n * sizeof(double);
        return p;
      }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, n * sizeof(double), cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return static_cast<double*>(p);
  }
  void put(double* p, size_t n) {
    if (!p) return;
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (pooled_ + n * sizeof(double) <= kMaxPooled) {
        free_[n].push_back(p);
        pooled_ += n * sizeof(double);
        return;
      }
    }
    cudaFreeHost(p);
  }
  ~HostPool() {
    for (auto& kv : free_)
      for (double* p : kv.second) cudaFreeHost(p);
  }

 private:
  static constexpr size_t kMaxPooled = (size_t)8 << 30;  // idle pinned bytes kept for reuse
  std::mutex mu_;
  std::map<size_t, std::vector<double*>> free_;
  size_t pooled_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  int N = 0;
  double L = 0.0;
  size_t n2 = 0;          // 2 N^2 doubles per field
  double* Q = nullptr;    // copied at submit (pool buffer), returned once the request is finished
  double k1 = 0.0, k2 = 0.0;
  int want_m = 0;
  int retries = 0;
  double t_submit = 0.0, t_start = -1.0, t_done = -1.0;
  int status = DBAR_EBUSY;
  int itot = 0, ncyc = 0;
  double resid = 0.0;
  double* S = nullptr;    // results (pool buffers), returned at release
  double* m = nullptr;
  bool released = false;
};

struct Lane {
  int N = 0;
  double L = 0.0;
  cudaStream_t stream = nullptr;  // own stream: one lane's cycle runs while others are serviced
  dbar_plan* plan = nullptr;
  int B = 0;
  size_t bytes = 0;
  std::deque<Request*> waiting;
  std::vector<Request*> slot;
  // completion of the last cycle part launched on `stream`: the worker steps a lane only
  // once that has finished, so a long cycle of one grid class never holds up the
  // cycle boundaries of the others
  cudaEvent_t done = nullptr;
  bool inflight = false;
  // the cycle in progress runs part by part (plan_step_part): the next part to launch,
  // -1 between cycles.  Once no slot iterates, the remaining chunks are skipped.
  int part = -1;
  bool ready() const { return !inflight || cudaEventQuery(done) != cudaErrorNotReady; }
  bool busy() const {
    if (!waiting.empty()) return true;
    for (Request* r : slot)
      if (r) return true;
    return false;
  }
};

}  // namespace

struct dbar_server {
  dbar_params defaults{};
  size_t budget = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  bool stop = false;
  int inject = 0;  // host-side fault injection: fail the next lane cycle
  std::thread worker;
  std::map<uint64_t, Request*> reqs;
  std::vector<Lane*> lanes;
  size_t used = 0;
  uint64_t next_ticket = 1;
  Clock::time_point t0;
  std::vector<double> latencies;
  double first_submit = -1.0, last_done = -1.0;
  uint64_t completed = 0;
  HostPool pool;

  double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

dbar_params lane_params(const dbar_server* S, int N, double L, int B) {
  dbar_params p = S->defaults;
  p.N = N;
  p.L = L;
  p.max_batch = B;
  p.mem_budget = 0;  // the server's own budget decides B
  return p;
}

// Creates the lane's plan with as many slots as the budget allows (caller holds mu).
bool open_lane(dbar_server* S, Lane* ln) {
  dbar_params p = lane_params(S, ln->N, ln->L, 1);
  const size_t per = plan_slot_bytes(&p, 1), fixed = plan_fixed_bytes(&p);
  auto room = [&]() -> int {
    if (S->used + fixed + per > S->budget) return 0;
    const size_t b = (S->budget - S->used - fixed) / per;
    const int cap = S->defaults.max_batch > 0 ? S->defaults.max_batch : 128;
    return (int)std::min<size_t>(b, (size_t)cap);
  };
  int B = room();
  if (B < 1) {  // drop idle lanes of other grid classes to make room
    for (Lane* o : S->lanes)
      if (o != ln && o->plan && !o->busy()) {
        cudaStreamSynchronize(o->stream);
        dbar_plan_destroy(o->plan);
        o->plan = nullptr;
        S->used -= o->bytes;
        o->bytes = 0;
      }
    B = room();
  }
  if (B < 1) return false;
  B = std::min<int>(B, (int)std::max<size_t>(1, ln->waiting.size() + 8));
  p.max_batch = B;
  dbar_plan* P = nullptr;
  if (!ln->stream) {
    // larger grids get the higher stream priority: their cycles are the longest, and the
    // latency tail is theirs; the small grids' short cycles fill the gaps
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);  // lo: least, hi: greatest (numerically lower)
    int lg = 0;
    while ((1 << (lg + 1)) <= ln->N) ++lg;
    const int prio = std::max(hi, lo - std::max(0, lg - 8));  // N <= 256: least; each doubling one step up
    if (cudaStreamCreateWithPriority(&ln->stream, cudaStreamNonBlocking, prio) != cudaSuccess) return false;
  }
  if (plan_create_ex(&p, 1, &P) != DBAR_OK) return false;
  ln->plan = P;
  ln->B = plan_batch(P);
  ln->bytes = plan_device_bytes(P);
  ln->slot.assign(ln->B, nullptr);
  S->used += ln->bytes;
  return true;
}

void finish(dbar_server* S, Request* r, int status) {
  r->status = status;
  r->t_done = S->now_ms();
  S->latencies.push_back(r->t_done - r->t_submit);
  S->last_done = r->t_done;
  S->completed += 1;
  S->pool.put(r->Q, r->n2);
  r->Q = nullptr;
}

// A lane's GPU work failed: re-queue its in-flight requests once, fail repeat
// offenders, and drop the plan (rebuilt when work arrives).  Caller holds mu.
void lane_failed(dbar_server* S, Lane* ln, int status) {
  ln->part = -1;
  for (Request*& r : ln->slot) {
    if (!r) continue;
    if (r->retries++ < 1) {
      r->t_start = -1.0;
      ln->waiting.push_front(r);
    } else {
      finish(S, r, status);
    }
    r = nullptr;
  }
  if (ln->plan) {
    dbar_plan_destroy(ln->plan);
    cudaGetLastError();
    ln->plan = nullptr;
    S->used -= ln->bytes;
    ln->bytes = 0;
  }
  S->done_cv.notify_all();
}

// One cycle boundary of one lane: retire, admit, start, advance.  Returns
// false when the lane could not run (no memory for its plan yet).
// Records the lane's completion event after what was just queued on its stream.
void mark_inflight(Lane* ln) {
  if (!ln->done && cudaEventCreateWithFlags(&ln->done, cudaEventDisableTiming) != cudaSuccess) ln->done = nullptr;
  ln->inflight = ln->done && cudaEventRecord(ln->done, ln->stream) == cudaSuccess;
}

bool step_lane(dbar_server* S, Lane* ln) {
  std::unique_lock<std::mutex> lk(S->mu);
  if (!ln->plan && !ln->waiting.empty() && !open_lane(S, ln)) return false;
  if (!ln->plan) return false;
  const int B = ln->B;
  if (ln->part >= 0) {  // the next part of the cycle in progress (its previous part has finished)
    lk.unlock();
    const int np = plan_cycle_parts(ln->plan);
    int next = ln->part;
    if (next < np && !plan_parts_running(ln->plan, B)) next = np;  // every slot done: the tail
    const dbar_status sp = plan_step_part(ln->plan, B, next, ln->stream);
    lk.lock();
    if (sp != DBAR_OK) {
      cudaStreamSynchronize(ln->stream);
      lane_failed(S, ln, sp);
      return true;
    }
    ln->part = next < np ? next + 1 : -1;
    mark_inflight(ln);
    return true;
  }
  std::vector<int> act(B, 0), mask(B, 0);
  lk.unlock();
  dbar_status st = plan_active(ln->plan, B, act.data(), ln->stream);
  lk.lock();
  if (st != DBAR_OK) {
    lane_failed(S, ln, st);
    return true;
  }
  // retire finished slots
  for (int s = 0; s < B; ++s) {
    Request* r = ln->slot[s];
    if (!r || act[s]) continue;
    lk.unlock();
    if (!r->S) r->S = S->pool.get(r->n2);
    if (r->want_m && !r->m) r->m = S->pool.get(r->n2);
    st = (!r->S || (r->want_m && !r->m))
             ? dbar_internal_fail(DBAR_ENOMEM, "page-locked host buffer for a result")
             : plan_read_slot(ln->plan, s, r->S, r->want_m ? r->m : nullptr, &r->itot, &r->ncyc, &r->resid,
                              ln->stream);
    lk.lock();
    if (st != DBAR_OK) {
      lane_failed(S, ln, st);
      return true;
    }
    finish(S, r, r->resid <= S->defaults.tol ? DBAR_OK : DBAR_ENOCONV);
    ln->slot[s] = nullptr;
  }
  S->done_cv.notify_all();
  // admit waiting requests into free slots
  std::vector<Request*> admit(B, nullptr);
  int nnew = 0;
  for (int s = 0; s < B && !ln->waiting.empty(); ++s) {
    if (ln->slot[s]) continue;
    Request* r = ln->waiting.front();
    ln->waiting.pop_front();
    ln->slot[s] = r;
    admit[s] = r;
    r->t_start = S->now_ms();
    mask[s] = 1;
    ++nnew;
  }
  int occupied = 0;
  for (Request* r : ln->slot) occupied += r != nullptr;
  const bool inject = S->inject != 0 && occupied > 0;
  if (inject) S->inject = 0;
  lk.unlock();
  st = DBAR_OK;
  for (int s = 0; s < B && st == DBAR_OK; ++s)
    if (admit[s]) st = plan_load_slot(ln->plan, s, admit[s]->Q, admit[s]->k1, admit[s]->k2, ln->stream);
  if (st == DBAR_OK && nnew) st = plan_begin(ln->plan, B, mask.data(), ln->stream);
  if (st == DBAR_OK && occupied) st = plan_step_part(ln->plan, B, 0, ln->stream);  // first part of a cycle
  if (st == DBAR_OK && occupied) {
    ln->part = 1;
    mark_inflight(ln);
  }
  if (st == DBAR_OK && inject) st = dbar_internal_fail(DBAR_ECUDA, "injected lane failure");
  if (st != DBAR_OK) {
    cudaStreamSynchronize(ln->stream);
    lk.lock();
    lane_failed(S, ln, st);
  }
  return true;
}

void worker_main(dbar_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Lane*> todo;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->work_cv.wait(lk, [&] {
        if (S->stop) return true;
        for (Lane* l : S->lanes)
          if (l->busy()) return true;
        return false;
      });
      if (S->stop) return;
      for (Lane* l : S->lanes)
        if (l->busy()) todo.push_back(l);
    }
    bool progressed = false;
    for (Lane* l : todo)
      if (l->ready()) progressed |= step_lane(S, l);  // lanes still running their cycle are skipped
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

// dst = src (n doubles); false if some entry is not finite
bool copy_finite(double* __restrict__ dst, const double* __restrict__ src, size_t n) {
  bool ok = true;
  for (size_t i = 0; i < n; ++i) {
    const double v = src[i];
    ok &= std::isfinite(v);
    dst[i] = v;
  }
  return ok;
}

void free_request(dbar_server* S, Request* r) {
  S->pool.put(r->Q, r->n2);
  S->pool.put(r->S, r->n2);
  S->pool.put(r->m, r->n2);
  delete r;
}

void fill_result(const dbar_server* S, const Request* r, dbar_result* out) {
  out->status = (dbar_status)r->status;
  out->iters = r->itot;
  out->cycles = r->ncyc;
  out->resid = r->resid;
  out->latency_ms = r->t_done - r->t_submit;
  out->queue_ms = r->t_start >= 0 ? r->t_start - r->t_submit : 0.0;
  out->run_ms = r->t_start >= 0 ? r->t_done - r->t_start : 0.0;
  out->S = r->t_done >= 0 ? r->S : nullptr;
  out->m = r->t_done >= 0 ? r->m : nullptr;
  (void)S;
}

}  // namespace

extern "C" dbar_status dbar_serve_create(const dbar_params* defaults, size_t mem_budget, dbar_server_t* out) {
  if (!out || !defaults) return dbar_internal_fail(DBAR_EINVAL, "dbar_serve_create: NULL argument");
  *out = nullptr;
  if (defaults->iterated)
    return dbar_internal_fail(DBAR_EINVAL, "dbar_serve_create: the server solves the Sec. 4 equation (iterated = 0)");
  if (defaults->regularisation != DBAR_REG_TAYLOR)
    return dbar_internal_fail(DBAR_EINVAL, "dbar_serve_create: the server uses the Taylor-Gaussian regularisation");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return dbar_internal_fail(DBAR_ECUDA, "no CUDA device is available");
  }
  dbar_server* S = new (std::nothrow) dbar_server();
  if (!S) return dbar_internal_fail(DBAR_ENOMEM, "host allocation failed");
  S->defaults = *defaults;
  S->budget = mem_budget;
  S->t0 = Clock::now();
  cudaGetDevice(&S->device);
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete S;
    return dbar_internal_fail(DBAR_ECUDA, "stream creation failed");
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_submit(dbar_server_t S, const dbar_request* rq, uint64_t* ticket) {
  if (!S || !rq || !ticket) return dbar_internal_fail(DBAR_EINVAL, "dbar_serve_submit: NULL argument");
  const int N = rq->N;
  if (N < 32 || N > 2048 || (N & (N - 1)))
    return dbar_internal_fail(DBAR_EINVAL, "request N must be a power of two in [32, 2048]");
  if (!(rq->L > 0.0) || !std::isfinite(rq->L)) return dbar_internal_fail(DBAR_EINVAL, "request L must be > 0");
  if (!rq->Q) return dbar_internal_fail(DBAR_EINVAL, "request Q is NULL");
  if (!std::isfinite(rq->k_re) || !std::isfinite(rq->k_im)) return dbar_internal_fail(DBAR_EINVAL, "k is not finite");
  const size_t n2 = 2 * (size_t)N * N;
  dbar_params p = lane_params(S, N, rq->L, 1);
  if (plan_fixed_bytes(&p) + plan_slot_bytes(&p, 1) > S->budget)
    return dbar_internal_fail(DBAR_ENOMEM, "one slot of this grid does not fit the memory budget");
  // copy into a page-locked pool buffer and check for non-finite entries in the same pass
  double* q = S->pool.get(n2);
  if (!q) return dbar_internal_fail(DBAR_ENOMEM, "page-locked host buffer for the potential");
  if (!copy_finite(q, rq->Q, n2)) {
    S->pool.put(q, n2);
    return dbar_internal_fail(DBAR_EINVAL, "Q has a non-finite entry");
  }
  Request* r = new (std::nothrow) Request();
  if (!r) {
    S->pool.put(q, n2);
    return dbar_internal_fail(DBAR_ENOMEM, "host allocation failed");
  }
  r->N = N;
  r->L = rq->L;
  r->n2 = n2;
  r->Q = q;
  r->k1 = rq->k_re;
  r->k2 = rq->k_im;
  r->want_m = rq->want_m;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    r->t_submit = S->now_ms();
    if (S->first_submit < 0) S->first_submit = r->t_submit;
    Lane* ln = nullptr;
    for (Lane* l : S->lanes)
      if (l->N == N && l->L == rq->L) ln = l;
    if (!ln) {
      ln = new Lane();
      ln->N = N;
      ln->L = rq->L;
      S->lanes.push_back(ln);
    }
    ln->waiting.push_back(r);
    S->reqs[r->ticket] = r;
    *ticket = r->ticket;
  }
  S->work_cv.notify_one();
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_poll(dbar_server_t S, uint64_t ticket, dbar_result* out) {
  if (!S || !out) return dbar_internal_fail(DBAR_EINVAL, "dbar_serve_poll: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end() || it->second->released) return dbar_internal_fail(DBAR_EINVAL, "unknown ticket");
  if (it->second->t_done < 0) return DBAR_EBUSY;
  fill_result(S, it->second, out);
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_wait(dbar_server_t S, uint64_t ticket, double timeout_s, dbar_result* out) {
  if (!S || !out) return dbar_internal_fail(DBAR_EINVAL, "dbar_serve_wait: NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end() || it->second->released) return dbar_internal_fail(DBAR_EINVAL, "unknown ticket");
  Request* r = it->second;
  const auto pred = [&] { return r->t_done >= 0; };
  if (timeout_s < 0) {
    S->done_cv.wait(lk, pred);
  } else if (!S->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return dbar_internal_fail(DBAR_ETIMEOUT, "request not finished within the timeout");
  }
  fill_result(S, r, out);
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_release(dbar_server_t S, uint64_t ticket) {
  if (!S) return dbar_internal_fail(DBAR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return dbar_internal_fail(DBAR_EINVAL, "unknown ticket");
  if (it->second->t_done < 0) return dbar_internal_fail(DBAR_EBUSY, "request still running");
  free_request(S, it->second);
  S->reqs.erase(it);
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_stats(dbar_server_t S, double* p50_ms, double* p99_ms, double* solves_per_s,
                                        uint64_t* completed, uint64_t* pending) {
  if (!S) return dbar_internal_fail(DBAR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const double pos = q * (double)(l.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < l.size() ? l[i] * (1.0 - f) + l[i + 1] * f : l[i];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (solves_per_s)
    *solves_per_s = (S->completed > 0 && S->last_done > S->first_submit)
                        ? (double)S->completed / ((S->last_done - S->first_submit) / 1e3)
                        : 0.0;
  if (completed) *completed = S->completed;
  if (pending) {
    uint64_t n = 0;
    for (auto& kv : S->reqs) n += kv.second->t_done < 0;
    *pending = n;
  }
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_inject_fault(dbar_server_t S) {
  if (!S) return dbar_internal_fail(DBAR_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  S->inject = 1;
  return DBAR_OK;
}

extern "C" dbar_status dbar_serve_destroy(dbar_server_t S) {
  if (!S) return DBAR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->work_cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  for (Lane* l : S->lanes) {
    if (l->stream) cudaStreamSynchronize(l->stream);
    if (l->plan) dbar_plan_destroy(l->plan);
    if (l->done) cudaEventDestroy(l->done);
    if (l->stream) cudaStreamDestroy(l->stream);
    delete l;
  }
  for (auto& kv : S->reqs) free_request(S, kv.second);
  cudaStreamDestroy(S->stream);
  delete S;
  return DBAR_OK;
}
