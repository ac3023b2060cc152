// serve.cu -- a request server with continuous batching over CBS plans.
//
// Requests (a grid, a permittivity, a source; optionally the adjoint of |E(r0)|^2 and the
// gradient) queue on submission.  One worker thread owns the GPU work: it admits queued
// requests into slots -- a slot is a plan with its own stream and field buffers for one grid
// shape -- while the device-memory budget and the limit on requests in flight allow, and
// advances every slot's series one block of iterations at a time without blocking on any of
// them.  Requests that arrive while others run are admitted as soon as a slot and memory are
// free, and their blocks interleave with the running ones on the GPU.  Idle slots are kept
// for requests of the same shape and evicted (least recently used) when memory is needed.
//
// A request's result is the same alone and in any mix: slots share no device memory, every
// kernel and reduction has a fixed order, and the stopping decision depends on the request's
// own residuals only.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <vector>

#include "plan.h"

namespace cbs {
const char* last_error_message();
}

using namespace cbs;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ShapeKey {
  int nx, ny, nz;
  double pitch, lam, nbg;
  int lo[3], hi[3];
  double layer_rt, layer_pow;
  int layer_corner;
  bool operator==(const ShapeKey& o) const {
    return nx == o.nx && ny == o.ny && nz == o.nz && pitch == o.pitch && lam == o.lam && nbg == o.nbg &&
           std::memcmp(lo, o.lo, sizeof(lo)) == 0 && std::memcmp(hi, o.hi, sizeof(hi)) == 0 &&
           layer_rt == o.layer_rt && layer_pow == o.layer_pow && layer_corner == o.layer_corner;
  }
};

ShapeKey key_of(const cbs_request& r) {
  ShapeKey k{r.nx, r.ny, r.nz, r.pitch_m, r.lambda_m, r.n_bg, {}, {},
             r.layer_round_trip, r.layer_power, r.layer_corner_max};
  for (int i = 0; i < 3; ++i) {
    k.lo[i] = r.pad_lo[i];
    k.hi[i] = r.pad_hi[i];
  }
  return k;
}

// Device bytes of a slot: the plan (V, W and the iterate at padded row pitch; twiddles and
// reduction scratch under 16 MB) and the slot's eps, E, E_adj and gradient.
size_t slot_bytes(const ShapeKey& k) {
  const size_t nxp = (size_t)((k.nx + 15) / 16 * 16);
  const size_t Nw = nxp * (k.ny + 1) * k.nz, N = (size_t)k.nx * k.ny * k.nz;   // planes may get a padding row
  return Nw * (8 + 24 + 24) + N * (4 + 24 + 24 + 4) + ((size_t)16 << 20);
}

struct Job {
  long long id = 0;
  cbs_request r{};
  double t_submit = 0;
  int passed = 0;          // later requests admitted while this one did not fit
};

// A queued request that does not fit yet lets later ones pass at most this many times; then
// nothing behind it is admitted until it fits (memory frees as running requests finish), so
// a large request in a stream of small ones waits a bounded time.
constexpr int kMaxPassed = 8;

enum class Phase { Idle, Forward, Adjoint, Output };

struct Slot {
  ShapeKey key{};
  cudaStream_t stream = nullptr;
  cbs_plan_s* plan = nullptr;
  float* eps = nullptr;
  float2* E = nullptr;
  float2* Ea = nullptr;
  float* grad = nullptr;
  double* obj_host = nullptr;       // pinned
  cudaEvent_t out_ev = nullptr;
  size_t bytes = 0;
  Phase phase = Phase::Idle;
  Job job;
  cbs_result res{};
  SeriesRun run;
  double last_used = 0;
};

void free_slot(Slot* s) {
  if (s->plan) cbs_destroy(s->plan);
  for (void* q : {(void*)s->eps, (void*)s->E, (void*)s->Ea, (void*)s->grad})
    if (q) cudaFree(q);
  if (s->obj_host) cudaFreeHost(s->obj_host);
  if (s->out_ev) cudaEventDestroy(s->out_ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // namespace

struct cbs_server_s {
  cbs_server_desc d{};
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> incoming;              // submitted, not yet seen by the worker
  std::list<Job> queue;                  // waiting for admission (worker only; a list, so
                                         // erasing one keeps pointers to the others valid)
  std::deque<cbs_result> done;           // completed, not yet taken
  long long next_id = 1;
  bool stop = false;
  long long n_queued = 0, n_active = 0;  // mirrors for cbs_server_info
  std::atomic<size_t> bytes_used{0};     // device bytes held by slots (written by the worker)
  std::list<Slot*> slots;                // worker only
  std::thread worker;
};

namespace {

bool fatal(int rc) { return !nonfatal(rc); }

void finish(cbs_server_s* S, Slot* s, int status) {
  s->res.status = status;
  s->res.t_done = now_s();
  if (fatal(status) && s->res.error[0] == 0)
    std::snprintf(s->res.error, sizeof(s->res.error), "%s", last_error_message());
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(s->res);
    S->n_active -= 1;
  }
  S->cv_done.notify_all();
  s->phase = Phase::Idle;
  s->last_used = now_s();
}

int make_slot(cbs_server_s* S, const ShapeKey& k, Slot** out) {
  auto* s = new Slot;
  s->key = k;
  s->bytes = slot_bytes(k);
  const size_t N = (size_t)k.nx * k.ny * k.nz;
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->out_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&s->obj_host, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->eps, N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->E, 3 * N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&s->Ea, 3 * N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&s->grad, N * sizeof(float));
  if (e != cudaSuccess) {
    free_slot(s);
    return fail(e == cudaErrorMemoryAllocation ? CBS_ERR_OOM : CBS_ERR_CUDA, "slot set-up: %s",
                cudaGetErrorString(e));
  }
  cbs_plan_desc pd{};
  pd.nx = k.nx;
  pd.ny = k.ny;
  pd.nz = k.nz;
  pd.pitch_m = k.pitch;
  pd.lambda_m = k.lam;
  pd.n_bg = k.nbg;
  for (int i = 0; i < 3; ++i) {
    pd.pad_lo[i] = k.lo[i];
    pd.pad_hi[i] = k.hi[i];
  }
  pd.layer_round_trip = k.layer_rt;
  pd.layer_power = k.layer_pow;
  pd.layer_corner_max = k.layer_corner;
  pd.tol = S->d.tol;
  pd.max_iter = S->d.max_iter;
  pd.check_every = S->d.check_every;
  pd.cuda_stream = s->stream;
  const int rc = cbs_plan(&s->plan, &pd);
  if (rc) {
    s->plan = nullptr;
    free_slot(s);
    return rc;
  }
  *out = s;
  return CBS_OK;
}

// Forward phase of an admitted request: permittivity, potential, first block.
int start_job(Slot* s) {
  cbs_plan_s* p = s->plan;
  const cbs_request& r = s->job.r;
  const size_t N = (size_t)r.nx * r.ny * r.nz;
  const float* eps = r.eps_dev;
  if (!eps) {
    CK(cudaMemcpyAsync(s->eps, r.eps_host, N * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    eps = s->eps;
  }
  int rc = cbs_set_permittivity(p, eps);
  if (rc) return rc;
  SourceArgs src;
  rc = make_source(p, &r.src, src);
  if (rc) return rc;
  series_begin(p, s->E, src, 0, s->run);
  s->phase = Phase::Forward;
  return CBS_OK;
}

// Objective, gradient and the copies of the requested outputs, then the slot's out event.
int enqueue_outputs(Slot* s) {
  cbs_plan_s* p = s->plan;
  const cbs_request& r = s->job.r;
  const size_t N = (size_t)r.nx * r.ny * r.nz;
  CK(launch_objective(s->E, N, r.nx, r.ny, r.r0[0], r.r0[1], r.r0[2], p->dobj, s->stream));
  CK(cudaMemcpyAsync(s->obj_host, p->dobj, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  if (r.adjoint) {
    CK(launch_gradient(s->E, s->Ea, N, (float)(2.0 * p->kvac * p->kvac), s->grad, s->stream));
    if (r.grad_dev) CK(cudaMemcpyAsync(r.grad_dev, s->grad, N * sizeof(float), cudaMemcpyDeviceToDevice, s->stream));
    if (r.grad_host) CK(cudaMemcpyAsync(r.grad_host, s->grad, N * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
  }
  if (r.E_dev) CK(cudaMemcpyAsync(r.E_dev, s->E, 3 * N * sizeof(float2), cudaMemcpyDeviceToDevice, s->stream));
  if (r.E_host) CK(cudaMemcpyAsync(r.E_host, s->E, 3 * N * sizeof(float2), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaEventRecord(s->out_ev, s->stream));
  s->phase = Phase::Output;
  return CBS_OK;
}

// Move a busy slot along without blocking; returns whether anything happened.
bool advance(cbs_server_s* S, Slot* s) {
  cbs_plan_s* p = s->plan;
  if (s->phase == Phase::Forward || s->phase == Phase::Adjoint) {
    const bool was_fwd = s->phase == Phase::Forward;
    const int it0 = s->run.it;
    if (!series_advance(p, s->run, false)) return s->run.it != it0;
    cbs_stats st{};
    const int rc = series_stats(p, s->run, &st);
    (was_fwd ? s->res.fwd : s->res.adj) = st;
    if (rc != CBS_OK && s->res.error[0] == 0)
      std::snprintf(s->res.error, sizeof(s->res.error), "%s: %s", was_fwd ? "forward" : "adjoint",
                    last_error_message());
    if (fatal(rc)) {
      finish(S, s, rc);
      return true;
    }
    int rc2 = CBS_OK;
    if (was_fwd && s->job.r.adjoint) {
      SourceArgs src;
      rc2 = adjoint_source(p, s->job.r.r0, s->E, src);
      if (!rc2) {
        series_begin(p, s->Ea, src, 0, s->run);
        s->phase = Phase::Adjoint;
      }
    } else {
      rc2 = enqueue_outputs(s);
    }
    if (rc2) finish(S, s, rc2);
    return true;
  }
  if (s->phase == Phase::Output) {
    const cudaError_t e = cudaEventQuery(s->out_ev);
    if (e == cudaErrorNotReady) return false;
    if (e != cudaSuccess) {
      finish(S, s, fail(CBS_ERR_CUDA, "output copies: %s", cudaGetErrorString(e)));
      return true;
    }
    s->res.objective = *s->obj_host;
    int st = CBS_OK;
    if (s->res.fwd.status != CBS_OK) st = s->res.fwd.status;
    else if (s->job.r.adjoint && s->res.adj.status != CBS_OK) st = s->res.adj.status;
    finish(S, s, st);
    return true;
  }
  return false;
}

// Admit queued requests in arrival order while the limits allow.  A request that does not fit
// yet lets later ones pass, kMaxPassed times at most; after that admission waits for it.
// Returns whether anything was admitted.
bool admit(cbs_server_s* S) {
  bool any = false;
  Job* blocked = nullptr;   // the oldest queued request that did not fit in this pass
  for (auto it = S->queue.begin(); it != S->queue.end();) {
    if (blocked && blocked->passed >= kMaxPassed) break;
    long long active;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      active = S->n_active;
    }
    if (active >= S->d.max_active) break;
    const ShapeKey k = key_of(it->r);
    Slot* slot = nullptr;
    for (Slot* s : S->slots)
      if (s->phase == Phase::Idle && s->key == k) {
        slot = s;
        break;
      }
    if (!slot) {
      const size_t need = slot_bytes(k);
      // evict idle slots of other shapes, least recently used first, until the new one fits
      while (S->bytes_used + need > S->budget) {
        Slot* lru = nullptr;
        for (Slot* s : S->slots)
          if (s->phase == Phase::Idle && (!lru || s->last_used < lru->last_used)) lru = s;
        if (!lru) break;
        S->slots.remove(lru);
        S->bytes_used -= lru->bytes;
        free_slot(lru);
      }
      if (S->bytes_used + need > S->budget) {
        bool none_busy = true;
        for (Slot* s : S->slots) none_busy = none_busy && s->phase == Phase::Idle;
        if (none_busy) {   // can never fit: fail it rather than wait forever
          cbs_result res{};
          res.id = it->id;
          res.t_submit = it->t_submit;
          res.t_admit = res.t_done = now_s();
          res.status = CBS_ERR_OOM;
          std::snprintf(res.error, sizeof(res.error), "request needs %zu bytes, over the server's budget of %zu",
                        need, S->budget);
          {
            std::lock_guard<std::mutex> lk(S->mu);
            S->done.push_back(res);
            S->n_queued -= 1;
          }
          S->cv_done.notify_all();
          it = S->queue.erase(it);
          any = true;
          continue;
        }
        if (!blocked) blocked = &*it;
        ++it;
        continue;
      }
      const int rc = make_slot(S, k, &slot);
      if (rc) {
        cbs_result res{};
        res.id = it->id;
        res.t_submit = it->t_submit;
        res.t_admit = res.t_done = now_s();
        res.status = rc;
        std::snprintf(res.error, sizeof(res.error), "%s", last_error_message());
        {
          std::lock_guard<std::mutex> lk(S->mu);
          S->done.push_back(res);
          S->n_queued -= 1;
        }
        S->cv_done.notify_all();
        it = S->queue.erase(it);
        any = true;
        continue;
      }
      S->slots.push_back(slot);
      S->bytes_used += slot->bytes;
    }
    if (blocked) blocked->passed += 1;
    slot->job = *it;
    slot->res = cbs_result{};
    slot->res.id = it->id;
    slot->res.t_submit = it->t_submit;
    slot->res.t_admit = now_s();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->n_queued -= 1;
      S->n_active += 1;
    }
    it = S->queue.erase(it);
    any = true;
    const int rc = start_job(slot);
    if (rc) finish(S, slot, rc);
  }
  return any;
}

void worker_main(cbs_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      const bool idle_gpu = S->n_active == 0;
      if (idle_gpu && S->queue.empty() && S->incoming.empty()) {
        if (S->stop) break;
        S->cv_work.wait(lk, [&] { return S->stop || !S->incoming.empty(); });
      }
      while (!S->incoming.empty()) {
        S->queue.push_back(S->incoming.front());
        S->incoming.pop_front();
      }
      if (S->stop && S->n_active == 0) {
        // closing: queued requests are not started
        for (const Job& j : S->queue) {
          cbs_result res{};
          res.id = j.id;
          res.t_submit = j.t_submit;
          res.t_admit = res.t_done = now_s();
          res.status = CBS_ERR_STATE;
          std::snprintf(res.error, sizeof(res.error), "server closed before the request started");
          S->done.push_back(res);
        }
        S->n_queued = 0;
        S->queue.clear();
        S->cv_done.notify_all();
        break;
      }
    }
    bool progressed = false;
    if (!S->stop) progressed = admit(S);
    for (Slot* s : S->slots)
      if (s->phase != Phase::Idle) progressed = advance(S, s) || progressed;
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  for (Slot* s : S->slots) {
    cudaStreamSynchronize(s->stream);
    free_slot(s);
  }
  S->slots.clear();
  S->bytes_used = 0;
}

}  // namespace

extern "C" {

int cbs_server_create(cbs_server_t* out, const cbs_server_desc* desc) {
  if (!out || !desc) return fail(CBS_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (desc->max_active < 1 || desc->max_iter < 1 || desc->check_every < 1)
    return fail(CBS_ERR_ARG, "max_active, max_iter and check_every must be >= 1");
  auto* S = new cbs_server_s;
  S->d = *desc;
  cudaError_t e = cudaGetDevice(&S->device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete S;
    return fail(CBS_ERR_CUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  S->budget = desc->hbm_budget_bytes ? (size_t)desc->hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return CBS_OK;
}

int cbs_server_submit(cbs_server_t S, const cbs_request* req, long long* id) {
  if (!S || !req) return fail(CBS_ERR_ARG, "NULL argument");
  const cbs_request& r = *req;
  if ((r.eps_host == nullptr) == (r.eps_dev == nullptr)) return fail(CBS_ERR_ARG, "give exactly one of eps_host, eps_dev");
  if (r.nx < 1 || r.ny < 1 || r.nz < 1) return fail(CBS_ERR_ARG, "bad grid %d x %d x %d", r.nx, r.ny, r.nz);
  if (r.r0[0] < 0 || r.r0[0] >= r.nx || r.r0[1] < 0 || r.r0[1] >= r.ny || r.r0[2] < 0 || r.r0[2] >= r.nz)
    return fail(CBS_ERR_ARG, "r0 (%d,%d,%d) outside the grid", r.r0[0], r.r0[1], r.r0[2]);
  if (r.src.warm_start != 0) return fail(CBS_ERR_ARG, "served solves start from zero (warm_start must be 0)");
  if (r.src.kind == CBS_SRC_USER) return fail(CBS_ERR_ARG, "served solves take plane-wave or point sources");
  Job j;
  j.r = r;
  j.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(CBS_ERR_STATE, "server is closing");
    j.id = S->next_id++;
    S->incoming.push_back(j);
    S->n_queued += 1;
  }
  S->cv_work.notify_one();
  if (id) *id = j.id;
  return CBS_OK;
}

int cbs_server_take(cbs_server_t S, cbs_result* out, int max, double timeout_s, int* n) {
  if (!S || !out || !n || max < 1) return fail(CBS_ERR_ARG, "bad argument");
  *n = 0;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && timeout_s > 0)
    S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return !S->done.empty(); });
  while (*n < max && !S->done.empty()) {
    out[(*n)++] = S->done.front();
    S->done.pop_front();
  }
  return CBS_OK;
}

int cbs_server_info(cbs_server_t S, long long* queued, long long* active, double* bytes_used) {
  if (!S) return fail(CBS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (queued) *queued = S->n_queued;
  if (active) *active = S->n_active;
  if (bytes_used) *bytes_used = (double)S->bytes_used;
  return CBS_OK;
}

void cbs_server_destroy(cbs_server_t S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  delete S;
}

}  // extern "C"
