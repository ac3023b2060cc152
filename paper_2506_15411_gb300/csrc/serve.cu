// serve.cu -- a request server with continuous batching over CBS plans.
//
// Requests (a grid, a permittivity, a source; optionally the adjoint of |E(r0)|^2 and the
// gradient) queue on submission.  One worker thread owns the GPU work.  Requests of the same
// grid shape share a batch: a plan whose arrays hold up to kMaxMembers requests side by side
// (seats), each with its own permittivity, splitting and source.  Every launch of a batch's
// block of iterations carries all of its iterating requests (the tile space has a request
// index), so same-shape requests in flight share each persistent launch instead of taking
// turns on the GPU.  The worker admits queued requests into free seats, or into a new batch,
// while the device-memory budget and the limit on requests in flight allow; a request that
// arrives while others run joins its batch at the next block of iterations, and one whose
// series has stopped leaves it there.  Batches of different shapes run on their own streams.
// Batches without requests are kept for later requests of their shape and evicted (least
// recently used) when memory is needed.
//
// A request's result is the same alone and in any mix: its blocks of a launch are the blocks
// of its own persistent grid (so its tiles and the order of its residual sums do not depend
// on the other members), seats share no device memory, and the stopping decision depends on
// the request's own residuals only.  Batches of smaller grids run on higher-priority streams.
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

// Device bytes of a seat: the plan's V, W and iterate at padded row pitch, and the request's
// eps, E, E_adj and gradient; a batch adds under 16 MB of tables and reduction scratch.
size_t seat_bytes(const ShapeKey& k) {
  const size_t nxp = (size_t)((k.nx + 15) / 16 * 16);
  const size_t Nw = nxp * k.ny * k.nz, N = (size_t)k.nx * k.ny * k.nz;
  return Nw * (8 + 24 + 24) + N * (4 + 24 + 24 + 4);
}
size_t batch_bytes(const ShapeKey& k, int seats) { return seats * seat_bytes(k) + ((size_t)16 << 20); }

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

// One request's place in a batch.
struct Seat {
  int idx = 0;                  // seat index in the plan's arrays
  Phase phase = Phase::Idle;
  Job job;
  cbs_result res{};
  float* eps = nullptr;         // the request's permittivity (copied here when given on the host)
  float2* E = nullptr;          // forward field, dense [3][nz][ny][nx]
  float2* Ea = nullptr;         // adjoint field, dense
  float* grad = nullptr;
  double* obj_host = nullptr;   // pinned
  cudaEvent_t out_ev = nullptr;
  Member mem{};                 // the request in a launch: source, splitting, seat
  SeriesRun run;                // its series (stopping rules; run.E is the field it fills)
  int blk = 0;                  // its iterations in the block in flight (0: not in it)
};

// A plan whose seats hold requests of one grid shape, with its own stream; `setup` is the
// stream of the seats' permittivity set-up, which runs beside the batch's iterations.
struct Batch {
  ShapeKey key{};
  cudaStream_t stream = nullptr, setup = nullptr;
  cbs_plan_s* plan = nullptr;
  std::vector<Seat> seats;
  size_t bytes = 0;
  bool in_flight = false;       // a block of iterations is enqueued (the plan's blk_ev ends it)
  double last_used = 0;
  int busy() const {
    int n = 0;
    for (const Seat& s : seats) n += s.phase != Phase::Idle;
    return n;
  }
};

void free_batch(Batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->setup) cudaStreamSynchronize(b->setup);
  if (b->plan) cbs_destroy(b->plan);
  for (Seat& s : b->seats) {
    for (void* q : {(void*)s.eps, (void*)s.E, (void*)s.Ea, (void*)s.grad})
      if (q) cudaFree(q);
    if (s.obj_host) cudaFreeHost(s.obj_host);
    if (s.out_ev) cudaEventDestroy(s.out_ev);
  }
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->setup) cudaStreamDestroy(b->setup);
  delete b;
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
  std::atomic<size_t> bytes_used{0};     // device bytes held by batches (written by the worker)
  long long n_launches = 0, n_member_iters = 0;   // launch sharing (under mu)
  int max_members = 0;
  std::list<Batch*> batches;             // worker only
  std::thread worker;
};

namespace {

bool fatal(int rc) { return !nonfatal(rc); }

void finish(cbs_server_s* S, Batch* b, Seat& s, int status) {
  s.res.status = status;
  s.res.t_done = now_s();
  if (fatal(status) && s.res.error[0] == 0)
    std::snprintf(s.res.error, sizeof(s.res.error), "%s", last_error_message());
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(s.res);
    S->n_active -= 1;
  }
  S->cv_done.notify_all();
  s.phase = Phase::Idle;
  s.blk = 0;
  b->last_used = now_s();
}

// Stream priority of a batch: smaller grids get higher priority (one level per factor of 4 in
// voxels above 2^20, as far as the device's range goes), so that when batches of different
// sizes are in flight the GPU picks a small request's next kernel before a large one's and
// short requests are not held to the pace of long ones.
int batch_priority(size_t voxels) {
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
  int level = 0;
  for (size_t v = (size_t)1 << 21; v < voxels && greatest + level < least; v <<= 2) ++level;
  return greatest + level;
}

int make_batch(cbs_server_s* S, const ShapeKey& k, int seats, Batch** out) {
  auto* b = new Batch;
  b->key = k;
  b->bytes = batch_bytes(k, seats);
  b->seats.resize(seats);
  const size_t N = (size_t)k.nx * k.ny * k.nz;
  const int prio = batch_priority(N);
  cudaError_t e = cudaStreamCreateWithPriority(&b->stream, cudaStreamNonBlocking, prio);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->setup, cudaStreamNonBlocking, prio);
  for (int i = 0; i < seats && e == cudaSuccess; ++i) {
    Seat& s = b->seats[i];
    s.idx = i;
    e = cudaEventCreateWithFlags(&s.out_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&s.obj_host, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s.eps, N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s.E, 3 * N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&s.Ea, 3 * N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&s.grad, N * sizeof(float));
  }
  if (e != cudaSuccess) {
    free_batch(b);
    return fail(e == cudaErrorMemoryAllocation ? CBS_ERR_OOM : CBS_ERR_CUDA, "batch set-up: %s",
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
  pd.cuda_stream = b->stream;
  const int rc = plan_create(&b->plan, &pd, seats);
  if (rc) {
    b->plan = nullptr;
    free_batch(b);
    return rc;
  }
  *out = b;
  return CBS_OK;
}

// Start the series of seat s (field `E` receives the result) with source `src`: the seat's
// iterate and residual counter are cleared and the series' first x pass is enqueued on the
// batch's stream, after whatever is in flight there; the seat takes part from the next block.
int seat_begin(Batch* b, Seat& s, float2* E, const SourceArgs& src, Phase phase) {
  cbs_plan_s* p = b->plan;
  s.run = SeriesRun{};
  s.run.t0 = std::chrono::steady_clock::now();
  s.run.E = E;
  s.mem.src = src;
  s.blk = 0;
  const size_t Nw = p->base.Nw;
  CK(cudaMemsetAsync(p->Ei + (size_t)s.idx * 3 * Nw, 0, 3 * Nw * sizeof(float2), b->stream));
  CK(cudaMemsetAsync(p->counter + s.idx, 0, sizeof(unsigned), b->stream));
  // the seat's own member slot (its previous copy completed with its previous series)
  p->mem_host[1 + s.idx] = s.mem;
  CK(cudaMemcpyAsync(p->mem_dev + 1 + s.idx, p->mem_host + 1 + s.idx, sizeof(Member), cudaMemcpyHostToDevice,
                     b->stream));
  IterArgs a = p->base;
  a.nmem = 1;
  a.mem = p->mem_dev + 1 + s.idx;
  CK(launch_xpass_fwd(a, b->stream));
  s.phase = phase;
  return CBS_OK;
}

// An admitted request: its permittivity and splitting (on the set-up stream), source, and the
// start of its forward series.
int start_job(Batch* b, Seat& s) {
  cbs_plan_s* p = b->plan;
  const cbs_request& r = s.job.r;
  const size_t N = (size_t)r.nx * r.ny * r.nz;
  const float* eps = r.eps_dev;
  if (!eps) {
    CK(cudaMemcpyAsync(s.eps, r.eps_host, N * sizeof(float), cudaMemcpyHostToDevice, b->setup));
    eps = s.eps;
  }
  int rc = seat_permittivity(p, s.idx, eps, b->setup);
  if (rc) return rc;
  s.mem = Member{};
  s.mem.seat = s.idx;
  s.mem.inv_eps = (float)(1.0 / p->seat_eps[s.idx]);
  s.mem.kt2 = make_float2((float)p->seat_k0sq[s.idx], (float)p->seat_eps[s.idx]);
  SourceArgs src;
  rc = make_source(p, &r.src, src);
  if (rc) return rc;
  return seat_begin(b, s, s.E, src, Phase::Forward);
}

// Objective, gradient and the copies of the requested outputs, then the seat's out event.
int enqueue_outputs(Batch* b, Seat& s) {
  cbs_plan_s* p = b->plan;
  const cbs_request& r = s.job.r;
  const size_t N = (size_t)r.nx * r.ny * r.nz;
  cudaStream_t st = b->stream;
  double* dobj = p->dobj + s.idx;
  CK(launch_objective(s.E, N, r.nx, r.ny, r.r0[0], r.r0[1], r.r0[2], dobj, st));
  CK(cudaMemcpyAsync(s.obj_host, dobj, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (r.adjoint) {
    CK(launch_gradient(s.E, s.Ea, N, (float)(2.0 * p->kvac * p->kvac), s.grad, st));
    if (r.grad_dev) CK(cudaMemcpyAsync(r.grad_dev, s.grad, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (r.grad_host) CK(cudaMemcpyAsync(r.grad_host, s.grad, N * sizeof(float), cudaMemcpyDeviceToHost, st));
  }
  if (r.E_dev) CK(cudaMemcpyAsync(r.E_dev, s.E, 3 * N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if (r.E_host) CK(cudaMemcpyAsync(r.E_host, s.E, 3 * N * sizeof(float2), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(s.out_ev, st));
  s.phase = Phase::Output;
  return CBS_OK;
}

// Enqueue the next block of iterations of every iterating seat: iteration k launches the
// seats that still have k iterations to go in this block (the same number a seat would run
// alone), then the residual sums of all seats and the error flag come back, and the plan's
// blk_ev marks the end.
int enqueue_block(cbs_server_s* S, Batch* b) {
  cbs_plan_s* p = b->plan;
  int L = 0;
  for (Seat& s : b->seats) {
    s.blk = 0;
    if (s.phase != Phase::Forward && s.phase != Phase::Adjoint) continue;
    s.blk = std::min(p->d.check_every, p->d.max_iter - s.run.it);
    L = std::max(L, s.blk);
  }
  if (L == 0) return CBS_OK;
  // the member lists of the block's iterations, staged and copied at once (the previous
  // block's copy has completed: its event was waited for)
  const size_t base = 1 + (size_t)p->seats;
  std::vector<int> nm(L);
  for (int k = 0; k < L; ++k) {
    Member* list = p->mem_host + base + (size_t)k * kMaxMembers;
    nm[k] = 0;
    for (const Seat& s : b->seats)
      if (s.blk > k) list[nm[k]++] = s.mem;
  }
  CK(cudaMemcpyAsync(p->mem_dev + base, p->mem_host + base, (size_t)L * kMaxMembers * sizeof(Member),
                     cudaMemcpyHostToDevice, b->stream));
  IterArgs a = p->base;
  for (int k = 0; k < L; ++k) {
    a.nmem = nm[k];
    a.mem = p->mem_dev + base + (size_t)k * kMaxMembers;
    a.slot = k;
    const int rc = launch_iteration(p, a, b->stream, nullptr);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(S->mu);
    S->n_launches += 1;
    S->n_member_iters += a.nmem;
    S->max_members = std::max(S->max_members, a.nmem);
  }
  const size_t nh = (size_t)p->seats * p->base.hist_cap;
  CK(cudaMemcpyAsync(p->hist_host, p->hist, nh * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaMemcpyAsync(p->err_host, p->err_dev, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaEventRecord(p->blk_ev, b->stream));
  b->in_flight = true;
  return CBS_OK;
}

// A seat's series has stopped (R.rc says how): copy its iterate out, then either start the
// adjoint series or enqueue the outputs; a fatal error ends the request.
void seat_series_end(cbs_server_s* S, Batch* b, Seat& s) {
  cbs_plan_s* p = b->plan;
  const bool was_fwd = s.phase == Phase::Forward;
  cbs_stats st{};
  int rc = series_stats(p, s.run, &st);
  (was_fwd ? s.res.fwd : s.res.adj) = st;
  if (rc != CBS_OK && s.res.error[0] == 0)
    std::snprintf(s.res.error, sizeof(s.res.error), "%s: %s", was_fwd ? "forward" : "adjoint", last_error_message());
  const cudaError_t e = field_copy(p, s.idx, s.run.E, true, b->stream);
  if (e != cudaSuccess && !fatal(rc)) rc = fail(CBS_ERR_CUDA, "field copy-out: %s", cudaGetErrorString(e));
  if (fatal(rc)) {
    finish(S, b, s, rc);
    return;
  }
  int rc2 = CBS_OK;
  if (was_fwd && s.job.r.adjoint) {
    const cbs_request& r = s.job.r;
    float2* amp = p->adj_amp + 3 * s.idx;
    const cudaError_t ea = launch_adjoint_amp(s.E, p->N, r.nx, r.ny, r.r0[0], r.r0[1], r.r0[2],
                                              (float)(p->pitch * p->pitch), amp, b->stream);
    if (ea != cudaSuccess) {
      rc2 = fail(CBS_ERR_CUDA, "adjoint source: %s", cudaGetErrorString(ea));
    } else {
      SourceArgs src{};
      src.kind = CBS_SRC_POINT;
      src.px = r.r0[0];
      src.py = r.r0[1];
      src.pz = r.r0[2];
      src.amp_dev = amp;
      rc2 = seat_begin(b, s, s.Ea, src, Phase::Adjoint);
    }
  } else {
    rc2 = enqueue_outputs(b, s);
  }
  if (rc2) finish(S, b, s, rc2);
}

// Move a batch along without blocking; returns whether anything happened.
bool advance(cbs_server_s* S, Batch* b) {
  cbs_plan_s* p = b->plan;
  bool any = false;
  if (b->in_flight) {
    const cudaError_t e = cudaEventQuery(p->blk_ev);
    if (e != cudaErrorNotReady) {
      b->in_flight = false;
      any = true;
      int err = CBS_OK;
      if (e != cudaSuccess) {
        err = fail(CBS_ERR_CUDA, "iteration block failed: %s", cudaGetErrorString(e));
      } else if (*p->err_host) {
        err = fail(CBS_ERR_CUDA, "a tensor-copy wait timed out in an FFT pass (device error %d)", *p->err_host);
        *p->err_host = 0;
        cudaMemsetAsync(p->err_dev, 0, sizeof(int), b->stream);
      }
      for (Seat& s : b->seats) {
        if (s.blk == 0) continue;
        bool over;
        if (err) {
          s.run.rc = err;
          over = true;
        } else {
          s.run.m = s.blk;
          over = series_absorb_residuals(p, s.run, p->hist_host + (size_t)s.idx * p->base.hist_cap);
        }
        s.blk = 0;
        if (over) seat_series_end(S, b, s);
      }
    }
  }
  for (Seat& s : b->seats) {
    if (s.phase != Phase::Output) continue;
    const cudaError_t e = cudaEventQuery(s.out_ev);
    if (e == cudaErrorNotReady) continue;
    any = true;
    if (e != cudaSuccess) {
      finish(S, b, s, fail(CBS_ERR_CUDA, "output copies: %s", cudaGetErrorString(e)));
      continue;
    }
    s.res.objective = *s.obj_host;
    int st = CBS_OK;
    if (s.res.fwd.status != CBS_OK) st = s.res.fwd.status;
    else if (s.job.r.adjoint && s.res.adj.status != CBS_OK) st = s.res.adj.status;
    finish(S, b, s, st);
  }
  if (!b->in_flight) {
    const int rc = enqueue_block(S, b);
    if (rc) {   // a launch failed: every seat of the block ends with the error
      for (Seat& s : b->seats)
        if (s.blk > 0) {
          s.run.rc = rc;
          s.blk = 0;
          seat_series_end(S, b, s);
        }
      any = true;
    }
  }
  return any;
}

// Post a result for a queued request that ends before admission.
void reject(cbs_server_s* S, const Job& j, int status, const char* msg) {
  cbs_result res{};
  res.id = j.id;
  res.t_submit = j.t_submit;
  res.t_admit = res.t_done = now_s();
  res.status = status;
  std::snprintf(res.error, sizeof(res.error), "%s", msg);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(res);
    S->n_queued -= 1;
  }
  S->cv_done.notify_all();
}

// Admit queued requests in arrival order while the limits allow: into a free seat of a batch
// of the same shape, else into a new batch with as many seats (up to the limit on requests
// in flight) as the memory budget leaves room for.  A request that does not fit yet lets
// later ones pass, kMaxPassed times at most; after that admission waits for it.  Returns
// whether anything was admitted.
bool admit(cbs_server_s* S) {
  bool any = false;
  Job* blocked = nullptr;   // the oldest queued request that did not fit in this pass
  const int max_seats = std::max(1, std::min<int>(kMaxMembers, S->d.max_active));
  for (auto it = S->queue.begin(); it != S->queue.end();) {
    if (blocked && blocked->passed >= kMaxPassed) break;
    long long active;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      active = S->n_active;
    }
    if (active >= S->d.max_active) break;
    const ShapeKey k = key_of(it->r);
    Batch* batch = nullptr;
    Seat* seat = nullptr;
    for (Batch* b : S->batches) {
      if (!(b->key == k)) continue;
      for (Seat& s : b->seats)
        if (s.phase == Phase::Idle) {
          seat = &s;
          break;
        }
      if (seat) {
        batch = b;
        break;
      }
    }
    if (!batch) {
      // evict batches without requests (other shapes, or full ones of this shape), least
      // recently used first, until a batch of this shape fits
      auto fits = [&](int n) { return S->bytes_used + batch_bytes(k, n) <= S->budget; };
      while (!fits(1)) {
        Batch* lru = nullptr;
        for (Batch* b : S->batches)
          if (b->busy() == 0 && !b->in_flight && (!lru || b->last_used < lru->last_used)) lru = b;
        if (!lru) break;
        S->batches.remove(lru);
        S->bytes_used -= lru->bytes;
        free_batch(lru);
      }
      if (!fits(1)) {
        bool none_busy = true;
        for (Batch* b : S->batches) none_busy = none_busy && b->busy() == 0;
        if (none_busy) {   // can never fit: fail it rather than wait forever
          char msg[160];
          std::snprintf(msg, sizeof(msg), "request needs %zu bytes, over the server's budget of %zu",
                        batch_bytes(k, 1), S->budget);
          reject(S, *it, CBS_ERR_OOM, msg);
          it = S->queue.erase(it);
          any = true;
          continue;
        }
        if (!blocked) blocked = &*it;
        ++it;
        continue;
      }
      int n = max_seats;
      while (n > 1 && !fits(n)) --n;
      const int rc = make_batch(S, k, n, &batch);
      if (rc) {
        reject(S, *it, rc, last_error_message());
        it = S->queue.erase(it);
        any = true;
        continue;
      }
      S->batches.push_back(batch);
      S->bytes_used += batch->bytes;
      seat = &batch->seats[0];
    }
    if (blocked) blocked->passed += 1;
    seat->job = *it;
    seat->res = cbs_result{};
    seat->res.id = it->id;
    seat->res.t_submit = it->t_submit;
    seat->res.t_admit = now_s();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->n_queued -= 1;
      S->n_active += 1;
    }
    it = S->queue.erase(it);
    any = true;
    seat->phase = Phase::Forward;   // taken (start_job sets it up)
    const int rc = start_job(batch, *seat);
    if (rc) finish(S, batch, *seat, rc);
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
    for (Batch* b : S->batches)
      if (b->busy() > 0 || b->in_flight) progressed = advance(S, b) || progressed;
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  for (Batch* b : S->batches) free_batch(b);
  S->batches.clear();
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

int cbs_server_sharing(cbs_server_t S, long long* launches, long long* request_iterations, int* max_members) {
  if (!S) return fail(CBS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (launches) *launches = S->n_launches;
  if (request_iterations) *request_iterations = S->n_member_iters;
  if (max_members) *max_members = S->max_members;
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
