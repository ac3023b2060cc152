// api.cu -- host side of the C ABI declared in include/cbs.h: plans, the iteration loop with
// its residual checks, the adjoint and gradient calls.
//
// One CBS iteration (refs. [25], [26] of arXiv 2506.15411) is these kernel passes on the
// plan's stream:
//   1. x pass     W = FFT_x(V E + S)
//   2. y pass     W = FFT_y(W)
//   3. z pass     W = IFFT_z(G(p) FFT_z(W)) / N
//   4. y pass     W = IFFT_y(W)
//   5. x pass     W = IFFT_x(W); delta = gamma (E - W); E -= delta; sum |delta|^2 (FP64)
// where pass 5 of one iteration and pass 1 of the next run as one kernel on each x tile, so a
// series launches pass 1 once and then four kernels per iteration.
// Every `check_every` iterations the host reads the FP64 residual sums and decides whether
// to stop; a full block of iterations is replayed from a CUDA graph.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cbs.h"
#include "absorber.h"
#include "axis_plan.h"
#include "plan.h"
#include "tma.cuh"

namespace cbs {
cudaError_t xpass_set_smem_limit(int bytes);
cudaError_t yzpass_set_smem_limit(int bytes);
}  // namespace cbs

using namespace cbs;

namespace {

thread_local std::string g_err;

constexpr double kPiD = 3.14159265358979323846;
#ifndef CBS_MAX_YZ_OCC
#define CBS_MAX_YZ_OCC 2
#endif
#ifndef CBS_MIN_OCC2_TX
#define CBS_MIN_OCC2_TX 8
#endif
#ifndef CBS_YZ_MAX_BUF
#define CBS_YZ_MAX_BUF 4
#endif
#ifndef CBS_X_SETS
#define CBS_X_SETS 3
#endif
#ifndef CBS_X_MIN_ROWS
#define CBS_X_MIN_ROWS 2
#endif
constexpr int kMaxYZOcc = CBS_MAX_YZ_OCC;    // a build with 1 keeps every y/z kernel at one block per SM
constexpr int kMinOcc2Tx = CBS_MIN_OCC2_TX;  // narrowest tile worth two blocks per SM
constexpr int kYZMaxBuf = CBS_YZ_MAX_BUF;    // most tile buffers of a y or z block
#ifndef CBS_Z_THREADS
#define CBS_Z_THREADS 512
#endif
constexpr int kZThreadsPlan = CBS_Z_THREADS;  // threads of a z block (as the kernel is built)
#ifndef CBS_YBLOCK
#define CBS_YBLOCK 128
#endif
constexpr int kYBlock = CBS_YBLOCK;          // target rows of a y block of the plan's arrays
constexpr int kXSets = CBS_X_SETS;           // most buffer sets of an x block ...
constexpr int kXMinRows = CBS_X_MIN_ROWS;    // ... while its tiles keep at least this many rows
#ifndef CBS_X_OCC
#define CBS_X_OCC 1
#endif
#ifndef CBS_Z_OCC
#define CBS_Z_OCC 1
#endif
#ifndef CBS_Z_GROUPS
#define CBS_Z_GROUPS 2
#endif
#ifndef CBS_X_GROUPS
#define CBS_X_GROUPS 2
#endif
constexpr int kXGroups = CBS_X_GROUPS;       // warp groups of the fused x block
constexpr int kXOcc = CBS_X_OCC;             // x blocks per SM (the kernels' launch bounds)
constexpr int kZOcc = CBS_Z_OCC;             // z blocks per SM
constexpr int kZGroups = CBS_Z_GROUPS;       // warp groups of a z block
constexpr int kMaxN = 1024;

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 5D map of the workspace W in its y-blocked layout, viewed as [3 seats][nyb][nz][yblk][nx]
// complex64 (8-byte elements) with row pitch nxp; box = {bx, by, bz, 1, 1} over (x, y in
// block, z).  Elements beyond nx or nz read as zero and are not written.
bool encode_w_map(CUtensorMap* tm, float2* W, int nx, int ny, int nz, int nxp, int yblk, int seats, int bx, int by,
                  int bz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[5] = {(cuuint64_t)nx, (cuuint64_t)yblk, (cuuint64_t)nz, (cuuint64_t)(ny / yblk),
                              (cuuint64_t)3 * seats};
  const cuuint64_t row = (cuuint64_t)nxp * sizeof(float2);
  const cuuint64_t strides[4] = {row, row * yblk, row * yblk * nz, row * ny * nz};
  const cuuint32_t box[5] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, W, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}




}  // namespace

namespace cbs {
// The calling thread's last error message.
const char* last_error_message() { return g_err.c_str(); }
// Message for cbs_last_error from other translation units.
const char* set_last_error(const char* msg) {
  g_err = msg;
  return g_err.c_str();
}
}  // namespace cbs


namespace cbs {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void drop_graphs(cbs_plan_s* p) {
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
}

int sync_in(cbs_plan_s* p) {
  CK(cudaSetDevice(p->device));
  if (p->own_stream) {
    CK(cudaEventRecord(p->ev, p->user_stream));
    CK(cudaStreamWaitEvent(p->stream, p->ev, 0));
  }
  return CBS_OK;
}

// The four launches of one iteration after the series' first (which k_xpass_fwd starts):
// y, z + Green, inverse y, then the x pass that finishes this iteration and forms the next
// one's W.  With ev != null, events ev[0..4] bracket them.
int launch_iteration(const cbs_plan_s* p, const IterArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  if (ev) CK(cudaEventRecord(ev[0], s));
  CK(launch_ypass(p->tmy, a, false, s));
  if (ev) CK(cudaEventRecord(ev[1], s));
  CK(launch_zpass_green(p->tmz, a, s));
  if (ev) CK(cudaEventRecord(ev[2], s));
  CK(launch_ypass(p->tmy, a, true, s));
  if (ev) CK(cudaEventRecord(ev[3], s));
  CK(launch_xpass_inv_fwd(a, s));
  if (ev) CK(cudaEventRecord(ev[4], s));
  return CBS_OK;
}

// Iterations k0 .. k1-1 of a block (residual slots k0 .. k1-1); with profiling on, the
// block's last iteration (slot m-1) is bracketed by the timing events.
int launch_range(cbs_plan_s* p, const IterArgs& a0, int k0, int k1, int m) {
  IterArgs a = a0;
  for (int k = k0; k < k1; ++k) {
    a.slot = k;
    int rc = launch_iteration(p, a, p->stream, (p->profiling && k == m - 1) ? p->pev : nullptr);
    if (rc) return rc;
  }
  return CBS_OK;
}

// After a block has completed: add its timed iteration to the per-pass totals.
int collect_pass_times(cbs_plan_s* p) {
  if (!p->profiling) return CBS_OK;
  for (int i = 0; i < 4; ++i) {   // passes 1..4; pass 0 (the first forward x) is not timed
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->pev[i], p->pev[i + 1]));
    p->pass_ms[i + 1] += ms;
    p->pass_n[i + 1] += 1;
  }
  return CBS_OK;
}

// Run iterations 0 .. n-1 of a block from a cached graph (captured on first use; event
// records are kept out of graphs because events recorded by graph nodes cannot be timed).
int graph_block(cbs_plan_s* p, const IterArgs& a, int n, bool& used) {
  used = false;
  cudaGraphExec_t exec = nullptr;
  for (auto& g : p->graphs)
    if (g.E == a.E && g.iters == n) exec = g.exec;
  if (!exec) {
    if (p->graphs.size() >= 8) drop_graphs(p);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_range(p, a, 0, n, n + 1);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->stream, &captured);
    if (rc) {
      if (captured) cudaGraphDestroy(captured);
      return rc;
    }
    if (e != cudaSuccess) return fail(CBS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    g = captured;
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CBS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    p->graphs.push_back(GraphEntry{a.E, n, ex});
    exec = ex;
  }
  CK(cudaGraphLaunch(exec, p->stream));
  used = true;
  return CBS_OK;
}

// Source in the kernels' scaled units (k^2 quantities times pitch^2).
int make_source(cbs_plan_s* p, const cbs_source* src, SourceArgs& s) {
  s = SourceArgs{};
  s.kind = src->kind;
  const double h = p->pitch;
  if (src->kind == CBS_SRC_PLANE_WAVE) {
    s.zp = src->z_plane < 0 ? p->d.pad_lo[2] : src->z_plane;
    if (s.zp >= p->d.nz) return fail(CBS_ERR_ARG, "z_plane %d outside the grid", s.zp);
    // S = pol * (-2 i k_b / pitch); scaled by pitch^2: pol * (-2 i k_b pitch)
    const double kb = p->kvac * p->d.n_bg * h;
    for (int c = 0; c < 3; ++c) {
      const double re = src->pol[c][0], im = src->pol[c][1];
      s.amp[c] = make_float2((float)(2.0 * kb * im), (float)(-2.0 * kb * re));
    }
  } else if (src->kind == CBS_SRC_POINT) {
    const int* r = src->r0;
    if (r[0] < 0 || r[0] >= p->d.nx || r[1] < 0 || r[1] >= p->d.ny || r[2] < 0 || r[2] >= p->d.nz)
      return fail(CBS_ERR_ARG, "point source (%d,%d,%d) outside the grid", r[0], r[1], r[2]);
    s.px = r[0];
    s.py = r[1];
    s.pz = r[2];
    for (int c = 0; c < 3; ++c)
      s.amp[c] = make_float2((float)(src->pol[c][0] * h * h), (float)(src->pol[c][1] * h * h));
  } else if (src->kind == CBS_SRC_USER) {
    if (!src->user_src_dev) return fail(CBS_ERR_ARG, "user source pointer is NULL");
    s.user = static_cast<const float2*>(src->user_src_dev);
    s.user_scale = (float)(h * h);
  } else {
    return fail(CBS_ERR_ARG, "unknown source kind %d", src->kind);
  }
  return CBS_OK;
}


// Copy a field between the caller's dense layout [3][nz][ny][nx] and the y-blocked iterate of
// seat `seat` (the row padding is never written here: it stays zero).
cudaError_t field_copy(const cbs_plan_s* p, int seat, float2* dense, bool to_dense, cudaStream_t s) {
  const IterArgs& a = p->base;
  float2* Ei = p->Ei + (size_t)seat * 3 * a.Nw;
  return to_dense ? launch_field_layout(Ei, dense, true, a.nx, a.ny, a.nz, a.nxp, a.yblk, s)
                  : launch_field_layout(dense, Ei, false, a.nx, a.ny, a.nz, a.nxp, a.yblk, s);
}

// Enqueue the next block of iterations, the copy of its residual sums and of the error flag,
// and the event the host waits on.
int series_enqueue_block(cbs_plan_s* p, SeriesRun& R) {
  R.m = std::min(p->d.check_every, p->d.max_iter - R.it);
  R.blk_range = nvtxRangeStartA("cbs: block of iterations");
  // full blocks replay a graph; with profiling the last iteration runs outside it
  const int ng = (R.m == p->d.check_every) ? (p->profiling ? R.m - 1 : R.m) : 0;
  bool used = false;
  int rc = CBS_OK;
  if (ng > 1) rc = graph_block(p, R.a, ng, used);
  if (!rc) rc = launch_range(p, R.a, used ? ng : 0, R.m, R.m);
  if (rc) return rc;
  CK(cudaMemcpyAsync(p->hist_host, p->hist, R.m * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(p->err_host, p->err_dev, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaEventRecord(p->blk_ev, p->stream));
  R.iterating = true;
  return CBS_OK;
}

// The stopping rules on a block's residual sums (one run; shared with the request server).
bool series_absorb_residuals(const cbs_plan_s* p, SeriesRun& R, const double* h) {
  for (int k = 0; k < R.m; ++k) {
    ++R.it;
    const double r = std::sqrt(h[k]);
    if (R.r0 < 0) R.r0 = r;
    R.rel = R.r0 > 0 ? r / R.r0 : 0.0;
    if (!std::isfinite(r) || R.rel > 1e4) {
      R.rc = fail(CBS_ERR_DIVERGED, "series diverged at iteration %d (relative residual %g)", R.it, R.rel);
      return true;
    }
    if (R.rel < 0.99 * R.best) {
      R.best = R.rel;
      R.best_it = R.it;
    }
  }
  // converged when the residual at the check (the block's last iteration) is within tol; a
  // dip below tol earlier in the block does not count (the residual is not monotone)
  const bool done = p->d.tol > 0 && R.rel <= p->d.tol;
  if (!done && p->time_limit_s > 0 && R.it < p->d.max_iter) {
    const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - R.t0).count();
    if (t >= p->time_limit_s) {
      R.rc = fail(CBS_ERR_TIME_LIMIT, "wall-clock limit %g s reached after %d iterations (relative residual %g)",
                  p->time_limit_s, R.it, R.rel);
      return true;
    }
  }
  // stagnation: the residual has sat at its rounding floor for a long stretch
  if (!done && p->d.tol > 0 && R.it - R.best_it >= std::max(1000, R.it / 4)) {
    R.rc = fail(CBS_ERR_STAGNATED, "residual stagnated at %g (best %g) after %d iterations, above tol %g", R.rel,
                R.best, R.it, p->d.tol);
    return true;
  }
  return done || R.it >= p->d.max_iter;
}

// Host side of a completed block: error flag, pass times, residuals, stopping rules.
// Sets R.rc on an error and returns whether iterating is over.
bool series_absorb_block(cbs_plan_s* p, SeriesRun& R) {
  R.iterating = false;
  nvtxRangeEnd(R.blk_range);
  R.blk_range = 0;
  if (*p->err_host) {
    R.rc = fail(CBS_ERR_CUDA, "a tensor-copy wait timed out in an FFT pass (device error %d)", *p->err_host);
    return true;
  }
  R.rc = collect_pass_times(p);
  if (R.rc) return true;
  return series_absorb_residuals(p, R, p->hist_host);
}

// Copy the iterate back into the caller's field (also after an error: E then holds the last
// iterate), with blk_ev marking its end.
void series_enqueue_copy_out(cbs_plan_s* p, SeriesRun& R) {
  cudaError_t e = field_copy(p, 0, R.E, true, p->stream);
  if (e == cudaSuccess) e = cudaEventRecord(p->blk_ev, p->stream);
  if (e != cudaSuccess) {
    if (R.rc == CBS_OK) R.rc = fail(CBS_ERR_CUDA, "field copy-out: %s", cudaGetErrorString(e));
    R.finished = true;
    return;
  }
  R.copying = true;
}

// Start a run: zero the iterate (and copy in the warm start), enqueue the first block.
// warm: 0 = start from E = 0; 1 = start from E, residuals relative to this run's first;
// 2 = start from E, residuals relative to the first residual of a start from 0 (one extra
// iteration from zero computes it, so a warm start converges in fewer iterations; that
// iteration is waited for here).  On an error before the first block R.finished is set.
void series_begin(cbs_plan_s* p, float2* E, const SourceArgs& src, int warm, SeriesRun& R) {
  R = SeriesRun{};
  R.t0 = std::chrono::steady_clock::now();
  R.E = E;
  if (!p->have_eps) {
    R.rc = fail(CBS_ERR_STATE, "cbs_set_permittivity has not been called");
    R.finished = true;
    return;
  }
  R.a = p->base;
  R.a.E = p->Ei;   // iterate on the plan's padded copy; the caller's E is read and written once
  R.a.nmem = 1;    // the plan's own solves use seat 0 and member 0
  R.a.mem = p->mem_dev;
  Member& m = p->mem_host[0];   // (the previous solve's copy of it has completed)
  m = Member{};
  m.src = src;
  m.inv_eps = (float)(1.0 / p->eps_s);
  m.kt2 = make_float2((float)p->k0sq_s, (float)p->eps_s);
  m.seat = 0;
  // every run starts from a clean error flag and residual counter: a run that a timed-out
  // tensor-copy wait ended left both behind, and everything else it touched (W, the
  // iterate, the partial sums) is recomputed from the plan's inputs below
  cudaError_t e = cudaMemcpyAsync(p->mem_dev, p->mem_host, sizeof(Member), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->Ei, 0, 3 * R.a.Nw * sizeof(float2), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->counter, 0, sizeof(unsigned), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->err_dev, 0, sizeof(int), p->stream);
  if (e != cudaSuccess) {
    R.rc = fail(CBS_ERR_CUDA, "field set-up: %s", cudaGetErrorString(e));
    R.finished = true;
    return;
  }
  if (warm == 2) {
    IterArgs a1 = R.a;
    a1.slot = 0;
    int rc = launch_xpass_fwd(a1, p->stream) == cudaSuccess ? CBS_OK : fail(CBS_ERR_CUDA, "x pass launch failed");
    if (!rc) rc = launch_iteration(p, a1, p->stream, nullptr);
    if (!rc) {
      e = cudaMemcpyAsync(p->hist_host, p->hist, sizeof(double), cudaMemcpyDeviceToHost, p->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(p->err_host, p->err_dev, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
      if (e != cudaSuccess)
        rc = fail(CBS_ERR_CUDA, "reference iteration: %s", cudaGetErrorString(e));
      else if (*p->err_host)
        rc = fail(CBS_ERR_CUDA, "a tensor-copy wait timed out in an FFT pass (device error %d)", *p->err_host);
    }
    if (rc) {
      R.rc = rc;
      R.finished = true;
      return;
    }
    R.r0 = std::sqrt(p->hist_host[0]);
    if (!(R.r0 > 0.0)) R.r0 = -1.0;   // a zero source: fall back to this run's first residual
    e = cudaMemsetAsync(p->Ei, 0, 3 * R.a.Nw * sizeof(float2), p->stream);
  }
  if (warm && e == cudaSuccess)
    e = field_copy(p, 0, E, false, p->stream);
  if (e == cudaSuccess) e = launch_xpass_fwd(R.a, p->stream);   // W of the first iteration
  if (e != cudaSuccess) {
    R.rc = fail(CBS_ERR_CUDA, "field copy-in: %s", cudaGetErrorString(e));
    R.finished = true;
    return;
  }
  R.rc = series_enqueue_block(p, R);
  if (R.rc) series_enqueue_copy_out(p, R);
}

// Advance a run: with wait, block until its current block (or copy-out) is done; without,
// return at once if it is still running.  Returns R.finished.
bool series_advance(cbs_plan_s* p, SeriesRun& R, bool wait) {
  if (R.finished) return true;
  cudaError_t e = wait ? cudaEventSynchronize(p->blk_ev) : cudaEventQuery(p->blk_ev);
  if (e == cudaErrorNotReady) return false;
  if (e != cudaSuccess) {
    if (R.rc == CBS_OK)
      R.rc = fail(CBS_ERR_CUDA, "%s failed: %s", R.copying ? "field copy-out" : "iteration block",
                  cudaGetErrorString(e));
    R.iterating = false;
    if (!R.copying) {
      series_enqueue_copy_out(p, R);
      return R.finished;
    }
    R.copying = false;
    R.finished = true;
    return true;
  }
  if (R.copying) {
    R.copying = false;
    R.finished = true;
    return true;
  }
  if (!series_absorb_block(p, R)) {
    R.rc = series_enqueue_block(p, R);
    if (R.rc == CBS_OK) return false;
  }
  series_enqueue_copy_out(p, R);
  return R.finished;
}

// Outcome of a finished run (NOT_CONVERGED when tol > 0 was not reached without another error).
int series_stats(const cbs_plan_s* p, SeriesRun& R, cbs_stats* S) {
  if (R.rc == CBS_OK && p->d.tol > 0 && !(R.rel <= p->d.tol))
    R.rc = fail(CBS_ERR_NOT_CONVERGED, "relative residual %g > tol %g after %d iterations", R.rel, p->d.tol, R.it);
  if (S) {
    S->iters = R.it;
    S->rel_resid = R.rel;
    S->resid0 = R.r0 < 0 ? 0.0 : R.r0;
    S->status = R.rc;
    S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - R.t0).count();
  }
  return R.rc;
}

int run_series(cbs_plan_s* p, float2* E, const SourceArgs& src, int warm, cbs_stats* st) {
  if (st) *st = cbs_stats{};
  SeriesRun R;
  series_begin(p, E, src, warm, R);
  while (!series_advance(p, R, true)) {
  }
  return series_stats(p, R, st);
}

int adjoint_source(cbs_plan_s* p, const int r0[3], const void* E_dev, SourceArgs& s) {
  if (r0[0] < 0 || r0[0] >= p->d.nx || r0[1] < 0 || r0[1] >= p->d.ny || r0[2] < 0 || r0[2] >= p->d.nz)
    return fail(CBS_ERR_ARG, "r0 (%d,%d,%d) outside the grid", r0[0], r0[1], r0[2]);
  CK(launch_adjoint_amp(static_cast<const float2*>(E_dev), p->N, p->d.nx, p->d.ny, r0[0], r0[1], r0[2],
                        (float)(p->pitch * p->pitch), p->adj_amp, p->stream));
  s = SourceArgs{};
  s.kind = CBS_SRC_POINT;
  s.px = r0[0];
  s.py = r0[1];
  s.pz = r0[2];
  s.amp_dev = p->adj_amp;
  return CBS_OK;
}

// Adjoint series of |E(r0)|^2 (source conj(E(r0)) at r0); warm as for run_series.
int adjoint_run(cbs_plan_s* p, const int r0[3], const void* E_dev, void* Eadj_dev, int warm, cbs_stats* stats) {
  if (stats) *stats = cbs_stats{};
  int rc = (!p || !r0 || !E_dev || !Eadj_dev) ? fail(CBS_ERR_ARG, "NULL argument") : sync_in(p);
  SourceArgs s;
  if (!rc) rc = adjoint_source(p, r0, E_dev, s);
  if (rc) {
    if (stats) stats->status = rc;
    return rc;
  }
  return run_series(p, static_cast<float2*>(Eadj_dev), s, warm, stats);
}

}  // namespace cbs

extern "C" {

const char* cbs_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace cbs {

// Splitting and potential of seat `seat` from a permittivity on the device (synchronous on
// stream s; uses the plan's set-up scratch): k0^2 the mid-range of k^2, epsilon the largest
// |k^2 - k0^2| over the grid (absorbing layers included), V = k^2 - k0^2 - i epsilon in the
// seat's slice.  The scaled k0^2 and epsilon land in seat_k0sq / seat_eps.
int seat_permittivity(cbs_plan_s* p, int seat, const float* eps, cudaStream_t s) {
  const int B = p->red_blocks;
  CK(launch_eps_minmax(eps, p->N, p->pmin, p->pmax, p->pbad, B, s));
  std::vector<float> mn(B), mx(B);
  std::vector<int> bad(B);
  CK(cudaMemcpyAsync(mn.data(), p->pmin, B * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(mx.data(), p->pmax, B * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(bad.data(), p->pbad, B * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double lo = 1e300, hi = -1e300;
  for (int b = 0; b < B; ++b) {
    if (bad[b]) return fail(CBS_ERR_ARG, "permittivity contains a non-finite value");
    lo = std::min(lo, (double)mn[b]);
    hi = std::max(hi, (double)mx[b]);
  }
  const double kv2 = (p->kvac * p->pitch) * (p->kvac * p->pitch);
  const double k0sq = 0.5 * kv2 * (lo + hi);
  CK(launch_k2_maxdev(eps, p->d.nx, p->d.ny, p->d.nz, p->sx, p->sy, p->sz, p->layers.corner_max, kv2, k0sq,
                      p->pdev, B, s));
  std::vector<double> dv(B);
  CK(cudaMemcpyAsync(dv.data(), p->pdev, B * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double epsilon = 0.0;
  for (int b = 0; b < B; ++b) epsilon = std::max(epsilon, dv[b]);
  if (!(epsilon > 0.0) || !std::isfinite(epsilon))
    return fail(CBS_ERR_ARG, "epsilon = %g: a lossless homogeneous grid has no convergent splitting", epsilon);
  CK(launch_build_v(eps, p->d.nx, p->d.ny, p->d.nz, p->base.nxp, p->base.yblk, p->sx, p->sy, p->sz,
                    p->layers.corner_max, kv2, k0sq, epsilon, p->V + (size_t)seat * p->base.Nw, s));
  CK(cudaStreamSynchronize(s));
  p->seat_k0sq[seat] = k0sq;
  p->seat_eps[seat] = epsilon;
  return CBS_OK;
}

// A plan whose arrays hold `seats` requests of the grid side by side (cbs_plan: one).
int plan_create(cbs_plan_s** out, const cbs_plan_desc* desc, int seats) {
  if (!out || !desc) return fail(CBS_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (seats < 1 || seats > kMaxMembers) return fail(CBS_ERR_ARG, "seats %d outside [1, %d]", seats, kMaxMembers);
  const cbs_plan_desc& d = *desc;
  const int dims[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1 || dims[a] > kMaxN) return fail(CBS_ERR_ARG, "axis %d size %d outside [1, %d]", a, dims[a], kMaxN);
    if (d.pad_lo[a] < 0 || d.pad_hi[a] < 0 || 2 * d.pad_lo[a] > dims[a] || 2 * d.pad_hi[a] > dims[a] ||
        d.pad_lo[a] + d.pad_hi[a] >= dims[a])
      return fail(CBS_ERR_ARG, "axis %d pads (%d, %d) do not fit size %d", a, d.pad_lo[a], d.pad_hi[a], dims[a]);
  }
  if (!(d.pitch_m > 0) || !(d.lambda_m > 0) || !(d.n_bg > 0))
    return fail(CBS_ERR_ARG, "pitch, wavelength and n_bg must be positive");
  if (d.max_iter < 1 || d.check_every < 1) return fail(CBS_ERR_ARG, "max_iter and check_every must be >= 1");
  const LayerSpec layers = layer_spec(d.layer_round_trip, d.layer_power, d.layer_corner_max);
  if (!layer_spec_valid(layers))
    return fail(CBS_ERR_ARG, "layer round trip %g, power %g or corner rule %d out of range", d.layer_round_trip,
                d.layer_power, d.layer_corner_max);
  // radices up to 11 where the axis allows (kernels built for them need fewer registers, and
  // the y pass then runs two blocks per SM: 256 = 8 8 4 beat 16 16 by 18 % per iteration on a
  // 256 x 256 x 192 grid), else up to 16 (axes with a factor 13)
  std::vector<int> rad[3];
  for (int a2 = 0; a2 < 3; ++a2)
    if (!factor_radices(dims[a2], 11, rad[a2]) && !factor_radices(dims[a2], 16, rad[a2]))
      return fail(CBS_ERR_ARG, "axis %d size %d is not a product of 2,3,5,7,11,13", a2, dims[a2]);

  cbs_plan_s* p = new cbs_plan_s();
  p->d = d;
  p->seats = seats;
  p->N = (size_t)d.nx * d.ny * d.nz;
  p->pitch = d.pitch_m;
  p->kvac = 2.0 * kPiD / d.lambda_m;
  p->layers = layers;
  p->user_stream = static_cast<cudaStream_t>(d.cuda_stream);
  auto bail = [&](int code) {
    cbs_destroy(p);
    return code;
  };
#define CKP(call)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      int code_ = (e_ == cudaErrorMemoryAllocation) ? CBS_ERR_OOM : CBS_ERR_CUDA;                \
      fail(code_, "%s failed: %s", #call, cudaGetErrorString(e_));                               \
      return bail(code_);                                                                        \
    }                                                                                            \
  } while (0)
  CKP(cudaGetDevice(&p->device));
  if (p->user_stream) {
    p->stream = p->user_stream;   // work (and graph capture) on the caller's stream
  } else {
    CKP(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
    p->own_stream = true;         // the legacy stream cannot be captured
  }
  CKP(cudaEventCreateWithFlags(&p->ev, cudaEventDisableTiming));
  CKP(cudaEventCreateWithFlags(&p->blk_ev, cudaEventDisableTiming));
  CKP(xpass_set_smem_limit(227 * 1024));
  CKP(yzpass_set_smem_limit(227 * 1024));

  IterArgs& a = p->base;
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.N = p->N;
  // launch shapes: persistent tile kernels with rings of tile buffers (the FFTs run in place,
  // so a tile needs no scratch): x tiles of rpb rows, y and z tiles of TX columns by whole
  // tensor-copy boxes
  const size_t kBlockBudget = 220 * 1024, kBlockBudget2 = 110 * 1024;
  const size_t kXBudget = kBlockBudget / kXOcc, kZBudget = kBlockBudget / kZOcc;
  a.nxp = round_up(d.nx, 16);
  a.Nw = (size_t)a.nxp * d.ny * d.nz;
  const int twb[3] = {round_up(d.nx * (int)sizeof(float2), 16), round_up(d.ny * (int)sizeof(float2), 16),
                      round_up(d.nz * (int)sizeof(float2), 16)};
  {
    // x: nset buffer sets of 7 arrays [rpb][nxp] (W and E of 3 components, V); the most sets
    // (up to kXSets) that still hold tiles of at least kXMinRows rows, then the most rows
    const size_t fixed = (size_t)twb[0] + 8 * 5 + 16 + 32 * 8;
    const size_t row7 = (size_t)7 * a.nxp * sizeof(float2);
    a.xgroups = kXGroups;
    a.nset_x = kXGroups + 1;   // a tile in hand per warp group and one more in flight
    for (int ns = std::max(kXSets, kXGroups + 1); ns >= kXGroups + 1; --ns)
      if ((kXBudget - fixed) / (ns * row7) >= (size_t)kXMinRows || ns == kXGroups + 1) {
        a.nset_x = ns;
        break;
      }
    a.rpb = (int)std::max<size_t>(1, std::min<size_t>(64, (kXBudget - fixed) / (a.nset_x * row7)));
    const size_t row4 = (size_t)4 * a.rpb * a.nxp * sizeof(float2);
    a.nset_xf = (int)std::max<size_t>(2, std::min<size_t>(4, (kXBudget - fixed) / row4));
  }
  // y and z tiles: TX columns x whole axis, brought in by boxes of B rows.  B is a divisor of
  // the axis in [16, 64] when one keeps every box's shared-memory offset (B TX 8 bytes) a
  // multiple of 128 bytes -- then no padded rows are held -- else 64 (rows past the axis
  // read as zero and are not stored); a short axis is one box.
  auto box_rows = [](int n, int tx) {
    if (n <= kBoxRows) return round_up(n, 4);
    for (int b = kBoxRows; b >= 16; --b)
      if (n % b == 0 && (b * tx) % 16 == 0) return b;
    return kBoxRows;
  };
  const int pqbz = round_up(d.nz * (int)sizeof(float2), 16);
  // y blocks of the arrays: the largest divisor of ny up to kYBlock rows whose tensor-copy box
  // keeps the y tile's shared-memory offsets on 128-byte boundaries (yblk TX 8 bytes), else
  // up to 256 rows (the box limit); 0 if none (then that tile width is not used)
  auto yblock_for = [&](int tx) {
    for (int lim : {kYBlock, 256})
      for (int b = std::min(lim, d.ny); b >= 1; --b)
        if (d.ny % b == 0 && (b * tx) % 16 == 0) return b;
    return 0;
  };
  // a y tile holds exactly ny rows (nyb boxes of yblk rows)
  auto ysmem = [&](int tx, int nb) {
    if (!yblock_for(tx)) return (size_t)1 << 40;
    return (size_t)nb * d.ny * tx * sizeof(float2) + twb[1] + 8 * nb + 8;
  };
  auto zsmem = [&](int tx, int nb) {
    return (size_t)3 * nb * round_up(d.nz, box_rows(d.nz, tx)) * tx * sizeof(float2) + twb[2] + pqbz + 8 * (nb + 1) +
           8;
  };
  auto max_radix = [](const std::vector<int>& r) { return *std::max_element(r.begin(), r.end()); };
  // Two blocks per SM (half the shared memory each) when the axis needs no radix above 11,
  // else one: the widest tile, then the most buffers (2 .. kYZMaxBuf), that fits.
  auto pick = [&](auto smem, int maxr, int& tx, int& nb, int& occ) {
    for (occ = (maxr <= 11 && kMaxYZOcc >= 2) ? 2 : 1; occ >= 1; --occ) {
      const size_t budget = occ == 2 ? kBlockBudget2 : kBlockBudget;
      for (tx = 16; tx >= (occ == 2 ? kMinOcc2Tx : 4); tx /= 2)
        for (nb = kYZMaxBuf; nb >= 2; --nb)
          if (smem(tx, nb) <= budget) return true;
    }
    return false;
  };
  // z: every warp group needs a tile in hand and one more in flight; two groups while the
  // tiles allow, else one
  auto pick_z = [&](int& tx, int& nb, int& groups) {
    for (groups = kZGroups; groups >= 1; --groups)
      for (tx = 16; tx >= 4; tx /= 2)
        for (nb = kYZMaxBuf; nb >= groups + 1; --nb)
          if (zsmem(tx, nb) <= kZBudget) return true;
    return false;
  };
  const bool fy = pick(ysmem, max_radix(rad[1]), a.tx_y, a.nbuf_y, a.occ_y);
  const bool fz = pick_z(a.tx_z, a.nbuf_z, a.zgroups);
  a.occ_z = kZOcc;
  if (!fy || !fz) {
    fail(CBS_ERR_ARG, "axis too long for the shared-memory tiles");
    return bail(CBS_ERR_ARG);
  }
  a.yblk = yblock_for(a.tx_y);
  a.nyb = d.ny / a.yblk;
  a.yb = a.yblk;
  a.nyr = d.ny;
  a.zb = box_rows(d.nz, a.tx_z);
  a.nzr = round_up(d.nz, a.zb);
  a.maxr_x = max_radix(rad[0]);
  a.maxr_z = max_radix(rad[2]);
  a.twbx = twb[0];
  a.twby = twb[1];
  a.twbz = twb[2];
  a.pqbz = pqbz;

  const size_t N = p->N;
  const size_t S = (size_t)seats;
  CKP(cudaMalloc(&p->V, S * a.Nw * sizeof(float2)));
  CKP(cudaMemset(p->V, 0, S * a.Nw * sizeof(float2)));        // row padding stays zero
  CKP(cudaMalloc(&p->Ei, S * 3 * a.Nw * sizeof(float2)));
  CKP(cudaMalloc(&p->W, S * 3 * a.Nw * sizeof(float2)));
  CKP(cudaMemset(p->W, 0, S * 3 * a.Nw * sizeof(float2)));   // row padding stays zero
  CKP(cudaMalloc(&p->err_dev, sizeof(int)));
  CKP(cudaMemset(p->err_dev, 0, sizeof(int)));
  CKP(cudaMallocHost(&p->err_host, sizeof(int)));
  if (!encode_w_map(&p->tmy, p->W, d.nx, d.ny, d.nz, a.nxp, a.yblk, seats, a.tx_y, a.yblk, 1) ||
      !encode_w_map(&p->tmz, p->W, d.nx, d.ny, d.nz, a.nxp, a.yblk, seats, a.tx_z, 1, a.zb)) {
    fail(CBS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the workspace");
    return bail(CBS_ERR_CUDA);
  }
  CKP(cudaMalloc(&p->partials, S * xpass_tiles(a) * sizeof(double)));   // >= seats x the x grid
  CKP(cudaMalloc(&p->counter, S * sizeof(unsigned)));
  CKP(cudaMemset(p->counter, 0, S * sizeof(unsigned)));
  CKP(cudaMalloc(&p->hist, S * d.check_every * sizeof(double)));
  CKP(cudaMallocHost(&p->hist_host, S * d.check_every * sizeof(double)));
  CKP(cudaMalloc(&p->mem_dev, members_len(seats, d.check_every) * sizeof(Member)));
  CKP(cudaMallocHost(&p->mem_host, members_len(seats, d.check_every) * sizeof(Member)));
  CKP(cudaMalloc(&p->adj_amp, S * 3 * sizeof(float2)));
  CKP(cudaMalloc(&p->dobj, S * sizeof(double)));
  p->seat_k0sq.assign(seats, 0.0);
  p->seat_eps.assign(seats, 0.0);
  CKP(cudaMalloc(&p->sx, d.nx * sizeof(double)));
  CKP(cudaMalloc(&p->sy, d.ny * sizeof(double)));
  CKP(cudaMalloc(&p->sz, d.nz * sizeof(double)));
  p->red_blocks = 152 * 4;
  CKP(cudaMalloc(&p->pmin, p->red_blocks * sizeof(float)));
  CKP(cudaMalloc(&p->pmax, p->red_blocks * sizeof(float)));
  CKP(cudaMalloc(&p->pbad, p->red_blocks * sizeof(int)));
  CKP(cudaMalloc(&p->pdev, p->red_blocks * sizeof(double)));

  // per-axis FFT tables (axis_plan.h): radix order for the axis' shared-memory layout, stage
  // table, per-stage twiddles (FP64, rounded; padded to n entries so that a fixed n * 8 bytes
  // are copied into the tiles) and the wave numbers of each spectrum position (padded to 16
  // entries); every table starts on a 128-byte boundary
  {
    const AxisLayout lay[3] = {AxisLayout::Rows, AxisLayout::Cols, AxisLayout::ColsZ};
    const int ncol[3] = {0, a.tx_y, a.tx_z};
    std::vector<int4> st_all(3 * 2 * kMaxAxisStages, make_int4(1, 1, 1, 0));
    std::vector<float2> tw_all, pq_all;
    int twoff[3], pqoff[3];
    for (int a2 = 0; a2 < 3; ++a2) {
      const int n = dims[a2];
      p->radix_order[a2] = a2 == 2 ? order_radices_z(rad[a2], n, a.tx_z, kZThreadsPlan / a.zgroups)
                                   : order_radices(rad[a2], n, lay[a2], ncol[a2]);
      std::vector<int4> st;
      std::vector<float2> tw, pq;
      axis_tables(n, p->radix_order[a2], st, tw, pq);
      std::copy(st.begin(), st.end(), st_all.begin() + a2 * 2 * kMaxAxisStages);
      twoff[a2] = (int)tw_all.size();
      tw.resize(round_up(n, 16), make_float2(0.f, 0.f));
      tw_all.insert(tw_all.end(), tw.begin(), tw.end());
      pqoff[a2] = (int)pq_all.size();
      pq.resize(round_up(n, 16), make_float2(0.f, 0.f));
      pq_all.insert(pq_all.end(), pq.begin(), pq.end());
      AxisIP& ap = a2 == 0 ? a.ax : (a2 == 1 ? a.ay : a.az);
      ap.n = n;
      ap.ns = (int)p->radix_order[a2].size();
    }
    CKP(cudaMalloc(&p->tw, tw_all.size() * sizeof(float2)));
    CKP(cudaMemcpy(p->tw, tw_all.data(), tw_all.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CKP(cudaMalloc(&p->pq, pq_all.size() * sizeof(float2)));
    CKP(cudaMemcpy(p->pq, pq_all.data(), pq_all.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CKP(cudaMalloc(&p->stages, st_all.size() * sizeof(int4)));
    CKP(cudaMemcpy(p->stages, st_all.data(), st_all.size() * sizeof(int4), cudaMemcpyHostToDevice));
    a.twx = p->tw + twoff[0];
    a.twy = p->tw + twoff[1];
    a.twz = p->tw + twoff[2];
    a.pqx = p->pq + pqoff[0];
    a.pqy = p->pq + pqoff[1];
    a.pqz = p->pq + pqoff[2];
    a.ax.st = p->stages;
    a.ay.st = p->stages + 2 * kMaxAxisStages;
    a.az.st = p->stages + 4 * kMaxAxisStages;
  }

  // persistent grid sizes (occupancy of each tile kernel at its shared-memory size)
  {
    int sms = 0;
    CKP(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    p->sms = sms;
    CKP(x_grid_size(a, sms));
    CKP(yz_grid_sizes(a, sms));
  }

  // every address the tile kernels bulk-copy from or to must be 16-byte aligned, every size
  // a multiple of 16 (checked here once: these pointers and sizes are fixed for the plan)
  {
    auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    const bool ok = a16(a.twx) && a16(a.twy) && a16(a.twz) && a16(a.pqz) && a16(p->Ei) && a16(p->V) && a16(p->W) &&
                    (a.twbx % 16 == 0) && (a.twby % 16 == 0) && (a.twbz % 16 == 0) &&
                    ((size_t)a.nxp * sizeof(float2)) % 16 == 0 && (a.Nw * sizeof(float2)) % 16 == 0;
    if (!ok) {
      fail(CBS_ERR_CUDA, "internal: a bulk-copy address or size is not 16-byte aligned");
      return bail(CBS_ERR_CUDA);
    }
  }

  // absorbing layers (absorber.h): sigma along each axis; the set-up kernels combine the three
  for (int a2 = 0; a2 < 3; ++a2) {
    const int n = dims[a2], lo = d.pad_lo[a2], hi = d.pad_hi[a2];
    const double slo = layer_sigma_max(p->layers, d.n_bg, p->kvac, lo, d.pitch_m);
    const double shi = layer_sigma_max(p->layers, d.n_bg, p->kvac, hi, d.pitch_m);
    std::vector<double> s(n, 0.0);
    for (int i = 0; i < n; ++i) s[i] = layer_axis_sigma(i, n, lo, hi, slo, shi, p->layers.power);
    double* dst = a2 == 0 ? p->sx : (a2 == 1 ? p->sy : p->sz);
    CKP(cudaMemcpy(dst, s.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  }

  a.W = p->W;
  a.V = p->V;
  a.E = p->Ei;
  a.seats = seats;
  a.nmem = 1;
  a.mem = p->mem_dev;
  a.err = p->err_dev;
  a.partials = p->partials;
  a.counter = p->counter;
  a.hist = p->hist;
  a.hist_cap = d.check_every;
  a.invN = (float)(1.0 / (double)N);
#undef CKP
  *out = p;
  return CBS_OK;
}

}  // namespace cbs

extern "C" {

int cbs_plan(cbs_plan_t* out, const cbs_plan_desc* desc) {
  g_err.clear();
  return plan_create(out, desc, 1);
}

void cbs_destroy(cbs_plan_t p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  drop_graphs(p);
  void* devs[] = {p->V, p->W, p->Ei, p->tw, p->pq, p->stages, p->partials, p->counter, p->hist, p->mem_dev,
                  p->adj_amp, p->dobj,
                  p->sx, p->sy, p->sz, p->pmin, p->pmax, p->pbad, p->pdev, p->eps_dev,
                  p->Ef, p->Ea, p->grad_dev, p->err_dev};
  for (void* q : devs)
    if (q) cudaFree(q);
  if (p->hist_host) cudaFreeHost(p->hist_host);
  if (p->mem_host) cudaFreeHost(p->mem_host);
  if (p->err_host) cudaFreeHost(p->err_host);
  if (p->ev) cudaEventDestroy(p->ev);
  if (p->blk_ev) cudaEventDestroy(p->blk_ev);
  for (cudaEvent_t e : p->pev)
    if (e) cudaEventDestroy(e);
  if (p->stream && p->own_stream) cudaStreamDestroy(p->stream);
  delete p;
}

int cbs_set_profiling(cbs_plan_t p, int on) {
  g_err.clear();
  if (!p) return fail(CBS_ERR_ARG, "NULL plan");
  CK(cudaSetDevice(p->device));
  if (on && !p->pev[0])
    for (cudaEvent_t& e : p->pev) CK(cudaEventCreate(&e));
  if ((on != 0) != p->profiling) {
    CK(cudaStreamSynchronize(p->stream));
    drop_graphs(p);
  }
  p->profiling = on != 0;
  return CBS_OK;
}

int cbs_pass_times(cbs_plan_t p, double ms_total[5], long long launches[5], int reset) {
  g_err.clear();
  if (!p) return fail(CBS_ERR_ARG, "NULL plan");
  for (int i = 0; i < 5; ++i) {
    if (ms_total) ms_total[i] = p->pass_ms[i];
    if (launches) launches[i] = p->pass_n[i];
    if (reset) {
      p->pass_ms[i] = 0.0;
      p->pass_n[i] = 0;
    }
  }
  return CBS_OK;
}

int cbs_set_solver(cbs_plan_t p, double tol, int max_iter, int check_every) {
  g_err.clear();
  if (!p) return fail(CBS_ERR_ARG, "NULL plan");
  if (max_iter < 1 || check_every < 1) return fail(CBS_ERR_ARG, "max_iter and check_every must be >= 1");
  if (check_every != p->d.check_every) {
    CK(cudaSetDevice(p->device));
    CK(cudaStreamSynchronize(p->stream));
    drop_graphs(p);
    double* h = nullptr;
    double* hh = nullptr;
    Member* md = nullptr;
    Member* mh = nullptr;
    const size_t n = (size_t)p->seats * check_every, nm = members_len(p->seats, check_every);
    cudaError_t e = cudaMalloc(&h, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&hh, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&md, nm * sizeof(Member));
    if (e == cudaSuccess) e = cudaMallocHost(&mh, nm * sizeof(Member));
    if (e != cudaSuccess) {
      if (h) cudaFree(h);
      if (hh) cudaFreeHost(hh);
      if (md) cudaFree(md);
      return fail(CBS_ERR_CUDA, "solver buffers: %s", cudaGetErrorString(e));
    }
    cudaFree(p->hist);
    cudaFreeHost(p->hist_host);
    cudaFree(p->mem_dev);
    cudaFreeHost(p->mem_host);
    p->hist = h;
    p->hist_host = hh;
    p->mem_dev = md;
    p->mem_host = mh;
    p->base.hist = h;
    p->base.hist_cap = check_every;
    p->base.mem = md;
  }
  p->d.tol = tol;
  p->d.max_iter = max_iter;
  p->d.check_every = check_every;
  return CBS_OK;
}

int cbs_set_time_limit(cbs_plan_t p, double seconds) {
  g_err.clear();
  if (!p) return fail(CBS_ERR_ARG, "NULL plan");
  if (!(seconds >= 0) || !std::isfinite(seconds)) return fail(CBS_ERR_ARG, "time limit %g s", seconds);
  p->time_limit_s = seconds;
  return CBS_OK;
}

int cbs_set_permittivity(cbs_plan_t p, const float* eps) {
  NvtxRange nv("cbs_set_permittivity");
  g_err.clear();
  if (!p || !eps) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(p);
  if (!rc) rc = seat_permittivity(p, 0, eps, p->stream);
  if (rc) return rc;
  p->k0sq_s = p->seat_k0sq[0];
  p->eps_s = p->seat_eps[0];
  p->have_eps = true;   // (the splitting reaches the kernels through the member array)
  return CBS_OK;
}

int cbs_get_splitting(cbs_plan_t p, double* k0sq, double* epsilon) {
  g_err.clear();
  if (!p) return fail(CBS_ERR_ARG, "NULL plan");
  if (!p->have_eps) return fail(CBS_ERR_STATE, "cbs_set_permittivity has not been called");
  const double s = 1.0 / (p->pitch * p->pitch);
  if (k0sq) *k0sq = p->k0sq_s * s;
  if (epsilon) *epsilon = p->eps_s * s;
  return CBS_OK;
}

int cbs_forward(cbs_plan_t p, const cbs_source* src, void* E_dev, cbs_stats* stats) {
  NvtxRange nv("cbs_forward");
  g_err.clear();
  if (stats) *stats = cbs_stats{};
  if (!p || !src || !E_dev) {
    if (stats) stats->status = CBS_ERR_ARG;
    return fail(CBS_ERR_ARG, "NULL argument");
  }
  if (src->warm_start < 0 || src->warm_start > 2) {
    if (stats) stats->status = CBS_ERR_ARG;
    return fail(CBS_ERR_ARG, "warm_start %d is not 0, 1 or 2", src->warm_start);
  }
  SourceArgs s;
  int rc = make_source(p, src, s);
  if (!rc) rc = sync_in(p);
  if (rc) {
    if (stats) stats->status = rc;
    return rc;
  }
  return run_series(p, static_cast<float2*>(E_dev), s, src->warm_start, stats);
}

int cbs_adjoint(cbs_plan_t p, const int r0[3], const void* E_dev, void* Eadj_dev, cbs_stats* stats) {
  NvtxRange nv("cbs_adjoint");
  g_err.clear();
  return adjoint_run(p, r0, E_dev, Eadj_dev, 0, stats);
}

int cbs_gradient(cbs_plan_t p, const void* E_dev, const void* Eadj_dev, const int r0[3], float* grad_dev,
                 double* objective) {
  NvtxRange nv("cbs_gradient");
  g_err.clear();
  if (!p || !E_dev || !Eadj_dev || !grad_dev) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(p);
  if (rc) return rc;
  const float coef = (float)(2.0 * p->kvac * p->kvac);
  CK(launch_gradient(static_cast<const float2*>(E_dev), static_cast<const float2*>(Eadj_dev), p->N, coef,
                     grad_dev, p->stream));
  if (r0 && objective) {
    if (r0[0] < 0 || r0[0] >= p->d.nx || r0[1] < 0 || r0[1] >= p->d.ny || r0[2] < 0 || r0[2] >= p->d.nz)
      return fail(CBS_ERR_ARG, "r0 (%d,%d,%d) outside the grid", r0[0], r0[1], r0[2]);
    CK(launch_objective(static_cast<const float2*>(E_dev), p->N, p->d.nx, p->d.ny, r0[0], r0[1], r0[2], p->dobj,
                        p->stream));
    CK(cudaMemcpyAsync(objective, p->dobj, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  }
  CK(cudaStreamSynchronize(p->stream));
  return CBS_OK;
}

int cbs_selftest_wait_timeout(int* device_status) {
  g_err.clear();
  if (!device_status) return fail(CBS_ERR_ARG, "NULL argument");
  *device_status = 0;
  int* err = nullptr;
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_wait_selftest(err, 2000, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(device_status, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  // the context must still take work after the timed-out wait
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (err) cudaFree(err);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail(CBS_ERR_CUDA, "self-test: %s", cudaGetErrorString(e));
  if (*device_status != kErrTmaTimeout)
    return fail(CBS_ERR_CUDA, "self-test: the bounded wait did not report its timeout (status %d)", *device_status);
  return CBS_OK;
}

int cbs_objective(cbs_plan_t p, const void* E_dev, const int r0[3], double* objective) {
  g_err.clear();
  if (!p || !E_dev || !r0 || !objective) return fail(CBS_ERR_ARG, "NULL argument");
  if (r0[0] < 0 || r0[0] >= p->d.nx || r0[1] < 0 || r0[1] >= p->d.ny || r0[2] < 0 || r0[2] >= p->d.nz)
    return fail(CBS_ERR_ARG, "r0 (%d,%d,%d) outside the grid", r0[0], r0[1], r0[2]);
  int rc = sync_in(p);
  if (rc) return rc;
  CK(launch_objective(static_cast<const float2*>(E_dev), p->N, p->d.nx, p->d.ny, r0[0], r0[1], r0[2], p->dobj,
                      p->stream));
  CK(cudaMemcpyAsync(objective, p->dobj, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return CBS_OK;
}

int cbs_design_step_host(cbs_plan_t p, const float* eps_host, const cbs_source* src, const int r0[3],
                         float* grad_host, double* objective, cbs_stats* fwd, cbs_stats* adj) {
  g_err.clear();
  if (!p || !eps_host || !src || !r0 || !grad_host || !objective) return fail(CBS_ERR_ARG, "NULL argument");
  CK(cudaSetDevice(p->device));
  const size_t N = p->N;
  if (!p->eps_dev) {
    CK(cudaMalloc(&p->eps_dev, N * sizeof(float)));
    CK(cudaMalloc(&p->grad_dev, N * sizeof(float)));
    CK(cudaMalloc(&p->Ef, 3 * N * sizeof(float2)));
    CK(cudaMalloc(&p->Ea, 3 * N * sizeof(float2)));
  }
  int rc = sync_in(p);
  if (rc) return rc;
  CK(cudaMemcpyAsync(p->eps_dev, eps_host, N * sizeof(float), cudaMemcpyHostToDevice, p->stream));
  rc = cbs_set_permittivity(p, p->eps_dev);
  if (rc) return rc;
  cbs_source s = *src;
  s.warm_start = 0;
  rc = cbs_forward(p, &s, p->Ef, fwd);
  if (rc) return rc;
  rc = cbs_adjoint(p, r0, p->Ef, p->Ea, adj);
  if (rc) return rc;
  rc = cbs_gradient(p, p->Ef, p->Ea, r0, p->grad_dev, objective);
  if (rc) return rc;
  CK(cudaMemcpyAsync(grad_host, p->grad_dev, N * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return CBS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ inverse design
struct cbs_design_s {
  cbs_plan_s* p = nullptr;
  cbs_design_desc d{};
  int nx = 0, ny = 0;
  double pitch_um = 0;
  int R = 0;                          // Gaussian half-width (0: no smoothing)
  float* w = nullptr;                 // 2R+1 weights
  float *t1 = nullptr, *t2 = nullptr, *heff = nullptr, *gh = nullptr, *m = nullptr, *v = nullptr;
  float *eps = nullptr, *grad = nullptr;
  int t = 0;                          // Adam steps taken
};

namespace {

int design_effective(cbs_design_s* D, const float* h, float* out) {
  cbs_plan_s* p = D->p;
  const size_t mb = (size_t)D->nx * D->ny * sizeof(float);
  const float* src = h;
  if (D->d.mirror) {
    CK(launch_mirror(h, D->t1, D->nx, D->ny, p->stream));
    src = D->t1;
  }
  if (D->R > 0) {
    CK(launch_filter(src, D->t2, D->nx, D->ny, D->w, D->R, 0, p->stream));
    CK(launch_filter(D->t2, out, D->nx, D->ny, D->w, D->R, 1, p->stream));
  } else if (src != out) {
    CK(cudaMemcpyAsync(out, src, mb, cudaMemcpyDeviceToDevice, p->stream));
  }
  return CBS_OK;
}

int design_permittivity(cbs_design_s* D, const float* heff, float* eps) {
  cbs_plan_s* p = D->p;
  const double eb = p->d.n_bg * p->d.n_bg, el = D->d.n_lens * D->d.n_lens;
  CK(launch_height_to_eps(heff, eps, D->nx, D->ny, p->d.nz, D->d.z_base, (float)(1.0 / D->pitch_um), (float)eb,
                          (float)(el - eb), p->sms, p->stream));
  return CBS_OK;
}

int design_height_gradient(cbs_design_s* D, const float* heff, const float* grad_eps, float* out) {
  cbs_plan_s* p = D->p;
  const double eb = p->d.n_bg * p->d.n_bg, el = D->d.n_lens * D->d.n_lens;
  const size_t mb = (size_t)D->nx * D->ny * sizeof(float);
  CK(launch_surface_grad(grad_eps, heff, D->t1, D->nx, D->ny, p->d.nz, D->d.z_base, (float)(1.0 / D->pitch_um),
                         (float)((el - eb) / D->pitch_um), p->stream));
  if (D->R > 0) {
    CK(launch_filter(D->t1, D->t2, D->nx, D->ny, D->w, D->R, 0, p->stream));
    CK(launch_filter(D->t2, D->t1, D->nx, D->ny, D->w, D->R, 1, p->stream));
  }
  if (D->d.mirror)
    CK(launch_mirror(D->t1, out, D->nx, D->ny, p->stream));
  else
    CK(cudaMemcpyAsync(out, D->t1, mb, cudaMemcpyDeviceToDevice, p->stream));
  return CBS_OK;
}

int design_adam(cbs_design_s* D, float* h, const float* gh) {
  cbs_plan_s* p = D->p;
  D->t += 1;
  const double c1 = 1.0 / (1.0 - std::pow(D->d.beta1, D->t));
  const double c2 = 1.0 / (1.0 - std::pow(D->d.beta2, D->t));
  const double r = 0.5 * D->d.aperture_um;
  CK(launch_adam(h, gh, D->m, D->v, D->nx, D->ny, D->pitch_um, r * r, (float)D->d.alpha, (float)D->d.beta1,
                 (float)D->d.beta2, (float)c1, (float)c2, (float)D->d.adam_eps, (float)D->d.h_max_um, p->stream));
  return CBS_OK;
}

}  // namespace

extern "C" {

int cbs_design_create(cbs_design_t* out, cbs_plan_t p, const cbs_design_desc* desc) {
  g_err.clear();
  if (!out || !p || !desc) return fail(CBS_ERR_ARG, "NULL argument");
  *out = nullptr;
  const cbs_design_desc& d = *desc;
  if (d.z_base < 0 || d.z_base >= p->d.nz) return fail(CBS_ERR_ARG, "z_base %d outside the grid", d.z_base);
  if (!(d.n_lens > 0) || !(d.aperture_um >= 0) || !(d.h_max_um >= 0) || !(d.sigma_um >= 0) || !(d.alpha > 0) ||
      !(d.beta1 >= 0 && d.beta1 < 1) || !(d.beta2 >= 0 && d.beta2 < 1) || !(d.adam_eps > 0))
    return fail(CBS_ERR_ARG, "design parameters out of range");
  auto* D = new cbs_design_s;
  D->p = p;
  D->d = d;
  D->nx = p->d.nx;
  D->ny = p->d.ny;
  D->pitch_um = p->d.pitch_m * 1e6;
  auto bail = [&](int rc) {
    cbs_design_destroy(D);
    return rc;
  };
  if (d.sigma_um > 0) {
    const double s = d.sigma_um / D->pitch_um;
    D->R = (int)std::ceil(4.0 * s);
    if (D->R > 256) {
      fail(CBS_ERR_ARG, "smoothing sigma of %g pixels: the filter half-width ceil(4 sigma) exceeds 256", s);
      return bail(CBS_ERR_ARG);
    }
  }
  const size_t M = (size_t)D->nx * D->ny;
  cudaError_t e = cudaSetDevice(p->device);
  for (float** q : {&D->t1, &D->t2, &D->heff, &D->gh, &D->m, &D->v})
    if (e == cudaSuccess) e = cudaMalloc(q, M * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&D->eps, p->N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&D->grad, p->N * sizeof(float));
  if (e == cudaSuccess && D->R > 0) {
    // w_0 .. w_R of the symmetric kernel exp(-k^2 / 2 s^2), |k| <= R, normalised to sum 1
    std::vector<double> wd(D->R + 1);
    const double s = d.sigma_um / D->pitch_um;
    double sum = 0;
    for (int k = 0; k <= D->R; ++k) {
      wd[k] = std::exp(-(double)k * k / (2.0 * s * s));
      sum += (k == 0 ? 1.0 : 2.0) * wd[k];
    }
    std::vector<float> wf(wd.size());
    for (size_t i = 0; i < wd.size(); ++i) wf[i] = (float)(wd[i] / sum);
    e = cudaMalloc(&D->w, wf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(D->w, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(D->m, 0, M * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(D->v, 0, M * sizeof(float));
  if (e != cudaSuccess) {
    fail(e == cudaErrorMemoryAllocation ? CBS_ERR_OOM : CBS_ERR_CUDA, "design set-up: %s", cudaGetErrorString(e));
    return bail(e == cudaErrorMemoryAllocation ? CBS_ERR_OOM : CBS_ERR_CUDA);
  }
  *out = D;
  return CBS_OK;
}

void cbs_design_destroy(cbs_design_t D) {
  if (!D) return;
  cudaSetDevice(D->p->device);
  if (D->p->stream) cudaStreamSynchronize(D->p->stream);
  for (float* q : {D->w, D->t1, D->t2, D->heff, D->gh, D->m, D->v, D->eps, D->grad})
    if (q) cudaFree(q);
  delete D;
}

int cbs_design_reset(cbs_design_t D) {
  g_err.clear();
  if (!D) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(D->p);
  if (rc) return rc;
  const size_t mb = (size_t)D->nx * D->ny * sizeof(float);
  CK(cudaMemsetAsync(D->m, 0, mb, D->p->stream));
  CK(cudaMemsetAsync(D->v, 0, mb, D->p->stream));
  CK(cudaStreamSynchronize(D->p->stream));
  D->t = 0;
  return CBS_OK;
}

int cbs_design_get_state(cbs_design_t D, float* m, float* v, int* t) {
  g_err.clear();
  if (!D || !m || !v || !t) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(D->p);
  if (rc) return rc;
  const size_t mb = (size_t)D->nx * D->ny * sizeof(float);
  CK(cudaMemcpyAsync(m, D->m, mb, cudaMemcpyDefault, D->p->stream));
  CK(cudaMemcpyAsync(v, D->v, mb, cudaMemcpyDefault, D->p->stream));
  CK(cudaStreamSynchronize(D->p->stream));
  *t = D->t;
  return CBS_OK;
}

int cbs_design_set_state(cbs_design_t D, const float* m, const float* v, int t) {
  g_err.clear();
  if (!D || !m || !v) return fail(CBS_ERR_ARG, "NULL argument");
  if (t < 0) return fail(CBS_ERR_ARG, "step count %d < 0", t);
  int rc = sync_in(D->p);
  if (rc) return rc;
  const size_t mb = (size_t)D->nx * D->ny * sizeof(float);
  CK(cudaMemcpyAsync(D->m, m, mb, cudaMemcpyDefault, D->p->stream));
  CK(cudaMemcpyAsync(D->v, v, mb, cudaMemcpyDefault, D->p->stream));
  CK(cudaStreamSynchronize(D->p->stream));
  D->t = t;
  return CBS_OK;
}

int cbs_design_permittivity(cbs_design_t D, const float* h_dev, float* h_eff_dev, float* eps_dev) {
  g_err.clear();
  if (!D || !h_dev || !eps_dev) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(D->p);
  if (rc) return rc;
  float* heff = h_eff_dev ? h_eff_dev : D->heff;
  rc = design_effective(D, h_dev, heff);
  if (!rc) rc = design_permittivity(D, heff, eps_dev);
  if (rc) return rc;
  CK(cudaStreamSynchronize(D->p->stream));
  return CBS_OK;
}

int cbs_design_height_gradient(cbs_design_t D, const float* h_dev, const float* grad_eps_dev, float* grad_h_dev) {
  g_err.clear();
  if (!D || !h_dev || !grad_eps_dev || !grad_h_dev) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(D->p);
  if (rc) return rc;
  rc = design_effective(D, h_dev, D->heff);
  if (!rc) rc = design_height_gradient(D, D->heff, grad_eps_dev, grad_h_dev);
  if (rc) return rc;
  CK(cudaStreamSynchronize(D->p->stream));
  return CBS_OK;
}

int cbs_design_adam(cbs_design_t D, float* h_dev, const float* grad_h_dev) {
  g_err.clear();
  if (!D || !h_dev || !grad_h_dev) return fail(CBS_ERR_ARG, "NULL argument");
  int rc = sync_in(D->p);
  if (!rc) rc = design_adam(D, h_dev, grad_h_dev);
  if (rc) return rc;
  CK(cudaStreamSynchronize(D->p->stream));
  return CBS_OK;
}

int cbs_design_step(cbs_design_t D, float* h_dev, const cbs_source* src, const int r0[3], void* E_dev,
                    void* Eadj_dev, float* grad_h_dev, double* objective, cbs_stats* fwd, cbs_stats* adj) {
  NvtxRange nv("cbs_design_step");
  g_err.clear();
  if (fwd) *fwd = cbs_stats{};
  if (adj) *adj = cbs_stats{};
  if (!D || !h_dev || !src || !r0 || !E_dev || !Eadj_dev || !objective) return fail(CBS_ERR_ARG, "NULL argument");
  if (src->warm_start < 0 || src->warm_start > 2) return fail(CBS_ERR_ARG, "warm_start %d is not 0, 1 or 2", src->warm_start);
  cbs_plan_s* p = D->p;
  int rc = sync_in(p);
  if (!rc) rc = design_effective(D, h_dev, D->heff);
  if (!rc) rc = design_permittivity(D, D->heff, D->eps);
  if (rc) return rc;
  rc = cbs_set_permittivity(p, D->eps);
  if (rc) return rc;
  SourceArgs s;
  rc = make_source(p, src, s);
  if (rc) return rc;
  cbs_stats f{}, a{};
  rc = run_series(p, static_cast<float2*>(E_dev), s, src->warm_start, &f);
  if (fwd) *fwd = f;
  if (!nonfatal(rc)) return rc;
  rc = adjoint_run(p, r0, E_dev, Eadj_dev, src->warm_start, &a);
  if (adj) *adj = a;
  if (!nonfatal(rc)) return rc;
  const float coef = (float)(2.0 * p->kvac * p->kvac);
  CK(launch_gradient(static_cast<const float2*>(E_dev), static_cast<const float2*>(Eadj_dev), p->N, coef, D->grad,
                     p->stream));
  CK(launch_objective(static_cast<const float2*>(E_dev), p->N, p->d.nx, p->d.ny, r0[0], r0[1], r0[2], p->dobj,
                      p->stream));
  rc = design_height_gradient(D, D->heff, D->grad, D->gh);
  if (!rc && grad_h_dev)
    CK(cudaMemcpyAsync(grad_h_dev, D->gh, (size_t)D->nx * D->ny * sizeof(float), cudaMemcpyDeviceToDevice,
                       p->stream));
  if (!rc) rc = design_adam(D, h_dev, D->gh);
  if (rc) return rc;
  CK(cudaMemcpyAsync(objective, p->dobj, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return CBS_OK;
}

}  // extern "C"
