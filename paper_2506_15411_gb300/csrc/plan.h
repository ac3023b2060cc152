// plan.h -- the plan object behind cbs_plan_t and the host-side series driver, shared by
// the C ABI (api.cu) and the request server (serve.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <vector>

#include "../../include/cbs.h"
#include "absorber.h"
#include "cbs_internal.h"

namespace cbs {

// Record a message for cbs_last_error (this thread) and return code.
int fail(int code, const char* fmt, ...);

}  // namespace cbs

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return cbs::fail(CBS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

namespace cbs {

// An NVTX range over a scope (host timeline of the API calls, for nsys and `ncu --nvtx`);
// without a tool attached the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Solves that return with the last iterate in E and do not stop a design step or a request.
inline bool nonfatal(int rc) {
  return rc == CBS_OK || rc == CBS_ERR_NOT_CONVERGED || rc == CBS_ERR_STAGNATED || rc == CBS_ERR_TIME_LIMIT;
}

// A captured block of iterations (the launches read the source and splitting from the plan's
// member array, so a graph serves every solve of the plan).
struct GraphEntry {
  float2* E;
  int iters;
  cudaGraphExec_t exec;
};

// Length of a plan's member array: [0] the plan's own solves, [1 + s] seat s alone (a series'
// first x pass), then check_every lists of kMaxMembers for a batch's block of iterations.
inline size_t members_len(int seats, int check_every) {
  return 1 + (size_t)seats + (size_t)check_every * kMaxMembers;
}

}  // namespace cbs

struct cbs_plan_s {
  cbs_plan_desc d{};
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;   // the caller's stream, or an owned one for NULL (legacy)
  bool own_stream = false;
  cudaEvent_t ev = nullptr;
  cudaEvent_t blk_ev = nullptr;    // end of the last enqueued block of iterations or copy-out
  CUtensorMap tmy{}, tmz{};        // W maps for the y pass and the z pass
  int* err_dev = nullptr;          // kernels' error flag
  int* err_host = nullptr;         // pinned copy
  cbs::IterArgs base{};
  int seats = 1;                   // requests the arrays hold side by side (cbs_plan: 1)
  size_t N = 0;
  double pitch = 0, kvac = 0;
  cbs::LayerSpec layers{};         // absorbing-layer profile (absorber.h)
  int sms = 0;
  // device memory owned by the plan
  float2* V = nullptr;
  float2* W = nullptr;
  float2* Ei = nullptr;            // the field being iterated, padded rows
  float2* tw = nullptr;             // per-stage twiddles of the three axes
  float2* pq = nullptr;             // wave numbers of the spectrum positions of the three axes
  int4* stages = nullptr;
  std::vector<int> radix_order[3];  // DIF radix order of each axis
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* hist = nullptr;
  cbs::Member* mem_dev = nullptr;   // launch members (members_len) and their pinned staging
  cbs::Member* mem_host = nullptr;
  float2* adj_amp = nullptr;
  double* dobj = nullptr;
  double *sx = nullptr, *sy = nullptr, *sz = nullptr;
  // set-up scratch
  float *pmin = nullptr, *pmax = nullptr;
  int* pbad = nullptr;
  double* pdev = nullptr;
  int red_blocks = 0;
  // host staging (pinned)
  double* hist_host = nullptr;
  // host-buffer design step
  float* eps_dev = nullptr;
  float2* Ef = nullptr;
  float2* Ea = nullptr;
  float* grad_dev = nullptr;
  // splitting (scaled units) of the plan's own solves (seat 0), and of every seat
  bool have_eps = false;
  double k0sq_s = 0, eps_s = 0;
  std::vector<double> seat_k0sq, seat_eps;
  // graphs of one block of check_every iterations, per (E, source) binding
  std::vector<cbs::GraphEntry> graphs;
  // pass timing (events around the launches of the last iteration of each block)
  double time_limit_s = 0;         // wall-clock limit of a solve (0: none)
  bool profiling = false;
  cudaEvent_t pev[6] = {};
  double pass_ms[5] = {};
  long long pass_n[5] = {};
};

namespace cbs {

// One run of the series on a plan, advanced a block of check_every iterations at a time, so
// that a caller can keep several plans' runs in flight on their own streams (the server) or
// wait on one (the blocking calls).
struct SeriesRun {
  float2* E = nullptr;     // caller's field: copied in (warm start) and out once
  IterArgs a{};
  int it = 0, best_it = 0, m = 0;
  double r0 = -1.0, rel = 0.0, best = 1e300;
  int rc = CBS_OK;
  bool iterating = false;  // a block is in flight (blk_ev marks its residuals on the host)
  bool copying = false;    // the copy-out is in flight (blk_ev marks its end)
  bool finished = false;
  nvtxRangeId_t blk_range = 0;   // NVTX range of the block in flight
  std::chrono::steady_clock::time_point t0;
};

// Plans with several seats and their set-up (api.cu).
int plan_create(cbs_plan_s** out, const cbs_plan_desc* desc, int seats);
int seat_permittivity(cbs_plan_s* p, int seat, const float* eps, cudaStream_t s);
cudaError_t field_copy(const cbs_plan_s* p, int seat, float2* dense, bool to_dense, cudaStream_t s);
// The launches of one iteration after a series' first, for the members in a (api.cu).
int launch_iteration(const cbs_plan_s* p, const IterArgs& a, cudaStream_t s, cudaEvent_t* ev);

// Series driver (api.cu).
int sync_in(cbs_plan_s* p);
int make_source(cbs_plan_s* p, const cbs_source* src, SourceArgs& s);
void series_begin(cbs_plan_s* p, float2* E, const SourceArgs& src, int warm, SeriesRun& R);
bool series_advance(cbs_plan_s* p, SeriesRun& R, bool wait);
int series_stats(const cbs_plan_s* p, SeriesRun& R, cbs_stats* S);
// The stopping rules on the residual sums h[0 .. R.m-1] of a block (sets R.rc on an error);
// returns whether the run is over.
bool series_absorb_residuals(const cbs_plan_s* p, SeriesRun& R, const double* h);
int run_series(cbs_plan_s* p, float2* E, const SourceArgs& src, int warm, cbs_stats* st);
// Source of the adjoint of |E(r0)|^2 (enqueues the read of conj(E(r0)) on the plan's stream).
int adjoint_source(cbs_plan_s* p, const int r0[3], const void* E_dev, SourceArgs& s);

}  // namespace cbs
