/*
 * cbs.h -- C ABI of the GB300 vector convergent Born series (CBS) solver.
 *
 * The solver computes the total electric field E of the monochromatic Maxwell problem
 *
 *     curl curl E - k(r)^2 E = S,        k(r)^2 = k_vac^2 (eps_r(r) + i sigma(r)),
 *
 * on a periodic voxel grid surrounded by absorbing layers, and the adjoint-field gradient
 * of the focal intensity |E(r0)|^2 with respect to eps_r.  This is the forward/adjoint
 * machinery of arXiv 2506.15411 (the CBS of its refs. [25], [26], run inside absorbing
 * layers [lambda, lambda, 6 lambda], Fig. 1 benchmark paragraph; figure of merit and its
 * gradient, Fig. 2 caption and the figure-of-merit paragraph).  The series is
 *
 *     gamma = (i / epsilon) V,   V = k^2 - k0^2 - i epsilon,
 *     E <- E - gamma [E - G (V E + S)],
 *
 * with G the dyadic Green operator of curl curl - (k0^2 + i epsilon), applied in k-space by
 * 3D FFTs of the three field components.
 *
 * Conventions shared by every call
 *   - Time factor exp(-i w t); outgoing waves go as exp(+i k r).
 *   - Grid arrays are C-order [nz][ny][nx] (x fastest).  Fields are complex64 (interleaved
 *     float re, im) of shape [3][nz][ny][nx], component order (x, y, z): 24 bytes a voxel.
 *   - Every pointer named *_dev is device memory of the plan's device, owned by the
 *     caller, contiguous, and at least 8-byte aligned; the plan never frees it.
 *   - Work is enqueued on desc.cuda_stream (blocks of iterations are captured there as CUDA
 *     graphs, so no other thread may use that stream during a call); with a NULL stream the
 *     plan owns a stream that first waits for the legacy stream.  The solve calls return
 *     when their result is complete on the device (the host needs the residual to decide
 *     convergence).
 *   - Return value: CBS_OK (0) or a negative CBS_ERR_* code; cbs_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef CBS_GB300_H
#define CBS_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define CBS_OK 0
#define CBS_ERR_ARG (-1)            /* bad argument: dims, radix, pads, null pointer, ... */
#define CBS_ERR_OOM (-2)            /* device allocation failed */
#define CBS_ERR_NOT_CONVERGED (-3)  /* tol > 0 and max_iter reached; E holds the last iterate */
#define CBS_ERR_DIVERGED (-4)       /* residual non-finite or grew 1e4-fold; E is garbage */
#define CBS_ERR_CUDA (-5)           /* a CUDA runtime call failed, or a kernel's bounded wait on
                                       a tensor copy timed out ("a tensor-copy wait timed
                                       out"): that solve's E is garbage, the plan stays usable
                                       and the next solve starts from a cleared error flag */
#define CBS_ERR_STATE (-6)          /* call out of order, e.g. no permittivity set yet */
#define CBS_ERR_STAGNATED (-7)      /* tol > 0 not reached and the residual stopped falling
                                       (no new 1 % minimum over max(1000, it/4) iterations):
                                       the FP32 rounding floor; E holds the last iterate */
#define CBS_ERR_TIME_LIMIT (-8)     /* the solve's wall-clock limit (cbs_set_time_limit) ran
                                       out before tol was reached; E holds the last iterate */

typedef struct cbs_plan_s* cbs_plan_t;

/* Problem and solver description (copied by cbs_plan). */
typedef struct {
  int nx, ny, nz;         /* grid, including the absorbing layers; each a product of
                             2, 3, 5, 7, 11, 13 and at most 1024 (cbs_plan returns
                             CBS_ERR_ARG for others) */
  double pitch_m;         /* voxel pitch [m] (isotropic) */
  double lambda_m;        /* vacuum wavelength [m] */
  double n_bg;            /* background index; sets the layer strength */
  int pad_lo[3];          /* absorbing-layer thickness in voxels on the low faces (x,y,z) */
  int pad_hi[3];          /* ... and on the high faces; each pad <= half the axis */
  double tol;             /* stop when ||delta_k|| / ||delta_0|| <= tol; tol <= 0 runs
                             exactly max_iter iterations */
  int max_iter;           /* > 0 */
  int check_every;        /* iterations between residual checks on the host (>= 1) */
  void* cuda_stream;      /* cudaStream_t the plan works on; NULL = legacy (see above) */
  /* Absorbing layers (the paper gives their thickness, not their profile).  A voxel at depth
   * t (1 .. L) into a layer of L voxels gets k^2 = k_vac^2 (eps_r + i sigma) with
   * sigma = sigma_max (t/L)^p and sigma_max = (p+1) n_bg ln(1/layer_round_trip) / (k_vac L pitch):
   * a normally incident plane wave keeps the amplitude layer_round_trip after crossing the
   * layer and back (weak-absorption estimate).  That bounds the reflection of a layer several
   * wavelengths thick (measured 1.2e-4 for 1e-4 at 6 lambda); a layer one wavelength thick
   * reflects more through its gradient (about 5 % for 1e-4, 0.4 - 2 % for 1e-2).  The
   * absorption raises the series' shift epsilon, and the iteration count with it: weaker or
   * non-adding layers converge in fewer iterations.  Zero-initialised fields select the
   * defaults. */
  double layer_round_trip;  /* in (0, 1); 0 selects 1e-4 */
  double layer_power;       /* ramp exponent p in (0, 16]; 0 selects 2 */
  int layer_corner_max;     /* where layers overlap: 0 their profiles add, 1 the largest applies */
} cbs_plan_desc;

#define CBS_SRC_PLANE_WAVE 0  /* current sheet on plane z_plane launching pol * exp(ik|z-z_s|) */
#define CBS_SRC_POINT 1       /* raw value pol at voxel r0 (a dipole p is pol = p / pitch^3) */
#define CBS_SRC_USER 2        /* caller's S, complex64 [3][nz][ny][nx] on the device */

/* Source term S of the forward problem. */
typedef struct {
  int kind;                 /* CBS_SRC_* */
  double pol[3][2];         /* complex polarisation (re, im) for x, y, z */
  int z_plane;              /* plane-wave sheet; < 0 selects pad_lo[2] */
  int r0[3];                /* point-source voxel (x, y, z) */
  const void* user_src_dev; /* CBS_SRC_USER only */
  int warm_start;           /* 0: E starts at 0.  1: E_dev holds the initial guess; residuals
                               are relative to this run's first.  2: as 1, but relative to
                               the first residual of a start from 0 (one extra iteration
                               computes it), so a good guess stops early. */
} cbs_source;

/* Outcome of one solve (always filled when the pointer is not NULL). */
typedef struct {
  int iters;         /* iterations run */
  double rel_resid;  /* ||delta_last|| / ||delta_0|| (FP64 sums on the device) */
  double resid0;     /* ||delta_0|| */
  double seconds;    /* host wall time of the call */
  int status;        /* return code of the call */
} cbs_stats;

/* Create a plan for one problem as the paper states it: a voxel grid of the given pitch,
 * the vacuum wavelength and absorbing layers of given thickness on every face (thickness
 * [lambda, lambda, 6 lambda] in the Fig. 1 benchmark paragraph; the 621 x 621 x 261-voxel
 * design volume at 177 nm of the Fig. 4 paragraph).  Checks the description, factors each
 * axis into FFT radices and allocates the plan's device memory (potential V: 8 B/voxel;
 * k-space workspace W and the iterate: 24 B/voxel each; twiddles and reduction scratch).
 * *out receives the plan.  Errors: CBS_ERR_ARG, CBS_ERR_OOM, CBS_ERR_CUDA. */
int cbs_plan(cbs_plan_t* out, const cbs_plan_desc* desc);

/* Set the relative permittivity (real, float32 [nz][ny][nx], layers included; the plan
 * adds the absorption inside the pads).  Computes the splitting
 * k0^2 = (min Re k^2 + max Re k^2)/2, epsilon = max |k^2 - k0^2| with FP64 reductions on the
 * device and stores V.  Errors: CBS_ERR_ARG (NULL, non-finite or zero-epsilon input),
 * CBS_ERR_CUDA. */
int cbs_set_permittivity(cbs_plan_t plan, const float* eps_real_dev);

/* The splitting chosen by the last cbs_set_permittivity, in SI units [1/m^2]. */
int cbs_get_splitting(cbs_plan_t plan, double* k0sq, double* epsilon);

/* Change the stopping rule of later solves (same meaning as in cbs_plan_desc). */
int cbs_set_solver(cbs_plan_t plan, double tol, int max_iter, int check_every);

/* Wall-clock limit of later solves, in seconds from the solve's start (0: none, the default).
 * It is checked on the host after each block of check_every iterations, so a solve may run
 * up to one block past it; it then ends with CBS_ERR_TIME_LIMIT and E holds the last
 * iterate.  Errors: CBS_ERR_ARG (NULL plan, negative or non-finite seconds). */
int cbs_set_time_limit(cbs_plan_t plan, double seconds);

/* Forward solve (the CBS solve of the Fig. 1 benchmark paragraph: the total field of a lens
 * under a normally incident x-polarised plane wave, Fig. 2 paragraph): iterate the series
 * for source *src into E_dev (complex64 [3][nz][ny][nx]).
 * Returns CBS_OK, CBS_ERR_NOT_CONVERGED (tol > 0 not reached in max_iter; E_dev holds the
 * last iterate), CBS_ERR_STAGNATED (residual at its FP32 floor above tol),
 * CBS_ERR_TIME_LIMIT, CBS_ERR_DIVERGED, CBS_ERR_ARG, CBS_ERR_STATE or CBS_ERR_CUDA. */
int cbs_forward(cbs_plan_t plan, const cbs_source* src, void* E_dev, cbs_stats* stats);

/* Adjoint solve for the figure of merit |E(r0)|^2 (the adjoint field of the figure-of-merit
 * paragraph): E_adj = A^{-1}[conj(E(r0)) delta_r0],
 * the same series with a raw point source conj(E(r0)) read from E_dev on the device
 * (A = curl curl - k^2 is complex symmetric).  r0 = (x, y, z) voxel.  Eadj_dev starts at 0.
 * Return codes as cbs_forward. */
int cbs_adjoint(cbs_plan_t plan, const int r0[3], const void* E_dev, void* Eadj_dev,
                cbs_stats* stats);

/* Gradient of the figure of merit L = |E(r0)|^2 (Fig. 2 caption) from the forward and the
 * adjoint field (the 3D gradient of the figure-of-merit paragraph, there taken with respect to
 * the shape S(r); per unit of permittivity here):
 * dL/d eps_r(r) = 2 k_vac^2 Re[E_adj(r) . E(r)] into grad_dev (float32
 * [nz][ny][nx]); when r0 and objective are not NULL also *objective = |E(r0)|^2 (FP64).
 * Errors: CBS_ERR_ARG, CBS_ERR_CUDA. */
int cbs_gradient(cbs_plan_t plan, const void* E_dev, const void* Eadj_dev, const int r0[3],
                 float* grad_dev, double* objective);

/* Figure of merit alone: *objective = |E(r0)|^2 (FP64) for a field on the device.
 * Errors: CBS_ERR_ARG, CBS_ERR_CUDA. */
int cbs_objective(cbs_plan_t plan, const void* E_dev, const int r0[3], double* objective);

/* One design iteration from HOST buffers: copies eps (float32 [nz][ny][nx]) to the device,
 * sets it, runs the forward solve for *src into a plan-owned field, the adjoint solve for
 * |E(r0)|^2 and the gradient, and copies the gradient back into grad_host (float32
 * [nz][ny][nx]) and the objective into *objective.  The plan allocates its two field
 * buffers (48 B/voxel) and staging on first use.  fwd/adj may be NULL.  Return codes as
 * cbs_forward (the first failing step). */
int cbs_design_step_host(cbs_plan_t plan, const float* eps_host, const cbs_source* src,
                         const int r0[3], float* grad_host, double* objective,
                         cbs_stats* fwd, cbs_stats* adj);

/* Pass timing.  A series launches the forward x pass (V E + S, FFT_x) once, then four
 * kernels per iteration: y forward, z + k-space multiply, y inverse, and an x pass that
 * finishes the iteration (IFFT_x, update, residual) and forms the next iteration's FFT_x of
 * V E + S.  With profiling on, each block of iterations records CUDA events on the plan's
 * stream around the four launches of its last iteration (kept out of the captured graphs);
 * cbs_pass_times returns, per slot (0 the series' first forward x pass -- not timed, always 0;
 * 1 y forward; 2 z + k-space multiply; 3 y inverse; 4 x inverse + update + next forward x),
 * the summed event time in ms and the number of timed launches since the last reset.
 * Toggling drops the cached graphs.  Errors: CBS_ERR_ARG, CBS_ERR_CUDA. */
int cbs_set_profiling(cbs_plan_t plan, int on);
int cbs_pass_times(cbs_plan_t plan, double ms_total[5], long long launches[5], int reset);

/* The splitting of a permittivity grid (what cbs_set_permittivity computes: k0^2 and
 * epsilon in SI units [1/m^2]) without a plan and without allocating any memory.  For
 * callers that cannot call cudaMalloc: code whose device memory is all handed out by another
 * allocator, or loops that must not pay for, or synchronise the device on, cudaMalloc and
 * cudaFree.  The paper has no counterpart; it is a service of this library.
 *   desc: nx, ny, nz, pitch_m, lambda_m, n_bg, pad_lo, pad_hi and cuda_stream are used (the
 *         kernels run on cuda_stream; NULL is the legacy stream); the solver fields are not.
 *   eps_real_dev: float32 [nz][ny][nx] on the current device, layers included.
 * Scratch: one ~80 KB array in device memory per device that loads the library, kept until
 * the process exits.  The first call on a device looks up its address and keeps it for the
 * life of the process: after a cudaDeviceReset of that device the kept address is stale, so
 * do not call this entry point again on a device that has been reset.  Every call shares the array and leaves its contents behind;
 * calls that overlap on the GPU (other streams or threads) race and give wrong results.
 * Limit: nx * ny * nz <= 268,435,456 voxels (4096 blocks of 65,536); larger grids return
 * CBS_ERR_ARG.  Other errors: CBS_ERR_ARG (NULL; dims or pads that cbs_plan rejects:
 * an axis outside [1, 1024], a pad over half its axis; non-finite eps; epsilon = 0),
 * CBS_ERR_CUDA.  Blocks the host until the result is back. */
int cbs_splitting_noalloc(const cbs_plan_desc* desc, const float* eps_real_dev, double* k0sq,
                          double* epsilon);

/* ---------------------------------------------------------------- inverse design
 * One gradient step of the lens design loop of Section 3 / Fig. 2(a) on the thickness map
 * h(x, y) (float32 [ny][nx] on the device, micrometres; x, y the plan's lateral grid):
 *     h_eff = G_sigma[M h]             M: mirror average over (+-x, +-y) about the grid
 *                                      centre; G_sigma: separable Gaussian of std sigma,
 *                                      weights exp(-k^2/2s^2) for |k| <= ceil(4s), s = sigma /
 *                                      pitch, normalised, zero outside the map
 *     eps_r = n_bg^2 + f (n_lens^2 - n_bg^2),  f = clamp(h_eff / pitch - (z - z_base), 0, 1)
 *                                      for z >= z_base, else 0 (shape Theta(h - z) with
 *                                      subpixel filling along z)
 *     forward and adjoint CBS, dL/d eps_r = 2 k_vac^2 Re[E_adj . E], L = |E(r0)|^2
 *     dL/dh = M G_sigma[(n_lens^2 - n_bg^2)/pitch * dL/d eps_r at z_base + floor(h_eff/pitch)]
 *     Adam (Kingma & Ba) ascent on L with step alpha [um], then 0 <= h <= h_max inside the
 *     aperture (pixel centre within D/2 of the grid centre) and h = 0 outside it.
 * A design object belongs to one plan (same device and stream; not thread-safe) and owns
 * Adam's moments (2 maps), four scratch maps and two volumes (eps_r, dL/d eps_r: 8 B/voxel). */
typedef struct cbs_design_s* cbs_design_t;

typedef struct {
  int z_base;           /* z index of the lens base plane (h = 0) */
  double n_lens;        /* lens index (the background is the plan's n_bg) */
  double aperture_um;   /* design-region diameter D */
  double h_max_um;      /* upper bound of h */
  double sigma_um;      /* Gaussian smoothing std; 0 = none (ceil(4 sigma/pitch) <= 256) */
  int mirror;           /* nonzero: impose h(x, y) = h(+-x, +-y) */
  double alpha;         /* Adam step [um] (0.3 in Section 3) */
  double beta1, beta2;  /* Adam decay rates (0.9, 0.999) */
  double adam_eps;      /* Adam regulariser (1e-6) */
} cbs_design_desc;

/* Create / free a design object for plan.  Errors: CBS_ERR_ARG, CBS_ERR_OOM, CBS_ERR_CUDA. */
int cbs_design_create(cbs_design_t* out, cbs_plan_t plan, const cbs_design_desc* desc);
void cbs_design_destroy(cbs_design_t design);

/* Zero Adam's moments and step count. */
int cbs_design_reset(cbs_design_t design);

/* Checkpoint / resume of the design loop.  Its state is the map h (held by the caller),
 * Adam's first and second moments (float32 [ny][nx] each) and the number of Adam steps
 * taken, t (the bias corrections use beta^t).  get copies the moments into m / v and writes
 * t; set loads them, so that the next cbs_design_adam or cbs_design_step on this object does
 * exactly what it would have done on the object the state came from (same plan shape and
 * desc).  m and v hold ny*nx floats each and may be device or host memory (any address CUDA
 * can copy from or to); both calls block until the copies are done.  Errors: CBS_ERR_ARG
 * (NULL argument, t < 0), CBS_ERR_CUDA. */
int cbs_design_get_state(cbs_design_t design, float* m, float* v, int* t);
int cbs_design_set_state(cbs_design_t design, const float* m, const float* v, int t);

/* h -> h_eff (into h_eff_dev when not NULL) -> eps_r (float32 [nz][ny][nx] into eps_dev). */
int cbs_design_permittivity(cbs_design_t design, const float* h_dev, float* h_eff_dev, float* eps_dev);

/* dL/dh (float32 [ny][nx] into grad_h_dev) from dL/d eps_r (float32 [nz][ny][nx]) at the
 * design h_dev: the surface derivative and the adjoints of G_sigma and M. */
int cbs_design_height_gradient(cbs_design_t design, const float* h_dev, const float* grad_eps_dev,
                               float* grad_h_dev);

/* One Adam ascent step on h_dev (in place) for the gradient dL/dh in grad_h_dev, with the
 * box and aperture constraints; counts one step. */
int cbs_design_adam(cbs_design_t design, float* h_dev, const float* grad_h_dev);

/* The whole step: eps_r from h_dev, cbs_set_permittivity, the forward solve of *src into
 * E_dev and the adjoint solve of |E(r0)|^2 into Eadj_dev (both warm-started from their
 * contents when src->warm_start is 1 or 2, with that meaning), the gradient, dL/dh (copied
 * into grad_h_dev when not NULL) and the Adam update of h_dev in place.  *objective =
 * |E(r0)|^2 before the update.  fwd/adj may be NULL.  A solve that ends NOT_CONVERGED,
 * STAGNATED or TIME_LIMIT does not stop the step (its status is in fwd/adj); other errors return at the
 * failing step, with h_dev not updated. */
int cbs_design_step(cbs_design_t design, float* h_dev, const cbs_source* src, const int r0[3],
                    void* E_dev, void* Eadj_dev, float* grad_h_dev, double* objective,
                    cbs_stats* fwd, cbs_stats* adj);

/* ---------------------------------------------------------------- serving
 * A request server with continuous batching.  Submitted requests queue; a worker thread
 * admits them while the device-memory budget and max_active allow.  Requests of one grid
 * shape share a batch: a plan whose arrays hold up to min(8, max_active) requests side by
 * side (seats), each with its own permittivity, splitting and source.  The worker advances
 * every batch one block of check_every iterations at a time without waiting on any one of
 * them; each launch of a block carries every iterating request of the batch (the kernels'
 * tile space has a request index), so same-shape requests in flight share the launches, and
 * batches of different shapes run side by side on their own streams, smaller grids at higher
 * stream priority (a short request's next kernel goes before a long one's).  A request arriving
 * while others run takes a free seat at the next block, or a new batch when memory allows;
 * a batch is created with as many seats as the budget leaves room for.  Batches without
 * requests are kept for later requests of their shape and evicted, least recently used
 * first, when memory is needed.  Fields stay in the seat's device memory; only the outputs a
 * request asks for are copied out.  A request's result does not depend on what else runs:
 * its blocks in a launch are those of its own persistent grid, so its tiles and the order of
 * its residual sums are fixed, seats share no device memory, and the stopping decision uses
 * its own residuals only.  The server works on the device current at creation.  Not a part
 * of the paper; the serving layer of this library. */
typedef struct cbs_server_s* cbs_server_t;

typedef struct {
  double hbm_budget_bytes;  /* device bytes the batches may hold; 0 = 80 % of the free memory */
  int max_active;           /* requests admitted at once (>= 1) */
  double tol;               /* solver settings of every request (as in cbs_plan_desc) */
  int max_iter;
  int check_every;
} cbs_server_desc;

typedef struct {
  int nx, ny, nz;           /* grid and physics as in cbs_plan_desc */
  double pitch_m, lambda_m, n_bg;
  int pad_lo[3], pad_hi[3];
  double layer_round_trip;  /* absorbing layers as in cbs_plan_desc (0: defaults) */
  double layer_power;
  int layer_corner_max;
  const float* eps_host;    /* permittivity float32 [nz][ny][nx]: exactly one of eps_host */
  const float* eps_dev;     /* (read with a blocking copy at admission) and eps_dev */
  cbs_source src;           /* plane wave or point source; warm_start 0 */
  int adjoint;              /* nonzero: also the adjoint solve of |E(r0)|^2 and the gradient */
  int r0[3];                /* objective voxel; |E(r0)|^2 is reported for every request */
  void* E_host;             /* optional outputs (NULL = not copied): the field, complex64 */
  void* E_dev;              /*   [3][nz][ny][nx], to host (pinned avoids a blocking copy) or */
  float* grad_host;         /*   device memory; the gradient dL/d eps_r, float32 [nz][ny][nx] */
  float* grad_dev;          /*   (adjoint requests only) */
} cbs_request;
/* Every pointer in a request must stay valid until its result has been taken. */

typedef struct {
  long long id;             /* as returned by cbs_server_submit */
  int status;               /* CBS_OK, the forward's or adjoint's NOT_CONVERGED / STAGNATED,
                               or the error that ended the request */
  double objective;         /* |E(r0)|^2 */
  cbs_stats fwd, adj;       /* adj is zero for forward-only requests */
  double t_submit, t_admit, t_done;   /* CLOCK_MONOTONIC seconds */
  char error[192];          /* message when status is an error */
} cbs_result;

/* Start / stop a server (stop finishes the admitted requests; queued ones end with
 * CBS_ERR_STATE).  Errors: CBS_ERR_ARG, CBS_ERR_CUDA. */
int cbs_server_create(cbs_server_t* out, const cbs_server_desc* desc);
void cbs_server_destroy(cbs_server_t server);

/* Queue a request (thread-safe); *id receives its number.  Errors: CBS_ERR_ARG (bad grid,
 * r0, source or eps pointers), CBS_ERR_STATE (closing).  Plan errors (unsupported sizes,
 * device memory) come back in the result. */
int cbs_server_submit(cbs_server_t server, const cbs_request* req, long long* id);

/* Take up to max completed results (in completion order), waiting up to timeout_s seconds
 * for the first; *n receives the count (0 on timeout). */
int cbs_server_take(cbs_server_t server, cbs_result* out, int max, double timeout_s, int* n);

/* Requests waiting for admission, requests admitted, device bytes held by batches. */
int cbs_server_info(cbs_server_t server, long long* queued, long long* active, double* bytes_used);

/* Launch sharing so far: *launches = iterations launched (each the four passes of one
 * iteration of one batch), *request_iterations = the request iterations they carried (their
 * sum of members), *max_members = the most requests one launch carried.  Any pointer may be
 * NULL. */
int cbs_server_sharing(cbs_server_t server, long long* launches, long long* request_iterations, int* max_members);

/* Self-test of the failure path of the tile kernels: every wait of theirs on a tensor copy is
 * bounded and, when it gives up, records an error the host reads after the block of
 * iterations (CBS_ERR_CUDA, "a tensor-copy wait timed out") instead of hanging the GPU.  This
 * runs that bounded wait on an mbarrier nothing completes, on the current device, and checks
 * that it gave up (*device_status = 1) and that the context still takes work.  Returns CBS_OK,
 * or CBS_ERR_CUDA with a message. */
int cbs_selftest_wait_timeout(int* device_status);

/* Free the plan and its device memory (NULL is a no-op). */
void cbs_destroy(cbs_plan_t plan);

/* Message of the last failed call on this thread ("" if none). */
const char* cbs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CBS_GB300_H */
