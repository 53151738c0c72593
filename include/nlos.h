/*
 * nlos.h -- C ABI of the GB300 (sm_103a) curvature-regularised confocal NLOS
 * reconstruction library (arXiv 2301.00406).
 *
 * The library computes, on one GPU, the per-iteration work of the paper's two
 * ADMM solvers: the confocal light-cone-transform operator A = R_t^{-1} H R_z
 * of Sec. 2 (Eq. 3) and its transpose, the scan-grid sampling D (A_D = D A,
 * Sec. 3.1.2), and the curvature-regularisation sub-steps of Algorithm 1
 * (Sec. 3, Eq. 4-12) and Algorithm 2 (Sec. 4.1, Eq. 13).
 *
 * Conventions shared by every entry point
 *  - Every function returns an nlos_status; NLOS_OK (0) is success and the
 *    other codes are negative.  No function aborts, throws or exits across
 *    the ABI.  nlos_last_error() copies a thread-local message describing the
 *    most recent failure on the calling thread.
 *  - Volumes (albedo u) and transients (tau) are float32, contiguous,
 *    row-major [nx][ny][nt] (time/depth fastest).  Pointers named *_dev are
 *    device pointers in the current CUDA context; *_host pointers are host
 *    memory.  The caller owns every pointer it passes and must keep it valid
 *    until the work queued on `stream` has completed.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Work is queued on that stream without host synchronisation
 *    unless the function says otherwise.
 *  - Sizes of plans (and of everything that takes a geometry): nx = ny, a
 *    power of two in [8, 128] (the lateral convolution uses the symmetry of
 *    the cone kernel's spectrum under exchange of x and y); nt is a power of
 *    two in [16, 1024].  Other
 *    sizes return NLOS_ERR_INVALID_ARG.  nlos_solve_static and
 *    nlos_midpoint_confocal state their own limits.
 *  - A plan is not thread-safe: serialise calls that use the same plan.
 *    The server entry points other than create and destroy (nlos_submit,
 *    nlos_poll, nlos_wait, nlos_job_times, nlos_server_info,
 *    nlos_server_prepare) are thread-safe.
 */
#ifndef NLOS_H
#define NLOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nlos_status;
#define NLOS_OK 0
#define NLOS_ERR_INVALID_ARG (-1) /* bad pointer, size or parameter            */
#define NLOS_ERR_OOM (-2)         /* device or host allocation failed          */
#define NLOS_ERR_CUDA (-3)        /* a CUDA runtime call or launch failed      */
#define NLOS_ERR_BUSY (-4)        /* server queue full                         */
#define NLOS_ERR_NOT_READY (-5)   /* job still queued or running               */
#define NLOS_ERR_TIMEOUT (-6)     /* a bounded wait gave up                    */
#define NLOS_ERR_DIVERGED (-7)    /* non-finite energy or backtracking gave up */

/* Radiometric weight of R_t^{-1} (the t-axis resampling of Eq. 3). */
#define NLOS_RADIOMETRY_COMPENSATED 0 /* transient pre-multiplied by t^4: weight rho   */
#define NLOS_RADIOMETRY_RAW 1         /* 1/d^4 fall-off of Eq. 2: weight rho^-3       */

/* Start of the ADMM iterations (nlos_params.init). */
#define NLOS_INIT_ZERO 0         /* u0 = 0 (Algorithms 1-2 as printed)                        */
#define NLOS_INIT_BACKPROJECT 1  /* u0 = s A_D^T tau0, s = ||A_D^T tau0||^2 / ||A_D A_D^T tau0||^2 */

/* phi(kappa) of Sec. 3 (below Eq. 4). */
#define NLOS_PHI_TSC 0 /* a + b kappa^2 (the paper's choice) */
#define NLOS_PHI_TAC 1 /* a + b |kappa|                      */
#define NLOS_PHI_TRV 2 /* sqrt(a + b kappa^2)                */

typedef struct nlos_plan_s* nlos_plan;
typedef struct nlos_server_s* nlos_server;

/* Scan geometry of one confocal scene (Sec. 2).  The voxel grid shares the
 * scan grid laterally (nx x ny points over a wall_width_m square) and the time
 * axis in depth: depth bin k and time bin k both sit at rho_k = (k + 1/2)/nt of
 * the range R = c * nt * bin_width_s / 2. */
typedef struct {
  int32_t nx, ny, nt;
  double bin_width_s;   /* time-bin width in seconds, > 0                      */
  double wall_width_m;  /* side of the scanned wall patch in metres, > 0       */
  int32_t radiometry;   /* NLOS_RADIOMETRY_*                                    */
  const uint8_t* mask;  /* host, nx*ny bytes, nonzero = scan point measured
                           (the complement is the missing region X); NULL =
                           fully sampled.  Copied by nlos_plan_create.         */
} nlos_geometry;

/* Solver parameters.  nlos_params_default() fills the paper's values. */
typedef struct {
  int32_t model;         /* 1 = object domain (Algorithm 1), 2 = dual domain (Algorithm 2) */
  int32_t phi;           /* NLOS_PHI_*                                                      */
  double a, b;           /* Algorithm 1 phi parameters                                      */
  double mu;             /* Algorithm 1 penalty (Eq. 5)                                     */
  double a_u, b_u, a_tau, b_tau, lambda; /* Algorithm 2 (Eq. 13)                            */
  double mu1, mu2, mu3;  /* Algorithm 2 penalties (Sec. 4.1)                                */
  int32_t iters;         /* T_max                                                           */
  double eps_stop;       /* relative-energy stop of Algorithms 1/2; 0 = run all iters       */
  double L0;             /* initial L; <= 0 means 2 ||A_D||_2^2 (below Eq. 10)              */
  double eta;            /* backtracking growth factor for L (> 1)                          */
  int32_t max_backtracks;/* rejections allowed in one iteration before NLOS_ERR_DIVERGED;
                            0..1000                                                        */
  double eps_normal;     /* regulariser of |grad u| in the normal field                     */
  int32_t restart;       /* FISTA restart on energy increase: 0 off, 1 on, -1 model default
                            (off for model 1, on for model 2)                              */
  int32_t warm_start_iters; /* model 2 only: first run this many Algorithm-1 iterations
                            (a, b, mu, default L0, no restart) and start Algorithm 2 from
                            their u (the remark after Algorithm 2; tau starts at 0);
                            0 = start from u = 0.  Ignored for model 1; < 0 is an error. */
  int32_t init;          /* NLOS_INIT_*: start of the first phase (the warm stage when
                            warm_start_iters > 0).  NLOS_INIT_BACKPROJECT starts from the
                            back-projection of the data (the direct method of Sec. 1) scaled
                            by the s that minimises 1/2 ||A_D (s g) - tau0||^2, g = A_D^T tau0
                            (s = 0 for zero data); phi and the initial energy are those of
                            u0; tau starts at 0 (model 2).  Computed on the device (no host
                            synchronisation). */
} nlos_params;

/* Per-reconstruction statistics (host struct, filled after the run). */
typedef struct {
  int32_t iters_done;
  int32_t backtracks;    /* total rejected L trials                           */
  int32_t restarts;      /* FISTA restarts taken                              */
  int32_t status;        /* NLOS_OK or the error that stopped the run         */
  double L;              /* final L                                           */
  double energy;         /* E at the last iteration (Eq. 4 or Eq. 13)         */
  double rel_change;     /* e = |E_prev - E| / |E| at the last iteration      */
  double data_fit;       /* 1/2 ||A_D u - tau0||^2 (model 1) or 1/2 ||A u - tau||^2 (model 2) */
  double primal_res;     /* ||v - grad u|| at the last iteration              */
} nlos_stats;

/* Copy the most recent error message of the calling thread into buf
 * (NUL-terminated, truncated to n bytes).  Returns NLOS_OK. */
nlos_status nlos_last_error(char* buf, size_t n);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t nlos_version(void);

/* Fill *out with the defaults for `model` (1 or 2): the Bowling 8x8
 * settings of Sec. 5.2.1 (a = 9e-5, b = 2e-5, mu = 0.1; lambda = 235,
 * a_tau = 4e-4, b_tau = 3e-2, a_u = 2e-4, b_u = 4.5e-4), mu1..3 = 1, 800, 2 and
 * T_max = 200 / 300 (Sec. 5.1), eps_stop = 0, L0 = 0 (= 2||A_D||^2), eta = 2,
 * max_backtracks = 30, eps_normal = 1e-6, restart = -1, warm_start_iters = 0,
 * init = NLOS_INIT_ZERO.
 * Host only. */
nlos_status nlos_params_default(int32_t model, nlos_params* out);

/* Create a plan for one geometry (Sec. 2, Eq. 3): builds the R_z and R_t^{-1}
 * two-tap tables in FP64 on the host, the sampled-column list of the mask,
 * and the cone-kernel spectrum H on the device (queued on `stream`, which is
 * synchronised before return).  All device memory the plan needs for the
 * operator is allocated here.  *out is set only on success.
 * The first plan of a time-axis length and sampled-column count in a process
 * times the candidate launch shapes of the t-passes (columns per CTA) on the
 * plan's own buffers and keeps the fastest; the choices are also written to
 * a tuning file ($NLOS_TUNE_CACHE, else $XDG_CACHE_HOME/nlos-gb300/
 * tpass_tuning, else $HOME/.cache/nlos-gb300/tpass_tuning; NLOS_TUNE_CACHE=off
 * disables it), keyed by device name, SM count and the library's compile time, from which
 * later processes read them instead of timing again. */
nlos_status nlos_plan_create(const nlos_geometry* geom, void* stream, nlos_plan* out);

/* Release a plan and all its device memory.  Synchronises the device first.
 * NULL is accepted. */
nlos_status nlos_plan_destroy(nlos_plan plan);

/* Select how the plan computes the lateral convolution of every kt plane
 * with the cone-kernel spectrum (the H of Eq. 3 and its conjugate in A^T):
 *   0  hand-written FFT kernels in FP32 (default);
 *   1  DFT-matrix products on the tensor cores (tcgen05.mma issued from a
 *      hand-written kernel, accumulators in tensor memory): every operand
 *      split into hi + lo BF16 terms and the products hi hi + hi lo + lo hi
 *      accumulated in FP32 (the split-BF16 variant of the precision
 *      comparison);
 *   2  the same with the hi terms only (one BF16 product, FP32 accumulate).
 * Modes 1 and 2 need nx = ny = 128.  The first non-zero mode builds the
 * block DFT constant and a copy of the kernel spectrum rearranged for the
 * kernel's reads (16 (nt + 1) 129 64 bytes of device memory, freed by mode 0
 * or nlos_plan_destroy) and synchronises `stream`.  Results are those of
 * mode 0 within the split's rounding.  Every MMA completion wait of the
 * kernel gives up after one second; the next call of this function then
 * returns NLOS_ERR_TIMEOUT (the output of that launch is undefined).  Not
 * thread-safe with other calls on the same plan.  Errors: invalid mode or
 * size (NLOS_ERR_INVALID_ARG), device memory (NLOS_ERR_OOM), CUDA
 * (NLOS_ERR_CUDA). */
nlos_status nlos_plan_set_lateral(nlos_plan plan, int32_t mode, void* stream);

/* ||A_D||_2^2 (masked != 0) or ||A||_2^2 by power iteration on A_D^T A_D from
 * the all-ones vector (up to 200 steps, relative change < 1e-12), as used for
 * L0 = 2 ||A_D||^2 (below Eq. 10).  Computed once per plan and cached;
 * synchronises `stream`. */
nlos_status nlos_plan_norm2(nlos_plan plan, int32_t masked, void* stream, double* out);

/* Host-side tables of a geometry, computed exactly as nlos_plan_create does
 * (FP64 on the host, no GPU needed), for inspection and testing:
 *   rz_i0[nt], rt_k0[nt] (int32): first tap of R_z / R_t^{-1} per bin;
 *   rz_w[3*nt] = (w0, w1, g) per v-bin, rt_w[3*nt] = (w0, w1, wt) per t-bin
 *   (float32, rounded from FP64);
 *   cols[nx*ny] (int32): sampled columns x*ny + y, ascending; *n_cols set.
 * Any output pointer may be NULL.  Same validation as nlos_plan_create. */
nlos_status nlos_geometry_tables(const nlos_geometry* geom, int32_t* rz_i0, float* rz_w, int32_t* rt_k0,
                                 float* rt_w, int32_t* cols, int32_t* n_cols);

/* tau = A u (apply_mask = 0) or tau = D A u with zeros on unsampled columns
 * (apply_mask != 0): Eq. 3 and A_D = D A (Sec. 3.1.2).  u_dev, tau_dev:
 * [nx][ny][nt] float32; they must not overlap. */
nlos_status nlos_forward(nlos_plan plan, const float* u_dev, float* tau_dev, int32_t apply_mask,
                         void* stream);

/* u = A^T tau (apply_mask = 0) or A_D^T tau = A^T D tau (apply_mask != 0,
 * unsampled columns of tau ignored): the transpose used in grad f = A_D^T
 * (A_D u - tau0) (Eq. 10-11). */
nlos_status nlos_adjoint(nlos_plan plan, const float* tau_dev, float* u_dev, int32_t apply_mask,
                         void* stream);

/* The directional (normal-weighted) confocal model of Sec. 2 for a given
 * normal field: tau(x', t) = sum over voxels x of u(x) ((x' - x) . n(x) / d)^2
 * / d^4 delta(2 d - t c), the confocal case (illumination and detection at
 * the same wall point x') of the paper's non-confocal direction-albedo
 * model, on the plan's discretisation of A (Eq. 3): the squared cosine is
 * expanded into six products of a voxel field and a scan-point weight, so
 * the operator is six applications of A.  normals_dev: device, float32
 * [3][nx][ny][nt] (the components n_x, n_y, n_z of each voxel's normal, the
 * wall at z = 0 and the scene at z > 0; any length: the weight scales with
 * |n|^2).  apply_mask as nlos_forward.  nlos_adjoint_directional is its
 * transpose in u for the same normals.  Two field-sized device buffers are
 * allocated in the plan on the first call.  The output must not overlap an
 * input (NLOS_ERR_INVALID_ARG); NLOS_ERR_OOM if the buffers cannot be
 * allocated.  Queued on `stream`, no host synchronisation. */
nlos_status nlos_forward_directional(nlos_plan plan, const float* u_dev, const float* normals_dev, float* tau_dev,
                                     int32_t apply_mask, void* stream);
nlos_status nlos_adjoint_directional(nlos_plan plan, const float* tau_dev, const float* normals_dev, float* u_dev,
                                     int32_t apply_mask, void* stream);

/* x = F^{-1}[F(rhs) / (c0 + c1 lambda(k))] on the periodic nx x ny x nt grid,
 * lambda(k) = sum_d 4 sin^2(pi k_d / N_d): the solve of (c0 I + c1 nabla^*
 * nabla) x = rhs of Eq. 11 (forward differences, unit spacing).  c0 > 0,
 * c1 >= 0.  rhs_dev and x_dev may alias. */
nlos_status nlos_solve(nlos_plan plan, const float* rhs_dev, float* x_dev, double c0, double c1,
                       void* stream);

/* phi_out = phi(kappa(u)) with kappa = div(grad u / sqrt(|grad u|^2 + eps^2))
 * (Sec. 3, below Eq. 4), forward-difference gradient and backward-difference
 * divergence, periodic; phi_kind = NLOS_PHI_*. */
nlos_status nlos_curvature_weight(nlos_plan plan, const float* u_dev, float* phi_dev, double a,
                                  double b, int32_t phi_kind, double eps, void* stream);

/* Reconstruct u from the measured transient tau0 (full grid [nx][ny][nt];
 * unsampled columns ignored) with Algorithm 1 or 2 (params->model).
 * u_out_dev receives u; tau_out_dev (nullable) receives Algorithm 2's
 * recovered signal tau.  stats_host (nullable) is filled after the run.
 * All iteration state lives on the device; device memory for it is allocated
 * on the first call with a given model and kept by the plan.  Synchronises
 * `stream` before returning (the statistics are read back). */
nlos_status nlos_reconstruct(nlos_plan plan, const nlos_params* params, const float* tau0_dev,
                             float* u_out_dev, float* tau_out_dev, nlos_stats* stats_host,
                             void* stream);

/* Prepare the reconstruction that nlos_reconstruct would run with exactly these
 * arguments (same parameters and the same device pointers) without running it:
 * allocate the solver state, compute the operator norm if the plan lacks it
 * (host synchronisation on `stream`), and capture and cache the CUDA graph of
 * the whole run (the plan keeps four).  A following nlos_reconstruct with the
 * same arguments is then one graph launch with no capture work, e.g. inside
 * a timed or latency-critical region.  Runs with a relative-energy stop
 * (eps_stop > 0) or a backtracking rule that can reject (L0 below
 * 1.5 ||A_D||^2) are graphs too: their iteration loop and backtracking loop
 * are conditional graph nodes decided on the device, with no host round trip.
 * *graphed (nullable) = 1 when a graph is cached, 0 when the run will not use
 * one (kernel timing enabled, or iters = 0).  Argument rules and errors as
 * nlos_reconstruct; nothing is written to u_out_dev or tau_out_dev. */
nlos_status nlos_reconstruct_prepare(nlos_plan plan, const nlos_params* params, const float* tau0_dev,
                                     float* u_out_dev, float* tau_out_dev, int32_t* graphed, void* stream);

/* nlos_reconstruct from host memory: tau0_host (nx*ny*nt float32) is
 * copied to a device buffer owned by the plan (three field-sized buffers,
 * allocated on the first call and reused), the reconstruction runs as
 * nlos_reconstruct does (one cached graph launch where possible), and u
 * (and, for model 2 when tau_out_host is not NULL, tau) is copied back to
 * u_out_host / tau_out_host.  Synchronises `stream` before returning.  Host
 * buffers may be pageable or page-locked (page-locked memory copies
 * asynchronously and faster); the caller owns them.  The end-to-end form of
 * the paper's reconstruction (Algorithms 1-2) for a caller whose data lives
 * on the host.  Errors as nlos_reconstruct, and NLOS_ERR_OOM if the device
 * buffers cannot be allocated. */
nlos_status nlos_reconstruct_host(nlos_plan plan, const nlos_params* params, const float* tau0_host,
                                  float* u_out_host, float* tau_out_host, nlos_stats* stats_host, void* stream);

/* Reconstruct n independent scenes at once.  plans[i] must be n distinct
 * plans (each owns its scratch; a plan appearing twice is rejected);
 * params[i], tau0[i] (device), u_out[i] (device) and tau_out[i] (device,
 * nullable array or entries) as for nlos_reconstruct (16-byte aligned).
 * Each scene runs on an internal stream forked from `stream` and joined back
 * to it, as one graph launch where possible, else with its iterations
 * enqueued round-robin, so the scenes' kernels overlap on the GPU.  A scene's
 * result does not depend on the other scenes of the batch.  Synchronises
 * before returning; stats (nullable) receives n entries.  The paper
 * reconstructs one scene at a time; this is the many-scene batched
 * execution. */
nlos_status nlos_reconstruct_batch(const nlos_plan* plans, const nlos_params* params, const float* const* tau0,
                                   float* const* u_out, float* const* tau_out, int32_t n, nlos_stats* stats,
                                   void* stream);

/* Serving.  A server owns a worker thread on the current device that admits
 * submitted reconstruction jobs in arrival order while fewer than max_slots
 * run and the device memory they need fits hbm_budget_bytes, keeps each
 * running job's state resident on the device, and advances all running jobs
 * together (continuous batching: a job submitted while others run joins them
 * as soon as a slot and memory free up).  A job that can never fit the budget
 * fails with NLOS_ERR_OOM.  nlos_submit copies tau0_host (full grid
 * [nx][ny][nt]) and the geometry (mask included) and returns at once;
 * u_out_host must stay valid until the job is reported done, when the result
 * has been written there.  nlos_poll returns NLOS_OK (done, *out filled),
 * NLOS_ERR_NOT_READY, or the job's error; nlos_wait blocks up to timeout_s.
 * nlos_job_times gives the seconds from submit to start and from submit to
 * completion of a finished job.  nlos_server_info fills 8 counters: queued,
 * running, completed, failed, peak running, device bytes in use, peak bytes,
 * budget.  nlos_server_destroy stops accepting jobs, cancels queued ones if
 * cancel_pending != 0 (they end with NLOS_ERR_TIMEOUT), waits at most
 * timeout_s for the rest, joins the worker and frees everything; it returns
 * NLOS_ERR_TIMEOUT if jobs were still unfinished at the deadline (queued ones
 * are then cancelled; running ones are finished by the worker before it
 * exits).  Submit, poll, wait, job_times and info are thread-safe. */
nlos_status nlos_server_create(size_t hbm_budget_bytes, int32_t max_slots, nlos_server* out);
nlos_status nlos_submit(nlos_server server, const nlos_geometry* geom, const nlos_params* params,
                        const float* tau0_host, float* u_out_host, uint64_t* job_id);
nlos_status nlos_poll(nlos_server server, uint64_t job_id, nlos_stats* out);
nlos_status nlos_wait(nlos_server server, uint64_t job_id, double timeout_s, nlos_stats* out);
nlos_status nlos_job_times(nlos_server server, uint64_t job_id, double* queued_s, double* total_s);
nlos_status nlos_server_info(nlos_server server, int64_t* counters8);
/* Warm-up before traffic.  The first job of a geometry makes the worker
 * build that geometry's plan (tables, kernel spectrum, tuned launch shapes,
 * ||A_D||^2 by power iteration), and the first job of each (geometry, model)
 * in a new job context also allocates the context and captures its graph;
 * while the worker does that no other job is admitted or retired.
 * nlos_server_prepare does this work ahead of time: it builds the plan of
 * `geom` and keeps `contexts` idle job contexts of the kind `params` needs,
 * each with the graph of a run of `params` captured, so later jobs with the
 * same geometry and parameters start at once.  Existing idle contexts of that
 * kind count towards `contexts`; new ones are created only while they fit the
 * HBM budget (nothing is evicted for them), and *ready (nullable) receives
 * how many are ready.  Blocks until the worker has done it or timeout_s has
 * passed (NLOS_ERR_TIMEOUT; the warm-up still completes).  Thread-safe;
 * NLOS_ERR_BUSY after nlos_server_destroy has begun. */
nlos_status nlos_server_prepare(nlos_server server, const nlos_geometry* geom, const nlos_params* params,
                                int32_t contexts, double timeout_s, int32_t* ready);
nlos_status nlos_server_destroy(nlos_server server, int32_t cancel_pending, double timeout_s);

/* The periodic FFT solve of nlos_solve for callers that cannot allocate
 * device memory when they solve: code whose device memory is owned by
 * another allocator (a framework's caching pool) or capped by a fixed
 * budget, and real-time loops that must stay off the driver's allocation
 * path, which can synchronise the whole device.  The paper has no
 * counterpart: this is a deployment variant of the solve above.
 *
 * No plan: pass the grid (nx == ny, powers of two, 8 <= nx <= 64,
 * 16 <= nt <= 512), rhs_dev and x_dev ([nx][ny][nt] float32, may alias),
 * c0 > 0 and c1 >= 0.  Nothing is allocated: the spectrum scratch is a
 * static device array of 64 * 64 * 257 complex values (8 MiB) that every
 * GPU loading the library holds until the process exits; larger grids
 * return NLOS_ERR_INVALID_ARG (use nlos_solve).  The first call on a device
 * (with that device current) is the set-up: it looks up the array's device
 * address, fills small twiddle tables, sets the kernels' shared-memory
 * limits and synchronises the device; later calls only launch kernels.
 * All calls share the scratch: calls whose kernels overlap on the GPU
 * (other streams or other host threads) race and must be serialised by the
 * caller.  It keeps the last call's contents, but no call reads a value an
 * earlier call left behind.  Queued on `stream`, no host synchronisation
 * after the set-up. */
nlos_status nlos_solve_static(int32_t nx, int32_t ny, int32_t nt, const float* rhs_dev, float* x_dev, double c0,
                              double c1, void* stream);

/* Midpoint conversion of non-confocal transients into confocal ones
 * (Sec. 4, evaluation on non-confocal data: the confocal solvers run on a
 * non-confocal measurement after the midpoint approximation, which the
 * paper cites from f-k migration without stating it).
 *
 * Input: tau_nc_dev, device, float32 [nx][ny][nt], the transients of a
 * non-confocal scan with the laser fixed at the wall point
 * (laser_x_m, laser_y_m) and the detector at the scan grid centres
 * x_i = (i + 1/2 - nx/2) wall_width_m / nx (y likewise), bins of
 * bin_width_s.  Output: tau_c_dev, device, float32 [nx][ny][nt], the
 * confocal transients at the midpoints m_ij = (laser + s_ij) / 2, i.e. a
 * confocal scan of wall width wall_width_m / 2 centred at laser / 2, to be
 * reconstructed with a plan of that wall width.  Confocal bin k (centre
 * t_k = (k + 1/2) dt) reads the non-confocal record at the time
 * sqrt(t_k^2 + |s_ij - laser|^2 / c^2), exact for scatterers on the wall
 * normal through the midpoint, by two-tap linear interpolation between bin
 * centres (zero past the last bin); the amplitude is not changed.  The tap
 * positions are accurate to about 1e-11 bins (FP32 with a compensated square
 * root), the interpolation is FP32.
 *
 * nx, ny, nt powers of two >= 2, nt <= 2048; bin_width_s > 0, wall_width_m > 0, finite
 * laser coordinates; the buffers 4-byte aligned and not overlapping
 * (NLOS_ERR_INVALID_ARG otherwise).  The caller owns both buffers.  Queued
 * on `stream`, no host synchronisation, no allocation. */
nlos_status nlos_midpoint_confocal(int32_t nx, int32_t ny, int32_t nt, double bin_width_s, double wall_width_m,
                                   double laser_x_m, double laser_y_m, const float* tau_nc_dev, float* tau_c_dev,
                                   void* stream);

/* Self-test of the bounded waits (failure detection without a GPU fault).
 * The kernels that wait on an mbarrier (the TMA tile loads of the t-passes,
 * the tensor-core lateral stage) give up after a time limit, record
 * NLOS_ERR_TIMEOUT and run to their end, so the context stays usable.  This
 * launches one CTA on `stream` that waits with the same code on an mbarrier
 * whose expected bytes no copy delivers; the wait gives up after wait_ms
 * milliseconds (1 to 5000) and the kernel writes NLOS_ERR_TIMEOUT to
 * *status_dev (a device int32 the caller owns; NLOS_OK had the wait
 * completed).  Queued on `stream`, no host synchronisation.  Errors: wait_ms
 * out of range or a null pointer (NLOS_ERR_INVALID_ARG), CUDA
 * (NLOS_ERR_CUDA). */
nlos_status nlos_selftest_wait_timeout(int32_t wait_ms, int32_t* status_dev, void* stream);

/* Per-launch timing of a plan's kernels, for profiling.  When enabled, every
 * kernel the plan launches is bracketed by a pair of CUDA events recorded on
 * its launch stream.  nlos_timing_read synchronises the device, returns per
 * category the summed milliseconds and launch counts (categories: 0 lateral
 * convolution, 1 forward t-pass, 2 inverse t-pass, 3 adjoint end / solve
 * rhs, 4 lateral solve, 5 periodic t-FFT, 6 periodic inverse t-FFT,
 * 7 pre-solve stencil, 8 post-solve stencil, 9 scalar and small kernels,
 * 10 kernel spectrum), fills n entries and resets the record. */
nlos_status nlos_timing_enable(nlos_plan plan, int32_t enable);
nlos_status nlos_timing_read(nlos_plan plan, double* ms, int32_t* launches, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* NLOS_H */
