// Shared definitions of the CUDA implementation: error plumbing, complex
// helpers, the plan structure and the device-side scalar block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/nlos.h"

namespace nlos {

// ---------------------------------------------------------------------------
// Errors: every internal failure becomes a status plus a thread-local message.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
nlos_status fail(nlos_status code, const std::string& msg);
nlos_status cuda_fail(cudaError_t e, const char* what);

#define NLOS_CUDA(call)                                              \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return ::nlos::cuda_fail(e_, #call);      \
  } while (0)

#define NLOS_LAUNCH_CHECK(name)                                      \
  do {                                                               \
    cudaError_t e_ = cudaGetLastError();                             \
    if (e_ != cudaSuccess) return ::nlos::cuda_fail(e_, name);       \
  } while (0)

#define NLOS_TRY(call)                                               \
  do {                                                               \
    nlos_status s_ = (call);                                         \
    if (s_ != NLOS_OK) return s_;                                    \
  } while (0)

// ---------------------------------------------------------------------------
// Complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
// On the device the complex add and subtract are single paired-FP32
// instructions (sm_100 and later): both components in one issue slot, each
// rounded to nearest exactly as a scalar add would be.  a - b is computed as
// the fused b * (-1) + a, whose one rounding of the exact a - b is the
// subtraction's result.
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Device scalar block of one reconstruction: everything the iteration's
// kernels need that changes from one iteration to the next lives here, so an
// iteration is a fixed launch sequence (graph-capturable).
// ---------------------------------------------------------------------------
struct DevScalars {
  double L;           // current Lipschitz estimate of the linearised u-step
  double t;           // FISTA t_k
  double beta_prev;   // weight that formed the current u-bar (cached A u-bar)
  double beta;        // weight for the next extrapolation (set after the test)
  double t_next, beta_next;  // what the next accepted test sets t and beta to ((1 + sqrt(1 + 4 t^2)) / 2 and
                             // (t - 1) / t_next from the current t): set at the start and at the end of
                             // every iteration, so the post stencil reads the extrapolation weight
                             // without waiting for the test
  double E_prev;      // energy before this iteration
  double E, dE;       // energy of the last iteration and its change E_prev - E (the relative change
                      // |dE| / |E| is formed on the host)
  double f_fit;       // data term of the last accepted iterate
  double L_norm_ok;   // L above which acceptance is guaranteed (||A_D||^2 (1 + margin))
  int32_t iter;       // iterations done
  int32_t backtracks; // total rejections
  int32_t restarts;   // FISTA restarts
  int32_t status;     // NLOS_OK or an error code
  int32_t accept;     // outcome of the last test (1 accepted)
  int32_t rej_iter;   // rejections in the current iteration
  int32_t stop;       // relative-energy stop reached
  int32_t trips;      // trips of a graph-resident iteration loop
  uint32_t arrivals;  // blocks of the fused Algorithm-1 post step that have finished (its last block ends
                      // the iteration and resets the count)
  double pres2;       // ||v - grad u||^2 of the last iteration (its root is taken on the host)
  double test_lhs, test_rhs;  // ||A d||^2 and L ||d||^2 of the last test
};

// Number of FP64 partial-sum slots per block used by the reductions.
constexpr int kMaxTerms = 8;

// Per-thread sums of T terms in compensated FP32 (Kahan: s - c carries the
// sum to about two roundings regardless of the term count), reduced across a
// warp without rounding loss (TwoSum on hi/lo pairs) and converted to FP64
// once per warp (block_reduce_acc).  FP64 instructions issue at a small
// fraction of the FP32 rate on this GPU: an FP64 add per term, or even per
// chunk of 16 terms, kept the FP64 pipe 40-60 % busy in the reduction
// epilogues of otherwise FP32 kernels.  The order of every operation is fixed,
// so the sums are reproducible bit for bit.
template <int T>
struct SumAcc {
  float s[T], c[T];
  __device__ __forceinline__ SumAcc() {
#pragma unroll
    for (int t = 0; t < T; ++t) {
      s[t] = 0.f;
      c[t] = 0.f;
    }
  }
  __device__ __forceinline__ void add(int t, float v) {
    const float y = v - c[t];
    const float u = s[t] + y;
    c[t] = (u - s[t]) - y;
    s[t] = u;
  }
};

// Block-wide sums of the accumulators of every thread; thread 0 writes
// partials[blockIdx.x * kMaxTerms + t].  Every thread of the block calls it
// (blockDim.x a multiple of 32).
template <int T>
__device__ __forceinline__ void block_reduce_acc(const SumAcc<T>& ca, double* partials) {
  __shared__ double red[32][T];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    float hi = ca.s[t], lo = -ca.c[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
      const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
      const float sum = hi + h2;  // TwoSum: sum + err = hi + h2 exactly
      const float bb = sum - hi;
      const float err = (hi - (sum - bb)) + (h2 - bb);
      hi = sum;
      lo = lo + l2 + err;
    }
    if (lane == 0) red[warp][t] = (double)hi + (double)lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int t = 0; t < T; ++t) {
      double acc = 0.0;
      for (int w = 0; w < nw; ++w) acc += red[w][t];
      partials[(size_t)blockIdx.x * kMaxTerms + t] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct SolverState;  // defined in admm.cu

struct LateralTC;  // optional tensor-core lateral stage (conv_tc.cu)

struct Plan {
  int nx, ny, nt;
  double bin_width_s, wall_width_m, range_m;
  int radiometry;
  int ncols;          // number of sampled columns
  bool full_mask;     // every column sampled
  int lattice_rx = -1;  // r when every sampled column has x = r (mod 4) and some column is unsampled, else -1
  int lattice_ry = -1;  // r' when the sampled columns are exactly x = lattice_rx, y = r' (mod 4), else -1
  int device;
  int sms;            // streaming multiprocessors of the device (queried at plan creation); sets the
                      // grid of the grid-stride reductions, hence their summation order

  // host tables (FP64-derived, stored as the device uses them)
  std::vector<int32_t> h_rz_i0, h_rt_k0, h_cols;
  std::vector<float> h_rz_w, h_rt_w;  // 3 per bin
  std::vector<uint8_t> h_mask;

  // device tables
  int32_t* d_rz_i0 = nullptr;    // [nt]
  float* d_rz_w = nullptr;       // [3 nt]: w0, w1, g
  int32_t* d_rzt_start = nullptr;// [nt+1]: v-bins j with i0_j == i are [start[i], start[i+1])
  int32_t* d_rt_k0 = nullptr;    // [nt]
  float* d_rt_w = nullptr;       // [3 nt]: w0, w1, wt
  int32_t* d_rtt_start = nullptr;// [nt+1]: t-bins k with k0_k == j are [start[j], start[j+1])
  int32_t* d_cols = nullptr;     // [ncols] sampled columns x*ny + y
  int32_t* d_colpos = nullptr;   // [nx*ny] position of a column in d_cols, -1 if unsampled
  float2* d_tw2t = nullptr;      // [2 nt]  exp(-2 pi i n / (2 nt))
  float2* d_twt = nullptr;       // [nt]    exp(-2 pi i n / nt)
  float2* d_twx = nullptr;       // [2 nx]  exp(-2 pi i n / (2 nx))
  float2* d_twy = nullptr;       // [2 ny]
  float* d_lamx = nullptr;       // [nx] 4 sin^2(pi k / nx)
  float* d_lamy = nullptr;       // [ny]
  float* d_lamt = nullptr;       // [nt]
  float2* d_H = nullptr;         // [(nt+1)][(nx+1)][(ny+1)] cone-kernel spectrum
  // device forms of the resampling, weights pre-multiplied (FP64 -> float):
  // forward taps {w0*g, w1*g, i0 (int bits), 0} per output bin, and the
  // transposes as CSR rows of {weight, input index (int bits)}
  float4* d_rz_f4 = nullptr;     // [nt]  R_z
  float4* d_rt_f4 = nullptr;     // [nt]  R_t^{-1}
  int32_t* d_rzT_ptr = nullptr;  // [nt+1]
  float2* d_rzT_ent = nullptr;   // [<= 2 nt]
  int32_t* d_rtT_ptr = nullptr;  // [nt+1]
  float2* d_rtT_ent = nullptr;   // [<= 2 nt]

  // scratch owned by the plan
  float2* d_S = nullptr;         // [(nt+1)][nx][ny] padded t-spectrum (adjoint side)
  float2* d_S2 = nullptr;        // [(nt+1)][nx][ny] padded t-spectrum (forward side)
  float2* d_Sc = nullptr;        // [(nt+1)][ncols] compact spectrum of sampled columns
  float2* d_Sp = nullptr;        // [(nt/2+1)][nx][ny] periodic spectrum (solve)
  float* d_tmpc = nullptr;       // [ncols][nt] compact transient scratch
  double* d_partials = nullptr;  // reduction partials
  float* d_io[3] = {nullptr, nullptr, nullptr};  // tau0, u, tau of nlos_reconstruct_host (allocated on use)
  float* d_dir[2] = {nullptr, nullptr};  // scratch fields of the directional model (allocated on use)
  int partial_blocks = 0;
  DevScalars* d_scal = nullptr;  // scratch scalars (norm, diagnostics)

  double norm2_masked = -1.0, norm2_full = -1.0;
  SolverState* solver[3] = {nullptr, nullptr, nullptr};
  bool owns_tables = true;  // false for a per-job workspace clone (tables and H shared)

  // CUDA graphs of whole reconstructions (init, iterations, finish), keyed by
  // the parameters and the caller's buffers; replayed with one launch.
  struct GraphEntry {
    nlos_params p;
    const float* tau0;
    float* u_out;
    float* tau_out;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t capture_stream = nullptr;
  // parallel branch of a captured iteration (JobRun::aux) and its events
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
  // streams that capture the bodies of conditional nodes (iteration loop,
  // pointer-phase switch, backtracking loop)
  cudaStream_t body_stream[3] = {nullptr, nullptr, nullptr};

  // lateral stage as DFT-matrix products on the tensor cores
  // (nlos_plan_set_lateral); nullptr: the FFT kernels
  LateralTC* lateral = nullptr;

  // optional per-launch timing (nlos_timing_enable): event pairs recorded
  // around every kernel launch on the launch stream, harvested on read.
  mutable bool timing = false;
  mutable std::vector<cudaEvent_t> ev;
  mutable std::vector<int> ev_cat;
  mutable size_t ev_used = 0;
};

// Launch categories of the timer (index into nlos_timing_read's arrays).
enum KernelCat {
  KC_CONV = 0,      // k_conv: lateral padded convolution per kt plane
  KC_TFWD = 1,      // k_tfwd: R_z or R_t^T + padded t-FFT
  KC_TINV = 2,      // k_tinv: padded inverse t-FFT + R_t^{-1} (+ fit)
  KC_TADJ = 3,      // k_tadj: inverse t-FFT + R_z^T (+ solve rhs, periodic t-FFT)
  KC_SXY = 4,       // k_sxy: lateral periodic solve
  KC_SFWD = 5,      // k_sfwd: periodic t-FFT of a field
  KC_SINV = 6,      // k_sinv: periodic inverse t-FFT (k_sinv_rz: + R_z forward t-pass)
  KC_PRE = 7,       // k_pre1 / k_pre2: shrinkage + nabla^* stencils
  KC_POST = 8,      // k_post1 / k_post2: multipliers, curvature, extrapolation
  KC_SMALL = 9,     // one-thread scalar kernels, fills, gathers, reductions
  KC_KSPEC = 10,    // k_kspec: cone-kernel spectrum (plan time)
  KC_COUNT = 11
};

// RAII timer: records an event pair around the launches in its scope when
// timing is enabled on the plan.
struct KTimer {
  const Plan& P;
  cudaStream_t st;
  size_t slot;
  bool on;
  KTimer(const Plan& p, int cat, cudaStream_t s);
  ~KTimer();
};

// The directional (normal-weighted) model of Sec. 2 for the normal field
// normals = [3][nx][ny][nt] (directional.cu): six applications of A.
nlos_status apply_forward_directional(Plan& P, const float* u, const float* normals, float* tau, bool masked,
                                      cudaStream_t st);
nlos_status apply_adjoint_directional(Plan& P, const float* tau, const float* normals, float* u, bool masked,
                                      cudaStream_t st);

// Operator applications (admm.cu)
nlos_status apply_forward(const Plan& P, const float* u, float* out, bool compact, cudaStream_t st);
nlos_status apply_adjoint(const Plan& P, const float* r, float* u, bool compact, cudaStream_t st);
nlos_status gather_columns(const Plan& P, const float* full, float* compact, cudaStream_t st);
nlos_status apply_solve(const Plan& P, const float* rhs, float* x, double c0, double c1, cudaStream_t st);
nlos_status apply_curvature_weight(const Plan& P, const float* u, float* ph, double a, double b, int kind, double eps,
                                   cudaStream_t st);
nlos_status plan_norm2(Plan& P, bool masked, cudaStream_t st, double* out);
nlos_status reconstruct(Plan& P, const nlos_params& p, const float* tau0, float* u_out, float* tau_out,
                        nlos_stats* stats, cudaStream_t st);
// The same from host memory through the plan's own device buffers (copies in
// and out on st, then synchronises).
nlos_status reconstruct_host(Plan& P, const nlos_params& p, const float* tau0_host, float* u_out_host,
                             float* tau_out_host, nlos_stats* stats, cudaStream_t st);
void free_solver(SolverState* s);

// Per-job workspace: a copy of `base` that shares its read-only device tables
// and kernel spectrum but owns fresh scratch spectra and solver state, so
// several jobs of one geometry can run concurrently (plan.cu).
Plan* plan_clone_workspace(const Plan& base, nlos_status* status);
void plan_release(Plan* P);
// Bytes of device memory a workspace clone plus the solver state of `model`
// occupy (the shared tables excluded), and of the shared tables alone.
// Device bytes of a workspace clone plus the solver state of `model` (1, 2,
// or 3 = both, a model-2 run with an Algorithm-1 warm stage).
size_t workspace_bytes(const Plan& P, int model);
size_t shared_table_bytes(const Plan& P);
nlos_status create_plan_internal(const nlos_geometry* g, cudaStream_t st, Plan** out);
// Pre-set the shared-memory limits of the stencil kernels (admm.cu).
nlos_status prepare_stencils();

// One reconstruction as a sequence of enqueued steps (admm.cu).
struct JobRun {
  Plan* P = nullptr;
  SolverState* s = nullptr;
  nlos_params p{};
  const float* tau0 = nullptr;  // device, full grid
  float* u_out = nullptr;       // device
  float* tau_out = nullptr;     // device, nullable (model 2)
  cudaStream_t st = nullptr;
  double norm2 = 0.0, L0 = 0.0, L_host = 0.0;
  int restart = 0;
  int it = 0;
  int cur = 0, prev = 1, nxt = 2;  // rotation of the cached A u iterates
  bool done = false;
  // Algorithm-1 warm stage of a model-2 run: while phase == 1, p holds the
  // warm-stage parameters and main_p the run's own; job_step switches to
  // Algorithm 2 (phase 2) when the warm stage is done.
  int phase = 0;
  nlos_params main_p{};
  // While a graph-resident loop is being captured: the stream on which the
  // backtracking loop body is captured (the u-step then repeats on the device
  // until the test accepts); nullptr otherwise.
  cudaStream_t bt_stream = nullptr;
  // While a graph is captured: a second stream and a fork/join event pair, so
  // that work of an iteration that does not depend on the rest of it (the
  // Algorithm-1 pre stencil next to the start of A_D^T) becomes a parallel
  // branch of the graph; nullptr otherwise (everything on st).
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};
// Allocates the solver state on first use, computes (once per plan) the
// operator norm with a host synchronisation, and enqueues the initial state.
nlos_status job_init(JobRun& j);
// Enqueues one iteration.  Needs the host only while the backtracking rule can
// still reject (L < 1.5 ||A_D||^2) or when eps_stop > 0.
nlos_status job_step(JobRun& j);
bool job_async(const JobRun& j);
// Enqueues the copies of the result and of the scalar block to the host.
nlos_status job_finish(JobRun& j);
// After the job's stream has completed: statistics and final status.
nlos_status job_collect(JobRun& j, nlos_stats* stats);
// Enqueue the whole reconstruction of j on `launch` as one CUDA-graph launch
// (captured on first use for these parameters and buffers, then cached in the
// plan).  Runs with a fixed iteration count and no possible rejection are
// captured unrolled; runs with a relative-energy stop or a backtracking rule
// that can reject are captured as a device-driven loop of conditional nodes.
// Sets *used = false, enqueuing nothing, only when the plan's kernels are
// being timed.
nlos_status job_enqueue_graph(JobRun& j, cudaStream_t launch, bool* used);
// Captures and caches j's graph without launching it (*ready = false when the
// run would not use a graph: kernel timing on, or no iterations).
nlos_status job_prepare_graph(JobRun& j, cudaStream_t st, bool* ready);
nlos_status reconstruct_prepare(Plan& P, const nlos_params& p, const float* tau0, float* u_out, float* tau_out,
                                bool* ready, cudaStream_t st);
// Checks the parameter rules of nlos_params (model, counts, factors, penalties).
nlos_status validate_params(const nlos_params& p, const char* who);
void free_graphs(Plan* P);

// Launch configuration helpers
inline int div_up(int a, int b) { return (a + b - 1) / b; }
// Streaming multiprocessors of the current device (queried once per device).
int device_sm_count();
// Grid of the grid-stride stencil and reduction kernels: eight blocks per SM,
// at most the 4096 partial-sum slots a solver state holds.
inline int stencil_blocks(const Plan& P) { return P.sms * 8 < 4096 ? P.sms * 8 : 4096; }

// Raise a kernel's dynamic shared-memory limit once per (device, kernel):
// the attribute call is not repeated on every launch (nor during a stream
// capture once the kernel has been launched before).
nlos_status ensure_smem_attr(const void* kernel, size_t bytes);
template <typename K>
inline nlos_status ensure_smem(K kernel, size_t bytes) {
  return ensure_smem_attr(reinterpret_cast<const void*>(kernel), bytes);
}

}  // namespace nlos
