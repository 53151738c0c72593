// Many reconstructions on one GPU: the batch entry point and the serving
// runtime (continuous batching with admission by free HBM).
//
// Each job runs its ADMM iterations (job_init / job_step / job_finish of
// admm.cu) on its own CUDA stream, with its own workspace (scratch spectra and
// solver state) and the read-only tables of its geometry shared with every
// other job of that geometry.  A host loop advances every active job by one
// enqueued iteration per round, so the kernels of all active jobs are queued
// side by side and overlap on the device; a job's arithmetic (launch
// sequence, reduction order) does not depend on its neighbours, so its result
// is the same alone, in a batch or in the served mix.
#include <atomic>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>

#include "passes.cuh"

namespace nlos {

// ---------------------------------------------------------------------------
// Batch: n independent plans, one stream each, iterations interleaved.
// ---------------------------------------------------------------------------
static nlos_status reconstruct_batch(Plan** plans, const nlos_params* params, const float* const* tau0,
                                     float* const* u_out, float* const* tau_out, int n, nlos_stats* stats,
                                     cudaStream_t caller) {
  std::vector<cudaStream_t> streams(n, nullptr);
  std::vector<JobRun> jobs(n);
  cudaEvent_t start_ev = nullptr;
  nlos_status st = NLOS_OK;
  auto cleanup = [&]() {
    for (cudaStream_t s : streams)
      if (s) cudaStreamDestroy(s);
    if (start_ev) cudaEventDestroy(start_ev);
  };
  if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(start_ev, caller) != cudaSuccess) {
    cleanup();
    return cuda_fail(cudaGetLastError(), "batch: start event");
  }
  // stream priorities by scene size: the smallest scenes (whose kernels are
  // short and cannot fill the GPU) highest, so their blocks are dispatched as
  // soon as the large scenes' blocks free an SM instead of waiting behind them
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  std::vector<size_t> vols(n);
  for (int i = 0; i < n; ++i) vols[i] = (size_t)plans[i]->nx * plans[i]->ny * plans[i]->nt;
  std::vector<size_t> sizes(vols);
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  for (int i = 0; i < n && st == NLOS_OK; ++i) {
    const int rank = (int)(std::lower_bound(sizes.begin(), sizes.end(), vols[i]) - sizes.begin());
    const int prio = std::min(prio_greatest + rank, prio_least);  // greatest is the numerically lowest
    cudaError_t e = cudaStreamCreateWithPriority(&streams[i], cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(streams[i], start_ev, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "batch: stream");
    JobRun& j = jobs[i];
    j.P = plans[i];
    j.p = params[i];
    j.tau0 = tau0[i];
    j.u_out = u_out[i];
    j.tau_out = tau_out ? tau_out[i] : nullptr;
    j.st = streams[i];
  }
  // whole reconstructions as graph launches where possible; the rest are
  // stepped round robin, one enqueued iteration of every unfinished job per round
  std::vector<char> graphed(n, 0);
  for (int i = 0; i < n && st == NLOS_OK; ++i) {
    bool used = false;
    st = job_enqueue_graph(jobs[i], streams[i], &used);
    graphed[i] = used;
    if (st == NLOS_OK && !used) st = job_init(jobs[i]);
    if (used) jobs[i].done = true;
  }
  bool left = st == NLOS_OK;
  while (left && st == NLOS_OK) {
    left = false;
    for (int i = 0; i < n && st == NLOS_OK; ++i) {
      if (jobs[i].done) continue;
      st = job_step(jobs[i]);
      left = left || !jobs[i].done;
    }
  }
  for (int i = 0; i < n && st == NLOS_OK; ++i)
    if (!graphed[i]) st = job_finish(jobs[i]);
  // join: the caller's stream waits for every job
  for (int i = 0; i < n; ++i) {
    if (!streams[i]) continue;
    cudaEvent_t done_ev;
    if (cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done_ev, streams[i]);
      cudaStreamWaitEvent(caller, done_ev, 0);
      cudaEventDestroy(done_ev);
    }
  }
  for (int i = 0; i < n; ++i)
    if (streams[i]) {
      cudaError_t e = cudaStreamSynchronize(streams[i]);
      if (e != cudaSuccess && st == NLOS_OK) st = cuda_fail(e, "batch: job stream");
    }
  nlos_status first_err = st;
  if (st == NLOS_OK)
    for (int i = 0; i < n; ++i) {
      nlos_status si = job_collect(jobs[i], stats ? &stats[i] : nullptr);
      if (si != NLOS_OK && first_err == NLOS_OK) first_err = si;
    }
  cleanup();
  return first_err;
}

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------
using Clock = std::chrono::steady_clock;

struct GeomKey {
  int nx, ny, nt, radiometry;
  double bw, wall;
  std::vector<uint8_t> mask;
  bool operator<(const GeomKey& o) const {
    if (nx != o.nx) return nx < o.nx;
    if (ny != o.ny) return ny < o.ny;
    if (nt != o.nt) return nt < o.nt;
    if (radiometry != o.radiometry) return radiometry < o.radiometry;
    if (bw != o.bw) return bw < o.bw;
    if (wall != o.wall) return wall < o.wall;
    return mask < o.mask;
  }
};

enum JobState { JOB_QUEUED = 0, JOB_RUNNING = 1, JOB_DONE = 2, JOB_FAILED = 3, JOB_CANCELLED = 4 };

// Reusable device context of one running job (recycled per geometry + model).
struct JobCtx {
  GeomKey key;
  int model = 0;
  Plan* ws = nullptr;       // workspace clone
  float* d_tau0 = nullptr;  // device copy of the measurement
  float* d_u = nullptr;     // device result
  float* h_u = nullptr;     // pinned staging of the result
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  size_t bytes = 0;
};

struct Job {
  uint64_t id = 0;
  GeomKey key;
  nlos_params params{};
  std::vector<float> tau0;  // host copy taken at submit
  float* u_out_host = nullptr;
  JobState state = JOB_QUEUED;
  nlos_status status = NLOS_OK;
  nlos_stats stats{};
  Clock::time_point t_submit, t_start, t_done;
  JobCtx* ctx = nullptr;
  JobRun run;
  bool finishing = false;
  bool graphed = false;  // the whole run was enqueued as one graph launch
};

struct BaseEntry {
  Plan* plan = nullptr;
  size_t bytes = 0;
};

// A warm-up request (nlos_server_prepare): the geometry's base plan and
// `want` idle job contexts whose graphs for `params` are already captured.
struct Prep {
  GeomKey key;
  nlos_params params{};
  int want = 0;
  int ready = 0;
  nlos_status status = NLOS_OK;
  bool done = false;
};

struct ServerInfo {
  int64_t queued = 0, active = 0, completed = 0, failed = 0, peak_active = 0;
  size_t bytes_in_use = 0, bytes_peak = 0;
};

struct Server {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker (new jobs, shutdown)
  std::condition_variable done_cv;  // wakes waiters (job finished)
  std::deque<Job*> incoming;
  std::deque<std::shared_ptr<Prep>> preps;  // warm-up requests, handled before admission
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_id = 1;
  bool stopping = false;
  bool cancel_pending = false;
  ServerInfo info;
  std::thread worker;
  // worker-owned
  std::deque<Job*> pending;
  std::vector<Job*> active;
  std::map<GeomKey, BaseEntry> bases;
  std::multimap<std::pair<GeomKey, int>, JobCtx*> idle;
  size_t used = 0;
  cudaStream_t setup_stream = nullptr;
};

static GeomKey make_key(const nlos_geometry& g) {
  GeomKey k{g.nx, g.ny, g.nt, g.radiometry, g.bin_width_s, g.wall_width_m, {}};
  if (g.mask) k.mask.assign(g.mask, g.mask + (size_t)g.nx * g.ny);
  return k;
}

static nlos_geometry geom_of(const GeomKey& k) {
  nlos_geometry g{};
  g.nx = k.nx;
  g.ny = k.ny;
  g.nt = k.nt;
  g.bin_width_s = k.bw;
  g.wall_width_m = k.wall;
  g.radiometry = k.radiometry;
  g.mask = k.mask.empty() ? nullptr : k.mask.data();
  return g;
}

static void free_ctx(JobCtx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->ws) plan_release(c->ws);
  if (c->d_tau0) cudaFree(c->d_tau0);
  if (c->d_u) cudaFree(c->d_u);
  if (c->h_u) cudaFreeHost(c->h_u);
  if (c->done) cudaEventDestroy(c->done);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

// Solver state a job needs: its model, or 3 for a model-2 job with an
// Algorithm-1 warm stage (both solver states live in its workspace).
static int ctx_kind(const nlos_params& p) { return p.model == 2 && p.warm_start_iters > 0 ? 3 : p.model; }

static size_t ctx_bytes(const Plan& base, int model) {
  const size_t F = (size_t)base.nx * base.ny * base.nt * sizeof(float);
  return workspace_bytes(base, model) + 2 * F;
}

// Base plan (tables, kernel spectrum, operator norms) of a geometry, created once.
static nlos_status get_base(Server* S, const GeomKey& key, int model, BaseEntry** out) {
  auto it = S->bases.find(key);
  if (it == S->bases.end()) {
    nlos_geometry g = geom_of(key);
    Plan* P = nullptr;
    NLOS_TRY(create_plan_internal(&g, S->setup_stream, &P));
    BaseEntry e;
    e.plan = P;
    e.bytes = shared_table_bytes(*P) + workspace_bytes(*P, 0);
    S->used += e.bytes;
    it = S->bases.emplace(key, e).first;
  }
  double n2 = 0.0;
  if (model != 2) NLOS_TRY(plan_norm2(*it->second.plan, true, S->setup_stream, &n2));
  if (model != 1) NLOS_TRY(plan_norm2(*it->second.plan, false, S->setup_stream, &n2));
  *out = &it->second;
  return NLOS_OK;
}

static void release_idle(Server* S, size_t need) {
  // free recycled contexts until `need` more bytes fit (oldest first)
  for (auto it = S->idle.begin(); it != S->idle.end() && S->used + need > S->budget;) {
    S->used -= it->second->bytes;
    free_ctx(it->second);
    it = S->idle.erase(it);
  }
}

static nlos_status create_ctx(Server* S, const GeomKey& key, int kind, BaseEntry* base, JobCtx** out) {
  JobCtx* c = new JobCtx();
  c->key = key;
  c->model = kind;
  c->bytes = ctx_bytes(*base->plan, c->model);
  const size_t F = (size_t)base->plan->nx * base->plan->ny * base->plan->nt * sizeof(float);
  nlos_status s = NLOS_OK;
  c->ws = plan_clone_workspace(*base->plan, &s);
  if (s == NLOS_OK && cudaMalloc(&c->d_tau0, F) != cudaSuccess) s = fail(NLOS_ERR_OOM, "server: device tau0");
  if (s == NLOS_OK && cudaMalloc(&c->d_u, F) != cudaSuccess) s = fail(NLOS_ERR_OOM, "server: device u");
  if (s == NLOS_OK && cudaMallocHost(&c->h_u, F) != cudaSuccess) s = fail(NLOS_ERR_OOM, "server: pinned staging");
  // smaller grids get higher stream priority (one level per factor 2 of
  // voxels above 2^20): their short kernels take SMs as soon as a large job's
  // blocks free them, which cuts the latency of small jobs in a mixed load
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  int lv = 0;
  for (size_t v = F / sizeof(float); v > ((size_t)1 << 20); v >>= 1) ++lv;
  const int prio = std::min(prio_greatest + lv, prio_least);
  if (s == NLOS_OK && cudaStreamCreateWithPriority(&c->st, cudaStreamNonBlocking, prio) != cudaSuccess)
    s = fail(NLOS_ERR_CUDA, "server: stream");
  if (s == NLOS_OK && cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess)
    s = fail(NLOS_ERR_CUDA, "server: event");
  if (s != NLOS_OK) {
    cudaGetLastError();
    free_ctx(c);
    return s;
  }
  S->used += c->bytes;
  *out = c;
  return NLOS_OK;
}

static nlos_status acquire_ctx(Server* S, Job* jb, BaseEntry* base, JobCtx** out) {
  const auto k = std::make_pair(jb->key, ctx_kind(jb->params));
  auto it = S->idle.find(k);
  if (it != S->idle.end()) {
    *out = it->second;
    S->idle.erase(it);
    return NLOS_OK;
  }
  return create_ctx(S, k.first, k.second, base, out);
}

// Captures (or finds cached) the graph of a run of `p` in context c, with the
// context's own buffers, exactly as start_job will enqueue it.
static nlos_status warm_ctx(JobCtx* c, const nlos_params& p) {
  JobRun r;
  r.P = c->ws;
  r.p = p;
  r.tau0 = c->d_tau0;
  r.u_out = c->d_u;
  r.tau_out = nullptr;
  r.st = c->st;
  bool ready = false;
  NLOS_TRY(job_prepare_graph(r, c->st, &ready));
  return cudaStreamSynchronize(c->st) == cudaSuccess ? NLOS_OK : fail(NLOS_ERR_CUDA, "server: warm-up");
}

// Serves one warm-up request: the base plan, then up to `want` idle contexts
// of the request's kind (existing idle ones first), each with its graph
// captured.  Contexts that would exceed the HBM budget are not created and
// nothing else is evicted for them.
static void run_prep(Server* S, Prep& pr) {
  const int kind = ctx_kind(pr.params);
  BaseEntry* base = nullptr;
  nlos_status s = get_base(S, pr.key, kind, &base);
  int ready = 0;
  if (s == NLOS_OK) {
    auto range = S->idle.equal_range(std::make_pair(pr.key, kind));
    for (auto it = range.first; it != range.second && ready < pr.want && s == NLOS_OK; ++it) {
      s = warm_ctx(it->second, pr.params);
      if (s == NLOS_OK) ++ready;
    }
  }
  while (s == NLOS_OK && ready < pr.want && S->used + ctx_bytes(*base->plan, kind) <= S->budget) {
    JobCtx* c = nullptr;
    s = create_ctx(S, pr.key, kind, base, &c);
    if (s != NLOS_OK) break;
    S->idle.emplace(std::make_pair(pr.key, kind), c);
    s = warm_ctx(c, pr.params);
    if (s == NLOS_OK) ++ready;
  }
  std::lock_guard<std::mutex> lock(S->mu);
  pr.ready = ready;
  pr.status = s;
  pr.done = true;
  S->info.bytes_in_use = S->used;
  S->info.bytes_peak = std::max(S->info.bytes_peak, S->used);
  S->done_cv.notify_all();
}

static void finish_job(Server* S, Job* jb, JobState state, nlos_status status) {
  std::lock_guard<std::mutex> lock(S->mu);
  jb->state = state;
  jb->status = status;
  jb->t_done = Clock::now();
  jb->tau0.clear();
  jb->tau0.shrink_to_fit();
  if (state == JOB_DONE)
    S->info.completed += 1;
  else
    S->info.failed += 1;
  S->done_cv.notify_all();
}

static void recycle(Server* S, Job* jb) {
  if (jb->ctx) {
    S->idle.emplace(std::make_pair(jb->ctx->key, jb->ctx->model), jb->ctx);
    jb->ctx = nullptr;
  }
}

static nlos_status start_job(Server* S, Job* jb, BaseEntry* base) {
  JobCtx* c = nullptr;
  NLOS_TRY(acquire_ctx(S, jb, base, &c));
  jb->ctx = c;
  const size_t F = jb->tau0.size() * sizeof(float);
  // the host copy is pageable: cudaMemcpyAsync stages it through the driver
  NLOS_CUDA(cudaMemcpyAsync(c->d_tau0, jb->tau0.data(), F, cudaMemcpyHostToDevice, c->st));
  JobRun& r = jb->run;
  r = JobRun();
  r.P = c->ws;
  r.p = jb->params;
  r.tau0 = c->d_tau0;
  r.u_out = c->d_u;
  r.tau_out = nullptr;
  r.st = c->st;
  bool used = false;
  NLOS_TRY(job_enqueue_graph(r, c->st, &used));
  jb->graphed = used;
  if (used)
    r.done = true;
  else
    NLOS_TRY(job_init(r));
  jb->t_start = Clock::now();
  return NLOS_OK;
}

static void worker_main(Server* S) {
  cudaSetDevice(S->device);
  cudaStreamCreateWithFlags(&S->setup_stream, cudaStreamNonBlocking);
  for (;;) {
    {
      std::unique_lock<std::mutex> lock(S->mu);
      if (S->active.empty() && S->pending.empty() && S->incoming.empty() && S->preps.empty() && !S->stopping)
        S->cv.wait_for(lock, std::chrono::milliseconds(50));
      while (!S->incoming.empty()) {
        S->pending.push_back(S->incoming.front());
        S->incoming.pop_front();
      }
      if (S->cancel_pending) {
        for (Job* jb : S->pending) {
          jb->state = JOB_CANCELLED;
          jb->status = NLOS_ERR_TIMEOUT;
          jb->t_done = Clock::now();
        }
        S->info.failed += (int64_t)S->pending.size();
        S->pending.clear();
        S->done_cv.notify_all();
      }
      if (S->stopping && S->pending.empty() && S->active.empty() && S->preps.empty()) break;
      S->info.queued = (int64_t)S->pending.size();
    }
    bool progressed = false;
    for (;;) {
      std::shared_ptr<Prep> pr;
      {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->preps.empty()) break;
        pr = S->preps.front();
        S->preps.pop_front();
      }
      run_prep(S, *pr);
      progressed = true;
    }
    // admission: in arrival order, while a slot and the HBM budget allow
    while (!S->pending.empty() && (int)S->active.size() < S->max_slots) {
      Job* jb = S->pending.front();
      BaseEntry* base = nullptr;
      nlos_status s = get_base(S, jb->key, ctx_kind(jb->params), &base);
      if (s != NLOS_OK) {
        S->pending.pop_front();
        finish_job(S, jb, JOB_FAILED, s);
        progressed = true;
        continue;
      }
      const auto k = std::make_pair(jb->key, ctx_kind(jb->params));
      const bool recycled = S->idle.count(k) > 0;
      const size_t need = recycled ? 0 : ctx_bytes(*base->plan, k.second);
      if (S->used + need > S->budget) release_idle(S, need);
      if (S->used + need > S->budget) {
        if (S->active.empty()) {  // can never fit: fail instead of waiting forever
          S->pending.pop_front();
          finish_job(S, jb, JOB_FAILED, fail(NLOS_ERR_OOM, "server: job exceeds the HBM budget"));
          progressed = true;
          continue;
        }
        break;
      }
      S->pending.pop_front();
      s = start_job(S, jb, base);
      if (s != NLOS_OK) {
        recycle(S, jb);
        finish_job(S, jb, JOB_FAILED, s);
        progressed = true;
        continue;
      }
      {
        std::lock_guard<std::mutex> lock(S->mu);
        jb->state = JOB_RUNNING;
      }
      S->active.push_back(jb);
      progressed = true;
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->info.active = (int64_t)S->active.size();
      S->info.peak_active = std::max(S->info.peak_active, S->info.active);
      S->info.bytes_in_use = S->used;
      S->info.bytes_peak = std::max(S->info.bytes_peak, S->used);
    }
    // advance every active job by one enqueued iteration
    for (Job* jb : S->active) {
      if (jb->finishing) continue;
      nlos_status s = NLOS_OK;
      if (!jb->run.done) {
        s = job_step(jb->run);
        progressed = true;
      }
      if (s == NLOS_OK && jb->run.done) {
        JobCtx* c = jb->ctx;
        if (!jb->graphed) s = job_finish(jb->run);
        const size_t F = (size_t)c->ws->nx * c->ws->ny * c->ws->nt * sizeof(float);
        if (s == NLOS_OK && cudaMemcpyAsync(c->h_u, c->d_u, F, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
          s = fail(NLOS_ERR_CUDA, "server: result copy");
        if (s == NLOS_OK && cudaEventRecord(c->done, c->st) != cudaSuccess) s = fail(NLOS_ERR_CUDA, "server: event");
        jb->finishing = true;
        if (s != NLOS_OK) jb->status = s;
      }
      if (s != NLOS_OK) {
        jb->finishing = true;
        jb->status = s;
      }
    }
    // retire finished jobs
    for (size_t i = 0; i < S->active.size();) {
      Job* jb = S->active[i];
      if (!jb->finishing) {
        ++i;
        continue;
      }
      cudaError_t q = jb->status == NLOS_OK ? cudaEventQuery(jb->ctx->done) : cudaSuccess;
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      nlos_status s = jb->status;
      if (s == NLOS_OK && q != cudaSuccess) s = cuda_fail(q, "server: job");
      if (s == NLOS_OK) {
        cudaStreamSynchronize(jb->ctx->st);
        std::memcpy(jb->u_out_host, jb->ctx->h_u,
                    (size_t)jb->ctx->ws->nx * jb->ctx->ws->ny * jb->ctx->ws->nt * sizeof(float));
        s = job_collect(jb->run, &jb->stats);
      }
      recycle(S, jb);
      finish_job(S, jb, s == NLOS_OK ? JOB_DONE : JOB_FAILED, s);
      S->active.erase(S->active.begin() + i);
      progressed = true;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  // shutdown: free everything the worker owns
  for (auto& kv : S->idle) free_ctx(kv.second);
  S->idle.clear();
  for (auto& kv : S->bases) plan_release(kv.second.plan);
  S->bases.clear();
  if (S->setup_stream) cudaStreamDestroy(S->setup_stream);
}

}  // namespace nlos

using namespace nlos;

struct nlos_server_s {
  Server impl;
};

extern "C" {

nlos_status nlos_reconstruct_batch(const nlos_plan* plans, const nlos_params* params, const float* const* tau0,
                                   float* const* u_out, float* const* tau_out, int32_t n, nlos_stats* stats,
                                   void* stream) {
  try {
    if (!plans || !params || !tau0 || !u_out || n <= 0)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_batch: null argument or n <= 0");
    std::vector<Plan*> P(n);
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < n; ++i) {
      P[i] = reinterpret_cast<Plan*>(plans[i]);
      if (!P[i] || !tau0[i] || !u_out[i]) return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_batch: null entry");
      if (((reinterpret_cast<uintptr_t>(tau0[i]) | reinterpret_cast<uintptr_t>(u_out[i]) |
            reinterpret_cast<uintptr_t>(tau_out ? tau_out[i] : nullptr)) & 15) != 0)
        return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_batch: device buffers must be 16-byte aligned");
      if (P[i]->device != dev) return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_batch: plan on another device");
      NLOS_TRY(validate_params(params[i], "nlos_reconstruct_batch"));
      for (int k = 0; k < i; ++k)
        if (P[k] == P[i]) return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_batch: a plan appears twice");
    }
    if (stats) std::memset(stats, 0, sizeof(nlos_stats) * n);
    return reconstruct_batch(P.data(), params, tau0, u_out, tau_out, n, stats, reinterpret_cast<cudaStream_t>(stream));
  } catch (...) {
    return fail(NLOS_ERR_OOM, "nlos_reconstruct_batch: host allocation failed");
  }
}

nlos_status nlos_server_create(size_t hbm_budget_bytes, int32_t max_slots, nlos_server* out) {
  try {
    if (!out || max_slots <= 0 || hbm_budget_bytes == 0)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_server_create: need a budget > 0 and max_slots > 0");
    auto* s = new nlos_server_s();
    s->impl.budget = hbm_budget_bytes;
    s->impl.max_slots = max_slots;
    cudaGetDevice(&s->impl.device);
    s->impl.worker = std::thread(worker_main, &s->impl);
    *out = s;
    return NLOS_OK;
  } catch (...) {
    return fail(NLOS_ERR_OOM, "nlos_server_create: failed");
  }
}

nlos_status nlos_submit(nlos_server server, const nlos_geometry* geom, const nlos_params* params,
                        const float* tau0_host, float* u_out_host, uint64_t* job_id) {
  try {
    if (!server || !geom || !params || !tau0_host || !u_out_host || !job_id)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_submit: null argument");
    int32_t n = 0;
    NLOS_TRY(nlos_geometry_tables(geom, nullptr, nullptr, nullptr, nullptr, nullptr, &n));
    NLOS_TRY(validate_params(*params, "nlos_submit"));
    Server& S = server->impl;
    auto jb = std::make_unique<Job>();
    jb->key = make_key(*geom);
    jb->params = *params;
    const size_t V = (size_t)geom->nx * geom->ny * geom->nt;
    jb->tau0.assign(tau0_host, tau0_host + V);
    jb->u_out_host = u_out_host;
    jb->t_submit = Clock::now();
    std::lock_guard<std::mutex> lock(S.mu);
    if (S.stopping) return fail(NLOS_ERR_BUSY, "nlos_submit: server is shutting down");
    if (S.incoming.size() + S.info.queued > 100000) return fail(NLOS_ERR_BUSY, "nlos_submit: queue full");
    jb->id = S.next_id++;
    *job_id = jb->id;
    S.incoming.push_back(jb.get());
    S.jobs.emplace(jb->id, std::move(jb));
    S.cv.notify_one();
    return NLOS_OK;
  } catch (...) {
    return fail(NLOS_ERR_OOM, "nlos_submit: host allocation failed");
  }
}

nlos_status nlos_server_prepare(nlos_server server, const nlos_geometry* geom, const nlos_params* params,
                                int32_t contexts, double timeout_s, int32_t* ready) {
  try {
    if (ready) *ready = 0;
    if (!server || !geom || !params || contexts < 0)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_server_prepare: null argument or contexts < 0");
    int32_t n = 0;
    NLOS_TRY(nlos_geometry_tables(geom, nullptr, nullptr, nullptr, nullptr, nullptr, &n));
    NLOS_TRY(validate_params(*params, "nlos_server_prepare"));
    Server& S = server->impl;
    auto pr = std::make_shared<Prep>();
    pr->key = make_key(*geom);
    pr->params = *params;
    pr->want = contexts;
    std::unique_lock<std::mutex> lock(S.mu);
    if (S.stopping) return fail(NLOS_ERR_BUSY, "nlos_server_prepare: server is shutting down");
    S.preps.push_back(pr);
    S.cv.notify_one();
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    while (!pr->done)
      if (S.done_cv.wait_until(lock, deadline) == std::cv_status::timeout && !pr->done)
        return fail(NLOS_ERR_TIMEOUT, "nlos_server_prepare: timed out (the warm-up still completes)");
    if (ready) *ready = pr->ready;
    return pr->status == NLOS_OK ? NLOS_OK : fail(pr->status, "nlos_server_prepare: warm-up failed");
  } catch (...) {
    return fail(NLOS_ERR_OOM, "nlos_server_prepare: host allocation failed");
  }
}

static nlos_status poll_locked(Server& S, uint64_t id, nlos_stats* out) {
  auto it = S.jobs.find(id);
  if (it == S.jobs.end()) return fail(NLOS_ERR_INVALID_ARG, "unknown job id");
  Job* jb = it->second.get();
  if (jb->state == JOB_QUEUED || jb->state == JOB_RUNNING) return NLOS_ERR_NOT_READY;
  if (out) *out = jb->stats;
  if (jb->state == JOB_DONE) return NLOS_OK;
  return fail(jb->status != NLOS_OK ? jb->status : NLOS_ERR_CUDA, "job failed or was cancelled");
}

nlos_status nlos_poll(nlos_server server, uint64_t job_id, nlos_stats* out) {
  if (!server) return fail(NLOS_ERR_INVALID_ARG, "null server");
  Server& S = server->impl;
  std::lock_guard<std::mutex> lock(S.mu);
  return poll_locked(S, job_id, out);
}

nlos_status nlos_wait(nlos_server server, uint64_t job_id, double timeout_s, nlos_stats* out) {
  if (!server) return fail(NLOS_ERR_INVALID_ARG, "null server");
  Server& S = server->impl;
  std::unique_lock<std::mutex> lock(S.mu);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  for (;;) {
    nlos_status s = poll_locked(S, job_id, out);
    if (s != NLOS_ERR_NOT_READY) return s;
    if (S.done_cv.wait_until(lock, deadline) == std::cv_status::timeout) {
      s = poll_locked(S, job_id, out);
      return s == NLOS_ERR_NOT_READY ? NLOS_ERR_NOT_READY : s;
    }
  }
}

nlos_status nlos_job_times(nlos_server server, uint64_t job_id, double* queued_s, double* total_s) {
  if (!server) return fail(NLOS_ERR_INVALID_ARG, "null server");
  Server& S = server->impl;
  std::lock_guard<std::mutex> lock(S.mu);
  auto it = S.jobs.find(job_id);
  if (it == S.jobs.end()) return fail(NLOS_ERR_INVALID_ARG, "unknown job id");
  Job* jb = it->second.get();
  if (jb->state != JOB_DONE && jb->state != JOB_FAILED && jb->state != JOB_CANCELLED) return NLOS_ERR_NOT_READY;
  auto sec = [](Clock::duration d) { return std::chrono::duration<double>(d).count(); };
  if (queued_s) *queued_s = jb->t_start.time_since_epoch().count() ? sec(jb->t_start - jb->t_submit) : 0.0;
  if (total_s) *total_s = sec(jb->t_done - jb->t_submit);
  return NLOS_OK;
}

nlos_status nlos_server_info(nlos_server server, int64_t* out8) {
  if (!server || !out8) return fail(NLOS_ERR_INVALID_ARG, "null argument");
  Server& S = server->impl;
  std::lock_guard<std::mutex> lock(S.mu);
  out8[0] = S.info.queued + (int64_t)S.incoming.size();
  out8[1] = S.info.active;
  out8[2] = S.info.completed;
  out8[3] = S.info.failed;
  out8[4] = S.info.peak_active;
  out8[5] = (int64_t)S.info.bytes_in_use;
  out8[6] = (int64_t)S.info.bytes_peak;
  out8[7] = (int64_t)S.budget;
  return NLOS_OK;
}

nlos_status nlos_server_destroy(nlos_server server, int32_t cancel_pending, double timeout_s) {
  if (!server) return NLOS_OK;
  Server& S = server->impl;
  {
    std::lock_guard<std::mutex> lock(S.mu);
    S.stopping = true;
    S.cancel_pending = cancel_pending != 0;
    S.cv.notify_all();
  }
  // bounded wait for the worker to drain
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
  bool drained = false;
  for (;;) {
    {
      std::lock_guard<std::mutex> lock(S.mu);
      drained = S.info.completed + S.info.failed >= (int64_t)S.jobs.size();
    }
    if (drained || Clock::now() > deadline) break;
    std::this_thread::sleep_for(std::chrono::milliseconds(2));
  }
  if (!drained) {
    // give up waiting: cancel what is still queued; running jobs finish on the device
    std::lock_guard<std::mutex> lock(S.mu);
    S.cancel_pending = true;
    S.cv.notify_all();
  }
  S.worker.join();
  delete server;
  return drained ? NLOS_OK : fail(NLOS_ERR_TIMEOUT, "nlos_server_destroy: timed out waiting for jobs");
}

}  // extern "C"
