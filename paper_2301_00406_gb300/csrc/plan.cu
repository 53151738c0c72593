// Plan construction (geometry tables of Eq. 3 in FP64 on the host, the
// cone-kernel spectrum on the device) and the extern "C" entry points.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "passes.cuh"

namespace nlos {

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    dev = 0;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

nlos_status fail(nlos_status code, const std::string& msg) {
  set_error(msg);
  return code;
}

nlos_status cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? NLOS_ERR_OOM : NLOS_ERR_CUDA;
}

KTimer::KTimer(const Plan& p, int cat, cudaStream_t s) : P(p), st(s), slot(0), on(p.timing) {
  if (!on) return;
  if (P.ev_used + 2 > P.ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      on = false;
      return;
    }
    P.ev.push_back(a);
    P.ev.push_back(b);
    P.ev_cat.push_back(0);
  }
  slot = P.ev_used / 2;
  P.ev_cat[slot] = cat;
  cudaEventRecord(P.ev[2 * slot], st);
  P.ev_used += 2;
}

KTimer::~KTimer() {
  if (on) cudaEventRecord(P.ev[2 * slot + 1], st);
}

nlos_status ensure_smem_attr(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[dev][kernel];
  if (bytes <= have) return NLOS_OK;
  NLOS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return NLOS_OK;
}

static const double kC = 299792458.0;  // speed of light, m/s
static const double kPi = 3.14159265358979323846;

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

// Two-tap clamped linear interpolation at position p on an n-grid.
static void two_tap(double p, int n, int32_t* i0, float* w0, float* w1) {
  if (p < 0.0) p = 0.0;
  if (p > n - 1.0) p = n - 1.0;
  double f = std::floor(p);
  if (f > n - 2.0) f = n - 2.0;
  const double frac = p - f;
  *i0 = (int32_t)f;
  *w0 = (float)(1.0 - frac);
  *w1 = (float)frac;
}

// Build the host tables of the plan.
//  R_z:     v-bin j samples the rho-grid at sqrt((j + 1/2) nt) - 1/2, weight
//           g_j = 1 / (2 sqrt((j + 1/2) / nt)).
//  R_t^-1:  t-bin k samples the v-grid at (k + 1/2)^2 / nt - 1/2, weight
//           rho_k (compensated) or rho_k^-3 (raw), rho_k = (k + 1/2) / nt.
static void build_tables(Plan& P) {
  const int nt = P.nt;
  P.h_rz_i0.resize(nt);
  P.h_rz_w.resize(3 * nt);
  P.h_rt_k0.resize(nt);
  P.h_rt_w.resize(3 * nt);
  for (int j = 0; j < nt; ++j) {
    const double p = std::sqrt((j + 0.5) * nt) - 0.5;
    two_tap(p, nt, &P.h_rz_i0[j], &P.h_rz_w[3 * j], &P.h_rz_w[3 * j + 1]);
    P.h_rz_w[3 * j + 2] = (float)(1.0 / (2.0 * std::sqrt((j + 0.5) / nt)));
  }
  for (int k = 0; k < nt; ++k) {
    const double q = (k + 0.5) * (k + 0.5) / nt - 0.5;
    two_tap(q, nt, &P.h_rt_k0[k], &P.h_rt_w[3 * k], &P.h_rt_w[3 * k + 1]);
    const double rho = (k + 0.5) / nt;
    P.h_rt_w[3 * k + 2] = (float)(P.radiometry == NLOS_RADIOMETRY_RAW ? 1.0 / (rho * rho * rho) : rho);
  }
}

// Device forms of a two-tap resampling out_k = s_k (w0_k in[i0_k] + w1_k in[i0_k + 1]):
// forward taps with pre-multiplied weights, and the transpose as CSR rows.
static void device_taps(const std::vector<int32_t>& i0, const std::vector<float>& w3, int n,
                        std::vector<float4>* fwd, std::vector<int32_t>* ptr, std::vector<float2>* ent) {
  fwd->resize(n);
  std::vector<std::vector<std::pair<int, double>>> rows(n);
  for (int k = 0; k < n; ++k) {
    const double a = (double)w3[3 * k] * w3[3 * k + 2], b = (double)w3[3 * k + 1] * w3[3 * k + 2];
    int32_t bits;
    std::memcpy(&bits, &i0[k], sizeof(bits));
    float fb;
    std::memcpy(&fb, &bits, sizeof(fb));
    (*fwd)[k] = make_float4((float)a, (float)b, fb, 0.f);
    if (a != 0.0) rows[i0[k]].push_back({k, a});
    if (b != 0.0) rows[i0[k] + 1].push_back({k, b});
  }
  ptr->assign(n + 1, 0);
  ent->clear();
  for (int i = 0; i < n; ++i) {
    (*ptr)[i] = (int32_t)ent->size();
    for (auto& e : rows[i]) {
      float fi;
      int32_t idx = e.first;
      std::memcpy(&fi, &idx, sizeof(fi));
      ent->push_back(make_float2((float)e.second, fi));
    }
  }
  (*ptr)[n] = (int32_t)ent->size();
}

// start[i] = first index j with tab[j] >= i (tab non-decreasing), i in [0, n].
static std::vector<int32_t> starts_of(const std::vector<int32_t>& tab, int n) {
  std::vector<int32_t> s(n + 1);
  int j = 0;
  for (int i = 0; i <= n; ++i) {
    while (j < (int)tab.size() && tab[j] < i) ++j;
    s[i] = j;
  }
  return s;
}

template <typename T>
static nlos_status upload(T** dst, const T* src, size_t n) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), n * sizeof(T));
  if (e != cudaSuccess) {
    *dst = nullptr;
    return cuda_fail(e, "cudaMalloc (plan table)");
  }
  if (src) NLOS_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return NLOS_OK;
}

template <typename T>
static nlos_status dalloc(T** dst, size_t n) {
  return upload<T>(dst, nullptr, n);
}

static std::vector<float2> roots(int n, int m) {
  // exp(-2 pi i k / n), k < m, from FP64
  std::vector<float2> w(m);
  for (int k = 0; k < m; ++k) {
    const double a = -2.0 * kPi * k / n;
    w[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return w;
}

static std::vector<float> lap_eigs(int n) {
  std::vector<float> l(n);
  for (int k = 0; k < n; ++k) {
    const double s = std::sin(kPi * k / n);
    l[k] = (float)(4.0 * s * s);
  }
  return l;
}

static void free_workspace(Plan* P) {
  free_graphs(P);
  for (int m = 0; m < 3; ++m) {
    free_solver(P->solver[m]);
    P->solver[m] = nullptr;
  }
  void* ws[] = {P->d_S, P->d_S2, P->d_Sc, P->d_Sp, P->d_tmpc, P->d_partials, P->d_scal, P->d_io[0], P->d_io[1],
                P->d_io[2], P->d_dir[0], P->d_dir[1]};
  for (void* p : ws)
    if (p) cudaFree(p);
  for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
  P->ev.clear();
}

static void destroy_plan(Plan* P) {
  if (!P) return;
  cudaDeviceSynchronize();
  free_workspace(P);
  free_lateral_tc(P);
  if (P->owns_tables) {
    void* ptrs[] = {P->d_rz_i0, P->d_rz_w, P->d_rzt_start, P->d_rt_k0, P->d_rt_w, P->d_rtt_start, P->d_cols,
                    P->d_colpos, P->d_tw2t, P->d_twt, P->d_twx, P->d_twy, P->d_lamx, P->d_lamy, P->d_lamt,
                    P->d_H, P->d_rz_f4, P->d_rt_f4, P->d_rzT_ptr, P->d_rzT_ent, P->d_rtT_ptr, P->d_rtT_ent};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  delete P;
}

static nlos_status alloc_workspace(Plan* P) {
  const size_t full = (size_t)P->nx * P->ny;
  const size_t S = (size_t)(P->nt + 1) * full;
  nlos_status s = dalloc(&P->d_S, S);
  if (s == NLOS_OK) s = dalloc(&P->d_S2, S);
  if (s == NLOS_OK) s = dalloc(&P->d_Sc, (size_t)(P->nt + 1) * P->ncols);
  if (s == NLOS_OK) s = dalloc(&P->d_Sp, (size_t)(P->nt / 2 + 1) * full);
  if (s == NLOS_OK) s = dalloc(&P->d_tmpc, (size_t)P->ncols * P->nt);
  P->partial_blocks = 4096;
  if (s == NLOS_OK) s = dalloc(&P->d_partials, (size_t)P->partial_blocks * kMaxTerms);
  if (s == NLOS_OK) s = dalloc(&P->d_scal, 1);
  return s;
}

Plan* plan_clone_workspace(const Plan& base, nlos_status* status) {
  Plan* P = new Plan(base);
  P->owns_tables = false;
  for (int m = 0; m < 3; ++m) P->solver[m] = nullptr;
  P->d_S = P->d_S2 = P->d_Sc = P->d_Sp = nullptr;
  P->d_tmpc = nullptr;
  P->d_partials = nullptr;
  P->d_scal = nullptr;
  for (auto& b : P->d_io) b = nullptr;
  for (auto& b : P->d_dir) b = nullptr;
  P->timing = false;
  P->ev.clear();
  P->ev_cat.clear();
  P->ev_used = 0;
  P->graphs.clear();
  P->capture_stream = nullptr;
  for (auto& b : P->body_stream) b = nullptr;  // the base's streams stay the base's
  P->aux_stream = nullptr;
  P->aux_ev[0] = P->aux_ev[1] = nullptr;
  P->lateral = nullptr;                         // a clone uses the FFT lateral stage
  nlos_status s = alloc_workspace(P);
  if (s != NLOS_OK) {
    destroy_plan(P);
    *status = s;
    return nullptr;
  }
  *status = NLOS_OK;
  return P;
}

void plan_release(Plan* P) { destroy_plan(P); }

size_t shared_table_bytes(const Plan& P) {
  return sizeof(float2) * (size_t)(P.nt + 1) * (P.nx + 1) * (P.ny + 1) + 64 * (size_t)P.nt + 16 * (size_t)P.nx * P.ny;
}

size_t workspace_bytes(const Plan& P, int model) {
  const size_t full = (size_t)P.nx * P.ny, V = full * P.nt, F = V * sizeof(float);
  const size_t C = (size_t)P.ncols * P.nt * sizeof(float);
  size_t b = sizeof(float2) * ((size_t)(P.nt + 1) * full * 2 + (size_t)(P.nt + 1) * P.ncols +
                               (size_t)(P.nt / 2 + 1) * full) +
             C + sizeof(double) * 4096 * kMaxTerms + 4096;
  const size_t partials = 3 * sizeof(double) * kMaxTerms * 4096;
  if (model == 1 || model == 3) b += 13 * F + 4 * C + partials;
  if (model == 2 || model == 3) b += 25 * F + partials;
  return b;
}

static nlos_status validate_geometry(const nlos_geometry* g) {
  if (!g) return fail(NLOS_ERR_INVALID_ARG, "null geometry");
  if (!pow2_in(g->nx, 8, 128) || g->ny != g->nx)
    return fail(NLOS_ERR_INVALID_ARG, "nx must equal ny and be a power of two in [8, 128]");
  if (!pow2_in(g->nt, 16, 1024)) return fail(NLOS_ERR_INVALID_ARG, "nt must be a power of two in [16, 1024]");
  if (!(g->bin_width_s > 0.0) || !(g->wall_width_m > 0.0) || !std::isfinite(g->bin_width_s) ||
      !std::isfinite(g->wall_width_m))
    return fail(NLOS_ERR_INVALID_ARG, "bin_width_s and wall_width_m must be finite and > 0");
  if (g->radiometry != NLOS_RADIOMETRY_COMPENSATED && g->radiometry != NLOS_RADIOMETRY_RAW)
    return fail(NLOS_ERR_INVALID_ARG, "unknown radiometry");
  return NLOS_OK;
}

// Host part of a plan: geometry, mask list and resampling tables.
static nlos_status host_plan(const nlos_geometry* g, Plan* P, std::vector<int32_t>* colpos) {
  NLOS_TRY(validate_geometry(g));
  P->nx = g->nx;
  P->ny = g->ny;
  P->nt = g->nt;
  P->bin_width_s = g->bin_width_s;
  P->wall_width_m = g->wall_width_m;
  P->range_m = kC * g->nt * g->bin_width_s / 2.0;
  P->radiometry = g->radiometry;
  const int full = P->nx * P->ny;
  P->h_mask.assign(full, 1);
  if (g->mask) std::memcpy(P->h_mask.data(), g->mask, full);
  colpos->assign(full, -1);
  P->h_cols.clear();
  for (int c = 0; c < full; ++c)
    if (P->h_mask[c]) {
      (*colpos)[c] = (int32_t)P->h_cols.size();
      P->h_cols.push_back(c);
    }
  P->ncols = (int)P->h_cols.size();
  P->full_mask = P->ncols == full;
  if (P->ncols == 0) return fail(NLOS_ERR_INVALID_ARG, "mask samples no scan point");
  P->lattice_rx = -1;
  P->lattice_ry = -1;
  if (!P->full_mask) {
    const int r = P->h_cols[0] / P->ny % 4;
    bool one_class = true;
    for (int c : P->h_cols) one_class = one_class && (c / P->ny) % 4 == r;
    if (one_class) P->lattice_rx = r;
    // the full Cartesian lattice x = r, y = r' (mod 4): its compact index is (x / 4) (ny / 4) + y / 4
    const int ry = P->h_cols[0] % P->ny % 4;
    bool cart = one_class && P->nx % 4 == 0 && P->ny % 4 == 0 && P->ncols == (P->nx / 4) * (P->ny / 4);
    for (int c : P->h_cols) cart = cart && c % P->ny % 4 == ry;
    if (cart) P->lattice_ry = ry;
  }
  build_tables(*P);
  return NLOS_OK;
}

static nlos_status create_plan(const nlos_geometry* g, cudaStream_t st, Plan** out) {
  if (!out) return fail(NLOS_ERR_INVALID_ARG, "nlos_plan_create: null output pointer");
  Plan* P = new Plan();
  std::vector<int32_t> colpos;
  {
    nlos_status hs = host_plan(g, P, &colpos);
    if (hs != NLOS_OK) {
      delete P;
      return hs;
    }
  }
  cudaGetDevice(&P->device);
  P->sms = device_sm_count();
  const int nx = P->nx, ny = P->ny, nt = P->nt, full = nx * ny;
  const auto rzs = starts_of(P->h_rz_i0, nt);
  const auto rts = starts_of(P->h_rt_k0, nt);
  const auto tw2t = roots(2 * nt, 2 * nt);
  const auto twt = roots(nt, nt);
  const auto twx = roots(2 * nx, 2 * nx);
  const auto twy = roots(2 * ny, 2 * ny);
  const auto lx = lap_eigs(nx), ly = lap_eigs(ny), lt = lap_eigs(nt);

  nlos_status s = NLOS_OK;
#define UP(dst, vec) \
  if (s == NLOS_OK) s = upload(&P->dst, vec.data(), vec.size())
  UP(d_rz_i0, P->h_rz_i0);
  UP(d_rz_w, P->h_rz_w);
  UP(d_rzt_start, rzs);
  UP(d_rt_k0, P->h_rt_k0);
  UP(d_rt_w, P->h_rt_w);
  UP(d_rtt_start, rts);
  UP(d_cols, P->h_cols);
  UP(d_colpos, colpos);
  UP(d_tw2t, tw2t);
  UP(d_twt, twt);
  UP(d_twx, twx);
  UP(d_twy, twy);
  UP(d_lamx, lx);
  UP(d_lamy, ly);
  UP(d_lamt, lt);
  std::vector<float4> rzf, rtf;
  std::vector<int32_t> rzp, rtp;
  std::vector<float2> rze, rte;
  device_taps(P->h_rz_i0, P->h_rz_w, nt, &rzf, &rzp, &rze);
  device_taps(P->h_rt_k0, P->h_rt_w, nt, &rtf, &rtp, &rte);
  rze.resize(2 * nt, make_float2(0.f, 0.f));   // kernels stage a fixed 2 nt entries
  rte.resize(2 * nt, make_float2(0.f, 0.f));
  UP(d_rz_f4, rzf);
  UP(d_rt_f4, rtf);
  UP(d_rzT_ptr, rzp);
  UP(d_rzT_ent, rze);
  UP(d_rtT_ptr, rtp);
  UP(d_rtT_ent, rte);
#undef UP
  if (s == NLOS_OK) s = dalloc(&P->d_H, (size_t)(nt + 1) * (nx + 1) * (ny + 1));
  if (s == NLOS_OK) s = alloc_workspace(P);
  if (s != NLOS_OK) {
    destroy_plan(P);
    return s;
  }

  // Cone kernel taps on the lateral-periodic (2nx, 2ny) grid: offset
  // (i, j) in (-nx, nx) x (-ny, ny) has w = nt ((i dx)^2 + (j dy)^2) / R^2 in
  // v-bins and a linear hat on floor(w), floor(w) + 1 (truncated at nt).
  const double dx = P->wall_width_m / nx, dy = P->wall_width_m / ny, R = P->range_m;
  std::vector<int32_t> m0(4 * full, 0);
  std::vector<float2> hw(4 * full, make_float2(0.f, 0.f));
  std::vector<double> h0(4 * full, 0.0), h1(4 * full, 0.0);
  double ss = 0.0;
  for (int a = 0; a < 2 * nx; ++a) {
    const int i = a < nx ? a : a - 2 * nx;
    if (i <= -nx) continue;
    for (int b = 0; b < 2 * ny; ++b) {
      const int j = b < ny ? b : b - 2 * ny;
      if (j <= -ny) continue;
      const double sq = (i * dx) * (i * dx) + (j * dy) * (j * dy);
      const double w = nt * sq / (R * R);
      const double fl = std::floor(w);
      if (fl >= nt) continue;
      const double f = w - fl;
      const int li = a * 2 * ny + b;
      m0[li] = (int32_t)fl;
      h0[li] = 1.0 - f;
      h1[li] = (fl + 1.0 < nt) ? f : 0.0;
      ss += h0[li] * h0[li] + h1[li] * h1[li];
    }
  }
  const double inv = ss > 0.0 ? 1.0 / std::sqrt(ss) : 0.0;
  for (int li = 0; li < 4 * full; ++li) hw[li] = make_float2((float)(h0[li] * inv), (float)(h1[li] * inv));
  int32_t* d_m0 = nullptr;
  float2* d_hw = nullptr;
  s = upload(&d_m0, m0.data(), m0.size());
  if (s == NLOS_OK) s = upload(&d_hw, hw.data(), hw.size());
  if (s == NLOS_OK) s = prepare_tpass(nt);
  if (s == NLOS_OK) s = prepare_xy(nx);
  if (s == NLOS_OK) s = prepare_stencils();
  if (s == NLOS_OK) s = autotune_tpass(*P, st);
  if (s == NLOS_OK) {
    KTimer kt_(*P, KC_KSPEC, st);
    s = launch_kernel_spectrum(*P, d_m0, d_hw, st);
  }
  if (s == NLOS_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "plan kernel spectrum");
  }
  if (d_m0) cudaFree(d_m0);
  if (d_hw) cudaFree(d_hw);
  if (s != NLOS_OK) {
    destroy_plan(P);
    return s;
  }
  *out = P;
  return NLOS_OK;
}

nlos_status create_plan_internal(const nlos_geometry* g, cudaStream_t st, Plan** out) {
  return create_plan(g, st, out);
}

static nlos_status check_plan(nlos_plan plan) {
  if (!plan) return fail(NLOS_ERR_INVALID_ARG, "null plan");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != reinterpret_cast<Plan*>(plan)->device)
    return fail(NLOS_ERR_INVALID_ARG, "plan was created on another device");
  return NLOS_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The parameter rules shared by every entry point that runs a reconstruction.
nlos_status validate_params(const nlos_params& p, const char* who) {
  const std::string w(who);
  if (p.model != 1 && p.model != 2) return fail(NLOS_ERR_INVALID_ARG, w + ": model must be 1 or 2");
  if (p.iters < 0 || !(p.eta > 1.0) || p.max_backtracks < 0 || p.max_backtracks > 1000 || p.phi < 0 ||
      p.phi > 2 || !(p.eps_normal >= 0.0) || !(p.eps_stop >= 0.0) || p.warm_start_iters < 0 ||
      (p.init != NLOS_INIT_ZERO && p.init != NLOS_INIT_BACKPROJECT))
    return fail(NLOS_ERR_INVALID_ARG, w + ": invalid iteration parameters");
  if ((p.model == 1 || p.warm_start_iters > 0) && !(p.mu > 0.0))
    return fail(NLOS_ERR_INVALID_ARG, w + ": mu must be > 0");
  if (p.model == 2 && !(p.mu1 > 0.0 && p.mu2 > 0.0 && p.mu3 > 0.0 && p.lambda >= 0.0))
    return fail(NLOS_ERR_INVALID_ARG, w + ": mu1, mu2, mu3 must be > 0 and lambda >= 0");
  return NLOS_OK;
}
}  // namespace nlos

using namespace nlos;

#define API_GUARD(body)                                              \
  try {                                                              \
    body                                                             \
  } catch (const std::bad_alloc&) {                                  \
    return fail(NLOS_ERR_OOM, "host allocation failed");             \
  } catch (...) {                                                    \
    return fail(NLOS_ERR_INVALID_ARG, "unexpected internal error");  \
  }

extern "C" {

nlos_status nlos_last_error(char* buf, size_t n) {
  if (buf && n > 0) {
    const size_t k = std::min(n - 1, g_last_error.size());
    std::memcpy(buf, g_last_error.data(), k);
    buf[k] = '\0';
  }
  return NLOS_OK;
}

int32_t nlos_version(void) { return 100; }

nlos_status nlos_params_default(int32_t model, nlos_params* out) {
  if (!out) return fail(NLOS_ERR_INVALID_ARG, "null params");
  if (model != 1 && model != 2) return fail(NLOS_ERR_INVALID_ARG, "model must be 1 or 2");
  std::memset(out, 0, sizeof(*out));
  out->model = model;
  out->phi = NLOS_PHI_TSC;
  out->a = 9e-5;
  out->b = 2e-5;
  out->mu = 0.1;
  out->a_u = 2e-4;
  out->b_u = 4.5e-4;
  out->a_tau = 4e-4;
  out->b_tau = 3e-2;
  out->lambda = 235.0;
  out->mu1 = 1.0;
  out->mu2 = 800.0;
  out->mu3 = 2.0;
  out->iters = model == 1 ? 200 : 300;
  out->eps_stop = 0.0;
  out->L0 = 0.0;
  out->eta = 2.0;
  out->max_backtracks = 30;
  out->eps_normal = 1e-6;
  out->restart = -1;
  out->warm_start_iters = 0;
  out->init = NLOS_INIT_ZERO;
  return NLOS_OK;
}


nlos_status nlos_plan_create(const nlos_geometry* geom, void* stream, nlos_plan* out) {
  API_GUARD({
    Plan* P = nullptr;
    nlos_status s = create_plan(geom, reinterpret_cast<cudaStream_t>(stream), &P);
    if (s != NLOS_OK) return s;
    *out = reinterpret_cast<nlos_plan>(P);
    return NLOS_OK;
  })
}

nlos_status nlos_plan_set_lateral(nlos_plan plan, int32_t mode, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    Plan& P = *reinterpret_cast<Plan*>(plan);
    free_graphs(&P);  // cached graphs hold the previous lateral stage
    return set_lateral_mode(P, mode, reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_plan_destroy(nlos_plan plan) {
  API_GUARD({
    destroy_plan(reinterpret_cast<Plan*>(plan));
    return NLOS_OK;
  })
}

nlos_status nlos_plan_norm2(nlos_plan plan, int32_t masked, void* stream, double* out) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!out) return fail(NLOS_ERR_INVALID_ARG, "null output");
    return plan_norm2(*reinterpret_cast<Plan*>(plan), masked != 0, reinterpret_cast<cudaStream_t>(stream), out);
  })
}

nlos_status nlos_geometry_tables(const nlos_geometry* geom, int32_t* rz_i0, float* rz_w, int32_t* rt_k0,
                                 float* rt_w, int32_t* cols, int32_t* n_cols) {
  API_GUARD({
    Plan P;
    std::vector<int32_t> colpos;
    NLOS_TRY(host_plan(geom, &P, &colpos));
    if (rz_i0) std::memcpy(rz_i0, P.h_rz_i0.data(), P.nt * sizeof(int32_t));
    if (rz_w) std::memcpy(rz_w, P.h_rz_w.data(), 3 * P.nt * sizeof(float));
    if (rt_k0) std::memcpy(rt_k0, P.h_rt_k0.data(), P.nt * sizeof(int32_t));
    if (rt_w) std::memcpy(rt_w, P.h_rt_w.data(), 3 * P.nt * sizeof(float));
    if (cols) std::memcpy(cols, P.h_cols.data(), P.ncols * sizeof(int32_t));
    if (n_cols) *n_cols = P.ncols;
    return NLOS_OK;
  })
}

nlos_status nlos_forward(nlos_plan plan, const float* u_dev, float* tau_dev, int32_t apply_mask, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!u_dev || !tau_dev || !aligned16(u_dev) || !aligned16(tau_dev))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_forward: null or non-16-byte-aligned pointer");
    const Plan& P = *reinterpret_cast<Plan*>(plan);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!apply_mask || P.full_mask) return apply_forward(P, u_dev, tau_dev, false, st);
    const size_t V = (size_t)P.nx * P.ny * P.nt;
    NLOS_CUDA(cudaMemsetAsync(tau_dev, 0, V * sizeof(float), st));
    const int full = P.nx * P.ny;
    NLOS_TRY(launch_tfwd_rz(P, u_dev, full, P.d_S2, full, st));
    NLOS_TRY(launch_conv(P, P.d_S2, false, P.d_Sc, true, false, st));
    return launch_tinv_store(P, P.d_Sc, P.ncols, P.ncols, tau_dev, P.d_cols, st);
  })
}

nlos_status nlos_adjoint(nlos_plan plan, const float* tau_dev, float* u_dev, int32_t apply_mask, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!u_dev || !tau_dev || !aligned16(u_dev) || !aligned16(tau_dev))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_adjoint: null or non-16-byte-aligned pointer");
    const Plan& P = *reinterpret_cast<Plan*>(plan);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!apply_mask || P.full_mask) return apply_adjoint(P, tau_dev, u_dev, false, st);
    NLOS_TRY(gather_columns(P, tau_dev, P.d_tmpc, st));
    return apply_adjoint(P, P.d_tmpc, u_dev, true, st);
  })
}

static nlos_status check_directional(nlos_plan plan, const void* in, const void* normals, const void* out,
                                     const char* who) {
  NLOS_TRY(check_plan(plan));
  const Plan& P = *reinterpret_cast<const Plan*>(plan);
  if (!in || !normals || !out) return fail(NLOS_ERR_INVALID_ARG, std::string(who) + ": null pointer");
  const size_t F = (size_t)P.nx * P.ny * P.nt * sizeof(float);
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), n = reinterpret_cast<uintptr_t>(normals),
                  o = reinterpret_cast<uintptr_t>(out);
  if ((o < a + F && a < o + F) || (o < n + 3 * F && n < o + F))
    return fail(NLOS_ERR_INVALID_ARG, std::string(who) + ": the output overlaps an input");
  return NLOS_OK;
}

nlos_status nlos_forward_directional(nlos_plan plan, const float* u_dev, const float* normals_dev, float* tau_dev,
                                     int32_t apply_mask, void* stream) {
  API_GUARD({
    NLOS_TRY(check_directional(plan, u_dev, normals_dev, tau_dev, "nlos_forward_directional"));
    return apply_forward_directional(*reinterpret_cast<Plan*>(plan), u_dev, normals_dev, tau_dev, apply_mask != 0,
                                     reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_adjoint_directional(nlos_plan plan, const float* tau_dev, const float* normals_dev, float* u_dev,
                                     int32_t apply_mask, void* stream) {
  API_GUARD({
    NLOS_TRY(check_directional(plan, tau_dev, normals_dev, u_dev, "nlos_adjoint_directional"));
    return apply_adjoint_directional(*reinterpret_cast<Plan*>(plan), tau_dev, normals_dev, u_dev, apply_mask != 0,
                                     reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_solve(nlos_plan plan, const float* rhs_dev, float* x_dev, double c0, double c1, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!rhs_dev || !x_dev) return fail(NLOS_ERR_INVALID_ARG, "nlos_solve: null pointer");
    if (!(c0 > 0.0) || !(c1 >= 0.0) || !std::isfinite(c0) || !std::isfinite(c1))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_solve: need c0 > 0 and c1 >= 0");
    return apply_solve(*reinterpret_cast<Plan*>(plan), rhs_dev, x_dev, c0, c1, reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_curvature_weight(nlos_plan plan, const float* u_dev, float* phi_dev, double a, double b,
                                  int32_t phi_kind, double eps, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!u_dev || !phi_dev || u_dev == phi_dev)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_curvature_weight: null or aliased pointers");
    if (phi_kind < 0 || phi_kind > 2) return fail(NLOS_ERR_INVALID_ARG, "unknown phi kind");
    return apply_curvature_weight(*reinterpret_cast<Plan*>(plan), u_dev, phi_dev, a, b, phi_kind, eps,
                                  reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_reconstruct(nlos_plan plan, const nlos_params* params, const float* tau0_dev, float* u_out_dev,
                             float* tau_out_dev, nlos_stats* stats_host, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!params || !tau0_dev || !u_out_dev || !aligned16(tau0_dev) || !aligned16(u_out_dev))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct: null or non-16-byte-aligned pointer");
    const nlos_params& p = *params;
    NLOS_TRY(validate_params(p, "nlos_reconstruct"));
    if (stats_host) std::memset(stats_host, 0, sizeof(*stats_host));
    return reconstruct(*reinterpret_cast<Plan*>(plan), p, tau0_dev, u_out_dev, tau_out_dev, stats_host,
                       reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_reconstruct_host(nlos_plan plan, const nlos_params* params, const float* tau0_host,
                                  float* u_out_host, float* tau_out_host, nlos_stats* stats_host, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!params || !tau0_host || !u_out_host)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_host: null pointer");
    const nlos_params& p = *params;
    NLOS_TRY(validate_params(p, "nlos_reconstruct_host"));
    if (stats_host) std::memset(stats_host, 0, sizeof(*stats_host));
    return reconstruct_host(*reinterpret_cast<Plan*>(plan), p, tau0_host, u_out_host, tau_out_host, stats_host,
                            reinterpret_cast<cudaStream_t>(stream));
  })
}

nlos_status nlos_reconstruct_prepare(nlos_plan plan, const nlos_params* params, const float* tau0_dev,
                                     float* u_out_dev, float* tau_out_dev, int32_t* graphed, void* stream) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (graphed) *graphed = 0;
    if (!params || !tau0_dev || !u_out_dev || !aligned16(tau0_dev) || !aligned16(u_out_dev))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_reconstruct_prepare: null or non-16-byte-aligned pointer");
    const nlos_params& p = *params;
    NLOS_TRY(validate_params(p, "nlos_reconstruct_prepare"));
    bool ready = false;
    NLOS_TRY(reconstruct_prepare(*reinterpret_cast<Plan*>(plan), p, tau0_dev, u_out_dev, tau_out_dev, &ready,
                                 reinterpret_cast<cudaStream_t>(stream)));
    if (graphed) *graphed = ready ? 1 : 0;
    return NLOS_OK;
  })
}

nlos_status nlos_selftest_wait_timeout(int32_t wait_ms, int32_t* status_dev, void* stream) {
  return selftest_wait_timeout(wait_ms, status_dev, reinterpret_cast<cudaStream_t>(stream));
}

nlos_status nlos_timing_enable(nlos_plan plan, int32_t enable) {
  API_GUARD({
    if (!plan) return fail(NLOS_ERR_INVALID_ARG, "null plan");
    Plan& P = *reinterpret_cast<Plan*>(plan);
    P.timing = enable != 0;
    P.ev_used = 0;
    return NLOS_OK;
  })
}

nlos_status nlos_timing_read(nlos_plan plan, double* ms, int32_t* launches, int32_t n) {
  API_GUARD({
    NLOS_TRY(check_plan(plan));
    if (!ms || !launches || n <= 0) return fail(NLOS_ERR_INVALID_ARG, "nlos_timing_read: bad output arrays");
    Plan& P = *reinterpret_cast<Plan*>(plan);
    NLOS_CUDA(cudaDeviceSynchronize());
    for (int i = 0; i < n; ++i) {
      ms[i] = 0.0;
      launches[i] = 0;
    }
    for (size_t k = 0; k < P.ev_used / 2; ++k) {
      float t = 0.f;
      NLOS_CUDA(cudaEventElapsedTime(&t, P.ev[2 * k], P.ev[2 * k + 1]));
      const int c = P.ev_cat[k];
      if (c < n) {
        ms[c] += t;
        launches[c] += 1;
      }
    }
    P.ev_used = 0;
    return NLOS_OK;
  })
}

}  // extern "C"
