// Runtime dispatch of the t-pass launchers to their per-size instances
// (tpass_*.cu), and the launch-shape tuner of the t-passes.
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "tpass.cuh"

namespace nlos {

extern template struct TpassOps<16>;
extern template struct TpassOps<32>;
extern template struct TpassOps<64>;
extern template struct TpassOps<128>;
extern template struct TpassOps<256>;
extern template struct TpassOps<512>;
extern template struct TpassOps<1024>;

#define NLOS_DISPATCH_NT(nt, call)                                  \
  switch (nt) {                                                      \
    case 16: return TpassOps<16>::call;                              \
    case 32: return TpassOps<32>::call;                              \
    case 64: return TpassOps<64>::call;                              \
    case 128: return TpassOps<128>::call;                            \
    case 256: return TpassOps<256>::call;                            \
    case 512: return TpassOps<512>::call;                            \
    case 1024: return TpassOps<1024>::call;                          \
  }                                                                  \
  return fail(NLOS_ERR_INVALID_ARG, "unsupported nt")

nlos_status prepare_tpass(int nt) {
  NLOS_TRY(prepare_tpass_warp(nt));
  NLOS_DISPATCH_NT(nt, prepare());
}

nlos_status launch_tfwd_rz(const Plan& P, const float* u, int ncols, float2* S, int pitch, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tfwd_rz(P, u, ncols, S, pitch, st));
}
nlos_status launch_tfwd_rtt(const Plan& P, const Lin3& r, int ncols, float2* S, int pitch, cudaStream_t st) {
  if (tpass_warp_applies(P, ncols, pitch)) return launch_tfwd_rtt_warp(P, r, S, pitch, st);
  NLOS_DISPATCH_NT(P.nt, tfwd_rtt(P, r, ncols, S, pitch, st));
}
nlos_status launch_tinv_store(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                              const int32_t* outmap, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tinv_store(P, S, pitch, ncols, out, outmap, st));
}
nlos_status launch_tinv_fit(const Plan& P, const float2* S, int pitch, int ncols, float* out, const FitArgs& fa,
                            int* nblocks, cudaStream_t st) {
  if (tpass_warp_applies_cols(P, ncols, pitch)) return launch_tinv_fit_warp(P, S, pitch, out, fa, nblocks, st);
  NLOS_DISPATCH_NT(P.nt, tinv_fit(P, S, pitch, ncols, out, fa, nblocks, st));
}
nlos_status launch_tadj_store(const Plan& P, const float2* S, int pitch, int ncols, float* out, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tadj_store(P, S, pitch, ncols, out, st));
}
nlos_status launch_tadj_solve(const Plan& P, const float2* S, int pitch, int ncols, const SolveRhs& sr, float2* Sp,
                              cudaStream_t st) {
  if (tpass_warp_applies(P, ncols, pitch)) return launch_tadj_solve_warp(P, S, pitch, sr, Sp, st);
  NLOS_DISPATCH_NT(P.nt, tadj_solve(P, S, pitch, ncols, sr, Sp, st));
}
nlos_status launch_sfwd(const Plan& P, const float* x, int ncols, float2* Sp, cudaStream_t st, const float* x2) {
  NLOS_DISPATCH_NT(P.nt, sfwd(P, x, x2, ncols, Sp, st));
}
nlos_status launch_sinv(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref, double* partials,
                        int* nblocks, cudaStream_t st) {
  if (tpass_warp_applies(P, ncols, ncols)) return launch_sinv_warp(P, Sp, ncols, x, ref, partials, nblocks, st);
  NLOS_DISPATCH_NT(P.nt, sinv(P, Sp, ncols, x, ref, partials, nblocks, st));
}
nlos_status launch_sinv_rz(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref,
                           double* partials, int* nblocks, float2* S, int pitch, cudaStream_t st, DevScalars* sc) {
  if (tpass_warp_applies(P, ncols, pitch))
    return launch_sinv_rz_warp(P, Sp, pitch, x, ref, partials, nblocks, S, sc, st);
  NLOS_DISPATCH_NT(P.nt, sinv_rz(P, Sp, ncols, x, ref, partials, nblocks, S, pitch, st));
}

}  // namespace nlos

namespace nlos {

// ---------------------------------------------------------------------------
// t-pass launch-shape tuning
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tp_mu;
std::map<std::tuple<int, int, int>, int> g_tp_cols;  // (kind, nt, ncols) -> cols | hb << 8
thread_local int g_tp_force = 0;                       // candidate under test (tuner only)
bool g_tp_loaded = false;                              // tuning file read (under g_tp_mu)

// Tuning file: the tuner's choices persist across processes, keyed by the
// device name, its SM count and the compile time of the library (a choice made for
// other kernels or another GPU is never reused).  Path: $NLOS_TUNE_CACHE, or
// $XDG_CACHE_HOME/nlos-gb300/tpass_tuning, or $HOME/.cache/nlos-gb300/
// tpass_tuning; NLOS_TUNE_CACHE=off (or empty) keeps the choices in the
// process only.  Read and write failures leave the in-process behaviour
// unchanged.
const char kTuneMagic[] = "nlos-gb300 t-pass tuning v1";
const char kBuildId[] = __DATE__ " " __TIME__;

std::string tune_path() {
  if (const char* e = std::getenv("NLOS_TUNE_CACHE")) {
    const std::string v(e);
    return v == "off" ? std::string() : v;
  }
  std::string dir;
  if (const char* x = std::getenv("XDG_CACHE_HOME"); x && *x)
    dir = std::string(x) + "/nlos-gb300";
  else if (const char* h = std::getenv("HOME"); h && *h)
    dir = std::string(h) + "/.cache/nlos-gb300";
  else
    return std::string();
  return dir + "/tpass_tuning";
}

std::string tune_key() {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return std::string();
  }
  return std::string(prop.name) + " | " + std::to_string(prop.multiProcessorCount) + " SMs | " + kBuildId;
}

void tune_load_locked() {
  g_tp_loaded = true;
  const std::string path = tune_path(), key = tune_key();
  if (path.empty() || key.empty()) return;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  char line[512];
  const bool ok = std::fgets(line, sizeof line, f) && std::string(line) == std::string(kTuneMagic) + "\n" &&
                  std::fgets(line, sizeof line, f) && std::string(line) == key + "\n";
  int kind = 0, nt = 0, ncols = 0, v = 0;
  while (ok && std::fscanf(f, "%d %d %d %d", &kind, &nt, &ncols, &v) == 4)
    g_tp_cols.emplace(std::make_tuple(kind, nt, ncols), v);
  std::fclose(f);
}

void tune_save_locked() {
  const std::string path = tune_path(), key = tune_key();
  if (path.empty() || key.empty()) return;
  for (size_t i = 1; i < path.size(); ++i)  // create the directories of the path
    if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "%s\n%s\n", kTuneMagic, key.c_str());
  for (const auto& e : g_tp_cols)
    std::fprintf(f, "%d %d %d %d\n", std::get<0>(e.first), std::get<1>(e.first), std::get<2>(e.first), e.second);
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) std::remove(tmp.c_str());
}
}  // namespace

int tp_cols_for(int kind, int nt, int ncols) {
  if (g_tp_force) return g_tp_force;
  std::lock_guard<std::mutex> lock(g_tp_mu);
  auto it = g_tp_cols.find(std::make_tuple(kind, nt, ncols));
  return it == g_tp_cols.end() ? 0 : it->second;
}

// Times every column count (and, for the kernels with two halves, both the
// sequential and the batched halves) for each t-pass kind the plan launches
// and keeps the fastest; likewise the two kernels of the lateral solve.  Inputs are the plan's scratch buffers with whatever they hold
// (the kernels' addressing depends only on the tables and the shape, so any
// contents are safe); nothing outside the plan is written.
nlos_status autotune_tpass(Plan& P, cudaStream_t st) {
  const int nt = P.nt, full = P.nx * P.ny;
  const size_t V = (size_t)full * nt;
  float* f1 = reinterpret_cast<float*>(P.d_S2);  // 2 (nt + 1) full floats: two fields
  float* f2 = f1 + V;
  float* f3 = reinterpret_cast<float*>(P.d_Sp);  // (nt + 2) full floats: one field
  DevScalars* dsc = nullptr;
  NLOS_CUDA(cudaMalloc(&dsc, sizeof(DevScalars)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  nlos_status status = NLOS_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemsetAsync(dsc, 0, sizeof(DevScalars), st) != cudaSuccess)
    status = fail(NLOS_ERR_CUDA, "autotune: setup");
  int nb = 0;
  struct Case {
    int kind, ncols;
    bool partials;
    std::function<nlos_status()> run;
  };
  const int nc = P.ncols;  // compact launches; captured by value below
  const Lin3 r_full{{f3, nullptr, nullptr}, {1.f, 0.f, 0.f}, nullptr};
  const Lin3 r_comp{{P.d_tmpc, nullptr, nullptr}, {1.f, 0.f, 0.f}, nullptr};
  const SolveRhs sr{f1, f2, nullptr, 1.0};
  const FitArgs fa_full{f1, f2, f1, dsc, P.d_partials};
  const FitArgs fa_comp{P.d_tmpc, P.d_tmpc, P.d_tmpc, dsc, P.d_partials};
  std::vector<Case> cases = {
      {TPK_TFWD_RZ, full, false, [&] { return launch_tfwd_rz(P, f3, full, P.d_S, full, st); }},
      {TPK_TFWD_RTT, full, false, [&] { return launch_tfwd_rtt(P, r_full, full, P.d_S, full, st); }},
      {TPK_TINV_STORE, full, false, [&] { return launch_tinv_store(P, P.d_S, full, full, f3, nullptr, st); }},
      {TPK_TINV_FIT, full, true, [&] { return launch_tinv_fit(P, P.d_S, full, full, f3, fa_full, &nb, st); }},
      {TPK_TADJ_STORE, full, false, [&] { return launch_tadj_store(P, P.d_S, full, full, f1, st); }},
      {TPK_TADJ_SOLVE, full, false, [&] { return launch_tadj_solve(P, P.d_S, full, full, sr, P.d_Sp, st); }},
      {TPK_SFWD, full, false, [&] { return launch_sfwd(P, f1, full, P.d_Sp, st); }},
      {TPK_SINV, full, true, [&] { return launch_sinv(P, P.d_Sp, full, f1, f2, P.d_partials, &nb, st); }},
      {TPK_SINV_RZ, full, true,
       [&] { return launch_sinv_rz(P, P.d_Sp, full, f1, f2, P.d_partials, &nb, P.d_S, full, st); }},
  };
  // the lateral solve's kernel (its input, the periodic spectrum scratch,
  // holds whatever it holds; the denominators c0 + c1 (...) are >= 1)
  if (P.nx >= 32)
    cases.push_back({TPK_SXY, P.nx, false, [&] { return launch_sxy(P, P.d_Sp, nullptr, 1.0, 1.0, st); }});
  if (nc < full) {
    cases.push_back({TPK_TFWD_RTT, nc, false, [&, nc] { return launch_tfwd_rtt(P, r_comp, nc, P.d_Sc, nc, st); }});
    cases.push_back(
        {TPK_TINV_FIT, nc, true, [&, nc] { return launch_tinv_fit(P, P.d_Sc, nc, nc, f1, fa_comp, &nb, st); }});
    cases.push_back(
        {TPK_TINV_STORE, nc, false, [&, nc] { return launch_tinv_store(P, P.d_Sc, nc, nc, f1, nullptr, st); }});
  }
  const int max_cols = nt >= 1024 ? 8 : 16;
  {
    std::lock_guard<std::mutex> lock(g_tp_mu);
    if (!g_tp_loaded) tune_load_locked();
  }
  bool added = false;
  for (const Case& c : cases) {
    if (status != NLOS_OK) break;
    {
      std::lock_guard<std::mutex> lock(g_tp_mu);
      if (g_tp_cols.count(std::make_tuple(c.kind, nt, c.ncols))) continue;
    }
    // the warp-per-pair kernels have a fixed shape: nothing to tune
    const bool warp_kind = c.kind == TPK_TADJ_SOLVE || c.kind == TPK_SINV_RZ || c.kind == TPK_SINV ||
                           c.kind == TPK_TINV_FIT || c.kind == TPK_TFWD_RTT;
    const bool compact_kind = c.kind == TPK_TINV_FIT;
    if (warp_kind && (compact_kind ? tpass_warp_applies_cols(P, c.ncols, c.ncols)
                                   : tpass_warp_applies(P, c.ncols, c.ncols)))
      continue;
    const bool halves = c.kind != TPK_SFWD && c.kind != TPK_SINV;  // sinv_rz: its forward half
    const bool variant = c.kind == TPK_SXY;  // a choice between two kernels, not a shape
    int best = 0;
    float best_ms = 0.f;
    for (int cand = 0; cand < 8 && status == NLOS_OK; ++cand) {
      const int cols = max_cols >> (cand >> 1), hb = cand & 1;
      if (variant) {
        if (cand >= 2) break;
        g_tp_force = cand == 0 ? kSxyHalfWarp : kSxyPasses;
      } else {
        if (cols < 2 || (hb && !halves)) continue;
        if (c.partials && (c.ncols + cols - 1) / cols > P.partial_blocks) continue;
        g_tp_force = cols | hb << 8;
      }
      float t = 0.f;
      status = c.run();  // warm-up
      // best of 2 timings of 2 back-to-back launches (the launch latency of a
      // short kernel, and any per-launch overhead of a tool, is amortised)
      for (int rep = 0; rep < 2 && status == NLOS_OK; ++rep) {
        float ms = 0.f;
        if (cudaEventRecord(e0, st) != cudaSuccess) status = fail(NLOS_ERR_CUDA, "autotune: event");
        for (int l = 0; l < 2 && status == NLOS_OK; ++l) status = c.run();
        if (status == NLOS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                  cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          status = fail(NLOS_ERR_CUDA, "autotune: timing");
        if (rep == 0 || ms < t) t = ms;
      }
      const int chosen = g_tp_force;
      g_tp_force = 0;
      if (status == NLOS_OK && (best == 0 || t < best_ms)) {
        best = chosen;
        best_ms = t;
      }
    }
    if (status == NLOS_OK && best) {
      std::lock_guard<std::mutex> lock(g_tp_mu);
      added = g_tp_cols.emplace(std::make_tuple(c.kind, nt, c.ncols), best).second || added;  // first plan decides
    }
  }
  if (status == NLOS_OK && added) {
    std::lock_guard<std::mutex> lock(g_tp_mu);
    tune_save_locked();
  }
  g_tp_force = 0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dsc);
  return status;
}

}  // namespace nlos
