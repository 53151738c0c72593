// nlos_solve_static: the periodic FFT solve of nlos_solve without any device
// allocation and without a plan.
//
// Who needs it: callers that cannot call cudaMalloc at the moment they solve.
// Code whose device memory is owned by another allocator (a framework's
// caching pool) or capped by a fixed budget has no room to take from the
// driver, and real-time loops must stay off the driver's allocation path,
// which can synchronise the whole device.  They pass only their input and
// output buffers.
//
// Scratch: the periodic spectrum lives in g_static_spectrum, a file-scope
// __device__ array of kStaticSpectrumMax complex values (8 MiB, enough for
// nx = ny <= 64 and nt <= 512).  Every GPU that loads this library keeps that
// array (and the small twiddle / eigenvalue tables next to it) until the
// process exits.  All calls share it: two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it and produce
// garbage, so serialise them.  The array keeps the previous call's contents;
// nothing has to start at zero because the forward pass writes every
// spectrum entry the solve later reads.
//
// Set-up: the first call on a device, with that device current, looks up
// the device addresses of the arrays (cudaGetSymbolAddress; host code may not
// use the array names as device pointers), fills the tables with
// cudaMemcpyToSymbol, sets the shared-memory limits of every kernel a later
// call can launch, and synchronises the device, so the tables are in place
// before any stream (also one that does not wait for the legacy default
// stream) runs a solve.  Later calls on that device only launch three
// kernels.
#include <cmath>
#include <mutex>

#include "passes.cuh"

namespace nlos {

constexpr int kStaticMaxN = 64;      // nx = ny <= 64
constexpr int kStaticMaxNt = 512;    // nt <= 512
constexpr size_t kStaticSpectrumMax = (size_t)kStaticMaxN * kStaticMaxN * (kStaticMaxNt / 2 + 1);
// tables for every supported size, concatenated: nt in 16..512, n in 8..64
constexpr int kTwTLen = 2 * (16 + 32 + 64 + 128 + 256 + 512);
constexpr int kTwXLen = 2 * (8 + 16 + 32 + 64);
constexpr int kLamTLen = 16 + 32 + 64 + 128 + 256 + 512;
constexpr int kLamXLen = 8 + 16 + 32 + 64;

static __device__ __align__(256) float2 g_static_spectrum[kStaticSpectrumMax];
static __device__ __align__(256) float2 g_static_tw_t[kTwTLen];
static __device__ __align__(256) float2 g_static_tw_x[kTwXLen];
static __device__ __align__(256) float g_static_lam_t[kLamTLen];
static __device__ __align__(256) float g_static_lam_x[kLamXLen];

namespace {

constexpr int kMaxDevices = 64;

struct StaticDevice {
  bool ready = false;
  float2* spectrum = nullptr;
  float2* tw_t = nullptr;
  float2* tw_x = nullptr;
  float* lam_t = nullptr;
  float* lam_x = nullptr;
};

std::mutex g_static_mu;
StaticDevice g_static_dev[kMaxDevices];

// Offset of size n's table inside the concatenation (sizes start at `first`).
int table_offset(int n, int first, int per_entry) {
  int off = 0;
  for (int m = first; m < n; m *= 2) off += per_entry * m;
  return off;
}

nlos_status setup_device(int dev, StaticDevice* d) {
  NLOS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d->spectrum), g_static_spectrum));
  NLOS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d->tw_t), g_static_tw_t));
  NLOS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d->tw_x), g_static_tw_x));
  NLOS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d->lam_t), g_static_lam_t));
  NLOS_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d->lam_x), g_static_lam_x));
  const double pi = 3.14159265358979323846;
  std::vector<float2> twt(kTwTLen), twx(kTwXLen);
  std::vector<float> lt(kLamTLen), lx(kLamXLen);
  for (int nt = 16; nt <= kStaticMaxNt; nt *= 2) {
    const int o2 = table_offset(nt, 16, 2), o1 = table_offset(nt, 16, 1);
    for (int k = 0; k < 2 * nt; ++k) {
      const double a = -2.0 * pi * k / (2.0 * nt);
      twt[o2 + k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int k = 0; k < nt; ++k) {
      const double s = std::sin(pi * k / nt);
      lt[o1 + k] = (float)(4.0 * s * s);
    }
  }
  for (int n = 8; n <= kStaticMaxN; n *= 2) {
    const int o2 = table_offset(n, 8, 2), o1 = table_offset(n, 8, 1);
    for (int k = 0; k < 2 * n; ++k) {
      const double a = -2.0 * pi * k / (2.0 * n);
      twx[o2 + k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int k = 0; k < n; ++k) {
      const double s = std::sin(pi * k / n);
      lx[o1 + k] = (float)(4.0 * s * s);
    }
  }
  NLOS_CUDA(cudaMemcpyToSymbol(g_static_tw_t, twt.data(), sizeof(float2) * kTwTLen));
  NLOS_CUDA(cudaMemcpyToSymbol(g_static_tw_x, twx.data(), sizeof(float2) * kTwXLen));
  NLOS_CUDA(cudaMemcpyToSymbol(g_static_lam_t, lt.data(), sizeof(float) * kLamTLen));
  NLOS_CUDA(cudaMemcpyToSymbol(g_static_lam_x, lx.data(), sizeof(float) * kLamXLen));
  for (int nt = 16; nt <= kStaticMaxNt; nt *= 2) NLOS_TRY(prepare_tpass(nt));
  for (int n = 8; n <= kStaticMaxN; n *= 2) NLOS_TRY(prepare_xy(n));
  // the copies above are ordered on the legacy stream only, and a copy from
  // pageable memory may return before it lands: finish them before any call
  // launches on another stream
  NLOS_CUDA(cudaDeviceSynchronize());
  d->ready = true;
  (void)dev;
  return NLOS_OK;
}

}  // namespace

}  // namespace nlos

using namespace nlos;

extern "C" nlos_status nlos_solve_static(int32_t nx, int32_t ny, int32_t nt, const float* rhs_dev, float* x_dev,
                                         double c0, double c1, void* stream) {
  try {
    auto pow2 = [](int n) { return n > 0 && (n & (n - 1)) == 0; };
    if (nx != ny || !pow2(nx) || nx < 8 || !pow2(nt) || nt < 16)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_solve_static: need nx == ny, powers of two, nx >= 8, nt >= 16");
    if (nx > kStaticMaxN || nt > kStaticMaxNt || (size_t)nx * ny * (nt / 2 + 1) > kStaticSpectrumMax)
      return fail(NLOS_ERR_INVALID_ARG,
                  "nlos_solve_static: grid exceeds the static scratch (nx = ny <= 64, nt <= 512); use nlos_solve");
    if (!rhs_dev || !x_dev) return fail(NLOS_ERR_INVALID_ARG, "nlos_solve_static: null pointer");
    if (!(c0 > 0.0) || !(c1 >= 0.0) || !std::isfinite(c0) || !std::isfinite(c1))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_solve_static: need c0 > 0 and c1 >= 0");
    int dev = 0;
    NLOS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NLOS_ERR_INVALID_ARG, "nlos_solve_static: device index too large");
    StaticDevice* d = &g_static_dev[dev];
    {
      std::lock_guard<std::mutex> lock(g_static_mu);
      if (!d->ready) NLOS_TRY(setup_device(dev, d));
    }
    // A plan-shaped view of the static arrays: the three solve passes only
    // read the geometry, the twiddle and eigenvalue tables and the spectrum.
    Plan P;
    P.nx = nx;
    P.ny = ny;
    P.nt = nt;
    P.device = dev;
    P.d_tw2t = d->tw_t + table_offset(nt, 16, 2);
    P.d_twx = d->tw_x + table_offset(nx, 8, 2);
    P.d_twy = P.d_twx;
    P.d_lamt = d->lam_t + table_offset(nt, 16, 1);
    P.d_lamx = d->lam_x + table_offset(nx, 8, 1);
    P.d_lamy = P.d_lamx;
    P.d_Sp = d->spectrum;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int full = nx * ny;
    NLOS_TRY(launch_sfwd(P, rhs_dev, full, P.d_Sp, st));
    NLOS_TRY(launch_sxy(P, P.d_Sp, nullptr, c0, c1, st));
    NLOS_TRY(launch_sinv(P, P.d_Sp, full, x_dev, nullptr, nullptr, nullptr, st));
    return NLOS_OK;
  } catch (...) {
    return fail(NLOS_ERR_INVALID_ARG, "nlos_solve_static: unexpected internal error");
  }
}
