// Midpoint conversion of non-confocal transients into confocal ones (Sec. 4,
// evaluation on non-confocal data: the confocal solvers run on a non-confocal
// measurement after the midpoint approximation of f-k migration, which the
// paper cites without stating).
//
// A measurement with the laser at the wall point l and the detector at s is
// treated as a confocal measurement at the midpoint m = (l + s) / 2.  For a
// scatterer on the wall normal through m at depth z the non-confocal path is
// 2 sqrt(z^2 + |s - l|^2 / 4) and the confocal one 2 z, so the arrival times
// satisfy t_nc^2 = t_c^2 + q2 with q2 = |s - l|^2 / c^2.  Confocal bin k
// (centre t_k = (k + 1/2) dt) therefore reads the non-confocal record at
//     p = sqrt(t_k^2 + q2) / dt - 1/2   bins,
// by two-tap linear interpolation between bin centres, zero past the last
// bin; the amplitude is not changed.  Detector (i, j) sits at the scan grid
// centre (x_i, y_j), x_i = (i + 1/2 - nx/2) W / nx.
//
// One warp per column: q2 once per column, then 32 consecutive bins per
// step, whose taps are nearly consecutive too (p(k + 1) - p(k) = t_k / t_nc
// <= 1).  The source position is formed in FP64 with explicitly rounded
// operations and no fused multiply-add, so tap index and weight come from the
// same sequence of IEEE operations as a host evaluation of the formula; the
// interpolation is FP32.  FP64 runs at a small fraction of the FP32 rate on
// this GPU, so the pass is bound by its FP64 work (one square root per bin),
// not by its two memory passes; it runs once per measurement, before the
// solver.
#include <cmath>

#include "common.cuh"

namespace nlos {

constexpr double kLightSpeedMps = 299792458.0;
constexpr int kMidThreads = 256;

__global__ void __launch_bounds__(kMidThreads)
    k_midpoint(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int nt, double dt,
               double inv_dt, double pitch_x, double pitch_y, double lx, double ly, double c2) {
  const int lane = threadIdx.x & 31;
  const int warps = (int)(gridDim.x * (kMidThreads / 32));
  const int ncols = nx * ny;
  for (int col = (int)(blockIdx.x * (kMidThreads / 32) + (threadIdx.x >> 5)); col < ncols; col += warps) {
    const int i = col / ny, j = col - (col / ny) * ny;
    const double xi = __dmul_rn((double)i + 0.5 - 0.5 * nx, pitch_x);
    const double yj = __dmul_rn((double)j + 0.5 - 0.5 * ny, pitch_y);
    const double dx = __dsub_rn(xi, lx), dy = __dsub_rn(yj, ly);
    const double q2 = __ddiv_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), c2);
    const float* s = src + (size_t)col * nt;
    float* d = dst + (size_t)col * nt;
    for (int k = lane; k < nt; k += 32) {
      const double tk = __dmul_rn((double)k + 0.5, dt);
      const double tp = __dsqrt_rn(__dadd_rn(__dmul_rn(tk, tk), q2));
      const double p = __dsub_rn(__dmul_rn(tp, inv_dt), 0.5);
      const double fl = floor(p);
      const float w = (float)(p - fl);  // exact in FP64, rounded once to FP32
      const long long i0 = (long long)fl;  // >= k >= 0: the warp never reads earlier times
      const float a = i0 < nt ? __ldg(s + i0) : 0.0f;
      const float b = i0 + 1 < nt ? __ldg(s + i0 + 1) : 0.0f;
      d[k] = (1.0f - w) * a + w * b;
    }
  }
}

}  // namespace nlos

using namespace nlos;

extern "C" nlos_status nlos_midpoint_confocal(int32_t nx, int32_t ny, int32_t nt, double bin_width_s,
                                              double wall_width_m, double laser_x_m, double laser_y_m,
                                              const float* tau_nc_dev, float* tau_c_dev, void* stream) {
  try {
    auto pow2 = [](int n) { return n > 0 && (n & (n - 1)) == 0; };
    if (!pow2(nx) || !pow2(ny) || !pow2(nt) || nx < 2 || ny < 2 || nt < 2)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: nx, ny, nt must be powers of two >= 2");
    if ((long long)nx * ny > (1LL << 30) || (long long)nx * ny * nt > (1LL << 40))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: grid too large");
    if (!(bin_width_s > 0.0) || !std::isfinite(bin_width_s) || !(wall_width_m > 0.0) || !std::isfinite(wall_width_m) ||
        !std::isfinite(laser_x_m) || !std::isfinite(laser_y_m))
      return fail(NLOS_ERR_INVALID_ARG,
                  "nlos_midpoint_confocal: need bin_width_s > 0, wall_width_m > 0 and a finite laser point");
    if (!tau_nc_dev || !tau_c_dev || (reinterpret_cast<uintptr_t>(tau_nc_dev) & 3) ||
        (reinterpret_cast<uintptr_t>(tau_c_dev) & 3))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: null or misaligned buffer");
    const size_t bytes = (size_t)nx * ny * nt * sizeof(float);
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(tau_nc_dev), b0 = reinterpret_cast<uintptr_t>(tau_c_dev);
    if (a0 < b0 + bytes && b0 < a0 + bytes)
      return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: input and output overlap");
    const int ncols = nx * ny;
    const int per_block = kMidThreads / 32;
    const int blocks = (int)std::min<long long>((ncols + per_block - 1) / per_block, 152LL * 16);
    k_midpoint<<<blocks, kMidThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        tau_nc_dev, tau_c_dev, nx, ny, nt, bin_width_s, 1.0 / bin_width_s, wall_width_m / nx, wall_width_m / ny,
        laser_x_m, laser_y_m, kLightSpeedMps * kLightSpeedMps);
    NLOS_LAUNCH_CHECK("k_midpoint");
    return NLOS_OK;
  } catch (...) {
    return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: unexpected internal error");
  }
}
