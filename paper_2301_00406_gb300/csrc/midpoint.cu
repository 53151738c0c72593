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
// One warp per column: the column's offset term once, in FP64, then 32
// consecutive bins per step, whose taps are nearly consecutive too
// (p(k + 1) - p(k) = t_k / t_nc <= 1).  FP64 runs at a small fraction of the
// FP32 rate on this GPU, so the per-bin position is formed in FP32 with a
// compensated square root: in bins, p = sqrt(a^2 + Q) - 1/2 with
// a = k + 1/2 (a^2 exact in FP32 for nt <= 2048) and Q = q2 / dt^2 carried as
// a two-float sum; one Newton correction from the exact FMA residual gives
// p to about 1e-11 bins, so the tap split matches the FP64 evaluation except
// where p lies within that of an integer, where the interpolation is
// continuous anyway.  The pass is then bound by its two memory passes.
#include <cmath>

#include "common.cuh"

namespace nlos {

constexpr double kLightSpeedMps = 299792458.0;
constexpr int kMidThreads = 256;

__global__ void __launch_bounds__(kMidThreads)
    k_midpoint(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, int nt, double inv_dt2,
               double pitch_x, double pitch_y, double lx, double ly, double inv_c2) {
  const int lane = threadIdx.x & 31;
  const int warps = (int)(gridDim.x * (kMidThreads / 32));
  const int ncols = nx * ny;
  for (int col = (int)(blockIdx.x * (kMidThreads / 32) + (threadIdx.x >> 5)); col < ncols; col += warps) {
    const int i = col / ny, j = col - (col / ny) * ny;
    const double dx = ((double)i + 0.5 - 0.5 * nx) * pitch_x - lx;
    const double dy = ((double)j + 0.5 - 0.5 * ny) * pitch_y - ly;
    const double Q = (dx * dx + dy * dy) * inv_c2 * inv_dt2;  // (|s - l| / (c dt))^2, in bins^2
    const float qh = (float)Q, ql = (float)(Q - (double)qh);
    const float* s = src + (size_t)col * nt;
    float* d = dst + (size_t)col * nt;
    for (int k = lane; k < nt; k += 32) {
      const float a = (float)k + 0.5f;
      const float a2 = a * a;  // exact
      // a2 + Q as sh + sl (two-sum of a2 and qh, plus ql)
      const float sh = a2 + qh;
      const float bv = sh - a2;
      const float sl = ((a2 - (sh - bv)) + (qh - bv)) + ql;
      // sqrt(sh + sl) = r + rl: rl from the exact residual sh - r^2
      const float r = sqrtf(sh);
      const float rl = (fmaf(-r, r, sh) + sl) * (0.5f / r);
      const float ph = r - 0.5f;  // exact: r >= 1/2 and ulp(r) <= 1/2 here
      float fl = floorf(ph);
      float w = (ph - fl) + rl;
      if (w < 0.0f) {
        fl -= 1.0f;
        w += 1.0f;
      } else if (w >= 1.0f) {
        fl += 1.0f;
        w -= 1.0f;
      }
      const int i0 = (int)fl;  // >= k: the warp never reads earlier times
      const float va = i0 < nt ? __ldg(s + i0) : 0.0f;
      const float vb = i0 + 1 < nt ? __ldg(s + i0 + 1) : 0.0f;
      d[k] = (1.0f - w) * va + w * vb;
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
    if (nt > 2048 || (long long)nx * ny > (1LL << 30) || (long long)nx * ny * nt > (1LL << 40))
      return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: grid too large (nt <= 2048)");
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
    const int blocks = (int)std::min<long long>((ncols + per_block - 1) / per_block, (long long)device_sm_count() * 16);
    k_midpoint<<<blocks, kMidThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        tau_nc_dev, tau_c_dev, nx, ny, nt, 1.0 / (bin_width_s * bin_width_s), wall_width_m / nx, wall_width_m / ny,
        laser_x_m, laser_y_m, 1.0 / (kLightSpeedMps * kLightSpeedMps));
    NLOS_LAUNCH_CHECK("k_midpoint");
    return NLOS_OK;
  } catch (...) {
    return fail(NLOS_ERR_INVALID_ARG, "nlos_midpoint_confocal: unexpected internal error");
  }
}
