// Finite-difference helpers of the curvature sub-steps (Sec. 3):
// forward-difference gradient with periodic wrap, the regularised normal
// field n = grad u / sqrt(|grad u|^2 + eps^2), curvature kappa = backward
// divergence of n, phi(kappa) and the isotropic shrinkage of Eq. 7.
#pragma once

#include "common.cuh"

namespace nlos {

struct Vox {
  int nx, ny, nt;          // powers of two
  int mx, my, mt;          // n - 1 masks
  int sx, sy;              // strides of x and y (sy = nt, sx = ny * nt)
  __device__ __forceinline__ int idx(int x, int y, int t) const { return x * sx + y * sy + t; }
};

inline Vox make_vox(int nx, int ny, int nt) {
  Vox v;
  v.nx = nx; v.ny = ny; v.nt = nt;
  v.mx = nx - 1; v.my = ny - 1; v.mt = nt - 1;
  v.sy = nt; v.sx = ny * nt;
  return v;
}

// grad u at (x, y, t): forward differences, periodic.
__device__ __forceinline__ float3 grad_at(const float* __restrict__ u, const Vox& g, int x, int y, int t) {
  const float c = __ldg(u + g.idx(x, y, t));
  return make_float3(__ldg(u + g.idx((x + 1) & g.mx, y, t)) - c, __ldg(u + g.idx(x, (y + 1) & g.my, t)) - c,
                     __ldg(u + g.idx(x, y, (t + 1) & g.mt)) - c);
}

// (rsqrtf: within 2 ulp, far inside the operator tolerance, and a fraction of
// the instructions of an IEEE square root followed by an IEEE division)
__device__ __forceinline__ float3 normal_of(float3 d, float eps2) {
  const float inv = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z + eps2);
  return make_float3(d.x * inv, d.y * inv, d.z * inv);
}

// kappa at (x, y, t) = sum_d n_d(c) - n_d(c - e_d)
__device__ __forceinline__ float curvature_at(const float* __restrict__ u, const Vox& g, int x, int y, int t,
                                              float eps2, float3* grad_c) {
  const float3 gc = grad_at(u, g, x, y, t);
  if (grad_c) *grad_c = gc;
  const float3 nc = normal_of(gc, eps2);
  const float3 nxm = normal_of(grad_at(u, g, (x - 1) & g.mx, y, t), eps2);
  const float3 nym = normal_of(grad_at(u, g, x, (y - 1) & g.my, t), eps2);
  const float3 ntm = normal_of(grad_at(u, g, x, y, (t - 1) & g.mt), eps2);
  return (nc.x - nxm.x) + (nc.y - nym.y) + (nc.z - ntm.z);
}

__device__ __forceinline__ float phi_of(float k, float a, float b, int kind) {
  if (kind == NLOS_PHI_TAC) return a + b * fabsf(k);
  if (kind == NLOS_PHI_TRV) return sqrtf(a + b * k * k);
  return a + b * k * k;
}

// shrinkage(a, th) = max(|a| - th, 0) a / |a|, shrink(0, th) = 0 (Eq. 7),
// as a scale max(1 - th / |a|, 0) with th / |a| = th rsqrt(|a|^2)
__device__ __forceinline__ float3 shrink3(float3 a, float th) {
  const float n2 = a.x * a.x + a.y * a.y + a.z * a.z;
  if (!(n2 > 0.0f)) return make_float3(0.f, 0.f, 0.f);
  const float s = fmaxf(1.0f - th * rsqrtf(n2), 0.0f);
  return make_float3(a.x * s, a.y * s, a.z * s);
}

// v = shrink(grad ubar - Lam/mu, phi/mu) at one voxel, Lam as three planes.
__device__ __forceinline__ float3 v_at(const float* __restrict__ ub, const float* __restrict__ lam, size_t vs,
                                       const float* __restrict__ ph, const Vox& g, int x, int y, int t, float inv_mu) {
  const int i = g.idx(x, y, t);
  const float3 gb = grad_at(ub, g, x, y, t);
  const float3 a = make_float3(gb.x - __ldg(lam + i) * inv_mu, gb.y - __ldg(lam + vs + i) * inv_mu,
                               gb.z - __ldg(lam + 2 * vs + i) * inv_mu);
  return shrink3(a, __ldg(ph + i) * inv_mu);
}

}  // namespace nlos
