// Shared-memory halo-tiled stencils of Algorithm 1 (Eq. 7, Eq. 12, the
// right-hand side of the PDE above Eq. 11, kappa and phi of Sec. 3).
//
// A block owns a TY x TT tile of the (y, t) plane (TT = 128 time bins along
// the contiguous axis, TY = 8 rows) and marches through XB consecutive x
// planes.  Per x plane it stages the fields that are read at neighbours
// (with their +-1 halos, periodic wrap) in shared memory, evaluates the
// per-point quantity whose backward differences are needed (the normal field
// n, or q = v + Lambda/mu) over the tile plus its -1 halo, and finishes the
// interior.  The x-direction backward difference uses the value the same
// thread computed on the previous plane, kept in registers.  Fields read
// only at the voxel itself go straight from HBM to registers (coalesced).
// Each thread owns 4 interior voxels t = t0 + lane + 32 j, so shared-memory
// reads of a warp are unit-stride.
#pragma once

#include "fft.cuh"
#include "stencil.cuh"

namespace nlos {

constexpr int kTT = 128;                  // tile extent along t
constexpr int kTY = 8;                    // tile extent along y
constexpr int kTileThreads = 256;         // 8 warps: warp = row iy, lane = t offset
constexpr int kUW = kTT + 2, kUH = kTY + 2;  // staged field with -1/+1 halos: (TY+2) x (TT+2)
constexpr int kRW = kTT + 1, kRH = kTY + 1;  // region of per-point quantities: (TY+1) x (TT+1)

// Stage plane x of field f over y in [y0 + ylo, y0 + ylo + H), t in
// [t0 + tlo, t0 + tlo + W) into tile[H][pitch] (periodic wrap).
__device__ __forceinline__ void stage_plane(float* __restrict__ tile, int H, int W, int pitch,
                                            const float* __restrict__ f, const Vox& g, int x, int y0, int ylo,
                                            int t0, int tlo) {
  batched_copy<8, float>(
      H * W, threadIdx.x, blockDim.x,
      [&](int i) {
        const int yy = i / W, tt = i - yy * W;
        const int y = (y0 + ylo + yy) & g.my, t = (t0 + tlo + tt) & g.mt;
        return __ldg(f + g.idx(x, y, t));
      },
      [&](int i, float v) {
        const int yy = i / W, tt = i - yy * W;
        tile[yy * pitch + tt] = v;
      });
}

// Tiled k_pre1: reg = -mu sum_d (q_d(c) - q_d(c - e_d)), q = v + Lam/mu,
// v = shrink(grad ubar - Lam/mu, phi/mu).
__global__ void __launch_bounds__(kTileThreads, 4)
    k_pre1_tiled(const float* __restrict__ ub, const float* __restrict__ lam, const float* __restrict__ ph,
                 float* __restrict__ reg, Vox g, int xb, float mu, size_t V) {
  __shared__ float U[2][kUH * kUW];     // ubar planes x and x+1 over [y0-1, y0+TY] x [t0-1, t0+TT]
  __shared__ float L[3][kRH * kRW];     // Lambda plane x over the region [y0-1, y0+TY) x [t0-1, t0+TT)
  __shared__ float F[kRH * kRW];        // phi plane x over the region
  __shared__ float Q[3][kRH * kRW];     // q over the region
  const int ntile = g.nt / kTT;
  const int t0 = (blockIdx.x % ntile) * kTT;
  const int y0 = (blockIdx.x / ntile) * kTY;
  const int x0 = blockIdx.y * xb;
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;

  // q_x on plane x0 - 1 at this thread's voxels (the backward neighbour of the first plane)
  float qx_prev[4];
  {
    const int xm = (x0 - 1) & g.mx, y = y0 + iy;
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + lane + 32 * j;
      qx_prev[j] = v_at(ub, lam, V, ph, g, xm, y, t, inv_mu).x + __ldg(lam + g.idx(xm, y, t)) * inv_mu;
    }
  }
  stage_plane(U[0], kUH, kUW, kUW, ub, g, x0, y0, -1, t0, -1);
  for (int s = 0; s < xb; ++s) {
    const int x = x0 + s;
    float* Ux = U[s & 1];
    float* Un = U[(s + 1) & 1];
    stage_plane(Un, kUH, kUW, kUW, ub, g, (x + 1) & g.mx, y0, -1, t0, -1);
    for (int c = 0; c < 3; ++c) stage_plane(L[c], kRH, kRW, kRW, lam + c * V, g, x, y0, -1, t0, -1);
    stage_plane(F, kRH, kRW, kRW, ph, g, x, y0, -1, t0, -1);
    __syncthreads();
    // q over the region (region point (yy, tt) <-> (y0 - 1 + yy, t0 - 1 + tt))
    for (int i = threadIdx.x; i < kRH * kRW; i += blockDim.x) {
      const int yy = i / kRW, tt = i - yy * kRW;
      const float c = Ux[yy * kUW + tt];
      const float l0 = L[0][i], l1 = L[1][i], l2 = L[2][i];
      const float3 a = make_float3(Un[yy * kUW + tt] - c - l0 * inv_mu, Ux[(yy + 1) * kUW + tt] - c - l1 * inv_mu,
                                   Ux[yy * kUW + tt + 1] - c - l2 * inv_mu);
      const float3 v = shrink3(a, F[i] * inv_mu);
      Q[0][i] = v.x + l0 * inv_mu;
      Q[1][i] = v.y + l1 * inv_mu;
      Q[2][i] = v.z + l2 * inv_mu;
    }
    __syncthreads();
    const int y = y0 + iy;
    for (int j = 0; j < 4; ++j) {
      const int it = lane + 32 * j;
      const int r = (iy + 1) * kRW + it + 1;
      const float qx = Q[0][r];
      const float div = (qx - qx_prev[j]) + (Q[1][r] - Q[1][r - kRW]) + (Q[2][r] - Q[2][r - 1]);
      reg[g.idx(x, y, t0 + it)] = -mu * div;
      qx_prev[j] = qx;
    }
    __syncthreads();
  }
}

// Tiled k_post1: Lam += mu (v - grad u+), phi = phi(kappa(u+)),
// ubar' = u+ + beta (u+ - u^k); partials 0 = sum phi |grad u+|, 1 = |v - grad u+|^2.
__global__ void __launch_bounds__(kTileThreads, 3)
    k_post1_tiled(const float* __restrict__ unew, const float* __restrict__ uk, const float* __restrict__ ub,
                  float* __restrict__ lam, float* __restrict__ ph, float* __restrict__ ubn,
                  const DevScalars* __restrict__ sc, Vox g, int xb, float mu, float a, float b, int kind, float eps2,
                  size_t V, double* __restrict__ partials) {
  __shared__ float U[2][kUH * kUW];     // u+ planes x, x+1 over [y0-1, y0+TY] x [t0-1, t0+TT]
  __shared__ float B[2][kRH * kRW];     // ubar planes x, x+1 over [y0, y0+TY] x [t0, t0+TT]
  __shared__ float N[3][kRH * kRW];     // normal field of plane x over [y0-1, y0+TY) x [t0-1, t0+TT)
  const int ntile = g.nt / kTT;
  const int t0 = (blockIdx.x % ntile) * kTT;
  const int y0 = (blockIdx.x / ntile) * kTY;
  const int x0 = blockIdx.y * xb;
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;
  const float beta = (float)sc->beta;

  float nx_prev[4];
  {
    const int xm = (x0 - 1) & g.mx, y = y0 + iy;
    for (int j = 0; j < 4; ++j) nx_prev[j] = normal_of(grad_at(unew, g, xm, y, t0 + lane + 32 * j), eps2).x;
  }
  stage_plane(U[0], kUH, kUW, kUW, unew, g, x0, y0, -1, t0, -1);
  stage_plane(B[0], kRH, kRW, kRW, ub, g, x0, y0, 0, t0, 0);
  double acc[2] = {0.0, 0.0};
  for (int s = 0; s < xb; ++s) {
    const int x = x0 + s;
    const float* Ux = U[s & 1];
    float* Un = U[(s + 1) & 1];
    const float* Bx = B[s & 1];
    float* Bn = B[(s + 1) & 1];
    stage_plane(Un, kUH, kUW, kUW, unew, g, (x + 1) & g.mx, y0, -1, t0, -1);
    stage_plane(Bn, kRH, kRW, kRW, ub, g, (x + 1) & g.mx, y0, 0, t0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < kRH * kRW; i += blockDim.x) {
      const int yy = i / kRW, tt = i - yy * kRW;
      const float c = Ux[yy * kUW + tt];
      const float3 n = normal_of(
          make_float3(Un[yy * kUW + tt] - c, Ux[(yy + 1) * kUW + tt] - c, Ux[yy * kUW + tt + 1] - c), eps2);
      N[0][i] = n.x;
      N[1][i] = n.y;
      N[2][i] = n.z;
    }
    __syncthreads();
    const int y = y0 + iy;
    // all per-voxel HBM loads first, so 20 are in flight per thread
    float l0[4], l1[4], l2[4], phv[4], ukv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const size_t gi = g.idx(x, y, t0 + lane + 32 * j);
      l0[j] = __ldg(lam + gi);
      l1[j] = __ldg(lam + V + gi);
      l2[j] = __ldg(lam + 2 * V + gi);
      phv[j] = __ldg(ph + gi);
      ukv[j] = __ldg(uk + gi);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int it = lane + 32 * j;
      const int r = (iy + 1) * kRW + it + 1;     // region index of the voxel
      const int u = (iy + 1) * kUW + it + 1;     // staged-u+ index of the voxel
      const int bq = iy * kRW + it;              // staged-ubar index of the voxel
      const float kap = (N[0][r] - nx_prev[j]) + (N[1][r] - N[1][r - kRW]) + (N[2][r] - N[2][r - 1]);
      nx_prev[j] = N[0][r];
      const float uc = Ux[u];
      const float3 gu = make_float3(Un[u] - uc, Ux[u + kUW] - uc, Ux[u + 1] - uc);
      const size_t gi = g.idx(x, y, t0 + it);
      const float bc = Bx[bq];
      const float3 av = make_float3(Bn[bq] - bc - l0[j] * inv_mu, Bx[bq + kRW] - bc - l1[j] * inv_mu,
                                    Bx[bq + 1] - bc - l2[j] * inv_mu);
      const float3 v = shrink3(av, phv[j] * inv_mu);
      const float3 d = make_float3(v.x - gu.x, v.y - gu.y, v.z - gu.z);
      lam[gi] = l0[j] + mu * d.x;
      lam[V + gi] = l1[j] + mu * d.y;
      lam[2 * V + gi] = l2[j] + mu * d.z;
      const float pn = phi_of(kap, a, b, kind);
      ph[gi] = pn;
      ubn[gi] = uc + beta * (uc - ukv[j]);
      acc[0] += (double)pn * (double)sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z);
      acc[1] += (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z;
    }
    __syncthreads();
  }
  // block partials (grid is 2-D: flatten the block index)
  __shared__ double red[kTileThreads / 32][2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    double v = acc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[t] = v;
  }
  if (lane == 0) {
    red[iy][0] = acc[0];
    red[iy][1] = acc[1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      s0 += red[w][0];
      s1 += red[w][1];
    }
    const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    partials[bid * kMaxTerms + 0] = s0;
    partials[bid * kMaxTerms + 1] = s1;
  }
}

}  // namespace nlos
