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

// ---------------------------------------------------------------------------
// Software-pipelined versions: the planes of step s + 1 are copied into shared
// memory with cp.async while step s computes, and a persistent grid walks the
// (t, y, x-chunk) tiles.  The shared-memory ring holds three halo planes of the
// neighbour-read fields (planes x, x + 1 in use, x + 2 in flight).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// async copy of a halo plane (periodic wrap), element by element
__device__ __forceinline__ void stage_plane_async(float* __restrict__ tile, int H, int W, int pitch,
                                                  const float* __restrict__ f, const Vox& g, int x, int y0, int ylo,
                                                  int t0, int tlo) {
  for (int i = threadIdx.x; i < H * W; i += blockDim.x) {
    const int yy = i / W, tt = i - yy * W;
    const int y = (y0 + ylo + yy) & g.my, t = (t0 + tlo + tt) & g.mt;
    cp_async4(tile + yy * pitch + tt, f + g.idx(x, y, t));
  }
}
// async copy of the TY x TT interior of plane x (rows are contiguous and 16-byte aligned)
__device__ __forceinline__ void stage_interior_async(float* __restrict__ tile, const float* __restrict__ f,
                                                     const Vox& g, int x, int y0, int t0) {
  for (int i = threadIdx.x; i < kTY * kTT / 4; i += blockDim.x) {
    const int yy = i / (kTT / 4), q = i - yy * (kTT / 4);
    cp_async16(tile + yy * kTT + 4 * q, f + g.idx(x, y0 + yy, t0 + 4 * q));
  }
}

constexpr int kPipeXB = 4;  // x planes per tile

struct TileIdx {
  int t0, y0, x0;
};
__device__ __forceinline__ TileIdx tile_of(int tile, const Vox& g) {
  const int ntt = g.nt / kTT, nty = g.ny / kTY;
  TileIdx r;
  r.t0 = (tile % ntt) * kTT;
  r.y0 = ((tile / ntt) % nty) * kTY;
  r.x0 = (tile / (ntt * nty)) * kPipeXB;
  return r;
}

// The ubar ring is padded to a whole number of float4 so that the interior
// region after it, the target of the 16-byte cp.async copies, starts on a
// 16-byte boundary (the U ring before it is 3900 floats, a multiple of 4).
constexpr int kPost1BPlanes = (3 * kRH * kRW + 3) & ~3;
static_assert((3 * kUH * kUW) % 4 == 0, "U ring must end on a 16-byte boundary");
static_assert((3 * kUH * kUW + kPost1BPlanes) % 4 == 0, "interior region must start on a 16-byte boundary");
static_assert((kTY * kTT) % 4 == 0, "interior planes must be whole float4 rows");

// Pipelined k_post1 (same arithmetic as k_post1_tiled).
__global__ void __launch_bounds__(kTileThreads, 2)
    k_post1_pipe(const float* __restrict__ unew, const float* __restrict__ uk, const float* __restrict__ ub,
                 float* __restrict__ lam, float* __restrict__ ph, float* __restrict__ ubn,
                 const DevScalars* __restrict__ sc, Vox g, int ntiles, float mu, float a, float b, int kind,
                 float eps2, size_t V, double* __restrict__ partials) {
  extern __shared__ float4 smem_f4[];
  float* U = reinterpret_cast<float*>(smem_f4);       // [3][kUH * kUW]  u+ planes
  float* B = U + 3 * kUH * kUW;                       // [3][kRH * kRW]  ubar planes
  float* I = B + kPost1BPlanes;                       // [2][5][kTY * kTT] lam0..2, phi, u^k interiors (16-byte aligned)
  float* N = I + 2 * 5 * kTY * kTT;                   // [3][kRH * kRW]  normal field
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;
  const float beta = (float)sc->beta;
  const float* ifields[5] = {lam, lam + V, lam + 2 * V, ph, uk};
  double acc[2] = {0.0, 0.0};
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileIdx T = tile_of(tile, g);
    const int y = T.y0 + iy;
    float nx_prev[4];
    for (int j = 0; j < 4; ++j) {
      const int xm = (T.x0 - 1) & g.mx;
      nx_prev[j] = normal_of(grad_at(unew, g, xm, y, T.t0 + lane + 32 * j), eps2).x;
    }
    // prologue: planes x0 (group 0) and x0 + 1 plus the interiors of x0 (group 1)
    stage_plane_async(U, kUH, kUW, kUW, unew, g, T.x0, T.y0, -1, T.t0, -1);
    stage_plane_async(B, kRH, kRW, kRW, ub, g, T.x0, T.y0, 0, T.t0, 0);
    cp_async_commit();
    stage_plane_async(U + kUH * kUW, kUH, kUW, kUW, unew, g, (T.x0 + 1) & g.mx, T.y0, -1, T.t0, -1);
    stage_plane_async(B + kRH * kRW, kRH, kRW, kRW, ub, g, (T.x0 + 1) & g.mx, T.y0, 0, T.t0, 0);
    for (int f = 0; f < 5; ++f) stage_interior_async(I + f * kTY * kTT, ifields[f], g, T.x0, T.y0, T.t0);
    cp_async_commit();
    for (int s = 0; s < kPipeXB; ++s) {
      const int x = T.x0 + s;
      // prefetch planes x + 2 and the interiors of x + 1
      if (s + 1 < kPipeXB) {
        stage_plane_async(U + ((s + 2) % 3) * kUH * kUW, kUH, kUW, kUW, unew, g, (x + 2) & g.mx, T.y0, -1, T.t0, -1);
        stage_plane_async(B + ((s + 2) % 3) * kRH * kRW, kRH, kRW, kRW, ub, g, (x + 2) & g.mx, T.y0, 0, T.t0, 0);
        for (int f = 0; f < 5; ++f)
          stage_interior_async(I + (((s + 1) & 1) * 5 + f) * kTY * kTT, ifields[f], g, x + 1, T.y0, T.t0);
      }
      cp_async_commit();
      cp_async_wait_all_but_one();
      __syncthreads();
      const float* Ux = U + (s % 3) * kUH * kUW;
      const float* Un = U + ((s + 1) % 3) * kUH * kUW;
      const float* Bx = B + (s % 3) * kRH * kRW;
      const float* Bn = B + ((s + 1) % 3) * kRH * kRW;
      const float* Ix = I + (s & 1) * 5 * kTY * kTT;
      for (int i = threadIdx.x; i < kRH * kRW; i += blockDim.x) {
        const int yy = i / kRW, tt = i - yy * kRW;
        const float c = Ux[yy * kUW + tt];
        const float3 n = normal_of(
            make_float3(Un[yy * kUW + tt] - c, Ux[(yy + 1) * kUW + tt] - c, Ux[yy * kUW + tt + 1] - c), eps2);
        N[i] = n.x;
        N[kRH * kRW + i] = n.y;
        N[2 * kRH * kRW + i] = n.z;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = lane + 32 * j;
        const int r = (iy + 1) * kRW + it + 1;
        const int u = (iy + 1) * kUW + it + 1;
        const int bq = iy * kRW + it;
        const int ii = iy * kTT + it;
        const float kap = (N[r] - nx_prev[j]) + (N[kRH * kRW + r] - N[kRH * kRW + r - kRW]) +
                          (N[2 * kRH * kRW + r] - N[2 * kRH * kRW + r - 1]);
        nx_prev[j] = N[r];
        const float uc = Ux[u];
        const float3 gu = make_float3(Un[u] - uc, Ux[u + kUW] - uc, Ux[u + 1] - uc);
        const float l0 = Ix[ii], l1 = Ix[kTY * kTT + ii], l2 = Ix[2 * kTY * kTT + ii];
        const float bc = Bx[bq];
        const float3 av = make_float3(Bn[bq] - bc - l0 * inv_mu, Bx[bq + kRW] - bc - l1 * inv_mu,
                                      Bx[bq + 1] - bc - l2 * inv_mu);
        const float3 v = shrink3(av, Ix[3 * kTY * kTT + ii] * inv_mu);
        const float3 d = make_float3(v.x - gu.x, v.y - gu.y, v.z - gu.z);
        const size_t gi = g.idx(x, y, T.t0 + it);
        lam[gi] = l0 + mu * d.x;
        lam[V + gi] = l1 + mu * d.y;
        lam[2 * V + gi] = l2 + mu * d.z;
        const float pn = phi_of(kap, a, b, kind);
        ph[gi] = pn;
        ubn[gi] = uc + beta * (uc - Ix[4 * kTY * kTT + ii]);
        acc[0] += (double)pn * (double)sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z);
        acc[1] += (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z;
      }
      __syncthreads();
    }
    cp_async_wait_all();
  }
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
    partials[(size_t)blockIdx.x * kMaxTerms + 0] = s0;
    partials[(size_t)blockIdx.x * kMaxTerms + 1] = s1;
  }
}
constexpr size_t kPost1PipeSmem = sizeof(float) * (3 * kUH * kUW + kPost1BPlanes + 2 * 5 * kTY * kTT + 3 * kRH * kRW);

// Extra term of Algorithm 2's tau right-hand side: + mu3 (f + Lambda_3/mu3) with
// f = (lambda M tau0 + mu3 tau-bar - Lambda_3) / (lambda M + mu3).
struct FTerm {
  const float* tau0;
  const float* lam3;
  const int32_t* colpos;  // nullptr: every column sampled
  float lam_w, mu3;
};

// Pipelined k_pre1 (same arithmetic as k_pre1_tiled); with FTERM it also adds
// the f term of Algorithm 2's tau right-hand side (ub is then tau-bar).
template <bool FTERM>
__global__ void __launch_bounds__(kTileThreads, 3)
    k_pre1_pipe(const float* __restrict__ ub, const float* __restrict__ lam, const float* __restrict__ ph,
                float* __restrict__ reg, Vox g, int ntiles, float mu, size_t V, FTerm ft) {
  extern __shared__ float4 smem_f4[];
  float* U = reinterpret_cast<float*>(smem_f4);  // [3][kUH * kUW]     ubar planes
  float* L = U + 3 * kUH * kUW;                  // [2][4][kRH * kRW]  lam0..2, phi over the region
  float* Q = L + 2 * 4 * kRH * kRW;              // [3][kRH * kRW]     q over the region
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;
  const float* lfields[4] = {lam, lam + V, lam + 2 * V, ph};
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileIdx T = tile_of(tile, g);
    const int y = T.y0 + iy;
    float qx_prev[4];
    {
      const int xm = (T.x0 - 1) & g.mx;
      for (int j = 0; j < 4; ++j) {
        const int t = T.t0 + lane + 32 * j;
        qx_prev[j] = v_at(ub, lam, V, ph, g, xm, y, t, inv_mu).x + __ldg(lam + g.idx(xm, y, t)) * inv_mu;
      }
    }
    stage_plane_async(U, kUH, kUW, kUW, ub, g, T.x0, T.y0, -1, T.t0, -1);
    cp_async_commit();
    stage_plane_async(U + kUH * kUW, kUH, kUW, kUW, ub, g, (T.x0 + 1) & g.mx, T.y0, -1, T.t0, -1);
    for (int f = 0; f < 4; ++f) stage_plane_async(L + f * kRH * kRW, kRH, kRW, kRW, lfields[f], g, T.x0, T.y0, -1, T.t0, -1);
    cp_async_commit();
    for (int s = 0; s < kPipeXB; ++s) {
      const int x = T.x0 + s;
      if (s + 1 < kPipeXB) {
        stage_plane_async(U + ((s + 2) % 3) * kUH * kUW, kUH, kUW, kUW, ub, g, (x + 2) & g.mx, T.y0, -1, T.t0, -1);
        for (int f = 0; f < 4; ++f)
          stage_plane_async(L + (((s + 1) & 1) * 4 + f) * kRH * kRW, kRH, kRW, kRW, lfields[f], g, x + 1, T.y0, -1,
                            T.t0, -1);
      }
      cp_async_commit();
      cp_async_wait_all_but_one();
      __syncthreads();
      const float* Ux = U + (s % 3) * kUH * kUW;
      const float* Un = U + ((s + 1) % 3) * kUH * kUW;
      const float* Lx = L + (s & 1) * 4 * kRH * kRW;
      for (int i = threadIdx.x; i < kRH * kRW; i += blockDim.x) {
        const int yy = i / kRW, tt = i - yy * kRW;
        const float c = Ux[yy * kUW + tt];
        const float l0 = Lx[i], l1 = Lx[kRH * kRW + i], l2 = Lx[2 * kRH * kRW + i];
        const float3 av = make_float3(Un[yy * kUW + tt] - c - l0 * inv_mu, Ux[(yy + 1) * kUW + tt] - c - l1 * inv_mu,
                                      Ux[yy * kUW + tt + 1] - c - l2 * inv_mu);
        const float3 v = shrink3(av, Lx[3 * kRH * kRW + i] * inv_mu);
        Q[i] = v.x + l0 * inv_mu;
        Q[kRH * kRW + i] = v.y + l1 * inv_mu;
        Q[2 * kRH * kRW + i] = v.z + l2 * inv_mu;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = lane + 32 * j;
        const int r = (iy + 1) * kRW + it + 1;
        const float qx = Q[r];
        const float div =
            (qx - qx_prev[j]) + (Q[kRH * kRW + r] - Q[kRH * kRW + r - kRW]) + (Q[2 * kRH * kRW + r] - Q[2 * kRH * kRW + r - 1]);
        const size_t gi = g.idx(x, y, T.t0 + it);
        float out = -mu * div;
        if (FTERM) {
          const float m = ft.colpos ? (__ldg(ft.colpos + x * g.ny + y) >= 0 ? 1.0f : 0.0f) : 1.0f;
          const float l3 = __ldg(ft.lam3 + gi);
          const float tb = Ux[(iy + 1) * kUW + it + 1];
          const float f = (ft.lam_w * m * __ldg(ft.tau0 + gi) + ft.mu3 * tb - l3) / (ft.lam_w * m + ft.mu3);
          out += ft.mu3 * (f + l3 / ft.mu3);
        }
        reg[gi] = out;
        qx_prev[j] = qx;
      }
      __syncthreads();
    }
    cp_async_wait_all();
  }
}
constexpr size_t kPre1PipeSmem = sizeof(float) * (3 * kUH * kUW + 2 * 4 * kRH * kRW + 3 * kRH * kRW);

}  // namespace nlos
