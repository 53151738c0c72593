// Shared-memory halo-tiled stencils of Algorithm 1 (Eq. 7, Eq. 12, the
// right-hand side of the PDE above Eq. 11, kappa and phi of Sec. 3), also run
// twice per iteration by Algorithm 2 (u and tau).
//
// A block owns a TY x TT tile of the (y, t) plane (TT = 128 time bins along
// the contiguous axis, TY = 8 rows) and marches through consecutive x planes.
// The (tile, x plane) steps, x fastest, are split into one contiguous run per
// block of a persistent grid, so a block pays the pipeline's prologue (the
// first two planes in flight, the x - 1 values from global memory) only where
// its run starts or enters the next tile, not every few planes.  Per x plane it
// stages the fields that are read at neighbours (with their +-1 halos,
// periodic wrap) in shared memory, evaluates the per-point quantity whose
// backward differences are needed (the normal field n, or q = v + Lambda/mu)
// over the tile plus its -1 halo, and finishes the interior.  The
// x-direction backward difference uses the value the same thread computed on
// the previous plane, kept in registers.  Each thread owns 4 interior voxels
// t = t0 + lane + 32 j, so shared-memory reads of a warp are unit-stride.
//
// Software pipeline: the planes of step s + 1 are copied with cp.async while
// step s computes (a ring of three halo planes: x, x + 1 in use, x + 2 in
// flight).  Staged rows have pitch kP with t0 at column kC (16-byte aligned),
// so the 128-bin interior of a row moves as 32 16-byte copies and only the
// t0 - 1 / t0 + TT halo columns as single floats.
#pragma once

#include "fft.cuh"
#include "iter_end.cuh"
#include "stencil.cuh"

namespace nlos {

constexpr int kTT = 128;                     // tile extent along t
constexpr int kTY = 8;                       // tile extent along y
constexpr int kTileThreads = 256;            // 8 warps: warp = row iy, lane = t offset
constexpr int kUH = kTY + 2;                 // rows of a field staged with -1/+1 y halos
constexpr int kRW = kTT + 1, kRH = kTY + 1;  // region of per-point quantities: (TY+1) x (TT+1)
constexpr int kP = kTT + 8;                  // staged row pitch (floats)
constexpr int kC = 4;                        // column of t0 in a staged row (t0 - 1 at kC - 1)
static_assert(kP % 4 == 0 && kC % 4 == 0, "staged rows must keep the interior 16-byte aligned");

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Stage plane x of f: rows y = y0 + ylo + r (periodic), r < H, into
// tile[r][kP]; columns t0 .. t0 + TT - 1 at kC .. kC + TT - 1, plus t0 - 1 at
// kC - 1 (LO) and t0 + TT at kC + TT (HI), wrapped in t.
template <bool LO, bool HI>
__device__ __forceinline__ void stage_rows_async(float* __restrict__ tile, int H, const float* __restrict__ f,
                                                 const Vox& g, int x, int y0, int ylo, int t0) {
  constexpr int Q = kTT / 4;
  for (int i = threadIdx.x; i < H * Q; i += kTileThreads) {
    const int r = i / Q, q = i - r * Q;
    const int y = (y0 + ylo + r) & g.my;
    cp_async16(tile + r * kP + kC + 4 * q, f + g.idx(x, y, t0 + 4 * q));
  }
  if (LO || HI) {
    constexpr int E = (LO ? 1 : 0) + (HI ? 1 : 0);
    for (int i = threadIdx.x; i < H * E; i += kTileThreads) {
      const int r = i / E;
      const int side = (LO && HI) ? i - r * E : (HI ? 1 : 0);
      const int y = (y0 + ylo + r) & g.my;
      const int t = side ? (t0 + kTT) & g.mt : (t0 - 1) & g.mt;
      cp_async4(tile + r * kP + (side ? kC + kTT : kC - 1), f + g.idx(x, y, t));
    }
  }
}
// Stage the TY x TT interior of plane x (rows contiguous, 16-byte aligned)
// into tile[TY][TT].
__device__ __forceinline__ void stage_interior_async(float* __restrict__ tile, const float* __restrict__ f,
                                                     const Vox& g, int x, int y0, int t0) {
  for (int i = threadIdx.x; i < kTY * kTT / 4; i += kTileThreads) {
    const int yy = i / (kTT / 4), q = i - yy * (kTT / 4);
    cp_async16(tile + yy * kTT + 4 * q, f + g.idx(x, y0 + yy, t0 + 4 * q));
  }
}

// Number of (tile, x plane) steps of a grid.
inline int stencil_steps(const Vox& g) { return (g.nt / kTT) * (g.ny / kTY) * g.nx; }

// The next run of this block's share [cur, end) of the steps: tile (t0, y0),
// first plane x0, cnt planes (within one tile).
struct TileRun {
  int t0, y0, x0, cnt;
};
__device__ __forceinline__ TileRun run_at(int cur, int end, const Vox& g) {
  const int ntt = g.nt / kTT;
  const int tile = cur / g.nx, x0 = cur - tile * g.nx;
  TileRun r;
  r.t0 = (tile % ntt) * kTT;
  r.y0 = (tile / ntt) * kTY;
  r.x0 = x0;
  r.cnt = min(end - cur, g.nx - x0);
  return r;
}
__device__ __forceinline__ void block_share(int nsteps, int& cur, int& end) {
  cur = (int)((long long)nsteps * blockIdx.x / gridDim.x);
  end = (int)((long long)nsteps * (blockIdx.x + 1) / gridDim.x);
}

// Shared layout of k_post1_pipe (floats; every region a multiple of 4):
//   U [3][kUH][kP]     u+ planes, rows y0 - 1 .. y0 + TY, t0 - 1 .. t0 + TT
//   B [3][kRH][kP]     ubar planes, rows y0 .. y0 + TY, t0 .. t0 + TT
//   I [2][5][TY][TT]   lam0..2, phi, u^k interiors of planes x and x + 1
//   N [3][kRH][kRW]    normal field over the region (y0 - 1.., t0 - 1..)
constexpr int kPostU = 3 * kUH * kP, kPostB = 3 * kRH * kP, kPostI = 2 * 5 * kTY * kTT;
static_assert(kPostU % 4 == 0 && kPostB % 4 == 0, "staging regions must keep 16-byte alignment");
constexpr size_t kPost1PipeSmem = sizeof(float) * (kPostU + kPostB + kPostI + 3 * kRH * kRW);

// The elementwise Lambda_3 part of Algorithm 2's multiplier update, done by
// the tau half of the post step (u+ there is tau+, ubar is tau-bar):
// f = (lambda M tau0 + mu3 tau-bar - Lambda_3) / (lambda M + mu3),
// Lambda_3 += mu3 (f - tau+).
struct L3Term {
  const float* tau0;
  const float* au;  // A u+
  float* lam3;
  const int32_t* colpos;  // nullptr: every column sampled
  float lam_w, mu3;
};

// lam += mu (v - grad u+), phi = phi(kappa(u+)), ubar_next = u+ + beta (u+ - u^k)
// (Algorithm 1); partials 0 = sum phi |grad u+|, 1 = sum |v - grad u+|^2,
// v = shrink(grad ubar - lam/mu, phi/mu).  With L3 also the Lambda_3 update
// above and partials 2 = sum (A u+ - tau+)^2, 3 = sum M (tau+ - tau0)^2,
// 4 = sum (f - tau+)^2.  KIND: the phi of the curvature (NLOS_PHI_*).
template <bool L3, int KIND>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_post1_pipe(const float* __restrict__ unew, const float* __restrict__ uk, const float* __restrict__ ub,
                 float* __restrict__ lam, float* __restrict__ ph, float* __restrict__ ubn,
                 const DevScalars* __restrict__ sc, Vox g, int nsteps, float mu, float a, float b, float eps2,
                 size_t V, double* __restrict__ partials, L3Term l3) {
  extern __shared__ float4 smem_f4[];
  float* U = reinterpret_cast<float*>(smem_f4);
  float* B = U + kPostU;
  float* I = B + kPostB;
  float* N = I + kPostI;
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;
  const float beta = (float)sc->beta_next;
  const float* ifields[5] = {lam, lam + V, lam + 2 * V, ph, uk};
  // 1 / (lambda M + mu3) for M = 1 and M = 0
  const float l3_d1 = L3 ? 1.0f / (l3.lam_w + l3.mu3) : 0.0f, l3_d0 = L3 ? 1.0f / l3.mu3 : 0.0f;
  SumAcc<L3 ? 5 : 2> ca;
  int cur, end;
  block_share(nsteps, cur, end);
  while (cur < end) {
    const TileRun T = run_at(cur, end, g);
    cur += T.cnt;
    const int y = T.y0 + iy;
    float nx_prev[4];
    for (int j = 0; j < 4; ++j) {
      const int xm = (T.x0 - 1) & g.mx;
      nx_prev[j] = normal_of(grad_at(unew, g, xm, y, T.t0 + lane + 32 * j), eps2).x;
    }
    // prologue: planes x0 (group 0) and x0 + 1 plus the interiors of x0 (group 1)
    stage_rows_async<true, true>(U, kUH, unew, g, T.x0, T.y0, -1, T.t0);
    stage_rows_async<false, true>(B, kRH, ub, g, T.x0, T.y0, 0, T.t0);
    cp_async_commit();
    stage_rows_async<true, true>(U + kUH * kP, kUH, unew, g, (T.x0 + 1) & g.mx, T.y0, -1, T.t0);
    stage_rows_async<false, true>(B + kRH * kP, kRH, ub, g, (T.x0 + 1) & g.mx, T.y0, 0, T.t0);
    for (int f = 0; f < 5; ++f) stage_interior_async(I + f * kTY * kTT, ifields[f], g, T.x0, T.y0, T.t0);
    cp_async_commit();
    for (int s = 0; s < T.cnt; ++s) {
      const int x = T.x0 + s;
      // prefetch planes x + 2 and the interiors of x + 1
      if (s + 1 < T.cnt) {
        stage_rows_async<true, true>(U + ((s + 2) % 3) * kUH * kP, kUH, unew, g, (x + 2) & g.mx, T.y0, -1, T.t0);
        stage_rows_async<false, true>(B + ((s + 2) % 3) * kRH * kP, kRH, ub, g, (x + 2) & g.mx, T.y0, 0, T.t0);
        for (int f = 0; f < 5; ++f)
          stage_interior_async(I + (((s + 1) & 1) * 5 + f) * kTY * kTT, ifields[f], g, (x + 1) & g.mx, T.y0,
                               T.t0);
      }
      cp_async_commit();
      cp_async_wait_all_but_one();
      __syncthreads();
      const float* Ux = U + (s % 3) * kUH * kP;
      const float* Un = U + ((s + 1) % 3) * kUH * kP;
      const float* Bx = B + (s % 3) * kRH * kP;
      const float* Bn = B + ((s + 1) % 3) * kRH * kP;
      const float* Ix = I + (s & 1) * 5 * kTY * kTT;
      // the Lambda_3 inputs of this row, loaded now so their latency overlaps
      // the region pass below
      float l3_t0[4], l3_au[4], l3_l[4];
      bool l3_sampled = true;
      if (L3) {
        l3_sampled = l3.colpos ? __ldg(l3.colpos + x * g.ny + y) >= 0 : true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const size_t gi = g.idx(x, y, T.t0 + lane + 32 * j);
          l3_t0[j] = __ldg(l3.tau0 + gi);
          l3_au[j] = __ldg(l3.au + gi);
          l3_l[j] = l3.lam3[gi];
        }
      }
      // normals over the region: point (yy, tt) is voxel (y0 - 1 + yy, t0 - 1 +
      // tt); columns 0 .. TT - 1 two rows per pass, then the last column
      auto normal_at = [&](int yy, int tt) {
        const int o = yy * kP + tt + kC - 1, i = yy * kRW + tt;
        const float c = Ux[o];
        const float3 n = normal_of(make_float3(Un[o] - c, Ux[o + kP] - c, Ux[o + 1] - c), eps2);
        N[i] = n.x;
        N[kRH * kRW + i] = n.y;
        N[2 * kRH * kRW + i] = n.z;
      };
      static_assert(kTileThreads == 2 * kTT, "two region rows per pass");
#pragma unroll
      for (int yy = threadIdx.x / kTT; yy < kRH; yy += 2) normal_at(yy, threadIdx.x % kTT);
      if (threadIdx.x < kRH) normal_at(threadIdx.x, kTT);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = lane + 32 * j;
        const int r = (iy + 1) * kRW + it + 1;  // region index of the voxel
        const int u = (iy + 1) * kP + it + kC;  // staged u+ index of the voxel
        const int bq = iy * kP + it + kC;       // staged ubar index of the voxel
        const int ii = iy * kTT + it;           // interior index of the voxel
        const float kap = (N[r] - nx_prev[j]) + (N[kRH * kRW + r] - N[kRH * kRW + r - kRW]) +
                          (N[2 * kRH * kRW + r] - N[2 * kRH * kRW + r - 1]);
        nx_prev[j] = N[r];
        const float uc = Ux[u];
        const float3 gu = make_float3(Un[u] - uc, Ux[u + kP] - uc, Ux[u + 1] - uc);
        const float l0 = Ix[ii], l1 = Ix[kTY * kTT + ii], l2 = Ix[2 * kTY * kTT + ii];
        const float bc = Bx[bq];
        const float3 av = make_float3(Bn[bq] - bc - l0 * inv_mu, Bx[bq + kP] - bc - l1 * inv_mu,
                                      Bx[bq + 1] - bc - l2 * inv_mu);
        const float3 v = shrink3(av, Ix[3 * kTY * kTT + ii] * inv_mu);
        const float3 d = make_float3(v.x - gu.x, v.y - gu.y, v.z - gu.z);
        const size_t gi = g.idx(x, y, T.t0 + it);
        lam[gi] = l0 + mu * d.x;
        lam[V + gi] = l1 + mu * d.y;
        lam[2 * V + gi] = l2 + mu * d.z;
        const float pn = phi_of(kap, a, b, KIND);
        ph[gi] = pn;
        ubn[gi] = uc + beta * (uc - Ix[4 * kTY * kTT + ii]);
        ca.add(0, pn * sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z));
        ca.add(1, d.x * d.x + d.y * d.y + d.z * d.z);
        if (L3) {
          const float m = l3_sampled ? 1.0f : 0.0f;
          const float f = (l3.lam_w * m * l3_t0[j] + l3.mu3 * bc - l3_l[j]) * (l3_sampled ? l3_d1 : l3_d0);
          l3.lam3[gi] = l3_l[j] + l3.mu3 * (f - uc);
          const float r = l3_au[j] - uc, sres = m * (uc - l3_t0[j]), fr = f - uc;
          ca.add(2, r * r);
          ca.add(3, sres * sres);
          ca.add(4, fr * fr);
        }
      }
      __syncthreads();
    }
    cp_async_wait_all();
  }
  block_reduce_acc(ca, partials);
}

// Extra term of Algorithm 2's tau right-hand side: + mu3 (f + Lambda_3/mu3) with
// f = (lambda M tau0 + mu3 tau-bar - Lambda_3) / (lambda M + mu3).
struct FTerm {
  const float* tau0;
  const float* lam3;
  const int32_t* colpos;  // nullptr: every column sampled
  float lam_w, mu3;
};

// Shared layout of k_pre1_pipe (floats):
//   U [3][kUH][kP]       ubar planes, rows y0 - 1 .. y0 + TY, t0 - 1 .. t0 + TT
//   L [2][4][kRH][kP]    lam0..2, phi over the region rows y0 - 1 .., t0 - 1 ..
//   Q [3][kRH][kRW]      q over the region
constexpr int kPreU = 3 * kUH * kP, kPreL = 2 * 4 * kRH * kP;
static_assert(kPreU % 4 == 0 && kPreL % 4 == 0, "staging regions must keep 16-byte alignment");
constexpr size_t kPre1PipeSmem = sizeof(float) * (kPreU + kPreL + 3 * kRH * kRW);

// reg = -mu sum_d (q_d(c) - q_d(c - e_d)), q = v + Lam/mu,
// v = shrink(grad ubar - Lam/mu, phi/mu); with FTERM it also adds the f term
// of Algorithm 2's tau right-hand side (ub is then tau-bar).
template <bool FTERM>
__global__ void __launch_bounds__(kTileThreads, 3)
    k_pre1_pipe(const float* __restrict__ ub, const float* __restrict__ lam, const float* __restrict__ ph,
                float* __restrict__ reg, Vox g, int nsteps, float mu, size_t V, FTerm ft) {
  extern __shared__ float4 smem_f4[];
  float* U = reinterpret_cast<float*>(smem_f4);
  float* L = U + kPreU;
  float* Q = L + kPreL;
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;
  const float* lfields[4] = {lam, lam + V, lam + 2 * V, ph};
  const float inv_d1 = 1.0f / (ft.lam_w + ft.mu3), inv_d0 = 1.0f / ft.mu3;
  int cur, end;
  block_share(nsteps, cur, end);
  while (cur < end) {
    const TileRun T = run_at(cur, end, g);
    cur += T.cnt;
    const int y = T.y0 + iy;
    float qx_prev[4];
    {
      const int xm = (T.x0 - 1) & g.mx;
      for (int j = 0; j < 4; ++j) {
        const int t = T.t0 + lane + 32 * j;
        qx_prev[j] = v_at(ub, lam, V, ph, g, xm, y, t, inv_mu).x + __ldg(lam + g.idx(xm, y, t)) * inv_mu;
      }
    }
    stage_rows_async<true, true>(U, kUH, ub, g, T.x0, T.y0, -1, T.t0);
    cp_async_commit();
    stage_rows_async<true, true>(U + kUH * kP, kUH, ub, g, (T.x0 + 1) & g.mx, T.y0, -1, T.t0);
    for (int f = 0; f < 4; ++f)
      stage_rows_async<true, false>(L + f * kRH * kP, kRH, lfields[f], g, T.x0, T.y0, -1, T.t0);
    cp_async_commit();
    for (int s = 0; s < T.cnt; ++s) {
      const int x = T.x0 + s;
      if (s + 1 < T.cnt) {
        stage_rows_async<true, true>(U + ((s + 2) % 3) * kUH * kP, kUH, ub, g, (x + 2) & g.mx, T.y0, -1, T.t0);
        for (int f = 0; f < 4; ++f)
          stage_rows_async<true, false>(L + (((s + 1) & 1) * 4 + f) * kRH * kP, kRH, lfields[f], g,
                                        (x + 1) & g.mx, T.y0, -1, T.t0);
      }
      cp_async_commit();
      cp_async_wait_all_but_one();
      __syncthreads();
      const float* Ux = U + (s % 3) * kUH * kP;
      const float* Un = U + ((s + 1) % 3) * kUH * kP;
      const float* Lx = L + (s & 1) * 4 * kRH * kP;
      // the f term's point inputs, loaded now so their latency overlaps the
      // region pass below
      float ft_t0[4], ft_l3[4];
      bool ft_sampled = true;
      if (FTERM) {
        ft_sampled = ft.colpos ? __ldg(ft.colpos + x * g.ny + y) >= 0 : true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const size_t gi = g.idx(x, y, T.t0 + lane + 32 * j);
          ft_t0[j] = __ldg(ft.tau0 + gi);
          ft_l3[j] = __ldg(ft.lam3 + gi);
        }
      }
      // q over the region: point (yy, tt) is voxel (y0 - 1 + yy, t0 - 1 + tt);
      // columns 0 .. TT - 1 two rows per pass, then the last column
      auto q_at = [&](int yy, int tt) {
        const int o = yy * kP + tt + kC - 1, i = yy * kRW + tt;
        const float c = Ux[o];
        const float l0 = Lx[o], l1 = Lx[kRH * kP + o], l2 = Lx[2 * kRH * kP + o];
        const float3 av = make_float3(Un[o] - c - l0 * inv_mu, Ux[o + kP] - c - l1 * inv_mu,
                                      Ux[o + 1] - c - l2 * inv_mu);
        const float3 v = shrink3(av, Lx[3 * kRH * kP + o] * inv_mu);
        Q[i] = v.x + l0 * inv_mu;
        Q[kRH * kRW + i] = v.y + l1 * inv_mu;
        Q[2 * kRH * kRW + i] = v.z + l2 * inv_mu;
      };
#pragma unroll
      for (int yy = threadIdx.x / kTT; yy < kRH; yy += 2) q_at(yy, threadIdx.x % kTT);
      if (threadIdx.x < kRH) q_at(threadIdx.x, kTT);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = lane + 32 * j;
        const int r = (iy + 1) * kRW + it + 1;
        const float qx = Q[r];
        const float div = (qx - qx_prev[j]) + (Q[kRH * kRW + r] - Q[kRH * kRW + r - kRW]) +
                          (Q[2 * kRH * kRW + r] - Q[2 * kRH * kRW + r - 1]);
        const size_t gi = g.idx(x, y, T.t0 + it);
        float out = -mu * div;
        if (FTERM) {
          // the denominator lambda M + mu3 takes two values: sampled or not
          const float m = ft_sampled ? 1.0f : 0.0f;
          const float l3 = ft_l3[j];
          const float tb = Ux[(iy + 1) * kP + it + kC];
          const float f = (ft.lam_w * m * ft_t0[j] + ft.mu3 * tb - l3) * (ft_sampled ? inv_d1 : inv_d0);
          out += ft.mu3 * f + l3;
        }
        reg[gi] = out;
        qx_prev[j] = qx;
      }
      __syncthreads();
    }
    cp_async_wait_all();
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1's post step fused with the next iteration's pre step.
//
// The post step of iteration k (Lambda, phi and u-bar of iteration k + 1,
// Eq. 12 and the extrapolation) and the pre step of iteration k + 1 (the
// right-hand side reg = -mu div q, q = v' + Lambda_{k+1}/mu with v' =
// shrink(grad u-bar_{k+1} - Lambda_{k+1}/mu, phi_{k+1}/mu), Eq. 7 and the
// PDE above Eq. 11) read the same neighbourhoods, so one pass forms q from
// the values it has just computed instead of storing them and reading them
// back in a second launch.  The backward divergence needs q at the tile's
// voxels and at its -1 halo: the row above the tile and the column before it
// (the plane before is the previous step of the march).  A halo voxel's q
// needs Lambda and phi there in their state before this step, while the
// block that owns the voxel writes the new values: Lambda and phi are
// therefore read from one pair of buffers and written to another (the caller
// swaps them after every iteration).
//
// Shared layout (floats):
//   U [3][TY+3][kP]     u+ planes, rows y0 - 2 .. y0 + TY, t0 - 2 .. t0 + TT
//   B [3][TY+2][kP]     u-bar planes, rows y0 - 1 .. y0 + TY, t0 - 1 .. t0 + TT
//   K [3][TY+2][kP]     u^k planes, same extent as B
//   N [3][TY+2][TT+2]   normal field of u+, rows y0 - 2 .., t0 - 2 ..
//   Q [3][TY+1][TT+1]   q, rows y0 - 1 .., t0 - 1 ..
//   H [kFusHalo]        n_x of u+ on the plane before, at the halo voxels of Q
constexpr int kFusUH = kTY + 3, kFusNH = kTY + 2, kFusNW = kTT + 2;
constexpr int kFusHalo = kRW + kTY;  // halo voxels of Q: its first row, then its first column below it
static_assert(kFusHalo <= kTileThreads, "one halo voxel per thread");
constexpr int kFusU = 3 * kFusUH * kP, kFusB = 3 * kUH * kP, kFusN = 3 * kFusNH * kFusNW, kFusQ = 3 * kRH * kRW;
static_assert(kFusU % 4 == 0 && kFusB % 4 == 0, "staging regions must keep 16-byte alignment");
constexpr size_t kPostPreSmem = sizeof(float) * (kFusU + 2 * kFusB + kFusN + kFusQ + ((kFusHalo + 3) & ~3));

// Stage rows y0 - 2 + r (r < H, periodic) of plane x: columns t0 .. t0 + TT -
// 1 at kC .., t0 - 2 and t0 - 1 at kC - 2 (one 8-byte copy: t0 - 2 is even,
// so the pair is aligned and never straddles the wrap), t0 + TT at kC + TT.
__device__ __forceinline__ void stage_rows_lo2_async(float* __restrict__ tile, int H, const float* __restrict__ f,
                                                     const Vox& g, int x, int y0, int t0) {
  constexpr int Q = kTT / 4;
  for (int i = threadIdx.x; i < H * Q; i += kTileThreads) {
    const int r = i / Q, q = i - r * Q;
    const int y = (y0 - 2 + r) & g.my;
    cp_async16(tile + r * kP + kC + 4 * q, f + g.idx(x, y, t0 + 4 * q));
  }
  for (int i = threadIdx.x; i < 2 * H; i += kTileThreads) {
    const int r = i >> 1;
    const int y = (y0 - 2 + r) & g.my;
    if (i & 1)
      cp_async4(tile + r * kP + kC + kTT, f + g.idx(x, y, (t0 + kTT) & g.mt));
    else
      cp_async8(tile + r * kP + kC - 2, f + g.idx(x, y, (t0 - 2) & g.mt));
  }
}

// One voxel c of the fused step.  u, b, k: u+, u-bar and u^k at c, c + e_x,
// c + e_y, c + e_t; l, ph: Lambda and phi at c before the step; kap:
// kappa(u+) at c.
// shrink3 with a select in place of its early return (same value for every
// input).
__device__ __forceinline__ float3 shrink3_nb(float3 a, float th) {
  const float n2 = a.x * a.x + a.y * a.y + a.z * a.z;
  const float s = n2 > 0.0f ? fmaxf(1.0f - th * rsqrtf(n2), 0.0f) : 0.0f;
  return make_float3(a.x * s, a.y * s, a.z * s);
}

struct FusedPoint {
  float3 lam;  // Lambda_{k+1} = Lambda + mu (v - grad u+)
  float phi;   // phi(kappa(u+))
  float ubn;   // u-bar_{k+1} = u+ + beta (u+ - u^k)
  float3 q;    // v' + Lambda_{k+1} / mu
  float gn;    // |grad u+|
  float d2;    // |v - grad u+|^2
};
template <int KIND>
__device__ __forceinline__ FusedPoint fused_point(float4 u, float4 b, float4 k, float3 l, float ph, float kap,
                                                  float mu, float inv_mu, float beta, float pa, float pb) {
  FusedPoint o;
  const float3 gu = make_float3(u.y - u.x, u.z - u.x, u.w - u.x);
  const float3 av = make_float3(b.y - b.x - l.x * inv_mu, b.z - b.x - l.y * inv_mu, b.w - b.x - l.z * inv_mu);
  const float3 v = shrink3_nb(av, ph * inv_mu);
  const float3 d = make_float3(v.x - gu.x, v.y - gu.y, v.z - gu.z);
  o.lam = make_float3(l.x + mu * d.x, l.y + mu * d.y, l.z + mu * d.z);
  o.phi = phi_of(kap, pa, pb, KIND);
  const float n0 = u.x + beta * (u.x - k.x), n1 = u.y + beta * (u.y - k.y), n2 = u.z + beta * (u.z - k.z),
              n3 = u.w + beta * (u.w - k.w);
  o.ubn = n0;
  const float3 an = make_float3(n1 - n0 - o.lam.x * inv_mu, n2 - n0 - o.lam.y * inv_mu, n3 - n0 - o.lam.z * inv_mu);
  const float3 vn = shrink3_nb(an, o.phi * inv_mu);
  o.q = make_float3(vn.x + o.lam.x * inv_mu, vn.y + o.lam.y * inv_mu, vn.z + o.lam.z * inv_mu);
  o.gn = sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z);
  o.d2 = d.x * d.x + d.y * d.y + d.z * d.z;
  return o;
}

// f at c, c + e_x, c + e_y, c + e_t from global memory (periodic).
__device__ __forceinline__ float4 fwd4(const float* __restrict__ f, const Vox& g, int x, int y, int t) {
  return make_float4(__ldg(f + g.idx(x, y, t)), __ldg(f + g.idx((x + 1) & g.mx, y, t)),
                     __ldg(f + g.idx(x, (y + 1) & g.my, t)), __ldg(f + g.idx(x, y, (t + 1) & g.mt)));
}

// q_x of the fused step at one voxel, every input from global memory (the
// plane before a run's first plane).
template <int KIND>
__device__ __forceinline__ float fused_qx_at(const float* __restrict__ unew, const float* __restrict__ uk,
                                             const float* __restrict__ ub, const float* __restrict__ lam,
                                             const float* __restrict__ ph, const Vox& g, size_t V, int x, int y,
                                             int t, float mu, float inv_mu, float beta, float pa, float pb,
                                             float eps2) {
  const int i = g.idx(x, y, t);
  const float3 l = make_float3(__ldg(lam + i), __ldg(lam + V + i), __ldg(lam + 2 * V + i));
  const float kap = curvature_at(unew, g, x, y, t, eps2, nullptr);
  return fused_point<KIND>(fwd4(unew, g, x, y, t), fwd4(ub, g, x, y, t), fwd4(uk, g, x, y, t), l, __ldg(ph + i),
                           kap, mu, inv_mu, beta, pa, pb)
      .q.x;
}

// lamo = Lambda_{k+1}, pho = phi(kappa(u+)), ubn = u-bar_{k+1} (as k_post1_pipe)
// and reg = -mu div q for the next iteration (as k_pre1_pipe on those
// outputs); lam, ph: Lambda and phi before the step (not written).
// Partials 0 = sum phi |grad u+|, 1 = sum |v - grad u+|^2; with
// ie.end_here the last block to finish sums every block's partials and ends
// the iteration on ie.sc (the work of k_finalize).  Also Algorithm 2's u
// half (Lambda_1, phi_u, u-bar, and reg of the next u-step).  KIND: the phi
// of the curvature (NLOS_PHI_*).
template <int KIND>
__global__ void __launch_bounds__(kTileThreads, 2)
    k_post1_pre(const float* __restrict__ unew, const float* __restrict__ uk, const float* __restrict__ ub,
                const float* __restrict__ lam, const float* __restrict__ ph, float* __restrict__ lamo,
                float* __restrict__ pho, float* __restrict__ ubn, float* __restrict__ reg, IterEnd ie, Vox g,
                int nsteps, float mu, float pa, float pb, float eps2, size_t V, double* __restrict__ partials) {
  extern __shared__ float4 smem_f4[];
  float* U = reinterpret_cast<float*>(smem_f4);
  float* B = U + kFusU;
  float* K = B + kFusB;
  float* N = K + kFusB;
  float* Q = N + kFusN;
  float* H = Q + kFusQ;
  constexpr int SN = kFusNH * kFusNW, SQ = kRH * kRW;
  constexpr int SU = kFusUH * kP, SB = kUH * kP;
  const int iy = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_mu = 1.0f / mu;
  const float beta = (float)ie.sc->beta_next;
  // this thread's halo voxel of Q (threads < kFusHalo): Q row hy, column ht
  const int h = threadIdx.x;
  const bool has_halo = h < kFusHalo;
  const int hy = h < kRW ? 0 : h - kRW + 1, ht = h < kRW ? h : 0;
  SumAcc<2> ca;
  int cur, end;
  block_share(nsteps, cur, end);
  while (cur < end) {
    const TileRun T = run_at(cur, end, g);
    cur += T.cnt;
    const int y = T.y0 + iy;
    const int hyv = (T.y0 - 1 + hy) & g.my, htv = (T.t0 - 1 + ht) & g.mt;
    // prologue: planes x0 (group 0) and x0 + 1 (group 1)
    stage_rows_lo2_async(U, kFusUH, unew, g, T.x0, T.y0, T.t0);
    stage_rows_async<true, true>(B, kUH, ub, g, T.x0, T.y0, -1, T.t0);
    stage_rows_async<true, true>(K, kUH, uk, g, T.x0, T.y0, -1, T.t0);
    cp_async_commit();
    stage_rows_lo2_async(U + SU, kFusUH, unew, g, (T.x0 + 1) & g.mx, T.y0, T.t0);
    stage_rows_async<true, true>(B + SB, kUH, ub, g, (T.x0 + 1) & g.mx, T.y0, -1, T.t0);
    stage_rows_async<true, true>(K + SB, kUH, uk, g, (T.x0 + 1) & g.mx, T.y0, -1, T.t0);
    cp_async_commit();
    // (while those copies are in flight) the plane before the run: n_x of u+ at the own and halo voxels, q_x at
    // the own voxels
    const int xm = (T.x0 - 1) & g.mx;
    float nx_prev[4], qx_prev[4];
    for (int j = 0; j < 4; ++j) {
      const int t = T.t0 + lane + 32 * j;
      nx_prev[j] = normal_of(grad_at(unew, g, xm, y, t), eps2).x;
      qx_prev[j] = fused_qx_at<KIND>(unew, uk, ub, lam, ph, g, V, xm, y, t, mu, inv_mu, beta, pa, pb, eps2);
    }
    if (has_halo) H[h] = normal_of(grad_at(unew, g, xm, hyv, htv), eps2).x;
    for (int s = 0; s < T.cnt; ++s) {
      const int x = T.x0 + s;
      if (s + 1 < T.cnt) {
        const int xn = (x + 2) & g.mx, sl = (s + 2) % 3;
        stage_rows_lo2_async(U + sl * SU, kFusUH, unew, g, xn, T.y0, T.t0);
        stage_rows_async<true, true>(B + sl * SB, kUH, ub, g, xn, T.y0, -1, T.t0);
        stage_rows_async<true, true>(K + sl * SB, kUH, uk, g, xn, T.y0, -1, T.t0);
      }
      cp_async_commit();
      // Lambda and phi before the step at the own and halo voxels, loaded
      // now so that their latency overlaps the normal pass
      float3 lj[4];
      float pj[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const size_t gi = g.idx(x, y, T.t0 + lane + 32 * j);
        lj[j] = make_float3(__ldg(lam + gi), __ldg(lam + V + gi), __ldg(lam + 2 * V + gi));
        pj[j] = __ldg(ph + gi);
      }
      float3 lh = make_float3(0.f, 0.f, 0.f);
      float phh = 0.f;
      if (has_halo) {
        const size_t hi = g.idx(x, hyv, htv);
        lh = make_float3(__ldg(lam + hi), __ldg(lam + V + hi), __ldg(lam + 2 * V + hi));
        phh = __ldg(ph + hi);
      }
      cp_async_wait_all_but_one();
      __syncthreads();
      const float* Ux = U + (s % 3) * SU;
      const float* Un = U + ((s + 1) % 3) * SU;
      const float* Bx = B + (s % 3) * SB;
      const float* Bn = B + ((s + 1) % 3) * SB;
      const float* Kx = K + (s % 3) * SB;
      const float* Kn = K + ((s + 1) % 3) * SB;
      // normals over rows y0 - 2 .. y0 + TY - 1, t0 - 2 .. t0 + TT - 1: columns
      // 0 .. TT - 1 of the region two rows per pass, then its last two
      // columns
      auto normal_at = [&](int yy, int tt) {
        const int o = yy * kP + tt + kC - 2, i = yy * kFusNW + tt;
        const float c = Ux[o];
        const float3 n = normal_of(make_float3(Un[o] - c, Ux[o + kP] - c, Ux[o + 1] - c), eps2);
        N[i] = n.x;
        N[SN + i] = n.y;
        N[2 * SN + i] = n.z;
      };
      static_assert(kTileThreads == 2 * kTT && kFusNH % 2 == 0, "two region rows per pass");
#pragma unroll
      for (int yy = threadIdx.x / kTT; yy < kFusNH; yy += 2) normal_at(yy, threadIdx.x % kTT);
      if (threadIdx.x < 2 * kFusNH) normal_at(threadIdx.x >> 1, kTT + (threadIdx.x & 1));
      __syncthreads();
      // the own voxels: outputs of the post step, q
      float3 qj[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = lane + 32 * j;
        const int u = (iy + 2) * kP + kC + it;   // staged u+ index
        const int bk = (iy + 1) * kP + kC + it;  // staged u-bar / u^k index
        const int r2 = (iy + 2) * kFusNW + it + 2;
        const int r1 = (iy + 1) * kRW + it + 1;
        const float kap = (N[r2] - nx_prev[j]) + (N[SN + r2] - N[SN + r2 - kFusNW]) + (N[2 * SN + r2] - N[2 * SN + r2 - 1]);
        nx_prev[j] = N[r2];
        const FusedPoint fp = fused_point<KIND>(make_float4(Ux[u], Un[u], Ux[u + kP], Ux[u + 1]),
                                                make_float4(Bx[bk], Bn[bk], Bx[bk + kP], Bx[bk + 1]),
                                                make_float4(Kx[bk], Kn[bk], Kx[bk + kP], Kx[bk + 1]), lj[j], pj[j],
                                                kap, mu, inv_mu, beta, pa, pb);
        const size_t gi = g.idx(x, y, T.t0 + it);
        lamo[gi] = fp.lam.x;
        lamo[V + gi] = fp.lam.y;
        lamo[2 * V + gi] = fp.lam.z;
        pho[gi] = fp.phi;
        ubn[gi] = fp.ubn;
        ca.add(0, fp.phi * fp.gn);
        ca.add(1, fp.d2);
        Q[r1] = fp.q.x;
        Q[SQ + r1] = fp.q.y;
        Q[2 * SQ + r1] = fp.q.z;
        qj[j] = fp.q;
      }
      // the halo voxel: q only
      if (has_halo) {
        const int u = (hy + 1) * kP + kC - 1 + ht;
        const int bk = hy * kP + kC - 1 + ht;
        const int r2 = (hy + 1) * kFusNW + ht + 1;
        const int r1 = hy * kRW + ht;
        const float kap = (N[r2] - H[h]) + (N[SN + r2] - N[SN + r2 - kFusNW]) + (N[2 * SN + r2] - N[2 * SN + r2 - 1]);
        H[h] = N[r2];
        const FusedPoint fp = fused_point<KIND>(make_float4(Ux[u], Un[u], Ux[u + kP], Ux[u + 1]),
                                                make_float4(Bx[bk], Bn[bk], Bx[bk + kP], Bx[bk + 1]),
                                                make_float4(Kx[bk], Kn[bk], Kx[bk + kP], Kx[bk + 1]), lh, phh, kap,
                                                mu, inv_mu, beta, pa, pb);
        Q[r1] = fp.q.x;
        Q[SQ + r1] = fp.q.y;
        Q[2 * SQ + r1] = fp.q.z;
      }
      __syncthreads();
      // reg = -mu sum_d (q_d(c) - q_d(c - e_d)) at the own voxels
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int it = lane + 32 * j;
        const int r1 = (iy + 1) * kRW + it + 1;
        const float div =
            (qj[j].x - qx_prev[j]) + (qj[j].y - Q[SQ + r1 - kRW]) + (qj[j].z - Q[2 * SQ + r1 - 1]);
        reg[g.idx(x, y, T.t0 + it)] = -mu * div;
        qx_prev[j] = qj[j].x;
      }
      // the next step's first shared writes (the prefetch into this step's
      // slots, then N and Q) all come after a barrier that follows every
      // read of them above
    }
    cp_async_wait_all();
  }
  block_reduce_acc(ca, partials);
  end_iteration_if_last(ie, partials);
}

}  // namespace nlos
