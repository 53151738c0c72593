// Curvature-regularisation sub-steps and the ADMM drivers of Algorithm 1
// (Sec. 3, Eq. 5-12) and Algorithm 2 (Sec. 4.1, Eq. 13), plus the operator
// norm by power iteration.
//
// Every iteration is a fixed sequence of launches on the caller's stream.
// Scalars that change between iterations (L, the FISTA t and beta, energies)
// live in a DevScalars block in device memory and are updated by one-thread
// kernels, so no host synchronisation is needed per iteration unless the
// backtracking rule can still reject a step (L below 1.5 ||A_D||^2).
#include <cmath>
#include <array>
#include <cstring>

#include "passes.cuh"
#include "stencil.cuh"
#include "stencil_tiled.cuh"

namespace nlos {

constexpr int kStencilThreads = 256;

__host__ __device__ inline int ilog2i(int n) {
  int r = 0;
  while ((1 << r) < n) ++r;
  return r;
}

struct VoxIter {
  int lt, ly;
  __device__ __forceinline__ void decode(size_t i, const Vox& g, int& x, int& y, int& t) const {
    t = (int)(i & g.mt);
    y = (int)((i >> lt) & g.my);
    x = (int)(i >> (lt + ly));
  }
};

// ---------------------------------------------------------------------------
// Elementwise and reduction utilities
// ---------------------------------------------------------------------------
__global__ void k_fill(float* __restrict__ a, float v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] = v;
}

__global__ void k_scale(float* __restrict__ a, const double* __restrict__ s, size_t n) {
  const float f = (float)(1.0 / *s);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] *= f;
}

// partials[b][0] = sum a^2 (optionally only over columns with colpos >= 0)
__global__ void __launch_bounds__(kStencilThreads)
    k_sumsq(const float* __restrict__ a, size_t n, double* __restrict__ partials) {
  SumAcc<1> ca;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = __ldg(a + i);
    ca.add(0, v * v);
  }
  block_reduce_acc(ca, partials);
}

// Deterministic block-wide sums of per-block partials: thread i adds the
// partials of blocks i, i + T, i + 2T, ... in order, then a fixed binary tree
// combines the threads.  Every thread of the (single) block gets the result.
constexpr int kSumThreads = 256;

template <int NTERMS>
__device__ __forceinline__ void sum_partials_block(const double* __restrict__ p, int nb, const int (&terms)[NTERMS],
                                                   double (&out)[NTERMS]) {
  __shared__ double red[NTERMS][kSumThreads];
  double acc[NTERMS];
#pragma unroll
  for (int t = 0; t < NTERMS; ++t) acc[t] = 0.0;
  for (int b = threadIdx.x; b < nb; b += kSumThreads)
#pragma unroll
    for (int t = 0; t < NTERMS; ++t) acc[t] += p[(size_t)b * kMaxTerms + terms[t]];
#pragma unroll
  for (int t = 0; t < NTERMS; ++t) red[t][threadIdx.x] = acc[t];
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int t = 0; t < NTERMS; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + w];
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < NTERMS; ++t) out[t] = red[t][0];
  __syncthreads();
}

__global__ void __launch_bounds__(kSumThreads) k_sum_to(const double* __restrict__ p, int nb, int term,
                                                        double* __restrict__ out) {
  const int terms[1] = {term};
  double r[1];
  sum_partials_block<1>(p, nb, terms, r);
  if (threadIdx.x == 0) *out = r[0];
}

// s = sum(pnum) / sum(pden) over nb block partials (0 when the denominator is
// 0), the back-projection scale, into *out.
__global__ void __launch_bounds__(kSumThreads) k_ratio(const double* __restrict__ pnum,
                                                       const double* __restrict__ pden, int nb,
                                                       double* __restrict__ out) {
  const int t0[1] = {0};
  double n[1], d[1];
  sum_partials_block<1>(pnum, nb, t0, n);
  sum_partials_block<1>(pden, nb, t0, d);
  if (threadIdx.x == 0) *out = d[0] > 0.0 ? n[0] / d[0] : 0.0;
}

// out = a x + b y
__global__ void k_axpby(const float* __restrict__ x, float a, const float* __restrict__ y, float b,
                        float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

// x *= s, y *= s for the device scalar s (FP64, applied in FP32).
__global__ void k_scale2(float* __restrict__ x, size_t nx, float* __restrict__ y, size_t ny,
                         const double* __restrict__ s) {
  const float f = (float)*s;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nx + ny; i += (size_t)gridDim.x * blockDim.x) {
    if (i < nx)
      x[i] *= f;
    else
      y[i - nx] *= f;
  }
}

// Copy the sampled columns of a full [nx*ny][nt] array into compact form.
__global__ void k_gather_cols(const float* __restrict__ full, const int32_t* __restrict__ cols, int ncols, int nt,
                              float* __restrict__ out) {
  const size_t n = (size_t)ncols * nt;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / nt), t = (int)(i % nt);
    out[i] = __ldg(full + (size_t)__ldg(cols + j) * nt + t);
  }
}

// ---------------------------------------------------------------------------
// Curvature weight phi(kappa(u)) (Sec. 3)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kStencilThreads)
    k_curv_weight(const float* __restrict__ u, float* __restrict__ ph, Vox g, VoxIter vi, float a, float b, int kind,
                  float eps2, size_t V) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, t;
    vi.decode(i, g, x, y, t);
    ph[i] = phi_of(curvature_at(u, g, x, y, t, eps2, nullptr), a, b, kind);
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1 stencils
// ---------------------------------------------------------------------------
// reg = mu nabla^*(v + Lam/mu), v = shrink(grad ubar - Lam/mu, phi/mu) (Eq. 7 and
// the right-hand side of the PDE above Eq. 11); nabla^* q = -div_b q.
__global__ void __launch_bounds__(kStencilThreads)
    k_pre1(const float* __restrict__ ub, const float* __restrict__ lam, const float* __restrict__ ph,
           float* __restrict__ reg, Vox g, VoxIter vi, float mu, size_t V) {
  const float inv_mu = 1.0f / mu;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, t;
    vi.decode(i, g, x, y, t);
    const float3 vc = v_at(ub, lam, V, ph, g, x, y, t, inv_mu);
    const int ixm = g.idx((x - 1) & g.mx, y, t), iym = g.idx(x, (y - 1) & g.my, t), itm = g.idx(x, y, (t - 1) & g.mt);
    const float qxm = v_at(ub, lam, V, ph, g, (x - 1) & g.mx, y, t, inv_mu).x + __ldg(lam + ixm) * inv_mu;
    const float qym = v_at(ub, lam, V, ph, g, x, (y - 1) & g.my, t, inv_mu).y + __ldg(lam + V + iym) * inv_mu;
    const float qtm = v_at(ub, lam, V, ph, g, x, y, (t - 1) & g.mt, inv_mu).z + __ldg(lam + 2 * V + itm) * inv_mu;
    const float qcx = vc.x + __ldg(lam + i) * inv_mu;
    const float qcy = vc.y + __ldg(lam + V + i) * inv_mu;
    const float qct = vc.z + __ldg(lam + 2 * V + i) * inv_mu;
    reg[i] = -mu * ((qcx - qxm) + (qcy - qym) + (qct - qtm));
  }
}

// After an accepted u-step: Lam += mu (v - grad u+) (Eq. 12), phi = phi(kappa(u+)),
// ubar_next = u+ + beta (u+ - u^k) (Algorithm 1); partials 0 = sum phi |grad u+|,
// 1 = sum |v - grad u+|^2.
__global__ void __launch_bounds__(kStencilThreads)
    k_post1(const float* __restrict__ unew, const float* __restrict__ uk, const float* __restrict__ ub,
            float* __restrict__ lam, float* __restrict__ ph, float* __restrict__ ubn, const DevScalars* __restrict__ sc,
            Vox g, VoxIter vi, float mu, float a, float b, int kind, float eps2, size_t V, double* __restrict__ partials) {
  const float inv_mu = 1.0f / mu;
  const float beta = (float)sc->beta_next;
  SumAcc<2> ca;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, t;
    vi.decode(i, g, x, y, t);
    const float3 v = v_at(ub, lam, V, ph, g, x, y, t, inv_mu);
    float3 gu;
    const float kap = curvature_at(unew, g, x, y, t, eps2, &gu);
    const float3 d = make_float3(v.x - gu.x, v.y - gu.y, v.z - gu.z);
    lam[i] += mu * d.x;
    lam[V + i] += mu * d.y;
    lam[2 * V + i] += mu * d.z;
    const float pn = phi_of(kap, a, b, kind);
    ph[i] = pn;
    const float un = __ldg(unew + i);
    ubn[i] = un + beta * (un - __ldg(uk + i));
    ca.add(0, pn * sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z));
    ca.add(1, d.x * d.x + d.y * d.y + d.z * d.z);
  }
  block_reduce_acc(ca, partials);
}

// ---------------------------------------------------------------------------
// Algorithm 2 stencils
// ---------------------------------------------------------------------------
struct Alg2Coef {
  float mu1, mu2, mu3, lam_w;
  float a_u, b_u, a_t, b_t;
  int kind;
  float eps2;
};

__device__ __forceinline__ float mask_at(const int32_t* __restrict__ colpos, const Vox& g, int x, int y) {
  return colpos ? (__ldg(colpos + x * g.ny + y) >= 0 ? 1.0f : 0.0f) : 1.0f;
}

// f = (lambda M tau0 + mu3 tau-bar - Lam3) / (lambda M + mu3)
__device__ __forceinline__ float f_at(float m, float t0, float tb, float l3, const Alg2Coef& c) {
  return (c.lam_w * m * t0 + c.mu3 * tb - l3) / (c.lam_w * m + c.mu3);
}

__global__ void __launch_bounds__(kStencilThreads)
    k_pre2(const float* __restrict__ ub, const float* __restrict__ tb, const float* __restrict__ lam1,
           const float* __restrict__ lam2, const float* __restrict__ lam3, const float* __restrict__ phu,
           const float* __restrict__ pht, const float* __restrict__ tau0, const int32_t* __restrict__ colpos,
           float* __restrict__ regu, float* __restrict__ regt, Vox g, VoxIter vi, Alg2Coef c, size_t V) {
  const float im1 = 1.0f / c.mu1, im2 = 1.0f / c.mu2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, t;
    vi.decode(i, g, x, y, t);
    const int xm = (x - 1) & g.mx, ym = (y - 1) & g.my, tm = (t - 1) & g.mt;
    const int ixm = g.idx(xm, y, t), iym = g.idx(x, ym, t), itm = g.idx(x, y, tm);
    {
      const float3 vc = v_at(ub, lam1, V, phu, g, x, y, t, im1);
      const float qxm = v_at(ub, lam1, V, phu, g, xm, y, t, im1).x + __ldg(lam1 + ixm) * im1;
      const float qym = v_at(ub, lam1, V, phu, g, x, ym, t, im1).y + __ldg(lam1 + V + iym) * im1;
      const float qtm = v_at(ub, lam1, V, phu, g, x, y, tm, im1).z + __ldg(lam1 + 2 * V + itm) * im1;
      regu[i] = -c.mu1 * ((vc.x + __ldg(lam1 + i) * im1 - qxm) + (vc.y + __ldg(lam1 + V + i) * im1 - qym) +
                          (vc.z + __ldg(lam1 + 2 * V + i) * im1 - qtm));
    }
    {
      const float3 wc = v_at(tb, lam2, V, pht, g, x, y, t, im2);
      const float pxm = v_at(tb, lam2, V, pht, g, xm, y, t, im2).x + __ldg(lam2 + ixm) * im2;
      const float pym = v_at(tb, lam2, V, pht, g, x, ym, t, im2).y + __ldg(lam2 + V + iym) * im2;
      const float ptm = v_at(tb, lam2, V, pht, g, x, y, tm, im2).z + __ldg(lam2 + 2 * V + itm) * im2;
      const float div = (wc.x + __ldg(lam2 + i) * im2 - pxm) + (wc.y + __ldg(lam2 + V + i) * im2 - pym) +
                        (wc.z + __ldg(lam2 + 2 * V + i) * im2 - ptm);
      const float l3 = __ldg(lam3 + i);
      const float f = f_at(mask_at(colpos, g, x, y), __ldg(tau0 + i), __ldg(tb + i), l3, c);
      regt[i] = -c.mu2 * div + c.mu3 * (f + l3 / c.mu3);
    }
  }
}

// Post step of Algorithm 2: multipliers, phi_u, phi_tau, extrapolation, and
// partials 0 sum phi_u|grad u|, 1 sum phi_t|grad tau|, 2 sum (A u - tau)^2,
// 3 sum M (tau - tau0)^2, 4 |v - grad u|^2, 5 |w - grad tau|^2, 6 (f - tau)^2.
__global__ void __launch_bounds__(kStencilThreads)
    k_post2(const float* __restrict__ unew, const float* __restrict__ uk, const float* __restrict__ ub,
            const float* __restrict__ tnew, const float* __restrict__ tk, const float* __restrict__ tb,
            float* __restrict__ lam1, float* __restrict__ lam2, float* __restrict__ lam3, float* __restrict__ phu,
            float* __restrict__ pht, float* __restrict__ ubn, float* __restrict__ tbn, const float* __restrict__ au,
            const float* __restrict__ tau0, const int32_t* __restrict__ colpos, const DevScalars* __restrict__ sc, Vox g,
            VoxIter vi, Alg2Coef c, size_t V, double* __restrict__ partials) {
  const float im1 = 1.0f / c.mu1, im2 = 1.0f / c.mu2;
  const float beta = (float)sc->beta_next;
  SumAcc<7> ca;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, t;
    vi.decode(i, g, x, y, t);
    const float3 v = v_at(ub, lam1, V, phu, g, x, y, t, im1);
    const float3 w = v_at(tb, lam2, V, pht, g, x, y, t, im2);
    const float m = mask_at(colpos, g, x, y);
    const float t0 = __ldg(tau0 + i);
    const float l3 = lam3[i];
    const float f = f_at(m, t0, __ldg(tb + i), l3, c);
    float3 gu, gt;
    const float ku = curvature_at(unew, g, x, y, t, c.eps2, &gu);
    const float kt = curvature_at(tnew, g, x, y, t, c.eps2, &gt);
    const float3 dv = make_float3(v.x - gu.x, v.y - gu.y, v.z - gu.z);
    const float3 dw = make_float3(w.x - gt.x, w.y - gt.y, w.z - gt.z);
    const float tn = __ldg(tnew + i), un = __ldg(unew + i);
    lam1[i] += c.mu1 * dv.x;
    lam1[V + i] += c.mu1 * dv.y;
    lam1[2 * V + i] += c.mu1 * dv.z;
    lam2[i] += c.mu2 * dw.x;
    lam2[V + i] += c.mu2 * dw.y;
    lam2[2 * V + i] += c.mu2 * dw.z;
    lam3[i] = l3 + c.mu3 * (f - tn);
    const float pu = phi_of(ku, c.a_u, c.b_u, c.kind), pt = phi_of(kt, c.a_t, c.b_t, c.kind);
    phu[i] = pu;
    pht[i] = pt;
    ubn[i] = un + beta * (un - __ldg(uk + i));
    tbn[i] = tn + beta * (tn - __ldg(tk + i));
    const float r = __ldg(au + i) - tn;
    const float s = m * (tn - t0);
    ca.add(0, pu * sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z));
    ca.add(1, pt * sqrtf(gt.x * gt.x + gt.y * gt.y + gt.z * gt.z));
    ca.add(2, r * r);
    ca.add(3, s * s);
    ca.add(4, dv.x * dv.x + dv.y * dv.y + dv.z * dv.z);
    ca.add(5, dw.x * dw.x + dw.y * dw.y + dw.z * dw.z);
    ca.add(6, (f - tn) * (f - tn));
  }
  block_reduce_acc(ca, partials);
}

// ---------------------------------------------------------------------------
// Scalar kernels (one thread)
// ---------------------------------------------------------------------------
// Backtracking test of the linearised u-step: f is quadratic, so
// f(u+) - f(ubar) - <grad f(ubar), d> = 1/2 ||A d||^2 and the rule
// f(u+) <= f(ubar) + <grad f, d> + L/2 ||d||^2 is ||A d||^2 <= L ||d||^2.
// With `set_redo` (inside a graph) it also sets the condition of the
// backtracking loop node `redo`: 1 only after a rejection that leaves the
// status OK, so the loop ends after at most max_bt + 1 trials.
__global__ void __launch_bounds__(kSumThreads)
    k_test(DevScalars* sc, const double* __restrict__ pd, int nbd, const double* __restrict__ pf, int nbf, double eta,
           int max_bt, int force_accept, cudaGraphConditionalHandle redo, int set_redo) {
  const int t0[1] = {0};
  const int t01[2] = {0, 1};
  double d[1], f[2];
  sum_partials_block<1>(pd, nbd, t0, d);
  sum_partials_block<2>(pf, nbf, t01, f);
  if (threadIdx.x != 0) return;
  if (set_redo) cudaGraphSetConditional(redo, 0);
  if (sc->status != NLOS_OK) return;
  const double dn2 = d[0], r2 = f[0], ad2 = f[1];
  sc->test_lhs = ad2;
  sc->test_rhs = sc->L * dn2;
  const bool ok = ad2 <= sc->L * dn2;
  if (ok || force_accept) {
    sc->accept = 1;
    sc->f_fit = 0.5 * r2;
    const double tn = (1.0 + sqrt(1.0 + 4.0 * sc->t * sc->t)) / 2.0;
    sc->beta = (sc->t - 1.0) / tn;
    sc->t = tn;
    sc->rej_iter = 0;
  } else {
    sc->accept = 0;
    sc->L *= eta;
    sc->backtracks += 1;
    sc->rej_iter += 1;
    if (sc->rej_iter > max_bt) sc->status = NLOS_ERR_DIVERGED;
    if (set_redo && sc->status == NLOS_OK) cudaGraphSetConditional(redo, 1);
  }
}

// Graph-resident iteration loop (one thread each).  Each trip of the loop
// body runs one iteration out of a switch over the six pointer phases of the
// solver state (the u / u-bar buffers alternate with period 2 and the cached
// A u iterates rotate with period 3); `trips` counts the trips.
__global__ void k_loop_begin(const DevScalars* sc, cudaGraphConditionalHandle phase) {
  cudaGraphSetConditional(phase, (unsigned)(sc->trips % 6));
}
// End of a trip: continue while the status is OK, the relative-energy stop
// has not fired and fewer than `iters` trips ran (the trip count alone bounds
// the loop).
__global__ void k_loop_end(DevScalars* sc, cudaGraphConditionalHandle cont, int iters) {
  sc->trips += 1;
  const bool go = sc->trips < iters && sc->status == NLOS_OK && !sc->stop;
  cudaGraphSetConditional(cont, go ? 1u : 0u);
}
// o = a after an even number of trips, b after an odd number.
__global__ void k_select_copy(float* __restrict__ o, const float* __restrict__ a, const float* __restrict__ b,
                              size_t n, const DevScalars* sc) {
  const float* src = (sc->trips & 1) ? b : a;
  const bool al = ((reinterpret_cast<uintptr_t>(o) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
  const size_t n4 = al ? n / 4 : 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    reinterpret_cast<float4*>(o)[i] = __ldg(reinterpret_cast<const float4*>(src) + i);
  for (size_t i = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    o[i] = __ldg(src + i);
}

// End of an iteration: energy, relative change, restart, bookkeeping.
// model 1: E = f_fit + sum phi |grad u|; model 2: E from the post partials.
// fold_test (model 1, a test that cannot reject): the accepting test's
// bookkeeping (k_test with force_accept) is done here first, from the fit
// partials pf of nbf blocks, so the iteration needs no separate k_test launch.
__global__ void __launch_bounds__(kSumThreads)
    k_finalize(DevScalars* sc, const double* __restrict__ pp, int nb, int model, double lam_w, int restart,
               double eps_stop, const double* __restrict__ pf, int nbf, int fold_test) {
  const int terms[7] = {0, 1, 2, 3, 4, 5, 6};
  double v[7];
  sum_partials_block<7>(pp, nb, terms, v);
  double f[2] = {0.0, 0.0};
  if (fold_test) {
    const int t01[2] = {0, 1};
    sum_partials_block<2>(pf, nbf, t01, f);
  }
  if (threadIdx.x != 0) return;
  if (model == 1) {
    finalize1(sc, v[0], v[1], f[0], f[1], fold_test, restart, eps_stop);
    return;
  }
  if (sc->status != NLOS_OK) return;
  const double fit = 0.5 * v[2];
  sc->f_fit = fit;
  finalize_tail(sc, fit + 0.5 * lam_w * v[3] + v[0] + v[1], v[4], restart, eps_stop);
}

// End of an Algorithm-2 iteration from the partials of the split post step
// (u: phi|grad u|, |v - grad u|^2; tau: phi|grad tau|, |w - grad tau|^2;
// elementwise, terms t3 .. t3 + 2 of p3: (A u - tau)^2, M (tau - tau0)^2,
// (f - tau)^2).
__global__ void __launch_bounds__(kSumThreads)
    k_finalize2(DevScalars* sc, const double* __restrict__ pu, int nbu, const double* __restrict__ pt, int nbt,
                const double* __restrict__ p3, int nb3, int t3, double lam_w, int restart, double eps_stop) {
  const int t01[2] = {0, 1};
  const int t012[3] = {t3, t3 + 1, t3 + 2};
  double u[2], t[2], e3[3];
  sum_partials_block<2>(pu, nbu, t01, u);
  sum_partials_block<2>(pt, nbt, t01, t);
  sum_partials_block<3>(p3, nb3, t012, e3);
  if (threadIdx.x != 0) return;
  if (sc->status != NLOS_OK) return;
  const double fit = 0.5 * e3[0];
  sc->f_fit = fit;
  finalize_tail(sc, fit + 0.5 * lam_w * e3[1] + u[0] + t[0], u[1], restart, eps_stop);
}

// Initial scalar block; E_prev = s0 sum(pe0) + s1 sum(pe1) + s2 sum(pe2) over
// the nb block partials of each (pe1, pe2 nullable).
__global__ void __launch_bounds__(kSumThreads)
    k_init_scalars(DevScalars* sc, double L0, int nb, const double* __restrict__ pe0, double s0,
                   const double* __restrict__ pe1, double s1, const double* __restrict__ pe2, double s2) {
  const int t0[1] = {0};
  double v0[1], v1[1] = {0.0}, v2[1] = {0.0};
  sum_partials_block<1>(pe0, nb, t0, v0);
  if (pe1) sum_partials_block<1>(pe1, nb, t0, v1);
  if (pe2) sum_partials_block<1>(pe2, nb, t0, v2);
  if (threadIdx.x != 0) return;
  memset(sc, 0, sizeof(DevScalars));
  sc->L = L0;
  sc->t = 1.0;
  sc->E_prev = s0 * v0[0] + s1 * v1[0] + s2 * v2[0];
  sc->status = NLOS_OK;
  set_next_step(sc);
}

// partials[b][0] = sum phi |grad u| (forward differences, periodic): the
// curvature-weighted TV term of the energy at a given u.
__global__ void __launch_bounds__(kStencilThreads)
    k_tv_weighted(const float* __restrict__ u, const float* __restrict__ ph, Vox g, VoxIter vi, size_t V,
                  double* __restrict__ partials) {
  SumAcc<1> ca;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, t;
    vi.decode(i, g, x, y, t);
    const float3 gu = grad_at(u, g, x, y, t);
    ca.add(0, __ldg(ph + i) * sqrtf(gu.x * gu.x + gu.y * gu.y + gu.z * gu.z));
  }
  block_reduce_acc(ca, partials);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct SolverState {
  int model = 0;
  size_t V = 0;
  float *uk = nullptr, *unew = nullptr, *ub = nullptr, *ubn = nullptr, *lam = nullptr, *ph = nullptr, *reg = nullptr;
  // the fused post and pre step (Algorithm 1; Algorithm 2's u half): Lambda
  // and phi of the next iteration (swapped with lam and ph after every
  // iteration)
  float *lamn = nullptr, *phn = nullptr;
  float *tk = nullptr, *tnew = nullptr, *tb = nullptr, *tbn = nullptr, *lam2 = nullptr, *lam3 = nullptr,
        *pht = nullptr, *regt = nullptr, *tmp = nullptr;
  float* tau0c = nullptr;
  float* cache[3] = {nullptr, nullptr, nullptr};
  double *pa = nullptr, *pb = nullptr, *pc = nullptr;
  DevScalars* sc = nullptr;
  DevScalars* h_sc = nullptr;
  std::vector<void*> allocs;
};

static nlos_status dalloc(SolverState* s, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(NLOS_ERR_OOM, std::string("cudaMalloc of solver state failed: ") + cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  return NLOS_OK;
}

void free_solver(SolverState* s) {
  if (!s) return;
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  delete s;
}

static nlos_status get_solver(Plan& P, int model, SolverState** out) {
  if (P.solver[model]) {
    *out = P.solver[model];
    return NLOS_OK;
  }
  SolverState* s = new SolverState();
  s->model = model;
  const size_t V = (size_t)P.nx * P.ny * P.nt;
  s->V = V;
  const size_t F = V * sizeof(float);
  nlos_status st = NLOS_OK;
  auto A = [&](float** p, size_t bytes) {
    if (st == NLOS_OK) st = dalloc(s, reinterpret_cast<void**>(p), bytes);
  };
  A(&s->uk, F); A(&s->unew, F); A(&s->ub, F); A(&s->ubn, F); A(&s->lam, 3 * F); A(&s->ph, F); A(&s->reg, F);
  const size_t cachesz = model == 1 ? (size_t)P.ncols * P.nt * sizeof(float) : F;
  for (int i = 0; i < 3; ++i) A(&s->cache[i], cachesz);
  A(&s->lamn, 3 * F); A(&s->phn, F);
  if (model == 1) {
    A(&s->tau0c, (size_t)P.ncols * P.nt * sizeof(float));
  } else {
    A(&s->tk, F); A(&s->tnew, F); A(&s->tb, F); A(&s->tbn, F); A(&s->lam2, 3 * F); A(&s->lam3, F);
    A(&s->pht, F); A(&s->regt, F); A(&s->tmp, F);
  }
  const size_t pbytes = sizeof(double) * kMaxTerms * 4096;
  if (st == NLOS_OK) st = dalloc(s, reinterpret_cast<void**>(&s->pa), pbytes);
  if (st == NLOS_OK) st = dalloc(s, reinterpret_cast<void**>(&s->pb), pbytes);
  if (st == NLOS_OK) st = dalloc(s, reinterpret_cast<void**>(&s->pc), pbytes);
  if (st == NLOS_OK) st = dalloc(s, reinterpret_cast<void**>(&s->sc), sizeof(DevScalars));
  if (st == NLOS_OK) {
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&s->h_sc), sizeof(DevScalars));
    if (e != cudaSuccess) st = fail(NLOS_ERR_OOM, "cudaMallocHost failed");
  }
  if (st != NLOS_OK) {
    free_solver(s);
    return st;
  }
  P.solver[model] = s;
  *out = s;
  return NLOS_OK;
}

static int elem_grid(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 16); }

// Operator applications shared by the C API and the solvers.
nlos_status apply_forward(const Plan& P, const float* u, float* out, bool compact, cudaStream_t st) {
  const int full = P.nx * P.ny;
  NLOS_TRY(launch_tfwd_rz(P, u, full, P.d_S, full, st));
  if (compact) {
    NLOS_TRY(launch_conv(P, P.d_S, false, P.d_Sc, true, false, st));
    NLOS_TRY(launch_tinv_store(P, P.d_Sc, P.ncols, P.ncols, out, nullptr, st));
  } else {
    NLOS_TRY(launch_conv(P, P.d_S, false, P.d_S, false, false, st));
    NLOS_TRY(launch_tinv_store(P, P.d_S, full, full, out, nullptr, st));
  }
  return NLOS_OK;
}

nlos_status apply_adjoint(const Plan& P, const float* r, float* u, bool compact, cudaStream_t st) {
  const int full = P.nx * P.ny;
  Lin3 src{{r, nullptr, nullptr}, {1.f, 0.f, 0.f}, nullptr};
  if (compact) {
    NLOS_TRY(launch_tfwd_rtt(P, src, P.ncols, P.d_Sc, P.ncols, st));
    NLOS_TRY(launch_conv(P, P.d_Sc, true, P.d_S, false, true, st));
  } else {
    NLOS_TRY(launch_tfwd_rtt(P, src, full, P.d_S, full, st));
    NLOS_TRY(launch_conv(P, P.d_S, false, P.d_S, false, true, st));
  }
  NLOS_TRY(launch_tadj_store(P, P.d_S, full, full, u, st));
  return NLOS_OK;
}

nlos_status gather_columns(const Plan& P, const float* full, float* compact, cudaStream_t st) {
  const size_t n = (size_t)P.ncols * P.nt;
  { KTimer kt_(P, KC_SMALL, st);
  k_gather_cols<<<elem_grid(n), 256, 0, st>>>(full, P.d_cols, P.ncols, P.nt, compact);
  }
  NLOS_LAUNCH_CHECK("k_gather_cols");
  return NLOS_OK;
}

nlos_status apply_solve(const Plan& P, const float* rhs, float* x, double c0, double c1, cudaStream_t st) {
  const int full = P.nx * P.ny;
  NLOS_TRY(launch_sfwd(P, rhs, full, P.d_Sp, st));
  NLOS_TRY(launch_sxy(P, P.d_Sp, nullptr, c0, c1, st));
  NLOS_TRY(launch_sinv(P, P.d_Sp, full, x, nullptr, nullptr, nullptr, st));
  return NLOS_OK;
}

nlos_status apply_curvature_weight(const Plan& P, const float* u, float* ph, double a, double b, int kind, double eps,
                                   cudaStream_t st) {
  const Vox g = make_vox(P.nx, P.ny, P.nt);
  VoxIter vi{ilog2i(P.nt), ilog2i(P.ny)};
  const size_t V = (size_t)P.nx * P.ny * P.nt;
  { KTimer kt_(P, KC_SMALL, st);
  k_curv_weight<<<stencil_blocks(P), kStencilThreads, 0, st>>>(u, ph, g, vi, (float)a, (float)b, kind,
                                                            (float)(eps * eps), V);
  }
  NLOS_LAUNCH_CHECK("k_curv_weight");
  return NLOS_OK;
}

// Sum of squares of n floats, read back to the host (synchronises st).
static nlos_status host_sumsq(const Plan& P, const float* a, size_t n, double* out, cudaStream_t st) {
  { KTimer kt_(P, KC_SMALL, st);
  k_sumsq<<<stencil_blocks(P), kStencilThreads, 0, st>>>(a, n, P.d_partials);
  }
  NLOS_LAUNCH_CHECK("k_sumsq");
  double* d_out = reinterpret_cast<double*>(P.d_scal);
  { KTimer kt_(P, KC_SMALL, st);
  k_sum_to<<<1, kSumThreads, 0, st>>>(P.d_partials, stencil_blocks(P), 0, d_out);
  }
  NLOS_LAUNCH_CHECK("k_sum_to");
  NLOS_CUDA(cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  NLOS_CUDA(cudaStreamSynchronize(st));
  return NLOS_OK;
}

// ||A_D||^2 by power iteration on A_D^T A_D from the all-ones vector.
nlos_status plan_norm2(Plan& P, bool masked, cudaStream_t st, double* out) {
  double& cached = masked ? P.norm2_masked : P.norm2_full;
  if (cached >= 0.0) {
    *out = cached;
    return NLOS_OK;
  }
  const size_t V = (size_t)P.nx * P.ny * P.nt;
  const bool compact = masked && !P.full_mask;
  const size_t ny_elems = compact ? (size_t)P.ncols * P.nt : V;
  float *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, V * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(NLOS_ERR_OOM, "power iteration buffers");
  }
  if (cudaMalloc(&y, ny_elems * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(x);
    return fail(NLOS_ERR_OOM, "power iteration buffers");
  }
  nlos_status s = NLOS_OK;
  double lam = 0.0, lam_new = 0.0;
  { KTimer kt_(P, KC_SMALL, st);
  k_fill<<<elem_grid(V), 256, 0, st>>>(x, (float)(1.0 / std::sqrt((double)V)), V);
  }
  for (int it = 1; it <= 200 && s == NLOS_OK; ++it) {
    s = apply_forward(P, x, y, compact, st);
    if (s != NLOS_OK) break;
    s = host_sumsq(P, y, ny_elems, &lam_new, st);
    if (s != NLOS_OK) break;
    s = apply_adjoint(P, y, x, compact, st);
    if (s != NLOS_OK) break;
    double nz2 = 0.0;
    s = host_sumsq(P, x, V, &nz2, st);
    if (s != NLOS_OK) break;
    if (nz2 == 0.0) {
      lam_new = 0.0;
      break;
    }
    const double nz = std::sqrt(nz2);
    double* d_nz = reinterpret_cast<double*>(P.d_scal) + 1;
    cudaMemcpyAsync(d_nz, &nz, sizeof(double), cudaMemcpyHostToDevice, st);
    { KTimer kt_(P, KC_SMALL, st);
    k_scale<<<elem_grid(V), 256, 0, st>>>(x, d_nz, V);
    }
    if (it > 1 && std::fabs(lam_new - lam) <= 1e-12 * lam_new) break;
    lam = lam_new;
  }
  cudaStreamSynchronize(st);
  cudaFree(x);
  cudaFree(y);
  if (s != NLOS_OK) return s;
  cached = lam_new;
  *out = lam_new;
  return NLOS_OK;
}

static nlos_status read_scalars(SolverState* s, cudaStream_t st) {
  NLOS_CUDA(cudaMemcpyAsync(s->h_sc, s->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
  NLOS_CUDA(cudaStreamSynchronize(st));
  return NLOS_OK;
}

static void fill_stats(const DevScalars& d, nlos_stats* o) {
  if (!o) return;
  o->iters_done = d.iter;
  o->backtracks = d.backtracks;
  o->restarts = d.restarts;
  o->status = d.status;
  o->L = d.L;
  o->energy = d.E;
  o->rel_change = d.E != 0.0 ? std::fabs(d.dE) / std::fabs(d.E) : 0.0;
  o->data_fit = d.f_fit;
  o->primal_res = std::sqrt(d.pres2);
}

template <typename T>
static void swap_ptr(T*& a, T*& b) {
  T* t = a;
  a = b;
  b = t;
}

// k_post1_pipe for a phi kind known at run time.
template <bool L3>
static auto post1_pipe_kernel(int kind) {
  return kind == NLOS_PHI_TAC   ? k_post1_pipe<L3, NLOS_PHI_TAC>
         : kind == NLOS_PHI_TRV ? k_post1_pipe<L3, NLOS_PHI_TRV>
                                : k_post1_pipe<L3, NLOS_PHI_TSC>;
}

nlos_status prepare_stencils() {
  NLOS_TRY(ensure_smem(k_pre1_pipe<false>, kPre1PipeSmem));
  NLOS_TRY(ensure_smem(k_pre1_pipe<true>, kPre1PipeSmem));
  NLOS_TRY(ensure_smem(post1_pipe_kernel<true>(NLOS_PHI_TSC), kPost1PipeSmem));
  NLOS_TRY(ensure_smem(post1_pipe_kernel<true>(NLOS_PHI_TAC), kPost1PipeSmem));
  NLOS_TRY(ensure_smem(post1_pipe_kernel<true>(NLOS_PHI_TRV), kPost1PipeSmem));
  NLOS_TRY(ensure_smem(k_post1_pre<NLOS_PHI_TSC>, kPostPreSmem));
  NLOS_TRY(ensure_smem(k_post1_pre<NLOS_PHI_TAC>, kPostPreSmem));
  NLOS_TRY(ensure_smem(k_post1_pre<NLOS_PHI_TRV>, kPostPreSmem));
  return NLOS_OK;
}

// The pipelined halo-tiled stencils apply when the grid tiles evenly (TT =
// 128 along t, TY = 8 rows in y); the plain per-voxel kernels otherwise.
// Tiled Algorithm-1 runs fuse each iteration's post step with the next
// iteration's pre step (k_post1_pre), so only the run's start launches the
// pre step by itself.
static bool stencils_tiled(const Plan& P) { return P.nt % kTT == 0 && P.ny % kTY == 0; }

// reg = -mu div (v + Lambda/mu), v = shrink(grad u-bar - Lambda/mu, phi/mu)
// (Algorithm 1's pre step, and Algorithm 2's for u with mu = mu1) on stream
// st.
static nlos_status pre1(Plan& P, SolverState* s, double mu, cudaStream_t st) {
  const Vox g = make_vox(P.nx, P.ny, P.nt);
  KTimer kt_(P, KC_PRE, st);
  if (stencils_tiled(P)) {
    const int ntiles = stencil_steps(g);
    k_pre1_pipe<false><<<std::min(ntiles, P.sms * 3), kTileThreads, kPre1PipeSmem, st>>>(
        s->ub, s->lam, s->ph, s->reg, g, ntiles, (float)mu, s->V, FTerm{});
  } else {
    const VoxIter vi{ilog2i(P.nt), ilog2i(P.ny)};
    k_pre1<<<stencil_blocks(P), kStencilThreads, 0, st>>>(s->ub, s->lam, s->ph, s->reg, g, vi, (float)mu, s->V);
  }
  NLOS_LAUNCH_CHECK("k_pre1");
  return NLOS_OK;
}

// One linearised u-step with the backtracking loop (shared by both
// algorithms): the adjoint end + solve rhs (the adjoint spectrum is in d_S),
// the lateral solve, the periodic inverse (u+ and ||u+ - ubar||^2), the
// forward operator on u+ (spectrum in d_S2) and the fit/test.
struct UStepArgs {
  const float* reg;
  double mu;
  bool compact;        // model 1: sampled columns only
  const float* data;   // model 1: compact tau0; model 2: tau-bar (full)
  double eta;
  int max_bt;
  float* au_out;       // cache slot receiving A u+
  const float* auk;
  const float* aukm1;
  // model 2: the tau-solve regulariser term; the fit pass then also writes
  // the periodic t-spectrum of A u+ + tau_reg to d_Sp (the tau-solve rhs)
  const float* tau_reg = nullptr;
};

// Helpers for conditional nodes added during a stream capture.
static nlos_status capture_graph_of(cudaStream_t st, cudaGraph_t* g) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NLOS_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return fail(NLOS_ERR_CUDA, "stream is not capturing");
  return NLOS_OK;
}

// A condition handle of the graph that st is capturing into.
static nlos_status cond_handle(cudaStream_t st, unsigned dflt, unsigned flags, cudaGraphConditionalHandle* h) {
  cudaGraph_t g = nullptr;
  NLOS_TRY(capture_graph_of(st, &g));
  NLOS_CUDA(cudaGraphConditionalHandleCreate(h, g, dflt, flags));
  return NLOS_OK;
}

// Appends a conditional node (after everything captured on st so far) and
// continues st's capture after it; bodies receives its `size` body graphs.
static nlos_status add_cond_node(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                 unsigned size, cudaGraph_t* bodies) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  NLOS_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
  if (cs != cudaStreamCaptureStatusActive) return fail(NLOS_ERR_CUDA, "stream is not capturing");
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = size;
  cudaGraphNode_t node = nullptr;
  NLOS_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
  for (unsigned i = 0; i < size; ++i) bodies[i] = np.conditional.phGraph_out[i];
  NLOS_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return NLOS_OK;
}

// Captures fn(bs) into the (empty) body graph `body` on stream bs.
template <typename Fn>
static nlos_status capture_body(cudaStream_t bs, cudaGraph_t body, Fn&& fn) {
  NLOS_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const nlos_status s = fn(bs);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(bs, &out);
  NLOS_TRY(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (conditional body)");
  return NLOS_OK;
}

// One trial of the linearised u-step: solve for u+ at the current L, A u+
// (sampled columns for model 1) and the partial sums of the test.
// One trial of the u-step.  test: the backtracking rule can reject, so the
// trial also forms the partial sums of ||d||^2 and ||A d||^2 it needs; when
// it cannot (L >= 1.5 ||A_D||^2, the descent lemma), those terms are skipped
// (one field pass fewer) and k_test sums no blocks for them.
static nlos_status u_trial(Plan& P, SolverState* s, const UStepArgs& a, bool test, int* nbd, int* nbf,
                           cudaStream_t st) {
  const int full = P.nx * P.ny;
  const int ncols = a.compact ? P.ncols : full;
  SolveRhs sr{s->ub, a.reg, s->sc, 0.0};
  NLOS_TRY(launch_tadj_solve(P, P.d_S, full, full, sr, P.d_Sp, st));
  NLOS_TRY(launch_sxy(P, P.d_Sp, s->sc, 0.0, a.mu, st));
  NLOS_TRY(launch_sinv_rz(P, P.d_Sp, full, s->unew, test ? s->ub : nullptr, test ? s->pa : nullptr, nbd, P.d_S2,
                          full, st, s->sc));
  if (!test) *nbd = 0;
  float2* Sfit = P.d_S2;
  if (a.compact) {
    NLOS_TRY(launch_conv(P, P.d_S2, false, P.d_Sc, true, false, st));
    Sfit = P.d_Sc;
  } else {
    NLOS_TRY(launch_conv(P, P.d_S2, false, P.d_S2, false, false, st));
  }
  FitArgs fa{a.data, a.auk, a.aukm1, s->sc, s->pb, a.tau_reg, a.tau_reg ? P.d_Sp : nullptr, test};
  NLOS_TRY(launch_tinv_fit(P, Sfit, ncols, ncols, a.au_out, fa, nbf, st));
  return NLOS_OK;
}

// The u-step with its backtracking rule.  host_check: the rule can still
// reject (L below 1.5 ||A_D||^2).  Then either the host reads the test after
// every trial, or, while a graph-resident loop is captured (bt_stream set),
// the trials repeat in a conditional loop node on the device.  Otherwise the
// trial is accepted without a host round trip.
static nlos_status u_step(Plan& P, SolverState* s, const UStepArgs& a, bool host_check, double* L_host,
                          cudaStream_t bt_stream, cudaStream_t st, int* nbf_fold = nullptr) {
  // a test that cannot reject: the iteration's end (k_finalize, or the last
  // block of the fused post and pre step) does its bookkeeping from the fit
  // partials (nbf_fold receives their block count)
  if (!host_check && nbf_fold) {
    int nbd = 0;
    return u_trial(P, s, a, false, &nbd, nbf_fold, st);
  }
  if (host_check && bt_stream) {
    cudaGraphConditionalHandle redo = 0;
    NLOS_TRY(cond_handle(st, 0, 0, &redo));
    int nbd = 0, nbf = 0;
    NLOS_TRY(u_trial(P, s, a, true, &nbd, &nbf, st));
    k_test<<<1, kSumThreads, 0, st>>>(s->sc, s->pa, nbd, s->pb, nbf, a.eta, a.max_bt, 0, redo, 1);
    NLOS_LAUNCH_CHECK("k_test");
    cudaGraph_t body = nullptr;
    NLOS_TRY(add_cond_node(st, redo, cudaGraphCondTypeWhile, 1, &body));
    return capture_body(bt_stream, body, [&](cudaStream_t bs) -> nlos_status {
      int nbd2 = 0, nbf2 = 0;
      NLOS_TRY(u_trial(P, s, a, true, &nbd2, &nbf2, bs));
      k_test<<<1, kSumThreads, 0, bs>>>(s->sc, s->pa, nbd2, s->pb, nbf2, a.eta, a.max_bt, 0, redo, 1);
      NLOS_LAUNCH_CHECK("k_test");
      return NLOS_OK;
    });
  }
  for (;;) {
    int nbd = 0, nbf = 0;
    NLOS_TRY(u_trial(P, s, a, host_check, &nbd, &nbf, st));
    { KTimer kt_(P, KC_SMALL, st);
    k_test<<<1, kSumThreads, 0, st>>>(s->sc, s->pa, nbd, s->pb, nbf, a.eta, a.max_bt, host_check ? 0 : 1, 0, 0);
    }
    NLOS_LAUNCH_CHECK("k_test");
    if (!host_check) return NLOS_OK;
    NLOS_TRY(read_scalars(s, st));
    if (s->h_sc->status != NLOS_OK) return fail(NLOS_ERR_DIVERGED, "backtracking did not terminate");
    if (s->h_sc->accept) return NLOS_OK;
    *L_host = s->h_sc->L;  // rejected: L grew on the device, solve again
  }
}

static nlos_status zero(float* p, size_t n, cudaStream_t st) {
  NLOS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(float), st));
  return NLOS_OK;
}

static nlos_status fill(float* p, float v, size_t n, cudaStream_t st) {
  k_fill<<<elem_grid(n), 256, 0, st>>>(p, v, n);
  NLOS_LAUNCH_CHECK("k_fill");
  return NLOS_OK;
}

static float phi_zero(double a, double b, int kind) {
  (void)b;
  return kind == NLOS_PHI_TRV ? (float)std::sqrt(a) : (float)a;
}

// E_prev = scale * sum(sumsq_src^2) (+ 1/2 ||A u0||^2 + sum phi |grad u0| when
// `au0` is given: the energy of a warm-started Algorithm 2 at (u0, tau = 0)).
static nlos_status init_scalars(Plan& P, SolverState* s, double L0, const float* sumsq_src, size_t n, double scale,
                                cudaStream_t st, const float* au0 = nullptr, const float* u0 = nullptr,
                                const float* ph0 = nullptr) {
  // (au0 == nullptr with u0 given: the sum phi |grad u0| term alone)
  { KTimer kt_(P, KC_SMALL, st);
  k_sumsq<<<stencil_blocks(P), kStencilThreads, 0, st>>>(sumsq_src, n, s->pc);
  }
  NLOS_LAUNCH_CHECK("k_sumsq");
  if (au0) {
    { KTimer kt_(P, KC_SMALL, st);
    k_sumsq<<<stencil_blocks(P), kStencilThreads, 0, st>>>(au0, s->V, s->pa);
    }
    NLOS_LAUNCH_CHECK("k_sumsq");
  }
  if (u0) {
    const Vox g = make_vox(P.nx, P.ny, P.nt);
    const VoxIter vi{ilog2i(P.nt), ilog2i(P.ny)};
    { KTimer kt_(P, KC_SMALL, st);
    k_tv_weighted<<<stencil_blocks(P), kStencilThreads, 0, st>>>(u0, ph0, g, vi, s->V, s->pb);
    }
    NLOS_LAUNCH_CHECK("k_tv_weighted");
  }
  { KTimer kt_(P, KC_SMALL, st);
  k_init_scalars<<<1, kSumThreads, 0, st>>>(s->sc, L0, stencil_blocks(P), s->pc, scale, au0 ? s->pa : nullptr, 0.5,
                                            u0 ? s->pb : nullptr, 1.0);
  }
  NLOS_LAUNCH_CHECK("k_init_scalars");
  return NLOS_OK;
}

// ---------------------------------------------------------------------------
// One reconstruction as a state machine: init, one enqueued iteration per
// step, an asynchronous finish and the collection of the statistics.  A
// single reconstruction runs the steps back to back; the batch and the
// server interleave the steps of many jobs on their own streams.
// ---------------------------------------------------------------------------
// Initial state of the run j.p (u0 = u_init for model 2 when given, else 0).
// u0 = s A_D^T tau0 into u (full field) and s A_D u0 / s into au (compact
// sampled columns) with s = ||g||^2 / ||A_D g||^2, g = A_D^T tau0, computed on
// the device from the compact data tau0c; partials pa / pb of the solver state
// and the plan's scalar scratch are used.
static nlos_status backproject(JobRun& j, const float* tau0c, float* u, float* au) {
  Plan& P = *j.P;
  SolverState* s = j.s;
  cudaStream_t st = j.st;
  const size_t V = s->V, C = (size_t)P.ncols * P.nt;
  NLOS_TRY(apply_adjoint(P, tau0c, u, true, st));
  NLOS_TRY(apply_forward(P, u, au, true, st));
  double* d_s = reinterpret_cast<double*>(P.d_scal);
  { KTimer kt_(P, KC_SMALL, st);
  k_sumsq<<<stencil_blocks(P), kStencilThreads, 0, st>>>(u, V, s->pa);
  k_sumsq<<<stencil_blocks(P), kStencilThreads, 0, st>>>(au, C, s->pb);
  k_ratio<<<1, kSumThreads, 0, st>>>(s->pa, s->pb, stencil_blocks(P), d_s);
  k_scale2<<<elem_grid(V + C), 256, 0, st>>>(u, V, au, C, d_s);
  }
  NLOS_LAUNCH_CHECK("back-projection start");
  return NLOS_OK;
}

static nlos_status init_run(JobRun& j, const float* u_init) {
  Plan& P = *j.P;
  const nlos_params& p = j.p;
  cudaStream_t st = j.st;
  NLOS_TRY(get_solver(P, p.model, &j.s));
  SolverState* s = j.s;
  const size_t V = s->V;
  NLOS_TRY(plan_norm2(P, p.model == 1, st, &j.norm2));
  j.L0 = p.L0 > 0.0 ? p.L0 : 2.0 * j.norm2;
  j.L_host = j.L0;
  j.restart = p.restart < 0 ? (p.model == 2 ? 1 : 0) : p.restart;
  j.it = 0;
  j.cur = 0;
  j.prev = 1;
  j.nxt = 2;
  j.done = p.iters == 0;
  if (p.model == 1) {
    const size_t C = (size_t)P.ncols * P.nt;
    NLOS_TRY(zero(s->lam, 3 * V, st));
    NLOS_TRY(gather_columns(P, j.tau0, s->tau0c, st));
    if (p.init == NLOS_INIT_BACKPROJECT) {
      // u0 = u-bar0 = s A_D^T tau0 with its cached A_D u0 (u^{-1} = u0),
      // phi = phi(kappa(u0)), E_prev = 1/2 ||A_D u0 - tau0||^2 + sum phi |grad u0|
      NLOS_TRY(backproject(j, s->tau0c, s->uk, s->cache[j.cur]));
      NLOS_CUDA(cudaMemcpyAsync(s->ub, s->uk, V * sizeof(float), cudaMemcpyDeviceToDevice, st));
      NLOS_CUDA(cudaMemcpyAsync(s->cache[j.prev], s->cache[j.cur], C * sizeof(float), cudaMemcpyDeviceToDevice,
                                st));
      NLOS_TRY(zero(s->cache[j.nxt], C, st));
      NLOS_TRY(apply_curvature_weight(P, s->uk, s->ph, p.a, p.b, p.phi, p.eps_normal, st));
      { KTimer kt_(P, KC_SMALL, st);
      k_axpby<<<elem_grid(C), 256, 0, st>>>(s->cache[j.cur], 1.f, s->tau0c, -1.f, P.d_tmpc, C);
      }
      NLOS_LAUNCH_CHECK("k_axpby");
      NLOS_TRY(init_scalars(P, s, j.L0, P.d_tmpc, C, 0.5, st, nullptr, s->uk, s->ph));
    } else {
      NLOS_TRY(zero(s->uk, V, st));
      NLOS_TRY(zero(s->ub, V, st));
      for (int i = 0; i < 3; ++i) NLOS_TRY(zero(s->cache[i], C, st));
      NLOS_TRY(fill(s->ph, phi_zero(p.a, p.b, p.phi), V, st));
      NLOS_TRY(init_scalars(P, s, j.L0, s->tau0c, C, 0.5, st));
    }
    // the first iteration's right-hand side term (later ones come from the
    // fused post and pre step)
    if (stencils_tiled(P)) NLOS_TRY(pre1(P, s, p.mu, st));
  } else {
    for (float* f : {s->tk, s->tb, s->lam3}) NLOS_TRY(zero(f, V, st));
    NLOS_TRY(zero(s->lam, 3 * V, st));
    NLOS_TRY(zero(s->lam2, 3 * V, st));
    if (!u_init && p.init == NLOS_INIT_BACKPROJECT) {
      // the back-projection start, from the compact data (into tmp and the
      // plan's compact scratch), then the warm-start path below
      NLOS_TRY(gather_columns(P, j.tau0, P.d_tmpc, st));
      NLOS_TRY(backproject(j, P.d_tmpc, s->tmp, s->cache[j.nxt]));
      u_init = s->tmp;
    }
    if (u_init) {
      // warm start: u0 = u-bar0 = u_init, cached A u0 (u-bar0 = u0, so A u^{-1} = A u0),
      // phi_u = phi(kappa(u0))
      NLOS_CUDA(cudaMemcpyAsync(s->uk, u_init, V * sizeof(float), cudaMemcpyDeviceToDevice, st));
      NLOS_CUDA(cudaMemcpyAsync(s->ub, u_init, V * sizeof(float), cudaMemcpyDeviceToDevice, st));
      NLOS_TRY(apply_forward(P, s->uk, s->cache[j.cur], false, st));
      NLOS_CUDA(cudaMemcpyAsync(s->cache[j.prev], s->cache[j.cur], V * sizeof(float), cudaMemcpyDeviceToDevice,
                                st));
      NLOS_TRY(zero(s->cache[j.nxt], V, st));
      NLOS_TRY(apply_curvature_weight(P, s->uk, s->ph, p.a_u, p.b_u, p.phi, p.eps_normal, st));
    } else {
      NLOS_TRY(zero(s->uk, V, st));
      NLOS_TRY(zero(s->ub, V, st));
      for (int i = 0; i < 3; ++i) NLOS_TRY(zero(s->cache[i], V, st));
      NLOS_TRY(fill(s->ph, phi_zero(p.a_u, p.b_u, p.phi), V, st));
    }
    NLOS_TRY(fill(s->pht, phi_zero(p.a_tau, p.b_tau, p.phi), V, st));
    // E(u0, 0) = lambda/2 ||tau0||^2 over the sampled columns (+ 1/2 ||A u0||^2
    // + sum phi_u |grad u0| for a warm start)
    NLOS_TRY(gather_columns(P, j.tau0, s->tmp, st));
    NLOS_TRY(init_scalars(P, s, j.L0, s->tmp, (size_t)P.ncols * P.nt, 0.5 * p.lambda, st,
                          u_init ? s->cache[j.cur] : nullptr, s->uk, s->ph));
    // the first iteration's u right-hand side term (later ones come from the
    // fused post and pre step of the u half)
    if (stencils_tiled(P)) NLOS_TRY(pre1(P, s, p.mu1, st));
  }
  return NLOS_OK;
}

// Parameters of the Algorithm-1 warm stage of model-2 parameters p.
static nlos_params warm_params(const nlos_params& p) {
  nlos_params w = p;
  w.model = 1;
  w.iters = p.warm_start_iters;
  w.eps_stop = 0.0;
  w.L0 = 0.0;
  w.restart = 0;
  w.warm_start_iters = 0;
  return w;
}

nlos_status job_init(JobRun& j) {
  j.phase = 0;
  if (j.p.model == 2 && j.p.warm_start_iters > 0) {
    j.main_p = j.p;
    j.p = warm_params(j.main_p);
    j.phase = 1;
  }
  return init_run(j, nullptr);
}

bool job_async(const JobRun& j) { return j.p.eps_stop <= 0.0 && j.L0 >= 1.5 * j.norm2; }

static nlos_status step_alg1(JobRun& j) {
  Plan& P = *j.P;
  SolverState* s = j.s;
  const nlos_params& p = j.p;
  cudaStream_t st = j.st;
  const size_t V = s->V;
  const Vox g = make_vox(P.nx, P.ny, P.nt);
  const VoxIter vi{ilog2i(P.nt), ilog2i(P.ny)};
  const float eps2 = (float)(p.eps_normal * p.eps_normal);
  const bool tiled = stencils_tiled(P);
  const int ntiles = tiled ? stencil_steps(g) : 0;  // (tile, x plane) steps
  const int post_grid = std::min(ntiles, P.sms * 2);
  const int post_blocks = tiled ? post_grid : stencil_blocks(P);
  // Untiled grids: the pre stencil (reads u-bar, Lambda, phi; writes reg) and
  // the start of A_D^T (reads the cached A u, tau0 and beta; writes the
  // spectrum scratch) are independent, so in a captured graph the pre
  // stencil is a parallel branch, joined before the u-step reads reg.  Tiled
  // grids have reg from the previous iteration's fused post and pre step.
  const bool fork = !tiled && j.aux;
  if (!tiled) {
    cudaStream_t pst = st;
    if (fork) {
      NLOS_CUDA(cudaEventRecord(j.ev_fork, st));
      NLOS_CUDA(cudaStreamWaitEvent(j.aux, j.ev_fork, 0));
      pst = j.aux;
    }
    NLOS_TRY(pre1(P, s, p.mu, pst));
    if (fork) NLOS_CUDA(cudaEventRecord(j.ev_join, pst));
  }
  Lin3 r{{s->cache[j.cur], s->cache[j.prev], s->tau0c}, {0.f, 0.f, 0.f}, s->sc};
  NLOS_TRY(launch_tfwd_rtt(P, r, P.ncols, P.d_Sc, P.ncols, st));
  NLOS_TRY(launch_conv(P, P.d_Sc, true, P.d_S, false, true, st));
  if (fork) NLOS_CUDA(cudaStreamWaitEvent(st, j.ev_join, 0));
  const bool host_check = j.L_host < 1.5 * j.norm2;
  UStepArgs ua{s->reg, p.mu, true, s->tau0c, p.eta, p.max_backtracks, s->cache[j.nxt], s->cache[j.cur],
               s->cache[j.prev]};
  int nbf_fold = 0;  // test folded into the iteration's end (it cannot reject): fit partial blocks
  NLOS_TRY(u_step(P, s, ua, host_check, &j.L_host, j.bt_stream, st, &nbf_fold));
  const int fold = host_check ? 0 : 1;
  if (tiled) {
    // the fused post and pre step; its last block ends the iteration
    KTimer kt_(P, KC_POST, st);
    auto kern = p.phi == NLOS_PHI_TAC   ? k_post1_pre<NLOS_PHI_TAC>
                : p.phi == NLOS_PHI_TRV ? k_post1_pre<NLOS_PHI_TRV>
                                        : k_post1_pre<NLOS_PHI_TSC>;
    const IterEnd ie{s->sc, 1, s->pb, nbf_fold, fold, j.restart, p.eps_stop};
    kern<<<post_grid, kTileThreads, kPostPreSmem, st>>>(s->unew, s->uk, s->ub, s->lam, s->ph, s->lamn, s->phn, s->ubn,
                                                       s->reg, ie, g, ntiles, (float)p.mu, (float)p.a, (float)p.b,
                                                       eps2, V, s->pc);
    NLOS_LAUNCH_CHECK("k_post1_pre");
  } else {
    { KTimer kt_(P, KC_POST, st);
    k_post1<<<stencil_blocks(P), kStencilThreads, 0, st>>>(s->unew, s->uk, s->ub, s->lam, s->ph, s->ubn, s->sc, g, vi,
                                                        (float)p.mu, (float)p.a, (float)p.b, p.phi, eps2, V, s->pc);
    }
    NLOS_LAUNCH_CHECK("k_post1");
    { KTimer kt_(P, KC_SMALL, st);
    k_finalize<<<1, kSumThreads, 0, st>>>(s->sc, s->pc, post_blocks, 1, 0.0, j.restart, p.eps_stop, s->pb, nbf_fold,
                                          fold);
    }
    NLOS_LAUNCH_CHECK("k_finalize");
  }
  swap_ptr(s->uk, s->unew);
  swap_ptr(s->ub, s->ubn);
  if (tiled) {
    swap_ptr(s->lam, s->lamn);
    swap_ptr(s->ph, s->phn);
  }
  return NLOS_OK;
}

static nlos_status step_alg2(JobRun& j) {
  Plan& P = *j.P;
  SolverState* s = j.s;
  const nlos_params& p = j.p;
  cudaStream_t st = j.st;
  const size_t V = s->V;
  const Vox g = make_vox(P.nx, P.ny, P.nt);
  const VoxIter vi{ilog2i(P.nt), ilog2i(P.ny)};
  const int full = P.nx * P.ny;
  const int32_t* colpos = P.full_mask ? nullptr : P.d_colpos;
  Alg2Coef c{(float)p.mu1, (float)p.mu2, (float)p.mu3, (float)p.lambda, (float)p.a_u, (float)p.b_u,
             (float)p.a_tau, (float)p.b_tau, p.phi, (float)(p.eps_normal * p.eps_normal)};
  const bool tiled = P.nt % kTT == 0 && P.ny % kTY == 0;
  const int ntiles = tiled ? stencil_steps(g) : 0;  // (tile, x plane) steps
  const int pre_grid = std::min(ntiles, P.sms * 3), post_grid = std::min(ntiles, P.sms * 2);
  { KTimer kt_(P, KC_PRE, st);
  if (tiled) {
    // the u half's reg comes from the previous iteration's fused post and pre
    // step (or the run's start)
    const FTerm ft{j.tau0, s->lam3, colpos, (float)p.lambda, (float)p.mu3};
    k_pre1_pipe<true><<<pre_grid, kTileThreads, kPre1PipeSmem, st>>>(s->tb, s->lam2, s->pht, s->regt, g, ntiles,
                                                                     (float)p.mu2, V, ft);
  } else {
    k_pre2<<<stencil_blocks(P), kStencilThreads, 0, st>>>(s->ub, s->tb, s->lam, s->lam2, s->lam3, s->ph, s->pht,
                                                       j.tau0, colpos, s->reg, s->regt, g, vi, c, V);
  }
  }
  NLOS_LAUNCH_CHECK("k_pre2");
  Lin3 r{{s->cache[j.cur], s->cache[j.prev], s->tb}, {0.f, 0.f, 0.f}, s->sc};
  NLOS_TRY(launch_tfwd_rtt(P, r, full, P.d_S, full, st));
  NLOS_TRY(launch_conv(P, P.d_S, false, P.d_S, false, true, st));
  const bool host_check = j.L_host < 1.5 * j.norm2;
  // the fit pass of the u-step also leaves the t-spectrum of the tau-solve
  // rhs, A u+ + regt, in d_Sp
  UStepArgs ua{s->reg, p.mu1, false, s->tb, p.eta, p.max_backtracks, s->cache[j.nxt], s->cache[j.cur],
               s->cache[j.prev], s->regt};
  NLOS_TRY(u_step(P, s, ua, host_check, &j.L_host, j.bt_stream, st));
  NLOS_TRY(launch_sxy(P, P.d_Sp, nullptr, 1.0 + p.mu3, p.mu2, st));
  NLOS_TRY(launch_sinv(P, P.d_Sp, full, s->tnew, nullptr, nullptr, nullptr, st));
  if (tiled) {
    // u and tau halves of the post step; the tau half also does the
    // elementwise Lambda_3 part.  The u-step partial buffer pa is free again
    // at this point.
    { KTimer kt_(P, KC_POST, st);
    auto kern = p.phi == NLOS_PHI_TAC   ? k_post1_pre<NLOS_PHI_TAC>
                : p.phi == NLOS_PHI_TRV ? k_post1_pre<NLOS_PHI_TRV>
                                        : k_post1_pre<NLOS_PHI_TSC>;
    const IterEnd ie{s->sc, 0, nullptr, 0, 0, 0, 0.0};  // k_finalize2 ends the iteration
    kern<<<post_grid, kTileThreads, kPostPreSmem, st>>>(s->unew, s->uk, s->ub, s->lam, s->ph, s->lamn, s->phn, s->ubn,
                                                       s->reg, ie, g, ntiles, (float)p.mu1, (float)p.a_u,
                                                       (float)p.b_u, c.eps2, V, s->pc);
    const L3Term l3{j.tau0, s->cache[j.nxt], s->lam3, colpos, (float)p.lambda, (float)p.mu3};
    post1_pipe_kernel<true>(p.phi)<<<post_grid, kTileThreads, kPost1PipeSmem, st>>>(
        s->tnew, s->tk, s->tb, s->lam2, s->pht, s->tbn, s->sc, g, ntiles, (float)p.mu2, (float)p.a_tau,
        (float)p.b_tau, c.eps2, V, s->pa, l3);
    }
    NLOS_LAUNCH_CHECK("k_post2");
    { KTimer kt_(P, KC_SMALL, st);
    k_finalize2<<<1, kSumThreads, 0, st>>>(s->sc, s->pc, post_grid, s->pa, post_grid, s->pa, post_grid, 2,
                                           p.lambda, j.restart, p.eps_stop);
    }
    NLOS_LAUNCH_CHECK("k_finalize2");
  } else {
    { KTimer kt_(P, KC_POST, st);
    k_post2<<<stencil_blocks(P), kStencilThreads, 0, st>>>(s->unew, s->uk, s->ub, s->tnew, s->tk, s->tb, s->lam,
                                                        s->lam2, s->lam3, s->ph, s->pht, s->ubn, s->tbn,
                                                        s->cache[j.nxt], j.tau0, colpos, s->sc, g, vi, c, V, s->pc);
    }
    NLOS_LAUNCH_CHECK("k_post2");
    { KTimer kt_(P, KC_SMALL, st);
    k_finalize<<<1, kSumThreads, 0, st>>>(s->sc, s->pc, stencil_blocks(P), 2, p.lambda, j.restart, p.eps_stop,
                                          nullptr, 0, 0);
    }
    NLOS_LAUNCH_CHECK("k_finalize");
  }
  swap_ptr(s->uk, s->unew);
  swap_ptr(s->ub, s->ubn);
  swap_ptr(s->tk, s->tnew);
  swap_ptr(s->tb, s->tbn);
  if (tiled) {
    swap_ptr(s->lam, s->lamn);
    swap_ptr(s->ph, s->phn);
  }
  return NLOS_OK;
}

// Enqueues one iteration and rotates the cached A u slots.
static nlos_status step_once(JobRun& j) {
  NLOS_TRY(j.p.model == 1 ? step_alg1(j) : step_alg2(j));
  const int t = j.prev;
  j.prev = j.cur;
  j.cur = j.nxt;
  j.nxt = t;
  return NLOS_OK;
}

nlos_status job_step(JobRun& j) {
  if (j.done) return NLOS_OK;
  NLOS_TRY(step_once(j));
  j.it += 1;
  if (j.it >= j.p.iters) j.done = true;
  if (j.p.eps_stop > 0.0 && !j.done) {
    NLOS_TRY(read_scalars(j.s, j.st));
    if (j.s->h_sc->stop || j.s->h_sc->status != NLOS_OK) j.done = true;
  }
  if (j.done && j.phase == 1) {
    // warm stage finished: Algorithm 2 from the Algorithm-1 result
    const float* u_warm = j.s->uk;
    j.p = j.main_p;
    j.phase = 2;
    NLOS_TRY(init_run(j, u_warm));
  }
  return NLOS_OK;
}

nlos_status job_finish(JobRun& j) {
  SolverState* s = j.s;
  const size_t F = s->V * sizeof(float);
  NLOS_CUDA(cudaMemcpyAsync(j.u_out, s->uk, F, cudaMemcpyDeviceToDevice, j.st));
  if (j.tau_out && s->model == 2) NLOS_CUDA(cudaMemcpyAsync(j.tau_out, s->tk, F, cudaMemcpyDeviceToDevice, j.st));
  NLOS_CUDA(cudaMemcpyAsync(s->h_sc, s->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, j.st));
  return NLOS_OK;
}

nlos_status job_collect(JobRun& j, nlos_stats* stats) {
  fill_stats(*j.s->h_sc, stats);
  if (j.s->h_sc->status != NLOS_OK)
    return fail(j.s->h_sc->status,
                "reconstruction stopped: non-finite energy, backtracking gave up, or a t-pass tile wait timed out");
  return NLOS_OK;
}

void free_graphs(Plan* P) {
  for (auto& g : P->graphs) cudaGraphExecDestroy(g.exec);
  P->graphs.clear();
  if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
  P->capture_stream = nullptr;
  for (auto& b : P->body_stream) {
    if (b) cudaStreamDestroy(b);
    b = nullptr;
  }
  if (P->aux_stream) cudaStreamDestroy(P->aux_stream);
  P->aux_stream = nullptr;
  for (auto& e : P->aux_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
}

// Captures (on c.st, which is capturing) a run whose iteration count is
// decided on the device: after the initial state (and the unrolled warm
// stage of a warm-started model-2 run), a while node runs one iteration per
// trip, chosen by a switch over the six pointer phases; k_loop_end stops it at
// `iters` trips, at the relative-energy stop or on an error.  A backtracking
// rule that can reject runs as a nested while node (u_step).  The result is
// copied from the buffer that the trip count's parity selects.
static nlos_status capture_looped(JobRun& c, cudaStream_t* bs) {
  NLOS_TRY(job_init(c));
  while (c.phase == 1) NLOS_TRY(job_step(c));  // warm stage: fixed count, no host decisions
  SolverState* s = c.s;
  if (c.p.iters <= 0) return job_finish(c);
  const float* u0 = s->uk;
  const float* u1 = s->unew;
  const float* t0 = s->tk;
  const float* t1 = s->tnew;
  const JobRun start = c;
  auto phase_ptrs = [s]() {
    return std::array<const float*, 13>{s->uk, s->unew, s->ub, s->ubn, s->tk, s->tnew, s->tb, s->tbn,
                                        s->cache[0], s->cache[1], s->cache[2], s->lam, s->ph};
  };
  const auto ptrs_start = phase_ptrs();
  cudaGraphConditionalHandle cont = 0;
  NLOS_TRY(cond_handle(c.st, 1, cudaGraphCondAssignDefault, &cont));
  cudaGraph_t loop_body = nullptr;
  NLOS_TRY(add_cond_node(c.st, cont, cudaGraphCondTypeWhile, 1, &loop_body));
  const cudaStream_t main_st = c.st;
  NLOS_TRY(capture_body(bs[0], loop_body, [&](cudaStream_t ls) -> nlos_status {
    cudaGraphConditionalHandle phase = 0;
    NLOS_TRY(cond_handle(ls, 0, 0, &phase));
    k_loop_begin<<<1, 1, 0, ls>>>(s->sc, phase);
    NLOS_LAUNCH_CHECK("k_loop_begin");
    cudaGraph_t bodies[6] = {};
    NLOS_TRY(add_cond_node(ls, phase, cudaGraphCondTypeSwitch, 6, bodies));
    for (int k = 0; k < 6; ++k) {
      NLOS_TRY(capture_body(bs[1], bodies[k], [&](cudaStream_t ps) -> nlos_status {
        c.st = ps;
        c.bt_stream = bs[2];
        const nlos_status r = step_once(c);
        c.st = main_st;
        c.bt_stream = nullptr;
        return r;
      }));
    }
    k_loop_end<<<1, 1, 0, ls>>>(s->sc, cont, c.p.iters);
    NLOS_LAUNCH_CHECK("k_loop_end");
    return NLOS_OK;
  }));
  // six iterations bring every rotated pointer back to its starting place
  if (c.cur != start.cur || c.prev != start.prev || c.nxt != start.nxt || phase_ptrs() != ptrs_start)
    return fail(NLOS_ERR_CUDA, "iteration pointer phases do not repeat after six iterations");
  const size_t V = s->V;
  k_select_copy<<<elem_grid(V), 256, 0, c.st>>>(c.u_out, u0, u1, V, s->sc);
  NLOS_LAUNCH_CHECK("k_select_copy");
  if (c.tau_out && s->model == 2) {
    k_select_copy<<<elem_grid(V), 256, 0, c.st>>>(c.tau_out, t0, t1, V, s->sc);
    NLOS_LAUNCH_CHECK("k_select_copy");
  }
  NLOS_CUDA(cudaMemcpyAsync(s->h_sc, s->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.st));
  return NLOS_OK;
}

// The cached graph of run j (same parameters and buffers), captured and
// cached on first use; *exec = nullptr when the plan's kernels are being
// timed or the run has no iterations.
static nlos_status job_graph(JobRun& j, cudaStream_t st, cudaGraphExec_t* exec) {
  *exec = nullptr;
  Plan& P = *j.P;
  const nlos_params& p = j.p;
  if (P.timing) return NLOS_OK;  // timed kernels: stepped
  // everything that may synchronise or allocate happens before the capture
  NLOS_TRY(get_solver(P, p.model, &j.s));
  NLOS_TRY(plan_norm2(P, p.model == 1, st, &j.norm2));
  if (p.model == 2 && p.warm_start_iters > 0) {
    SolverState* s1 = nullptr;
    double n1 = 0.0;
    NLOS_TRY(get_solver(P, 1, &s1));
    NLOS_TRY(plan_norm2(P, true, st, &n1));
  }
  const double L0 = p.L0 > 0.0 ? p.L0 : 2.0 * j.norm2;
  if (p.iters <= 0) return NLOS_OK;
  const bool looped = p.eps_stop > 0.0 || L0 < 1.5 * j.norm2;
  for (auto& g : P.graphs)
    if (std::memcmp(&g.p, &p, sizeof(nlos_params)) == 0 && g.tau0 == j.tau0 && g.u_out == j.u_out &&
        g.tau_out == j.tau_out) {
      *exec = g.exec;
      return NLOS_OK;
    }
  if (!P.capture_stream) NLOS_CUDA(cudaStreamCreateWithFlags(&P.capture_stream, cudaStreamNonBlocking));
  if (looped)
    for (auto& b : P.body_stream)
      if (!b) NLOS_CUDA(cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking));
  if (!P.aux_stream) NLOS_CUDA(cudaStreamCreateWithFlags(&P.aux_stream, cudaStreamNonBlocking));
  for (auto& e : P.aux_ev)
    if (!e) NLOS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  JobRun c = j;
  c.st = P.capture_stream;
  c.aux = P.aux_stream;
  c.ev_fork = P.aux_ev[0];
  c.ev_join = P.aux_ev[1];
  NLOS_CUDA(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
  nlos_status s = NLOS_OK;
  if (looped) {
    s = capture_looped(c, P.body_stream);
  } else {
    s = job_init(c);
    while (s == NLOS_OK && !c.done) s = job_step(c);
    if (s == NLOS_OK) s = job_finish(c);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c.st, &graph);
  if (s != NLOS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  if (P.graphs.size() >= 4) {
    cudaGraphExecDestroy(P.graphs.front().exec);
    P.graphs.erase(P.graphs.begin());
  }
  P.graphs.push_back(Plan::GraphEntry{p, j.tau0, j.u_out, j.tau_out, ge});
  j.s = c.s;
  *exec = ge;
  return NLOS_OK;
}

nlos_status job_enqueue_graph(JobRun& j, cudaStream_t launch, bool* used) {
  *used = false;
  cudaGraphExec_t exec = nullptr;
  NLOS_TRY(job_graph(j, launch, &exec));
  if (!exec) return NLOS_OK;
  NLOS_CUDA(cudaGraphLaunch(exec, launch));
  *used = true;
  return NLOS_OK;
}

nlos_status job_prepare_graph(JobRun& j, cudaStream_t st, bool* ready) {
  cudaGraphExec_t exec = nullptr;
  NLOS_TRY(job_graph(j, st, &exec));
  *ready = exec != nullptr;
  return NLOS_OK;
}

nlos_status reconstruct_prepare(Plan& P, const nlos_params& p, const float* tau0, float* u_out, float* tau_out,
                                bool* ready, cudaStream_t st) {
  if (p.model != 1 && p.model != 2) return fail(NLOS_ERR_INVALID_ARG, "params->model must be 1 or 2");
  JobRun j;
  j.P = &P;
  j.p = p;
  j.tau0 = tau0;
  j.u_out = u_out;
  j.tau_out = tau_out;
  j.st = st;
  return job_prepare_graph(j, st, ready);
}

nlos_status reconstruct(Plan& P, const nlos_params& p, const float* tau0, float* u_out, float* tau_out,
                        nlos_stats* stats, cudaStream_t st) {
  if (p.model != 1 && p.model != 2) return fail(NLOS_ERR_INVALID_ARG, "params->model must be 1 or 2");
  JobRun j;
  j.P = &P;
  j.p = p;
  j.tau0 = tau0;
  j.u_out = u_out;
  j.tau_out = tau_out;
  j.st = st;
  bool graphed = false;
  NLOS_TRY(job_enqueue_graph(j, st, &graphed));
  if (!graphed) {
    NLOS_TRY(job_init(j));
    while (!j.done) NLOS_TRY(job_step(j));
    NLOS_TRY(job_finish(j));
  }
  NLOS_CUDA(cudaStreamSynchronize(st));
  return job_collect(j, stats);
}

}  // namespace nlos

namespace nlos {

nlos_status reconstruct_host(Plan& P, const nlos_params& p, const float* tau0_host, float* u_out_host,
                             float* tau_out_host, nlos_stats* stats, cudaStream_t st) {
  if (p.model != 1 && p.model != 2) return fail(NLOS_ERR_INVALID_ARG, "params->model must be 1 or 2");
  const size_t F = (size_t)P.nx * P.ny * P.nt * sizeof(float);
  for (int i = 0; i < 3; ++i)
    if (!P.d_io[i]) {
      if (cudaMalloc(&P.d_io[i], F) != cudaSuccess) {
        cudaGetLastError();
        P.d_io[i] = nullptr;
        return fail(NLOS_ERR_OOM, "nlos_reconstruct_host: device buffers");
      }
    }
  JobRun j;
  j.P = &P;
  j.p = p;
  j.tau0 = P.d_io[0];
  j.u_out = P.d_io[1];
  j.tau_out = P.d_io[2];
  j.st = st;
  NLOS_CUDA(cudaMemcpyAsync(P.d_io[0], tau0_host, F, cudaMemcpyHostToDevice, st));
  bool graphed = false;
  NLOS_TRY(job_enqueue_graph(j, st, &graphed));
  if (!graphed) {
    NLOS_TRY(job_init(j));
    while (!j.done) NLOS_TRY(job_step(j));
    NLOS_TRY(job_finish(j));
  }
  NLOS_CUDA(cudaMemcpyAsync(u_out_host, P.d_io[1], F, cudaMemcpyDeviceToHost, st));
  if (tau_out_host && p.model == 2)
    NLOS_CUDA(cudaMemcpyAsync(tau_out_host, P.d_io[2], F, cudaMemcpyDeviceToHost, st));
  NLOS_CUDA(cudaStreamSynchronize(st));
  return job_collect(j, stats);
}

}  // namespace nlos
