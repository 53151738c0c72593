// The end of an ADMM iteration on the device scalar block (Algorithms 1-2):
// energy, relative change, the FISTA restart, bookkeeping and the next
// extrapolation step, from block partial sums.  Used by the single-block
// finalize kernels and by the last block of the fused Algorithm-1 post and
// pre step.
#pragma once

#include "common.cuh"

namespace nlos {

// The FISTA step (t_next, beta_next) that the next accepted test takes from
// t: ((1 + sqrt(1 + 4 t^2)) / 2, (t - 1) / t_next).
__device__ __forceinline__ double2 next_step_of(double t) {
  const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
  return make_double2(tn, (t - 1.0) / tn);
}
__device__ __forceinline__ void set_next_step(DevScalars* sc) {
  const double2 s = next_step_of(sc->t);
  sc->t_next = s.x;
  sc->beta_next = s.y;
}

// Energy E and squared primal residual pres2 of the finished iteration into
// the scalar block: divergence check, restart (t = 1 when E grew),
// bookkeeping, relative-energy stop, next step.  pre (nullable): the next step
// already computed from the t this iteration ends with when no restart
// happens.  One thread.
__device__ __forceinline__ void finalize_tail(DevScalars* sc, double E, double pres2, int restart, double eps_stop,
                                              const double2* pre = nullptr) {
  const double dE = sc->E_prev - E;
  if (!isfinite(E)) sc->status = NLOS_ERR_DIVERGED;
  bool restarted = false;
  if (restart && E > sc->E_prev) {
    sc->t = 1.0;
    sc->restarts += 1;
    restarted = true;
  }
  sc->beta_prev = sc->beta;
  sc->E = E;
  sc->dE = dE;
  sc->E_prev = E;
  sc->pres2 = pres2;
  sc->iter += 1;
  if (eps_stop > 0.0) {
    const double e = E != 0.0 ? fabs(dE) / fabs(E) : 0.0;
    if (e <= eps_stop) sc->stop = 1;
  }
  if (pre && !restarted) {
    sc->t_next = pre->x;
    sc->beta_next = pre->y;
  } else {
    set_next_step(sc);
  }
}

// Algorithm 1: pg = sum phi |grad u+|, pres2 = sum |v - grad u+|^2 from the
// post step; with fold_test, f0 = sum (A u+ - tau0)^2 and f1 = ||A d||^2 from
// the fit pass of a test that cannot reject, whose accepting bookkeeping is
// done here.  One thread.
__device__ __forceinline__ void finalize1(DevScalars* sc, double pg, double pres2, double f0, double f1,
                                          int fold_test, int restart, double eps_stop,
                                          const double2* pre = nullptr) {
  if (sc->status != NLOS_OK) return;
  if (fold_test) {
    sc->test_lhs = f1;
    sc->test_rhs = sc->L * 0.0;
    sc->accept = 1;
    sc->f_fit = 0.5 * f0;
    sc->beta = sc->beta_next;
    sc->t = sc->t_next;
    sc->rej_iter = 0;
  }
  finalize_tail(sc, sc->f_fit + pg, pres2, restart, eps_stop, pre);
}

// Terms 0 and 1 of the partials of na blocks at pa (into out[0], out[1]) and
// of nb blocks at pb (into out[2], out[3]; pb may be null), summed in a fixed
// order: per thread over the blocks tid, tid + blockDim, ..., then across the
// warp by shuffles, then over the warps as a binary tree; valid in thread 0.
// Every load is issued before the first add (one L2 round trip), and the four
// sums advance together (FP64 latency is long on this GPU).  Every thread of
// the block calls it.  The partials are read through L2 (other blocks of the
// running kernel may have written them).
__device__ __forceinline__ void block_sum_2x2(const double* pa, int na, const double* pb, int nb, double (&out)[4]) {
  __shared__ double wsum[4][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int kPer = 2;  // blocks per thread held in flight (more are summed in further rounds)
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int nmax = na > nb ? na : nb;
  for (int b0 = threadIdx.x; b0 < nmax; b0 += kPer * blockDim.x) {
    double v[kPer][4];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int b = b0 + k * blockDim.x;
      const bool ia = b < na, ib = pb != nullptr && b < nb;
      v[k][0] = ia ? __ldcg(pa + (size_t)b * kMaxTerms) : 0.0;
      v[k][1] = ia ? __ldcg(pa + (size_t)b * kMaxTerms + 1) : 0.0;
      v[k][2] = ib ? __ldcg(pb + (size_t)b * kMaxTerms) : 0.0;
      v[k][3] = ib ? __ldcg(pb + (size_t)b * kMaxTerms + 1) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] += v[k][t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < 4; ++t) wsum[t][warp] = acc[t];
  __syncthreads();
  if (warp == 0) {
    // the warp sums as a binary tree over lanes < nw (nw a power of two <= 32)
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t] = lane < nw ? wsum[t][lane] : 0.0;
    for (int o = nw >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] += __shfl_down_sync(0xffffffffu, acc[t], o);
    if (lane == 0)
#pragma unroll
      for (int t = 0; t < 4; ++t) out[t] = acc[t];
  }
  __syncthreads();
}

// What the last block of the fused post and pre step needs to end the
// iteration (Algorithm 1; Algorithm 2's u half leaves that to k_finalize2,
// which also needs the tau half's sums).
struct IterEnd {
  DevScalars* sc;
  int end_here;      // 1: the last block ends the iteration
  const double* pf;  // fit partials of a folded test
  int nbf;           // their block count
  int fold;          // 1: the test cannot reject and is folded in here
  int restart;
  double eps_stop;
};

// Called by every thread of every block after the block has written its
// partials (thread 0 wrote them last): the block that arrives last sums all
// blocks' partials and ends the iteration.  No block waits for another: each
// takes a ticket after a fence, and only the holder of the last ticket reads
// the others' partials.  The arrival counter is zero at the start of a run
// and is reset by the last block.
__device__ __forceinline__ void end_iteration_if_last(const IterEnd& ie, const double* partials) {
  if (!ie.end_here) return;
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ie.sc->arrivals, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the next step from the t this iteration ends with (t_next when the test
  // is folded in, else the t the test set), computed by another warp while
  // the sums run; used unless a restart resets t
  __shared__ double2 s_pre;
  if (threadIdx.x == 32) s_pre = next_step_of(ie.fold ? ie.sc->t_next : ie.sc->t);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  block_sum_2x2(partials, gridDim.x, ie.fold ? ie.pf : nullptr, ie.nbf, v);  // ends with a barrier
  if (threadIdx.x == 0) {
    ie.sc->arrivals = 0;
    const double2 pre = s_pre;
    finalize1(ie.sc, v[0], v[1], v[2], v[3], ie.fold, ie.restart, ie.eps_stop, &pre);
  }
}

}  // namespace nlos
