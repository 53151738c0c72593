// Hand-written FFT building blocks for sm_103a.
//
// Two levels:
//  * dft_reg<R, INV>: a length-R DFT (R = 1..64, power of two) held entirely
//    in registers, radix-2 decimation in frequency with compile-time twiddles
//    (every index is a constant after unrolling, so the twiddles fold into
//    the multiply instructions as immediates).
//  * team_fft<R1, R2, INV>: B independent length-N transforms (N = R1 R2) in
//    shared memory, by the two-step Cooley-Tukey split: R2 threads per
//    transform run length-R1 register DFTs on stride-R2 subsequences,
//    multiply by the inter-step twiddles exp(-2 pi i n2 k1 / N), and R1 threads
//    per transform finish with length-R2 register DFTs on contiguous runs.
//    Forward: natural order in, "digit-transposed" order out (position
//    p = R2 k1 + k2 holds frequency k1 + R1 k2).  Inverse: that order in,
//    natural order out, unnormalised.  The convolution and solve kernels only
//    ever multiply pointwise in the frequency domain, so no permutation pass
//    is needed; they map positions to frequencies with kfreq().
//    Thread-to-work mapping puts consecutive lanes on consecutive transforms,
//    so with an odd transform pitch (or unit transform stride) the shared
//    memory accesses of a warp fall in distinct banks.
#pragma once

#include "common.cuh"

namespace nlos {

// cos(2 pi k / 64), k = 0..16 (quarter wave), from FP64, rounded to float.
__host__ __device__ __forceinline__ constexpr float cos64_q(int k) {
  return k == 0    ? 1.0f
         : k == 1  ? 9.951847267e-01f
         : k == 2  ? 9.807852804e-01f
         : k == 3  ? 9.569403357e-01f
         : k == 4  ? 9.238795325e-01f
         : k == 5  ? 8.819212643e-01f
         : k == 6  ? 8.314696123e-01f
         : k == 7  ? 7.730104534e-01f
         : k == 8  ? 7.071067812e-01f
         : k == 9  ? 6.343932842e-01f
         : k == 10 ? 5.555702330e-01f
         : k == 11 ? 4.713967368e-01f
         : k == 12 ? 3.826834324e-01f
         : k == 13 ? 2.902846773e-01f
         : k == 14 ? 1.950903220e-01f
         : k == 15 ? 9.801714033e-02f
                   : 0.0f;
}

// exp(-2 pi i k / 64) (forward) or its conjugate (inverse), k in [0, 64).
template <bool INV>
__host__ __device__ __forceinline__ constexpr float2 root64(int k) {
  // theta = 2 pi k / 64; c = cos theta, s = sin theta by quarter-wave symmetry
  float c = k <= 16 ? cos64_q(k) : k <= 32 ? -cos64_q(32 - k) : k <= 48 ? -cos64_q(k - 32) : cos64_q(64 - k);
  float s = k <= 16 ? cos64_q(16 - k) : k <= 32 ? cos64_q(k - 16) : k <= 48 ? -cos64_q(48 - k) : -cos64_q(k - 48);
  return INV ? make_float2(c, s) : make_float2(c, -s);
}

// d * exp(-+2 pi i k / 64) with the trivial rotations special-cased.
template <bool INV>
__device__ __forceinline__ float2 twmul64(float2 d, int k) {
  if (k == 0) return d;
  if (k == 16) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
  if (k == 32) return make_float2(-d.x, -d.y);
  if (k == 48) return INV ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
  const float2 w = root64<INV>(k);
  return make_float2(d.x * w.x - d.y * w.y, d.x * w.y + d.y * w.x);
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

template <int R>
__host__ __device__ __forceinline__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 0; b < ilog2c(R); ++b) r |= ((i >> b) & 1) << (ilog2c(R) - 1 - b);
  return r;
}

// In-register length-R DFT, natural order in and out.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&a)[R]) {
  static_assert(R >= 1 && R <= 64 && (R & (R - 1)) == 0, "R must be a power of two <= 64");
  if (R == 1) return;
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 x0 = a[blk + j];
        const float2 x1 = a[blk + j + span];
        a[blk + j] = cadd(x0, x1);
        a[blk + j + span] = twmul64<INV>(csub(x0, x1), j * (64 / (2 * span)));
      }
    }
  }
  float2 t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = a[bitrev<R>(i)];
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = t[i];
}

// Factorisation N = R1 * R2 (* R3) used for each transform length.  Lengths
// up to 128 use two steps (the lateral passes rely on that); longer ones use
// three balanced steps so every step keeps all threads busy with small
// register DFTs.
template <int N> struct FftPlan;
template <> struct FftPlan<8>    { static constexpr int R1 = 4,  R2 = 2, R3 = 1; };
template <> struct FftPlan<16>   { static constexpr int R1 = 4,  R2 = 4, R3 = 1; };
template <> struct FftPlan<32>   { static constexpr int R1 = 8,  R2 = 4, R3 = 1; };
template <> struct FftPlan<64>   { static constexpr int R1 = 8,  R2 = 8, R3 = 1; };
template <> struct FftPlan<128>  { static constexpr int R1 = 16, R2 = 8, R3 = 1; };
template <> struct FftPlan<256>  { static constexpr int R1 = 8,  R2 = 8, R3 = 4; };
template <> struct FftPlan<512>  { static constexpr int R1 = 8,  R2 = 8, R3 = 8; };
template <> struct FftPlan<1024> { static constexpr int R1 = 16, R2 = 8, R3 = 8; };

// Position in the forward output of natural frequency k, and the inverse map:
// position k1 R2 R3 + k2 R3 + k3 holds frequency k1 + R1 (k2 + R2 k3).
template <int N>
__device__ __forceinline__ int fpos(int k) {
  constexpr int R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2, R3 = FftPlan<N>::R3;
  const int k1 = k % R1, kk = k / R1;
  return k1 * (R2 * R3) + (kk % R2) * R3 + kk / R2;
}
template <int N>
__device__ __forceinline__ int kfreq(int p) {
  constexpr int R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2, R3 = FftPlan<N>::R3;
  const int k1 = p / (R2 * R3), rem = p % (R2 * R3);
  return k1 + R1 * (rem / R3 + R2 * (rem % R3));
}

// B transforms of length N (B a power of two) in shared memory; element e of
// transform b lives at buf[addr(b, e)] (addr: any bijective layout, e.g. a
// strided plane or a bank-swizzled one).  The steps call addr(b, er, ec) for
// e = er + ec where er (the same for all of a task's elements) and ec (a
// compile-time constant after unrolling) have disjoint bits, so a layout can
// compute the part of er once per task.  tw[j * tws] = exp(-2 pi i j / N)
// for j < N (tw: a pointer, or any table type with operator[]).  All
// threads of the block call these; they end with __syncthreads().
//
// Three-step version (R3 > 1): N = R1 M, M = R2 R3.
//   step 1 (b, n23): R1-point DFT over n1 of x[n1 M + n23], twiddle w_N^(n23 k1);
//   step 2 (b, k1, n3): R2-point DFT over n2 of y[k1 M + n2 R3 + n3],
//          twiddle w_M^(n3 k2) = w_N^(R1 n3 k2);
//   step 3 (b, k1, k2): R3-point DFT over the contiguous n3.
// The inverse runs the steps backwards with conjugate twiddles.
template <int N, bool INV, typename Addr, typename TwT>
__device__ __forceinline__ void team_fft3a(float2* buf, int B, const Addr& addr, const TwT& tw, int tws, int tid,
                                           int nthr) {
  constexpr int R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2, R3 = FftPlan<N>::R3, M = R2 * R3;
  const int lb = __ffs(B) - 1;
  auto step1 = [&]() {
    for (int it = tid; it < B * M; it += nthr) {
      const int b = it & (B - 1), n23 = it >> lb;
      float2 a[R1];
#pragma unroll
      for (int n = 0; n < R1; ++n) a[n] = buf[addr(b, n23, n * M)];
      if (!INV) {
        dft_reg<R1, false>(a);
#pragma unroll
        for (int k = 1; k < R1; ++k) a[k] = cmul(a[k], tw[((n23 * k) & (N - 1)) * tws]);
      } else {
#pragma unroll
        for (int k = 1; k < R1; ++k) a[k] = cmulc(a[k], tw[((n23 * k) & (N - 1)) * tws]);
        dft_reg<R1, true>(a);
      }
#pragma unroll
      for (int n = 0; n < R1; ++n) buf[addr(b, n23, n * M)] = a[n];
    }
    __syncthreads();
  };
  auto step2 = [&]() {
    for (int it = tid; it < B * R1 * R3; it += nthr) {
      const int b = it & (B - 1), r = it >> lb;
      const int n3 = r % R3, k1 = r / R3;
      const int e0 = k1 * M + n3;
      float2 a[R2];
#pragma unroll
      for (int n = 0; n < R2; ++n) a[n] = buf[addr(b, e0, n * R3)];
      if (!INV) {
        dft_reg<R2, false>(a);
#pragma unroll
        for (int k = 1; k < R2; ++k) a[k] = cmul(a[k], tw[((R1 * n3 * k) & (N - 1)) * tws]);
      } else {
#pragma unroll
        for (int k = 1; k < R2; ++k) a[k] = cmulc(a[k], tw[((R1 * n3 * k) & (N - 1)) * tws]);
        dft_reg<R2, true>(a);
      }
#pragma unroll
      for (int n = 0; n < R2; ++n) buf[addr(b, e0, n * R3)] = a[n];
    }
    __syncthreads();
  };
  auto step3 = [&]() {
    for (int it = tid; it < B * R1 * R2; it += nthr) {
      const int b = it & (B - 1), r = it >> lb;
      const int e0 = r * R3;
      float2 a[R3];
#pragma unroll
      for (int n = 0; n < R3; ++n) a[n] = buf[addr(b, e0, n)];
      dft_reg<R3, INV>(a);
#pragma unroll
      for (int n = 0; n < R3; ++n) buf[addr(b, e0, n)] = a[n];
    }
    __syncthreads();
  };
  if (!INV) {
    step1();
    step2();
    step3();
  } else {
    step3();
    step2();
    step1();
  }
}

// Two-step version (R3 = 1; dispatches to the three-step one otherwise).
template <int N, bool INV, typename Addr, typename TwT>
__device__ __forceinline__ void team_fft_a(float2* buf, int B, const Addr& addr, const TwT& tw, int tws, int tid,
                                           int nthr) {
  constexpr int R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2;
  if constexpr (FftPlan<N>::R3 > 1) {
    team_fft3a<N, INV>(buf, B, addr, tw, tws, tid, nthr);
    return;
  }
  const int lb = __ffs(B) - 1;
  if (!INV) {
    for (int it = tid; it < B * R2; it += nthr) {
      const int b = it & (B - 1), n2 = it >> lb;
      float2 a[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) a[n1] = buf[addr(b, n2, n1 * R2)];
      dft_reg<R1, false>(a);
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmul(a[k1], tw[((n2 * k1) & (N - 1)) * tws]);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) buf[addr(b, n2, k1 * R2)] = a[k1];
    }
    __syncthreads();
    if (R2 > 1) {
      for (int it = tid; it < B * R1; it += nthr) {
        const int b = it & (B - 1), k1 = it >> lb;
        float2 a[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) a[n2] = buf[addr(b, k1 * R2, n2)];
        dft_reg<R2, false>(a);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) buf[addr(b, k1 * R2, k2)] = a[k2];
      }
      __syncthreads();
    }
  } else {
    if (R2 > 1) {
      for (int it = tid; it < B * R1; it += nthr) {
        const int b = it & (B - 1), k1 = it >> lb;
        float2 a[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) a[k2] = buf[addr(b, k1 * R2, k2)];
        dft_reg<R2, true>(a);
#pragma unroll
        for (int n2 = 1; n2 < R2; ++n2) a[n2] = cmulc(a[n2], tw[((n2 * k1) & (N - 1)) * tws]);
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) buf[addr(b, k1 * R2, n2)] = a[n2];
      }
      __syncthreads();
    }
    for (int it = tid; it < B * R2; it += nthr) {
      const int b = it & (B - 1), n2 = it >> lb;
      float2 a[R1];
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) a[k1] = buf[addr(b, n2, k1 * R2)];
      dft_reg<R1, true>(a);
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) buf[addr(b, n2, n1 * R2)] = a[n1];
    }
    __syncthreads();
  }
}

// Strided layout: element e of transform b at buf[b * ts + e * es].
struct StridedAddr {
  int ts, es;
  __device__ __forceinline__ int operator()(int b, int e) const { return b * ts + e * es; }
  __device__ __forceinline__ int operator()(int b, int er, int ec) const { return b * ts + (er + ec) * es; }
};
template <int N, bool INV>
__device__ __forceinline__ void team_fft(float2* buf, int B, int ts, int es, const float2* tw, int tws, int tid,
                                         int nthr) {
  team_fft_a<N, INV>(buf, B, StridedAddr{ts, es}, tw, tws, tid, nthr);
}

// Global -> shared staging with U independent loads in flight per thread:
// item i is produced by ld(i) and consumed by st(i, value).  A plain
// "load, store, next" loop keeps one load per thread in flight and is bound
// by memory latency, not bandwidth.
template <int U, typename T, typename LoadF, typename StoreF>
__device__ __forceinline__ void batched_copy(int total, int tid, int nthr, LoadF ld, StoreF st) {
  for (int base = tid; base < total; base += U * nthr) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * nthr;
      if (i < total) v[u] = ld(i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * nthr;
      if (i < total) st(i, v[u]);
    }
  }
}

}  // namespace nlos
