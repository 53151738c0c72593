// Register-resident complex FFTs run by a group of L lanes of one warp (L =
// 32: a whole warp, L = 16: each half of a warp on its own sequence).
//
// A length-N transform (N = L V) is held V values per lane, natural order in
// (lane l of the group, register m: element l + L m), and factored as N = V x
// L: a V-point register DFT over the stride-L elements of each lane, the
// twiddles w_N^(l k1), an exchange through the group's shared scratch that
// gives each run of G = L / V lanes one of the V length-L sequences, a V-point
// register DFT over the stride-G elements, the twiddles w_L^(g a), and a
// G-point DFT across the G lanes by shuffles (radix 2, decimation in
// frequency).  Lane k1 G + g, register a then holds frequency
// k1 + V a + V^2 rev_G(g) (rev_G: bit reversal of log2 G bits); the inverse
// runs the same steps backwards with conjugate twiddles, from that order back
// to natural order (unnormalised).
//
// Tables (shared or global memory): tw1[k1 L + l] = w_N^(l k1) for k1 < V,
// l < L (the second step reads it only when G > 2; for G = 2 its twiddles
// are compile-time roots); twc[n] = w_2N^n for n < N (only read when G > 2).  Scratch: V (L + G)
// float2 per group; the pitch L + G puts the strided reads of the exchange
// in distinct banks.
#pragma once

#include "fft.cuh"

namespace nlos {

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

template <int G>
__device__ __forceinline__ int rev_bits(int g) {
  int r = 0;
#pragma unroll
  for (int b = 1; b < G; b <<= 1) r = (r << 1) | ((g & b) ? 1 : 0);
  return r;
}

// The second-step twiddle w_N^(V g q) = w_L^(g q) when G = 2: 1 on the lanes
// g = 0, the compile-time root w_L^q on the lanes g = 1 (q a constant after
// unrolling), so no table read.
template <int L, bool INV>
__device__ __forceinline__ float2 twiddle_g2(float2 v, int q, int g) {
  const float2 r = twmul64<INV>(v, (64 / L) * q);
  return g ? r : v;
}

// G-point DFT across the lanes g of each sequence (every register a), radix
// 2.  Forward: decimation in frequency, natural lane order in, bit-reversed
// out; each stage of half-size h takes (u, v) = (lane g, lane g + h) to
// (u + v, (u - v) w_2h^(g mod h)).  Inverse: the stages backwards with
// conjugate twiddles (unnormalised).  The twiddle w_2h^j is w_2N^(j N / h).
// Every lane of the warp calls it (the shuffles span the whole warp; their
// xor masks stay inside a group).
template <int V, bool INV, int L = 32>
__device__ __forceinline__ void lane_dft(float2 (&b)[V], int g, const float2* twc) {
  constexpr int G = L / V, N = L * V;
  if constexpr (G > 1) {
    if constexpr (!INV) {
#pragma unroll
      for (int h = G / 2; h >= 1; h >>= 1) {
        const bool up = (g & h) != 0;
        const float s = up ? -1.0f : 1.0f;
        const float2 w = h > 1 && up ? twc[(g & (h - 1)) * (N / h)] : make_float2(1.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < V; ++a) {
          const float2 p = shfl_xor2(b[a], h);
          // lower lane: u + v; upper lane: u - v (u the lower lane's value)
          const float2 r = __ffma2_rn(b[a], make_float2(s, s), p);
          b[a] = h > 1 ? cmul(r, w) : r;
        }
      }
    } else {
#pragma unroll
      for (int h = 1; h < G; h <<= 1) {
        const bool up = (g & h) != 0;
        const float s = up ? -1.0f : 1.0f;
        const float2 w = h > 1 && up ? twc[(g & (h - 1)) * (N / h)] : make_float2(1.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < V; ++a) {
          const float2 t = h > 1 ? cmulc(b[a], w) : b[a];
          const float2 p = shfl_xor2(t, h);
          b[a] = __ffma2_rn(t, make_float2(s, s), p);
        }
      }
    }
  }
}

// Forward length-N transform of the group's sequence: natural order in, the
// order of the header out.  scr: the group's scratch; lane: index in the group.
template <int V, int L = 32>
__device__ __forceinline__ void wfft_fwd(float2 (&a)[V], float2* scr, const float2* tw1, const float2* twc,
                                         int lane) {
  constexpr int G = L / V, XP = L + G;
  dft_reg<V, false>(a);
#pragma unroll
  for (int k1 = 1; k1 < V; ++k1) a[k1] = cmul(a[k1], tw1[k1 * L + lane]);
#pragma unroll
  for (int k1 = 0; k1 < V; ++k1) scr[k1 * XP + lane] = a[k1];
  __syncwarp();
  const int k1 = lane / G, g = lane % G;
#pragma unroll
  for (int j = 0; j < V; ++j) a[j] = scr[k1 * XP + g + G * j];
  __syncwarp();
  dft_reg<V, false>(a);
  if constexpr (G == 2) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = twiddle_g2<L, false>(a[q], q, g);
  } else if constexpr (G > 1) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = cmul(a[q], tw1[q * L + V * g]);
  }
  lane_dft<V, false, L>(a, g, twc);
}

// Inverse of wfft_fwd (times N): the header's order in, natural order out.
template <int V, int L = 32>
__device__ __forceinline__ void wfft_inv(float2 (&a)[V], float2* scr, const float2* tw1, const float2* twc,
                                         int lane) {
  constexpr int G = L / V, XP = L + G;
  const int k1 = lane / G, g = lane % G;
  lane_dft<V, true, L>(a, g, twc);
  if constexpr (G == 2) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = twiddle_g2<L, true>(a[q], q, g);
  } else if constexpr (G > 1) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = cmulc(a[q], tw1[q * L + V * g]);
  }
  dft_reg<V, true>(a);
#pragma unroll
  for (int j = 0; j < V; ++j) scr[k1 * XP + g + G * j] = a[j];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < V; ++q) a[q] = scr[q * XP + lane];
  __syncwarp();
#pragma unroll
  for (int q = 1; q < V; ++q) a[q] = cmulc(a[q], tw1[q * L + lane]);
  dft_reg<V, true>(a);
}

// The twiddles one lane of a group multiplies by, held in registers for
// kernels that run many transforms per lane: t1[k1] = w_N^(lane k1) (first
// step), t2[q] = w_N^(V g q) (second step, g = lane mod G).
template <int V>
struct WTwid {
  float2 t1[V], t2[V];
};
template <int V, int L>
__device__ __forceinline__ void wtwid_load(WTwid<V>& t, const float2* tw1, int lane) {
  constexpr int G = L / V;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    t.t1[k] = tw1[k * L + lane];
    if constexpr (G != 2) t.t2[k] = tw1[k * L + V * (lane % G)];
  }
}

// wfft_fwd / wfft_inv with the lane's twiddles from registers.
template <int V, int L>
__device__ __forceinline__ void wfft_fwd(float2 (&a)[V], float2* scr, const WTwid<V>& t, const float2* twc,
                                         int lane) {
  constexpr int G = L / V, XP = L + G;
  dft_reg<V, false>(a);
#pragma unroll
  for (int k1 = 1; k1 < V; ++k1) a[k1] = cmul(a[k1], t.t1[k1]);
#pragma unroll
  for (int k1 = 0; k1 < V; ++k1) scr[k1 * XP + lane] = a[k1];
  __syncwarp();
  const int k1 = lane / G, g = lane % G;
#pragma unroll
  for (int j = 0; j < V; ++j) a[j] = scr[k1 * XP + g + G * j];
  __syncwarp();
  dft_reg<V, false>(a);
  if constexpr (G == 2) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = twiddle_g2<L, false>(a[q], q, g);
  } else if constexpr (G > 1) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = cmul(a[q], t.t2[q]);
  }
  lane_dft<V, false, L>(a, g, twc);
}
template <int V, int L>
__device__ __forceinline__ void wfft_inv(float2 (&a)[V], float2* scr, const WTwid<V>& t, const float2* twc,
                                         int lane) {
  constexpr int G = L / V, XP = L + G;
  const int k1 = lane / G, g = lane % G;
  lane_dft<V, true, L>(a, g, twc);
  if constexpr (G == 2) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = twiddle_g2<L, true>(a[q], q, g);
  } else if constexpr (G > 1) {
#pragma unroll
    for (int q = 1; q < V; ++q) a[q] = cmulc(a[q], t.t2[q]);
  }
  dft_reg<V, true>(a);
#pragma unroll
  for (int j = 0; j < V; ++j) scr[k1 * XP + g + G * j] = a[j];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < V; ++q) a[q] = scr[q * XP + lane];
  __syncwarp();
#pragma unroll
  for (int q = 1; q < V; ++q) a[q] = cmulc(a[q], t.t1[q]);
  dft_reg<V, true>(a);
}

}  // namespace nlos
