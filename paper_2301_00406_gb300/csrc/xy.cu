// FFT passes of the light-cone-transform operator A = R_t^{-1} H R_z (Eq. 3),
// of its transpose, and of the periodic solve of Eq. 11.
//
// Data layout in HBM (row-major, t fastest): volumes and transients are
// [nx][ny][nt] float32, i.e. one contiguous column of nt values per scan
// point.  Spectra are stored transposed, [kt][col] complex64, so that the
// lateral passes read whole kt planes.
//
// The zero-padded 3-D FFT of the convolution is factored into
//  * a t-pass per column: real signal of length nt zero-padded to 2 nt.
//    Two real columns a, b are packed as z = a + i b; the even and odd bins of
//    the padded length-2nt DFT of z are two length-nt DFTs (of z and of
//    z * exp(-i pi n / nt)), and the bins of a and b are separated with
//    Hermitian symmetry.  Only kt in [0, nt] is kept.
//  * a lateral pass per kt plane on a pair of CTAs in a thread-block cluster:
//    CTA r handles the ky bins of parity r of the 2 ny-point padded DFT
//    (again an ny-point DFT of a twisted row), runs the 2 nx-point padded
//    transform along x as two nx-point DFTs per column, multiplies by the
//    kernel spectrum, transforms back, and the pair sums its two halves of
//    the result through distributed shared memory.
// No padded array ever reaches HBM.
#include <cooperative_groups.h>

#include <type_traits>

#include "fft.cuh"
#include "passes.cuh"
#include "wfft.cuh"

namespace cg = cooperative_groups;

namespace nlos {

// ---------------------------------------------------------------------------
// Lateral convolution per kt plane on a CTA pair (cluster of 2).
// ---------------------------------------------------------------------------
template <int N>
struct CV {
  static constexpr int P = N + 1;                 // odd row pitch of the plane
  static constexpr int CH = N >= 32 ? 32 : N;     // columns per x-chunk
  static constexpr int SP = 2 * CH + 1;           // pitch of the chunk scratch (2 CH transforms)
  static constexpr size_t smem = sizeof(float2) * (N * P + N * SP + 2 * N);
};
constexpr int kConvThreads = 512;

// x-direction padded convolution of CH plane columns starting at c0 (the
// columns are ky' positions of the y-transformed plane; ky = 2 ky_nat + r).
// For each column and each x-parity ax the 2N-point padded DFT bin
// kx = 2 kx' + ax is the N-point DFT of the column twisted by
// exp(-i pi ax x / N); after the multiply by H the two inverse transforms are
// untwisted and summed back into the plane.  The split N = R1 R2 runs as
//   A  (per column, ax, n2): R1-point DFT of the stride-R2 subsequence,
//      twiddles, into the scratch;
//   B  (per transform, k1): R2-point DFT, multiply by H, inverse R2-point DFT
//      and inverse twiddles, all in registers;
//   A' (per column, n2): inverse R1-point DFTs of both parities, untwist,
//      sum, back into the plane.
template <int N>
__device__ __forceinline__ void xconv_chunk(float2* __restrict__ plane, float2* __restrict__ scr, int c0, int r,
                                            const float2* __restrict__ Hk, int adj, const float2* __restrict__ tw,
                                            int tid, int nthr) {
  constexpr int R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2, P = CV<N>::P, CH = CV<N>::CH, SP = CV<N>::SP;
  // A: forward first step of both parities
  for (int it = tid; it < 2 * CH * R2; it += nthr) {
    const int t = it % (2 * CH), n2 = it / (2 * CH);
    const int ax = t / CH, j = t % CH;
    float2 a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int x = R2 * n1 + n2;
      float2 v = plane[x * P + c0 + j];
      if (ax) v = cmul(v, tw[x]);
      a[n1] = v;
    }
    dft_reg<R1, false>(a);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmul(a[k1], tw[2 * ((n2 * k1) & (N - 1))]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) scr[(R2 * k1 + n2) * SP + t] = a[k1];
  }
  __syncthreads();
  // B: second step, kernel multiply, inverse second step
  for (int it = tid; it < 2 * CH * R1; it += nthr) {
    const int t = it % (2 * CH), k1 = it / (2 * CH);
    const int ax = t / CH, j = t % CH;
    float2 b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = scr[(R2 * k1 + n2) * SP + t];
    dft_reg<R2, false>(b);
    int ky = 2 * kfreq<N>(c0 + j) + r;
    if (ky > N) ky = 2 * N - ky;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      int kx = 2 * (k1 + R1 * k2) + ax;
      if (kx > N) kx = 2 * N - kx;
      const float2 h = __ldg(Hk + kx * (N + 1) + ky);
      b[k2] = adj ? cmulc(b[k2], h) : cmul(b[k2], h);
    }
    dft_reg<R2, true>(b);
#pragma unroll
    for (int n2 = 1; n2 < R2; ++n2) b[n2] = cmulc(b[n2], tw[2 * ((n2 * k1) & (N - 1))]);
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) scr[(R2 * k1 + n2) * SP + t] = b[n2];
  }
  __syncthreads();
  // A': inverse first step of both parities, untwist, sum into the plane
  for (int it = tid; it < CH * R2; it += nthr) {
    const int j = it % CH, n2 = it / CH;
    float2 e[R1], o[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      e[k1] = scr[(R2 * k1 + n2) * SP + j];
      o[k1] = scr[(R2 * k1 + n2) * SP + CH + j];
    }
    dft_reg<R1, true>(e);
    dft_reg<R1, true>(o);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int x = R2 * n1 + n2;
      plane[x * P + c0 + j] = cadd(e[n1], cmulc(o[n1], tw[x]));
    }
  }
  __syncthreads();
}

template <int N>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kConvThreads)
    k_conv(const float2* __restrict__ Sin, int in_pitch, const int32_t* __restrict__ in_cols, int in_n,
           float2* __restrict__ Sout, int out_pitch, const int32_t* __restrict__ out_cols, int out_n,
           const float2* __restrict__ H, int adj, const float2* __restrict__ twg) {
  constexpr int P = CV<N>::P, CH = CV<N>::CH, SP = CV<N>::SP;
  extern __shared__ float4 smem_f4[];
  float2* plane = reinterpret_cast<float2*>(smem_f4);   // [N][P]
  float2* scr = plane + N * P;                           // [N][SP]
  float2* tw = scr + N * SP;                             // [2N]: exp(-2 pi i n / 2N)
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int kt = blockIdx.x >> 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < 2 * N; i += nthr) tw[i] = __ldg(twg + i);
  __syncthreads();

  // 1. load the plane with the y-twist of parity r
  const float2* src = Sin + (size_t)kt * in_pitch;
  if (in_cols == nullptr) {
    batched_copy<8, float2>(
        N * N, tid, nthr, [&](int i) { return __ldg(src + i); },
        [&](int i, float2 v) {
          const int x = i / N, y = i % N;
          plane[x * P + y] = r ? cmul(v, tw[y]) : v;
        });
  } else {
    for (int i = tid; i < N * P; i += nthr) plane[i] = make_float2(0.f, 0.f);
    __syncthreads();
    batched_copy<4, float2>(
        in_n, tid, nthr, [&](int j) { return __ldg(src + j); },
        [&](int j, float2 v) {
          const int col = __ldg(in_cols + j);
          const int x = col / N, y = col % N;
          plane[x * P + y] = r ? cmul(v, tw[y]) : v;
        });
  }
  __syncthreads();

  // 2. y-DFT of every row (ky' positions, permuted)
  team_fft<N, false>(plane, N, P, 1, tw, 2, tid, nthr);

  // 3. x-direction padded convolution, CH columns at a time
  const float2* Hk = H + (size_t)kt * (N + 1) * (N + 1);
  for (int c0 = 0; c0 < N; c0 += CH) xconv_chunk<N>(plane, scr, c0, r, Hk, adj, tw, tid, nthr);

  // 4. inverse y-DFT of every row (natural y order)
  team_fft<N, true>(plane, N, P, 1, tw, 2, tid, nthr);

  // 5. sum the two parities across the pair: out = s (O_0 + O_1 exp(+i pi y / N))
  cluster.sync();
  const float2* p0 = r == 0 ? plane : cluster.map_shared_rank(plane, 0);
  const float2* p1 = r == 1 ? plane : cluster.map_shared_rank(plane, 1);
  const float s = 1.0f / (4.0f * N * N);
  float2* dst = Sout + (size_t)kt * out_pitch;
  if (out_cols == nullptr) {
    const int i0 = r * (N * N / 2);
    batched_copy<8, float4>(
        N * N / 2, tid, nthr,
        [&](int ii) {
          const int i = i0 + ii, x = i / N, y = i % N;
          const float2 a = p0[x * P + y], b = p1[x * P + y];
          return make_float4(a.x, a.y, b.x, b.y);
        },
        [&](int ii, float4 v) {
          const int i = i0 + ii, y = i % N;
          dst[i] = cscale(cadd(make_float2(v.x, v.y), cmulc(make_float2(v.z, v.w), tw[y])), s);
        });
  } else {
    const int half = (out_n + 1) / 2;
    const int jb = r * half, je = r ? out_n : half;
    batched_copy<4, float4>(
        je - jb, tid, nthr,
        [&](int jj) {
          const int col = __ldg(out_cols + jb + jj);
          const int x = col / N, y = col % N;
          const float2 a = p0[x * P + y], b = p1[x * P + y];
          return make_float4(a.x, a.y, b.x, b.y);
        },
        [&](int jj, float4 v) {
          const int y = __ldg(out_cols + jb + jj) % N;
          dst[jb + jj] = cscale(cadd(make_float2(v.x, v.y), cmulc(make_float2(v.z, v.w), tw[y])), s);
        });
  }
  cluster.sync();
}

// ---------------------------------------------------------------------------
// Periodic lateral solve per kt' plane.
// ---------------------------------------------------------------------------
// Column (x) pass of the periodic solve: forward first step, then per
// (column, k1) the second step, the division by c0 + c1 lambda(k) and the
// inverse second step in registers, then the inverse first step.
template <int N>
__device__ __forceinline__ void xsolve_pass(float2* __restrict__ plane, float c0, float c1, float lt,
                                            const float* __restrict__ lamx, const float2* __restrict__ tw, int tid,
                                            int nthr) {
  constexpr int R1 = FftPlan<N>::R1, R2 = FftPlan<N>::R2, P = N + 1;
  for (int it = tid; it < N * R2; it += nthr) {
    const int j = it % N, n2 = it / N;
    float2 a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) a[n1] = plane[(R2 * n1 + n2) * P + j];
    dft_reg<R1, false>(a);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmul(a[k1], tw[2 * ((n2 * k1) & (N - 1))]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) plane[(R2 * k1 + n2) * P + j] = a[k1];
  }
  __syncthreads();
  for (int it = tid; it < N * R1; it += nthr) {
    const int j = it % N, k1 = it / N;
    float2 b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = plane[(R2 * k1 + n2) * P + j];
    dft_reg<R2, false>(b);
    const float ly = __ldg(lamx + kfreq<N>(j)) + lt;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const float den = c0 + c1 * (__ldg(lamx + k1 + R1 * k2) + ly);
      b[k2] = cscale(b[k2], 1.0f / den);
    }
    dft_reg<R2, true>(b);
#pragma unroll
    for (int n2 = 1; n2 < R2; ++n2) b[n2] = cmulc(b[n2], tw[2 * ((n2 * k1) & (N - 1))]);
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) plane[(R2 * k1 + n2) * P + j] = b[n2];
  }
  __syncthreads();
  for (int it = tid; it < N * R2; it += nthr) {
    const int j = it % N, n2 = it / N;
    float2 a[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[k1] = plane[(R2 * k1 + n2) * P + j];
    dft_reg<R1, true>(a);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) plane[(R2 * n1 + n2) * P + j] = a[n1];
  }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kConvThreads)
    k_sxy(float2* __restrict__ Sp, int nt, const float* __restrict__ lamx, const float* __restrict__ lamt,
          const DevScalars* __restrict__ sc, double c0_host, double c1, const float2* __restrict__ twg) {
  constexpr int P = N + 1;
  extern __shared__ float4 smem_f4[];
  float2* plane = reinterpret_cast<float2*>(smem_f4);
  float2* tw = plane + N * P;
  const int kt = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < 2 * N; i += nthr) tw[i] = __ldg(twg + i);
  float2* g = Sp + (size_t)kt * N * N;
  const float s = 1.0f / (float)(N * N);
  batched_copy<8, float2>(
      N * N, tid, nthr, [&](int i) { return g[i]; },
      [&](int i, float2 v) { plane[(i / N) * P + (i % N)] = cscale(v, s); });
  __syncthreads();
  team_fft<N, false>(plane, N, P, 1, tw, 2, tid, nthr);   // rows (y)
  const float c0 = sc ? (float)sc->L : (float)c0_host;
  xsolve_pass<N>(plane, c0, (float)c1, __ldg(lamt + kt), lamx, tw, tid, nthr);
  team_fft<N, true>(plane, N, P, 1, tw, 2, tid, nthr);
  for (int i = tid; i < N * N; i += nthr) g[i] = plane[(i / N) * P + (i % N)];
}

// The same solve for N >= 32 with every transform held in registers by a
// half-warp (wfft.cuh with L = 16 lanes, V = N / 16 values per lane): 32
// groups of 16 lanes per CTA, N / 32 rows (then columns, then rows) per
// group, so a plane passes through shared memory three times with two CTA
// barriers, instead of once per transform step.
//  1. rows: load row x (lane l: elements l + 16 m, coalesced), forward
//     transform over y, store in the transform's output order (position
//     l + 16 m) into the plane (pitch N + 1: the column reads of step 2 fall
//     in distinct banks);
//  2. columns (one output position q = ky slot per group pass): forward
//     transform over x, divide by c0 + c1 (lambda(kx) + lambda(ky) +
//     lambda_t(kt)) and by N^2, inverse transform, back into the plane;
//  3. rows: inverse transform over y from the output order, store in
//     natural order.
template <int N>
struct SW {
  static constexpr int L = 16, V = N / L, G = L / V, XP = L + G;
  static constexpr int P = N + 1;                  // plane row pitch (float2)
  static constexpr int SCR = V * XP;               // exchange scratch per group
  static constexpr int THREADS = 512, GROUPS = THREADS / L;
  static constexpr int PER = N / GROUPS;           // rows or columns per group
  static constexpr size_t smem = sizeof(float2) * (N * P + GROUPS * SCR + 2 * N) + sizeof(float) * N;
  static_assert(N >= 32 && PER >= 1, "half-warp solve needs N >= 32");
};

// Frequency held by lane l (of a group), register m after the forward
// transform.
template <int N>
__device__ __forceinline__ int sw_freq(int l, int m) {
  using W = SW<N>;
  return l / W::G + W::V * m + W::V * W::V * rev_bits<W::G>(l % W::G);
}

template <int N>
__global__ void __launch_bounds__(SW<N>::THREADS, 1)
    k_sxy_w(float2* __restrict__ Sp, const float* __restrict__ lamx, const float* __restrict__ lamt,
            const DevScalars* __restrict__ sc, double c0_host, double c1, const float2* __restrict__ twg) {
  using W = SW<N>;
  constexpr int V = W::V, L = W::L, P = W::P;
  extern __shared__ float4 smem_f4[];
  float2* plane = reinterpret_cast<float2*>(smem_f4);
  float2* scr = plane + N * P + (threadIdx.x / L) * W::SCR;
  float2* tw1 = plane + N * P + W::GROUPS * W::SCR;
  float2* twc = tw1 + N;
  float* lx = reinterpret_cast<float*>(twc + N);
  const int grp = threadIdx.x / L, l = threadIdx.x % L;
  // tw1[k1 L + l] = w_N^(l k1) = w_2N^(2 l k1), twc[n] = w_2N^n
  for (int i = threadIdx.x; i < N; i += W::THREADS) {
    tw1[i] = __ldg(twg + ((2 * (i % L) * (i / L)) & (2 * N - 1)));
    twc[i] = __ldg(twg + i);
    lx[i] = __ldg(lamx + i);
  }
  const int kt = blockIdx.x;
  float2* g = Sp + (size_t)kt * N * N;
  // 1. rows, forward; the next row's loads are issued before this row's
  // transform
  float2 nxt[V];
#pragma unroll
  for (int m = 0; m < V; ++m) nxt[m] = g[grp * N + l + L * m];
  __syncthreads();  // tables staged
  WTwid<V> tw;
  wtwid_load<V, L>(tw, tw1, l);
#pragma unroll 1
  for (int r = 0; r < W::PER; ++r) {
    const int x = grp + W::GROUPS * r;
    float2 a[V];
#pragma unroll
    for (int m = 0; m < V; ++m) a[m] = nxt[m];
    if (r + 1 < W::PER) {
#pragma unroll
      for (int m = 0; m < V; ++m) nxt[m] = g[(x + W::GROUPS) * N + l + L * m];
    }
    wfft_fwd<V, L>(a, scr, tw, twc, l);
#pragma unroll
    for (int m = 0; m < V; ++m) plane[x * P + l + L * m] = a[m];
  }
  __syncthreads();
  // 2. columns: forward over x, division, inverse
  const float c0 = sc ? (float)sc->L : (float)c0_host;
  const float c1f = (float)c1, lt = __ldg(lamt + kt), s = 1.0f / (float)(N * N);
  float lk[V];
#pragma unroll
  for (int m = 0; m < V; ++m) lk[m] = lx[sw_freq<N>(l, m)];
#pragma unroll 1
  for (int r = 0; r < W::PER; ++r) {
    const int q = grp + W::GROUPS * r;
    const float ly = lx[sw_freq<N>(q % L, q / L)] + lt;
    float2 b[V];
#pragma unroll
    for (int m = 0; m < V; ++m) b[m] = plane[(l + L * m) * P + q];
    wfft_fwd<V, L>(b, scr, tw, twc, l);
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const float den = c0 + c1f * (lk[m] + ly);
      b[m] = cscale(b[m], __frcp_rn(den) * s);
    }
    wfft_inv<V, L>(b, scr, tw, twc, l);
#pragma unroll
    for (int m = 0; m < V; ++m) plane[(l + L * m) * P + q] = b[m];
  }
  __syncthreads();
  // 3. rows, inverse, natural order out
#pragma unroll 1
  for (int r = 0; r < W::PER; ++r) {
    const int x = grp + W::GROUPS * r;
    float2 a[V];
#pragma unroll
    for (int m = 0; m < V; ++m) a[m] = plane[x * P + l + L * m];
    wfft_inv<V, L>(a, scr, tw, twc, l);
#pragma unroll
    for (int m = 0; m < V; ++m) g[x * N + l + L * m] = a[m];
  }
}

// ---------------------------------------------------------------------------
// Cone-kernel spectrum: H(kx, ky, kt) for kx, ky in [0, N], kt in [0, nt], the
// DFT of h over the (2N, 2N, 2nt) grid.  One CTA per (kt, parity quadrant).
// Lateral tap (i, j) of h has two nonzero t-taps m0, m0 + 1 with weights hw.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kConvThreads)
    k_kspec(float2* __restrict__ H, int nt, const int32_t* __restrict__ m0t, const float2* __restrict__ hw,
            const float2* __restrict__ tw2t, const float2* __restrict__ twg) {
  constexpr int P = N + 1;
  extern __shared__ float4 smem_f4[];
  float2* plane = reinterpret_cast<float2*>(smem_f4);
  float2* tw = plane + N * P;
  const int kt = blockIdx.x >> 2, ax = (blockIdx.x >> 1) & 1, ay = blockIdx.x & 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < 2 * N; i += nthr) tw[i] = __ldg(twg + i);
  __syncthreads();
  const int n2 = 2 * nt;
  for (int i = tid; i < N * N; i += nthr) {
    const int x = i / N, y = i % N;
    float2 acc = make_float2(0.f, 0.f);
    for (int sx = 0; sx < 2; ++sx)
      for (int sy = 0; sy < 2; ++sy) {
        const int li = (x + sx * N) * (2 * N) + (y + sy * N);
        const int m = __ldg(m0t + li);
        const float2 w = __ldg(hw + li);
        // G = w0 exp(-2 pi i m kt / 2nt) + w1 exp(-2 pi i (m + 1) kt / 2nt)
        const long long ph0 = ((long long)m * kt) % n2;
        const long long ph1 = ((long long)(m + 1) * kt) % n2;
        float2 gv = cadd(cscale(__ldg(tw2t + ph0), w.x), cscale(__ldg(tw2t + ph1), w.y));
        const float sgn = ((ax & sx) ^ (ay & sy)) ? -1.0f : 1.0f;
        acc = cadd(acc, cscale(gv, sgn));
      }
    // twist exp(-i pi (ax x + ay y) / N)
    float2 t = make_float2(1.f, 0.f);
    if (ax) t = cmul(t, tw[x]);
    if (ay) t = cmul(t, tw[y]);
    plane[x * P + y] = cmul(acc, t);
  }
  __syncthreads();
  team_fft<N, false>(plane, N, P, 1, tw, 2, tid, nthr);
  team_fft<N, false>(plane, N, 1, P, tw, 2, tid, nthr);
  for (int i = tid; i < N * N; i += nthr) {
    const int xp = i / N, yp = i % N;
    const int kx = 2 * kfreq<N>(xp) + ax, ky = 2 * kfreq<N>(yp) + ay;
    if (kx <= N && ky <= N) H[((size_t)kt * (N + 1) + kx) * (N + 1) + ky] = plane[xp * P + yp];
  }
}

// ---------------------------------------------------------------------------
// Launchers (runtime size -> template instance)
// ---------------------------------------------------------------------------
template <typename F>
static nlos_status dispatch_n(int n, F&& f) {
  switch (n) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    case 128: return f(std::integral_constant<int, 128>{});
  }
  return fail(NLOS_ERR_INVALID_ARG, "unsupported nx/ny");
}

template <typename K>
static nlos_status set_smem(K kernel, size_t bytes) {
  return ensure_smem(kernel, bytes);
}

nlos_status prepare_xy(int n) {
  return dispatch_n(n, [&](auto nc) -> nlos_status {
    constexpr int N = decltype(nc)::value;
    if (N >= 32)
      NLOS_TRY(prepare_conv4(N));
    else
      NLOS_TRY(set_smem(k_conv<N>, CV<N>::smem));
    NLOS_TRY(set_smem(k_sxy<N>, sizeof(float2) * (N * (N + 1) + 2 * N)));
    if constexpr (N >= 32) NLOS_TRY(set_smem(k_sxy_w<N>, SW<N>::smem));
    NLOS_TRY(set_smem(k_kspec<N>, sizeof(float2) * (N * (N + 1) + 2 * N)));
    return NLOS_OK;
  });
}

nlos_status launch_conv(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact, bool adj,
                        cudaStream_t st) {
  KTimer kt_(P, KC_CONV, st);
  if (P.lateral) return launch_conv_tc(P, Sin, in_compact, Sout, out_compact, adj, st);
  if (P.nx >= 32) return launch_conv4(P, Sin, in_compact, Sout, out_compact, adj, st);
  return dispatch_n(P.nx, [&](auto nc) -> nlos_status {
    constexpr int N = decltype(nc)::value;
    auto kern = k_conv<N>;
    NLOS_TRY(set_smem(kern, CV<N>::smem));
    const int full = P.nx * P.ny;
    kern<<<2 * (P.nt + 1), kConvThreads, CV<N>::smem, st>>>(
        Sin, in_compact ? P.ncols : full, in_compact ? P.d_cols : nullptr, P.ncols, Sout,
        out_compact ? P.ncols : full, out_compact ? P.d_cols : nullptr, P.ncols, P.d_H, adj ? 1 : 0, P.d_twx);
    NLOS_LAUNCH_CHECK("k_conv");
    return NLOS_OK;
  });
}

nlos_status launch_sxy(const Plan& P, float2* Sp, const DevScalars* sc, double c0_host, double c1, cudaStream_t st) {
  KTimer kt_(P, KC_SXY, st);
  return dispatch_n(P.nx, [&](auto nc) -> nlos_status {
    constexpr int N = decltype(nc)::value;
    // the tuned choice for this plane size (the half-warp kernel unless the
    // plan's timing found the shared-memory passes faster)
    if constexpr (N >= 32) {
      if (tp_cols_for(TPK_SXY, P.nt, N) != kSxyPasses) {
        NLOS_TRY(set_smem(k_sxy_w<N>, SW<N>::smem));
        k_sxy_w<N><<<P.nt / 2 + 1, SW<N>::THREADS, SW<N>::smem, st>>>(Sp, P.d_lamx, P.d_lamt, sc, c0_host, c1,
                                                                       P.d_twx);
        NLOS_LAUNCH_CHECK("k_sxy_w");
        return NLOS_OK;
      }
    }
    auto kern = k_sxy<N>;
    const size_t sm = sizeof(float2) * (N * (N + 1) + 2 * N);
    NLOS_TRY(set_smem(kern, sm));
    kern<<<P.nt / 2 + 1, kConvThreads, sm, st>>>(Sp, P.nt, P.d_lamx, P.d_lamt, sc, c0_host, c1, P.d_twx);
    NLOS_LAUNCH_CHECK("k_sxy");
    return NLOS_OK;
  });
}

nlos_status launch_kernel_spectrum(const Plan& P, const int32_t* m0, const float2* hw, cudaStream_t st) {
  return dispatch_n(P.nx, [&](auto nc) -> nlos_status {
    constexpr int N = decltype(nc)::value;
    auto kern = k_kspec<N>;
    const size_t sm = sizeof(float2) * (N * (N + 1) + 2 * N);
    NLOS_TRY(set_smem(kern, sm));
    kern<<<4 * (P.nt + 1), kConvThreads, sm, st>>>(P.d_H, P.nt, m0, hw, P.d_tw2t, P.d_twx);
    NLOS_LAUNCH_CHECK("k_kspec");
    return NLOS_OK;
  });
}

}  // namespace nlos
