// Lateral convolution of the light-cone transform (the H of Eq. 3 applied to
// every kt plane of the t-transformed volume) for N = nx = ny in {32, 64, 128}:
// a cluster of four CTAs per kt plane, two CTAs resident per SM.
//
// The plane (N x N complex, zero-padded to 2N x 2N by the convolution) is
// split by lateral frequency: CTA q of the cluster owns the padded y bins
// ky = 4 k + q, k in [0, M), M = N / 2.  Because the input occupies only the
// first N of the 2N padded samples, those bins are an M-point DFT of the row
// folded once,
//     Y[4 k + q] = DFT_M( w^(q n) (row[n] + (-i)^q row[n + M]) )[k],
//     w = exp(-2 pi i / 2N),
// and the same fold by x parity p = kx mod 4 turns the padded 2N-point
// transform along x of each column into four M-point transforms.  After the
// multiply by H and the inverse transforms, the four parities (and, for y,
// the four CTAs) recombine as
//     out[n] = sum_p w^(-p n) I_p[n],  out[n + M] = sum_p i^p w^(-p n) I_p[n].
// Every M-point transform runs as two register DFTs (8 x R2, R2 = M / 8) with
// one exchange through shared memory.
//
// Phases of one CTA (q = rank in the cluster):
//  1. compact input only: scatter the sampled values of rows
//     [q N/4, (q+1) N/4) into a zeroed staging buffer;
//  2. y transform of all N rows (a dense input plane read from global
//     memory, a compact one from the four CTAs' staging buffers through
//     distributed shared memory) -> plane[x][k], k < M;
//  3. x convolution, one warp per column: fold by the four x parities,
//     forward M-point transforms, multiply by H, inverse, recombine across
//     the parity lanes with warp shuffles, back into the column;
//  4. inverse y transform of every row, untwisted by w^(-q n);
//  5. CTA q sums the four CTAs' results for its rows and writes them.
// Only cluster barriers separate the CTA-wide phases; inside a phase each
// warp owns whole rows or columns and synchronises with __syncwarp.
//
// The multiply reads H(kx, ky) as H(ky, kx): the cone kernel depends on
// (i dx)^2 + (j dy)^2 with dx = dy (nx = ny over one wall width), so its
// spectrum is symmetric in the two lateral frequencies, and the transposed
// lookup makes the 32 lanes of a warp read 32 consecutive kx.
#include <cooperative_groups.h>

#include <type_traits>

#include "fft.cuh"
#include "passes.cuh"

namespace cg = cooperative_groups;

namespace nlos {

template <int N>
struct C4 {
  static constexpr int M = N / 2;            // points per folded transform
  static constexpr int R2 = M / 8;           // second-step radix (first step is 8)
  static constexpr int RW = 32 / R2;         // rows per warp in the y phases
  static constexpr int CW = 8 / R2;          // columns per warp in the x phase
  static constexpr int ROWS = N / 4;         // input rows staged per CTA
  static constexpr int SP = N + R2;          // stage row pitch (float2)
  static constexpr int SPX = N == 128 ? 72 : N == 64 ? 40 : 18;  // x scratch pitch per (column, parity)
  static constexpr int WSCR = CW * 4 * SPX;  // x scratch per warp (float2)
  static constexpr int WARPS = 8, THREADS = 256;
  static constexpr int ZB = N == 128 ? 4 * 72 : 0;  // folded-bin buffer per warp (lattice modes)
  static constexpr int REGION = ROWS * SP > WARPS * (WSCR + ZB) ? ROWS * SP : WARPS * (WSCR + ZB);
  static constexpr size_t smem = sizeof(float2) * (N * M + REGION + 2 * N) + sizeof(int) * 2 * N;
};

// Row swizzle of the plane: element (x, k) lives at x M + (k ^ swz(x)), swz
// linear over GF(2) in the bits of x.  The coefficients make every access
// pattern of the three phases hit distinct banks, at N = 128 also those that
// visit only the rows x = 4 v + r0 of a stride-4 lattice (the y transforms
// four lattice rows per warp step, the lattice x passes eight rows 4 apart
// times two columns 8 apart): bits 2-4, which alone vary there, map to
// independent slot offsets (a bank model of every pattern chose them).
template <int N>
__host__ __device__ constexpr int swc(int bit) {
  return N == 128 ? (bit == 0 ? 8 : bit == 1 ? 1 : bit == 2 ? 14 : bit == 3 ? 15 : bit == 4 ? 13 : bit == 5 ? 8 : bit == 6 ? 4 : 0)
         : N == 64 ? (bit == 0 ? 8 : bit == 1 ? 15 : bit == 2 ? 10 : bit == 3 ? 8 : bit == 4 ? 3 : bit == 5 ? 14 : 0)
                   : (bit == 0 ? 8 : bit == 1 ? 3 : bit == 2 ? 12 : bit == 3 ? 11 : bit == 4 ? 15 : 0);
}
template <int N>
__host__ __device__ __forceinline__ constexpr int swz(int x) {
  int v = 0;
#pragma unroll
  for (int b = 0; (1 << b) < N; ++b)
    if ((x >> b) & 1) v ^= swc<N>(b);
  return v;
}
// swz is linear over GF(2): for x = a + b with disjoint bits, swz(x) =
// swz(a) ^ swz(b).  The phases below split row indices into a lane-constant
// part and an iteration (or compile-time) part and combine the two.

// In-row position of the intermediate value (n2, k1) between the two steps
// of a y transform, and within a (column, parity) slot of the x scratch.
__device__ __forceinline__ constexpr int ipos(int n2, int k1) { return 8 * n2 + (k1 ^ (n2 & 7)); }

// v * (-i)^p and v * i^p for a runtime p in [0, 4)
__device__ __forceinline__ float2 rot_mi(float2 v, int p) {
  const float2 r = (p & 1) ? make_float2(v.y, -v.x) : v;
  return (p & 2) ? make_float2(-r.x, -r.y) : r;
}
__device__ __forceinline__ float2 rot_i(float2 v, int p) {
  const float2 r = (p & 1) ? make_float2(-v.y, v.x) : v;
  return (p & 2) ? make_float2(-r.x, -r.y) : r;
}
// index of the padded frequency k in [0, 2N) within the stored [0, N] half
template <int N>
__device__ __forceinline__ int fold_k(int k) {
  return k <= N ? k : 2 * N - k;
}

// Phase 2: forward y transform of every row for bins ky = 4 k + Q.  LAT:
// only the rows x = 4 v + r0 (v < N / 4) hold input, and each warp step
// takes four such rows (the swizzle of x = 4 v + r0 is swz(4 v) ^ swz(r0),
// the bits of 4 v and r0 being disjoint).
// csrc (LAT only, nullable): the compact input of a full stride-4 lattice
// (sampled columns x = 4 mx + r0, y = 4 my + ry, compact index mx N/4 + my),
// read in place of the staging buffers.
template <int N, int Q, bool LAT>
__device__ __forceinline__ void c4_yfwd(float2* __restrict__ plane, const float2* const (&stage)[4],
                                        const float2* __restrict__ gsrc, const float2* __restrict__ csrc, int ry,
                                        const float2* __restrict__ tw, const int* __restrict__ rowin, int r0,
                                        int warp, int lane) {
  using C = C4<N>;
  constexpr int M = C::M, R2 = C::R2, RW = C::RW, SP = C::SP, ROWS = C::ROWS;
  constexpr int NR = LAT ? N / 4 : N;  // rows visited
  auto xr = [&](int v) { return LAT ? 4 * v + r0 : v; };
  auto sw = [&](int v) { return LAT ? swz<N>(4 * v) : swz<N>(v); };
  const int rsub = lane / R2, n2 = lane % R2;
  // inter-step twiddles w^(n2 (Q + 4 k1)), k1 = 0..7 (the fold twist w^(Q n2) merged in)
  float2 twa[8];
  {
    const float2 st = tw[(4 * n2) & (2 * N - 1)];
    twa[0] = tw[(Q * n2) & (2 * N - 1)];
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) twa[k1] = cmul(twa[k1 - 1], st);
  }
  // Rows come from global memory (gsrc, a dense plane) or from the four
  // CTAs' staging buffers (distributed shared memory); either way the next
  // row group's 16 values per lane are fetched while the current one computes.
  float2 pu[8], pv[8];
  auto fetch = [&](int it) {
    const int x = xr(it * RW + rsub);
    if (it < NR / RW && rowin[x]) {
      if (LAT && csrc) {
        // this lane's y = n2 + R2 n1 (+ M) are lattice columns only when n2 = ry (mod 4)
        const bool live = (n2 & 3) == ry;
        const float2* rowc = csrc + (it * RW + rsub) * (N / 4) + (n2 >> 2);
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
          pu[n1] = live ? __ldg(rowc + (R2 / 4) * n1) : make_float2(0.f, 0.f);
          pv[n1] = live ? __ldg(rowc + (R2 / 4) * n1 + M / 4) : make_float2(0.f, 0.f);
        }
      } else if (gsrc) {
        const float2* row = gsrc + x * N;
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
          pu[n1] = __ldg(row + n2 + R2 * n1);
          pv[n1] = __ldg(row + n2 + R2 * n1 + M);
        }
      } else {
        const int o = x / ROWS;
        const float2* row =
            (o == 0 ? stage[0] : o == 1 ? stage[1] : o == 2 ? stage[2] : stage[3]) + (x % ROWS) * SP;
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
          pu[n1] = row[n2 + R2 * n1];
          pv[n1] = row[n2 + R2 * n1 + M];
        }
      }
    }
  };
  // swizzles of the lane's row offsets within a row group (rsub, and the
  // step-2 items' rows lane / 8 + 4 j)
  const int s_rsub = sw(rsub);
  int s_item[8 / R2];
#pragma unroll
  for (int j = 0; j < 8 / R2; ++j) s_item[j] = sw((lane + 32 * j) / 8);
  fetch(warp);
  for (int it = warp; it < NR / RW; it += C::WARPS) {
    const int s_it = sw(it * RW) ^ (LAT ? swz<N>(r0) : 0);
    {
      const int x = xr(it * RW + rsub);
      float2 cu[8], cv[8];
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) {
        cu[n1] = pu[n1];
        cv[n1] = pv[n1];
      }
      fetch(it + C::WARPS);
      if (rowin[x]) {
        float2 a[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
          const float2 u = cu[n1], v = cv[n1];
          // (-i)^Q v and the fold twist w^(Q R2 n1) = exp(-2 pi i Q n1 / 32)
          const float2 r = Q == 0 ? v : Q == 1 ? make_float2(v.y, -v.x) : Q == 2 ? make_float2(-v.x, -v.y)
                                                                             : make_float2(-v.y, v.x);
          a[n1] = twmul64<false>(cadd(u, r), (2 * Q * n1) & 63);
        }
        dft_reg<8, false>(a);
        float2* prow = plane + x * M;
        const int s = s_it ^ s_rsub;
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) prow[ipos(n2, k1) ^ s] = cmul(a[k1], twa[k1]);
      }
    }
    __syncwarp();
    // second step: item (row rs, k1); 8 / R2 items per lane
    float2 b[8 / R2][R2];
#pragma unroll
    for (int j = 0; j < 8 / R2; ++j) {
      const int i = lane + 32 * j, xx = xr(it * RW + i / 8), k1 = i % 8;
      if (rowin[xx]) {
        const float2* pr = plane + xx * M;
        const int ss = s_it ^ s_item[j];
#pragma unroll
        for (int m = 0; m < R2; ++m) b[j][m] = pr[ipos(m, k1) ^ ss];
        dft_reg<R2, false>(b[j]);
      } else {
#pragma unroll
        for (int m = 0; m < R2; ++m) b[j][m] = make_float2(0.f, 0.f);
      }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8 / R2; ++j) {
      const int i = lane + 32 * j, xx = xr(it * RW + i / 8), k1 = i % 8;
      float2* pr = plane + xx * M;
      const int ss = s_it ^ s_item[j];
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) pr[(k1 + 8 * k2) ^ ss] = b[j][k2];
    }
    __syncwarp();
  }
}

// Phase 4: inverse y transform of every row, times w^(-Q n) (n < M).  LAT:
// only the rows x = 4 v + r0 are wanted, four of them per warp step.
template <int N, int Q, bool LAT>
__device__ __forceinline__ void c4_yinv(float2* __restrict__ plane, const float2* __restrict__ tw,
                                        const int* __restrict__ rowout, int r0, int warp, int lane) {
  using C = C4<N>;
  constexpr int M = C::M, R2 = C::R2, RW = C::RW;
  constexpr int NR = LAT ? N / 4 : N;  // rows visited
  auto xr = [&](int v) { return LAT ? 4 * v + r0 : v; };
  auto sw = [&](int v) { return LAT ? swz<N>(4 * v) : swz<N>(v); };
  const int rsub = lane / R2, n2 = lane % R2;
  const int k1l = lane % 8;
  // w^(-m (4 k1 + Q)), m < R2, for this lane's k1
  float2 twi[R2];
  {
    const float2 st = cconj(tw[(4 * k1l + Q) & (2 * N - 1)]);
    twi[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int m = 1; m < R2; ++m) twi[m] = cmul(twi[m - 1], st);
  }
  const int s_rsub = sw(rsub);
  int s_item[8 / R2];
#pragma unroll
  for (int j = 0; j < 8 / R2; ++j) s_item[j] = sw((lane + 32 * j) / 8);
  for (int it = warp; it < NR / RW; it += C::WARPS) {
    const int s_it = sw(it * RW) ^ (LAT ? swz<N>(r0) : 0);
    float2 b[8 / R2][R2];
#pragma unroll
    for (int j = 0; j < 8 / R2; ++j) {
      const int i = lane + 32 * j, xx = xr(it * RW + i / 8), k1 = i % 8;
      if (rowout[xx]) {
        const float2* pr = plane + xx * M;
        const int ss = s_it ^ s_item[j];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) b[j][k2] = pr[(k1 + 8 * k2) ^ ss];
        dft_reg<R2, true>(b[j]);
#pragma unroll
        for (int m = 1; m < R2; ++m) b[j][m] = cmul(b[j][m], twi[m]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8 / R2; ++j) {
      const int i = lane + 32 * j, xx = xr(it * RW + i / 8), k1 = i % 8;
      if (rowout[xx]) {
        float2* pr = plane + xx * M;
        const int ss = s_it ^ s_item[j];
#pragma unroll
        for (int m = 0; m < R2; ++m) pr[ipos(m, k1) ^ ss] = b[j][m];
      }
    }
    __syncwarp();
    const int x = xr(it * RW + rsub);
    float2 e[8];
    const bool live = rowout[x] != 0;
    float2* prow = plane + x * M;
    const int s = s_it ^ s_rsub;
    if (live) {
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) e[k1] = prow[ipos(n2, k1) ^ s];
      dft_reg<8, true>(e);
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) prow[(n2 + R2 * n1) ^ s] = twmul64<true>(e[n1], (2 * Q * n1) & 63);
    }
    __syncwarp();
  }
}

// Phase 3: x convolution of the CTA's M columns (ky = 4 c + q).
//
// XM 0: any input and output rows.  XM 1 (N = 128): the output is needed at
// the sampled rows x = 4 m + r0 only (a lattice of stride 4), so after the
// forward steps and H the lane's eight bins kx = 4 k1B + pB + 32 k2 fold to
// two, Z[k''] = w^(-k'' r0) sum_j Y[k'' + 64 j] i^(j r0) for k'' = 4 k1B +
// pB + 32 e (w = exp(-2 pi i / 2N)), and the 64-point inverse of Z at m < 32
// is the output at x = 4 m + r0; a warp folds four columns, then runs their
// inverses together, eight lanes per column.  XM 2 (N = 128): the input
// holds the lattice rows only, so the padded x spectrum is w^(kx r0)
// S[kx mod 64] with S the 64-point transform of the column's 32 lattice
// samples (computed four columns at a time, eight lanes per column); the
// lane's eight bins follow from two values of S by quarter turns, and H and
// the inverse steps are those of XM 0.
template <int N, int XM>
__device__ __forceinline__ void c4_xconv(float2* __restrict__ plane, float2* __restrict__ scr,
                                         float2* __restrict__ zbuf, const float2* __restrict__ tw,
                                         const float2* __restrict__ Hk, int q, int adj, int r0, int warp, int lane) {
  static_assert(XM == 0 || N == 128, "lattice modes are written for N = 128 (CW = 1, R2 = 8)");
  using C = C4<N>;
  constexpr int M = C::M, R2 = C::R2, CW = C::CW, SPX = C::SPX;
  const int cs = lane / (4 * R2), p = (lane / R2) % 4, n2 = lane % R2;
  const int pB = (lane / 8) % 4, k1B = lane % 8;   // step-B item of this lane
  // fold twist exp(-2 pi i p n1 / 32), n1 = 0..7
  float2 w32[8];
  {
    const float2 st = tw[p * (2 * N / 32)];
    w32[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int n1 = 1; n1 < 8; ++n1) w32[n1] = cmul(w32[n1 - 1], st);
  }
  // inter-step twiddles w^(n2 (p + 4 k1))
  float2 twa[8];
  {
    const float2 st = tw[(4 * n2) & (2 * N - 1)];
    twa[0] = tw[(p * n2) & (2 * N - 1)];
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) twa[k1] = cmul(twa[k1 - 1], st);
  }
  // inverse inter-step twiddles w^(-m (4 k1 + p)) for the step-B item
  float2 twb[R2];
  {
    const float2 st = cconj(tw[(4 * k1B + pB) & (2 * N - 1)]);
    twb[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int m = 1; m < R2; ++m) twb[m] = cmul(twb[m - 1], st);
  }
  const int sn2 = swz<N>(n2);
  float2* myscr = scr + (cs * 4 + p) * SPX;
  // H of this lane's step-B items (CW columns x R2 bins), fetched before step A
  // so the global-load latency overlaps it; conjugated for the adjoint
  auto fetch_h = [&](int cb, float2 (&h)[CW][R2]) {
#pragma unroll
    for (int j = 0; j < CW; ++j) {
      const float2* hrow = Hk + fold_k<N>(4 * (cb + j) + q) * (N + 1);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        float2 v = __ldg(hrow + fold_k<N>(4 * (k1B + 8 * k2) + pB));
        if (adj) v.y = -v.y;
        h[j][k2] = v;
      }
    }
  };

  if constexpr (XM == 0) {
    for (int cb = warp * CW; cb < M; cb += C::WARPS * CW) {
      const int c = cb + cs;
      float2 hv[CW][R2];
      fetch_h(cb, hv);
      // A: fold, first step, twiddles -> scratch
      {
        float2 a[8];
  #pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
          const int r0 = n2 + R2 * n1;
          const float2 u = plane[r0 * M + (c ^ sn2 ^ swz<N>(R2 * n1))];
          const float2 v = plane[(r0 + M) * M + (c ^ sn2 ^ swz<N>(R2 * n1) ^ swz<N>(M))];
          a[n1] = cmul(cadd(u, rot_mi(v, p)), w32[n1]);
        }
        dft_reg<8, false>(a);
  #pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) myscr[ipos(n2, k1)] = cmul(a[k1], twa[k1]);
      }
      __syncwarp();
      // B: second step, multiply by H, inverse second step, inverse twiddles
  #pragma unroll
      for (int j = 0; j < CW; ++j) {
        float2* s = scr + (j * 4 + pB) * SPX;
        float2 b[R2];
  #pragma unroll
        for (int m = 0; m < R2; ++m) b[m] = s[ipos(m, k1B)];
        dft_reg<R2, false>(b);
  #pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) b[k2] = cmul(b[k2], hv[j][k2]);
        dft_reg<R2, true>(b);
  #pragma unroll
        for (int m = 0; m < R2; ++m) s[ipos(m, k1B)] = m == 0 ? b[0] : cmul(b[m], twb[m]);
      }
      __syncwarp();
      // A': inverse first step, untwist, recombine the four parities
      {
        float2 e[8];
  #pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) e[k1] = myscr[ipos(n2, k1)];
        dft_reg<8, true>(e);
        // v_p[n] = w^(-p n) I_p[n]; the w^(-p n2) part is already applied in B
        float2 keep[8];
  #pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
          const float2 v = cmulc(e[n1], w32[n1]);
          const float2 v1 = rot_i(v, p);        // contribution to out[n + M]
          const float2 send = (p & 1) ? v : v1;  // the half this lane gives away
          const float2 mine = (p & 1) ? v1 : v;
          const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, send.x, R2),
                                         __shfl_xor_sync(0xffffffffu, send.y, R2));
          keep[n1] = cadd(mine, got);
        }
        const int h = p & 1, hi = p >> 1;
        const int s_out = sn2 ^ swz<N>(R2 * 4 * hi + M * h);  // row bits fixed per lane
  #pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const float2 send = hi ? keep[jj] : keep[4 + jj];
          const float2 mine = hi ? keep[4 + jj] : keep[jj];
          const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 2 * R2),
                                         __shfl_xor_sync(0xffffffffu, send.y, 2 * R2));
          const int x = n2 + R2 * (4 * hi + jj) + M * h;
          plane[x * M + (c ^ s_out ^ swz<N>(R2 * jj))] = cadd(mine, got);
        }
      }
      __syncwarp();
    }

  } else {
    // zbuf: four columns of 64 bins (pitch 72) per warp; entry (r, c) of the
    // 8 x 8 exchange of column jj at jj * 72 + 8 r + (c ^ r)
    constexpr int ZP = 72;
    const int jz = lane >> 3, tz = lane & 7;
    float2* zc = zbuf + jz * ZP;
    const int kk0 = 4 * k1B + pB;  // the lane's two folded bins kk0, kk0 + 32
#pragma unroll 1
    for (int g = 0; g < M / (4 * C::WARPS); ++g) {
      if constexpr (XM == 2) {
        // S = 64-point transform of the lattice samples s[m] = col[4 m + r0], m < 32
        const int c = warp + C::WARPS * (4 * g + jz);
        float2 a[8];
#pragma unroll
        for (int m1 = 0; m1 < 8; ++m1) {
          if (m1 < 4) {
            const int x = 4 * (8 * m1 + tz) + r0;
            a[m1] = plane[x * M + (c ^ swz<N>(x))];
          } else {
            a[m1] = make_float2(0.f, 0.f);
          }
        }
        dft_reg<8, false>(a);
#pragma unroll
        for (int k1 = 1; k1 < 8; ++k1) a[k1] = cmul(a[k1], tw[(4 * k1 * tz) & (2 * N - 1)]);
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) zc[8 * k1 + (tz ^ k1)] = a[k1];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 8; ++t) a[t] = zc[8 * tz + (t ^ tz)];
        __syncwarp();
        dft_reg<8, false>(a);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) zc[tz + 8 * k2] = a[k2];  // S[tz + 8 k2], natural order
        __syncwarp();
      }
#pragma unroll 1
      for (int jj = 0; jj < 4; ++jj) {
        const int c = warp + C::WARPS * (4 * g + jj);
        float2 hv[CW][R2];
        fetch_h(c, hv);
        float2* s = scr + pB * SPX;
        float2 b[R2];
        if constexpr (XM == 1) {
          // A: fold, first step, twiddles -> scratch (as XM 0)
          float2 a[8];
#pragma unroll
          for (int n1 = 0; n1 < 8; ++n1) {
            const int rr = n2 + R2 * n1;
            const float2 u = plane[rr * M + (c ^ sn2 ^ swz<N>(R2 * n1))];
            const float2 v = plane[(rr + M) * M + (c ^ sn2 ^ swz<N>(R2 * n1) ^ swz<N>(M))];
            a[n1] = cmul(cadd(u, rot_mi(v, p)), w32[n1]);
          }
          dft_reg<8, false>(a);
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) myscr[ipos(n2, k1)] = cmul(a[k1], twa[k1]);
          __syncwarp();
#pragma unroll
          for (int m = 0; m < R2; ++m) b[m] = s[ipos(m, k1B)];
          dft_reg<R2, false>(b);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) b[k2] = cmul(b[k2], hv[0][k2]);
          // fold the four j of each e, then the twist w^(-k'' r0)
          float2 z0 = b[0], z1 = b[1];
#pragma unroll
          for (int j = 1; j < 4; ++j) {
            z0 = cadd(z0, rot_i(b[2 * j], (j * r0) & 3));
            z1 = cadd(z1, rot_i(b[2 * j + 1], (j * r0) & 3));
          }
          float2* zj = zbuf + jj * ZP;
          zj[kk0] = cmulc(z0, tw[(kk0 * r0) & (2 * N - 1)]);
          zj[kk0 + 32] = cmulc(z1, tw[((kk0 + 32) * r0) & (2 * N - 1)]);
          __syncwarp();
        } else {
          // the lane's bins from S: b[e + 2 j] = w^(kk r0) S[kk] (-i)^(j r0), kk = kk0 + 32 e
          const float2* zj = zbuf + jj * ZP;
          const float2 s0 = cmul(zj[kk0], tw[(kk0 * r0) & (2 * N - 1)]);
          const float2 s1 = cmul(zj[kk0 + 32], tw[((kk0 + 32) * r0) & (2 * N - 1)]);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            b[2 * j] = cmul(rot_mi(s0, (j * r0) & 3), hv[0][2 * j]);
            b[2 * j + 1] = cmul(rot_mi(s1, (j * r0) & 3), hv[0][2 * j + 1]);
          }
          // inverse second step and inverse twiddles -> scratch, then A' as XM 0
          dft_reg<R2, true>(b);
#pragma unroll
          for (int m = 0; m < R2; ++m) s[ipos(m, k1B)] = m == 0 ? b[0] : cmul(b[m], twb[m]);
          __syncwarp();
          float2 e[8];
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) e[k1] = myscr[ipos(n2, k1)];
          dft_reg<8, true>(e);
          float2 keep[8];
#pragma unroll
          for (int n1 = 0; n1 < 8; ++n1) {
            const float2 v = cmulc(e[n1], w32[n1]);
            const float2 v1 = rot_i(v, p);
            const float2 send = (p & 1) ? v : v1;
            const float2 mine = (p & 1) ? v1 : v;
            const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, send.x, R2),
                                           __shfl_xor_sync(0xffffffffu, send.y, R2));
            keep[n1] = cadd(mine, got);
          }
          const int h = p & 1, hi = p >> 1;
          const int s_out = sn2 ^ swz<N>(R2 * 4 * hi + M * h);
#pragma unroll
          for (int j4 = 0; j4 < 4; ++j4) {
            const float2 send = hi ? keep[j4] : keep[4 + j4];
            const float2 mine = hi ? keep[4 + j4] : keep[j4];
            const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 2 * R2),
                                           __shfl_xor_sync(0xffffffffu, send.y, 2 * R2));
            const int x = n2 + R2 * (4 * hi + j4) + M * h;
            plane[x * M + (c ^ s_out ^ swz<N>(R2 * j4))] = cadd(mine, got);
          }
          __syncwarp();
        }
      }
      if constexpr (XM == 1) {
        // 64-point inverses of the four folded columns: lane (jz, tz) holds
        // Z[tz + 8 u]; out[mu1 + 8 mu2] for mu2 < 4 is the value at x = 4 (mu1 + 8 mu2) + r0
        float2 a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = zc[tz + 8 * u];
        __syncwarp();
        dft_reg<8, true>(a);
#pragma unroll
        for (int mu1 = 1; mu1 < 8; ++mu1) a[mu1] = cmulc(a[mu1], tw[(4 * tz * mu1) & (2 * N - 1)]);
#pragma unroll
        for (int mu1 = 0; mu1 < 8; ++mu1) zc[8 * mu1 + (tz ^ mu1)] = a[mu1];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 8; ++t) a[t] = zc[8 * tz + (t ^ tz)];
        __syncwarp();
        dft_reg<8, true>(a);
        const int c = warp + C::WARPS * (4 * g + jz);
#pragma unroll
        for (int mu2 = 0; mu2 < 4; ++mu2) {
          const int x = 4 * (tz + 8 * mu2) + r0;
          plane[x * M + (c ^ swz<N>(x))] = a[mu2];
        }
      }
    }
  }
}

template <int N, int XM>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(256, 2)
    k_conv4(const float2* __restrict__ Sin, int in_pitch, const int32_t* __restrict__ in_cols, int in_n,
            float2* __restrict__ Sout, int out_pitch, const int32_t* __restrict__ out_cols, int out_n,
            const float2* __restrict__ H, int adj, const float2* __restrict__ twg, int r0, int ry) {
  using C = C4<N>;
  constexpr int M = C::M, ROWS = C::ROWS, SP = C::SP;
  extern __shared__ float4 smem_f4[];
  float2* plane = reinterpret_cast<float2*>(smem_f4);  // [N][M], swizzled rows
  float2* region = plane + N * M;                      // stage [ROWS][SP]; later the x scratch
  float2* tw = region + C::REGION;                     // [2N]: exp(-2 pi i e / 2N)
  int* rowin = reinterpret_cast<int*>(tw + 2 * N);     // rows holding input samples
  int* rowout = rowin + N;                             // rows holding output samples
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int kt = blockIdx.x >> 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = q * ROWS;

  for (int i = tid; i < 2 * N; i += C::THREADS) tw[i] = __ldg(twg + i);
  for (int i = tid; i < N; i += C::THREADS) {
    rowin[i] = in_cols ? 0 : 1;
    rowout[i] = out_cols ? 0 : 1;
  }
  __syncthreads();
  if (in_cols)
    for (int j = tid; j < in_n; j += C::THREADS) rowin[__ldg(in_cols + j) / N] = 1;
  if (out_cols)
    for (int j = tid; j < out_n; j += C::THREADS) rowout[__ldg(out_cols + j) / N] = 1;

  // 1-2. forward y transform.  A dense input plane is read straight from
  // global memory (each row by the four CTAs, the three later reads mostly
  // L2 hits); a compact one (sampled columns) is first scattered, a quarter
  // of the rows per CTA, into the staging buffers and read from there
  // through distributed shared memory.
  const float2* src = Sin + (size_t)kt * in_pitch;
  const float2* stage[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) stage[r] = cluster.map_shared_rank(region, r);
  const float2* gsrc = nullptr;
  const float2* csrc = nullptr;  // full lattice: compact rows read in place
  if (in_cols == nullptr) {
    gsrc = src;
    __syncthreads();
  } else if (XM == 2 && ry >= 0) {
    csrc = src;
    __syncthreads();
  } else {
    for (int i = tid; i < ROWS * SP; i += C::THREADS) region[i] = make_float2(0.f, 0.f);
    __syncthreads();
    batched_copy<4, float2>(
        in_n, tid, C::THREADS, [&](int j) { return __ldg(src + j); },
        [&](int j, float2 v) {
          const int col = __ldg(in_cols + j), x = col / N;
          if (x >= x0 && x < x0 + ROWS) region[(x - x0) * SP + col % N] = v;
        });
    cluster.sync();
  }
  switch (q) {
    case 0: c4_yfwd<N, 0, XM == 2>(plane, stage, gsrc, csrc, ry, tw, rowin, r0, warp, lane); break;
    case 1: c4_yfwd<N, 1, XM == 2>(plane, stage, gsrc, csrc, ry, tw, rowin, r0, warp, lane); break;
    case 2: c4_yfwd<N, 2, XM == 2>(plane, stage, gsrc, csrc, ry, tw, rowin, r0, warp, lane); break;
    default: c4_yfwd<N, 3, XM == 2>(plane, stage, gsrc, csrc, ry, tw, rowin, r0, warp, lane); break;
  }
  if (in_cols == nullptr || csrc)
    __syncthreads();  // plane complete
  else
    cluster.sync();   // plane complete; no CTA reads the staging buffers any more

  // 3. x convolution
  const float2* Hk = H + (size_t)kt * (N + 1) * (N + 1);
  c4_xconv<N, XM>(plane, region + warp * C::WSCR, region + C::WARPS * C::WSCR + warp * C::ZB, tw, Hk, q, adj, r0,
                  warp, lane);
  __syncthreads();

  // 4. inverse y transform
  switch (q) {
    case 0: c4_yinv<N, 0, XM == 1>(plane, tw, rowout, r0, warp, lane); break;
    case 1: c4_yinv<N, 1, XM == 1>(plane, tw, rowout, r0, warp, lane); break;
    case 2: c4_yinv<N, 2, XM == 1>(plane, tw, rowout, r0, warp, lane); break;
    default: c4_yinv<N, 3, XM == 1>(plane, tw, rowout, r0, warp, lane); break;
  }
  cluster.sync();

  // 5. out[x][n + M h] = s sum_r i^(r h) P_r[x][n] over the four CTAs' planes
  const float2* pr[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) pr[r] = cluster.map_shared_rank(plane, r);
  const float s = 1.0f / (4.0f * N * N);
  float2* dst = Sout + (size_t)kt * out_pitch;
  if (out_cols == nullptr) {
    constexpr int ITEMS = ROWS * M, U = 4;
    static_assert(ITEMS % (U * C::THREADS) == 0 || ITEMS < U * C::THREADS, "combine unroll");
    for (int i0 = tid; i0 < ITEMS; i0 += U * C::THREADS) {
      float2 v[U][4];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * C::THREADS;
        if (i < ITEMS) {
          const int x = x0 + i / M, n = i % M;
          const int a = x * M + (n ^ swz<N>(x));
#pragma unroll
          for (int r = 0; r < 4; ++r) v[u][r] = pr[r][a];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * C::THREADS;
        if (i < ITEMS) {
          const int x = x0 + i / M, n = i % M;
          const float2 e02 = cadd(v[u][0], v[u][2]), d02 = csub(v[u][0], v[u][2]);
          const float2 e13 = cadd(v[u][1], v[u][3]), d13 = csub(v[u][1], v[u][3]);
          // h = 0: v0 + v1 + v2 + v3; h = 1: v0 + i v1 - v2 - i v3
          dst[x * N + n] = cscale(cadd(e02, e13), s);
          dst[x * N + n + M] = cscale(make_float2(d02.x - d13.y, d02.y + d13.x), s);
        }
      }
    }
  } else {
    for (int j = tid; j < out_n; j += C::THREADS) {
      const int col = __ldg(out_cols + j), x = col / N;
      if (x < x0 || x >= x0 + ROWS) continue;
      const int y = col % N, n = y % M, h = y / M;
      const int a = x * M + (n ^ swz<N>(x));
      const float2 v0 = pr[0][a], v1 = pr[1][a], v2 = pr[2][a], v3 = pr[3][a];
      float2 o;
      if (h == 0) {
        o = cadd(cadd(v0, v2), cadd(v1, v3));
      } else {
        const float2 d02 = csub(v0, v2), d13 = csub(v1, v3);
        o = make_float2(d02.x - d13.y, d02.y + d13.x);
      }
      dst[j] = cscale(o, s);
    }
  }
  cluster.sync();  // keep this CTA's plane alive until the others have read it
}

size_t conv4_smem_bytes(int n) {
  switch (n) {
    case 32: return C4<32>::smem;
    case 64: return C4<64>::smem;
    case 128: return C4<128>::smem;
  }
  return 0;
}

nlos_status prepare_conv4(int n) {
  switch (n) {
    case 32: return ensure_smem(k_conv4<32, 0>, C4<32>::smem);
    case 64: return ensure_smem(k_conv4<64, 0>, C4<64>::smem);
    case 128:
      NLOS_TRY(ensure_smem(k_conv4<128, 1>, C4<128>::smem));
      NLOS_TRY(ensure_smem(k_conv4<128, 2>, C4<128>::smem));
      return ensure_smem(k_conv4<128, 0>, C4<128>::smem);
  }
  return NLOS_OK;
}

nlos_status launch_conv4(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact, bool adj,
                         cudaStream_t st) {
  const int full = P.nx * P.ny;
  const int in_pitch = in_compact ? P.ncols : full, out_pitch = out_compact ? P.ncols : full;
  if ((reinterpret_cast<uintptr_t>(Sin) & 7) != 0 || (reinterpret_cast<uintptr_t>(Sout) & 7) != 0)
    return fail(NLOS_ERR_INVALID_ARG, "conv4: spectra must be 8-byte aligned");
  auto go = [&](auto kern, size_t smem) -> nlos_status {
    NLOS_TRY(ensure_smem(kern, smem));
    kern<<<4 * (P.nt + 1), 256, smem, st>>>(Sin, in_pitch, in_compact ? P.d_cols : nullptr, P.ncols, Sout,
                                            out_pitch, out_compact ? P.d_cols : nullptr, P.ncols, P.d_H,
                                            adj ? 1 : 0, P.d_twx, P.lattice_rx, P.lattice_ry);
    NLOS_LAUNCH_CHECK("k_conv4");
    return NLOS_OK;
  };
  switch (P.nx) {
    case 32: return go(k_conv4<32, 0>, C4<32>::smem);
    case 64: return go(k_conv4<64, 0>, C4<64>::smem);
    case 128:
      // sampled rows on one residue class mod 4: fold the x work to the lattice
      if (P.lattice_rx >= 0 && out_compact && !in_compact) return go(k_conv4<128, 1>, C4<128>::smem);
      if (P.lattice_rx >= 0 && in_compact && !out_compact) return go(k_conv4<128, 2>, C4<128>::smem);
      return go(k_conv4<128, 0>, C4<128>::smem);
  }
  return fail(NLOS_ERR_INVALID_ARG, "conv4: unsupported nx");
}

}  // namespace nlos
