// Full-grid t-passes of the iterations with one warp per column pair, for
// nt = 128, 256, 512: the adjoint end of A^T fused with the solve right-hand
// side (the tadj pass: inverse padded t-FFT, R_z^T, rhs = L u-bar - A^T r +
// reg, periodic t-FFT), the solve's inverse fused with the forward start of A
// (the sinv_rz pass: periodic inverse t-FFT to u+, R_z, padded t-FFT) or alone
// (the sinv pass), the end of A with the fit terms (the tinv pass: inverse
// padded t-FFT, R_t^{-1}, residual sums, and for Algorithm 2 the periodic
// t-FFT of the tau-solve right-hand side) and the start of A^T (the tfwd pass:
// residual, R_t^{-T}, padded t-FFT).
//
// Layout.  A CTA owns 16 consecutive columns (8 pairs, 8 warps).  The
// spectra are stored [bin][column] (float2), so the CTA's part of one bin is
// one 128-byte row segment; the CTA's whole spectrum tile (nt + 1 or nt/2 + 1
// rows) arrives in shared memory by TMA tile loads with the 128-byte swizzle
// (16-byte chunk c of row r at chunk c ^ (r mod 8)) and the output tile
// leaves by TMA tile stores from the same region.  The last row of each
// spectrum (bin nt or nt/2) moves by plain loads and stores, so the boxes
// stay a power of two high.  The real columns (u-bar, reg, u+) are stored
// [column][bin]; a warp reads and writes its two columns as 128-byte runs.
//
// Transforms.  Warp w transforms the packed pair z = x_{2w} + i x_{2w+1}.
// A length-N transform (N = 32 V) is held in registers, V values per lane,
// and factored as N = V x 32: a V-point register DFT over the stride-32
// elements of each lane, the twiddles w_N^(l k1), an exchange through the
// warp's shared scratch that gives each group of G = 32 / V lanes one of the
// V length-32 sequences, a V-point register DFT over the stride-G elements,
// the twiddles w_32^(g a), and a G-point DFT across the G lanes by shuffles
// (radix-2, decimation in frequency).  Input in natural order (lane l,
// register m: element l + 32 m) gives frequency k1 + V a + V^2 rev_G(g) in
// lane k1 G + g, register a (rev_G: bit reversal of log2 G bits); the
// inverse runs the same steps backwards with conjugate twiddles, from that
// order back to natural order (unnormalised).  The padded real transform of
// length 2N splits into the even and odd bins, two length-N transforms of
// z and z w_2N^n; the two real columns of a pair separate by Hermitian
// symmetry.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "fft.cuh"
#include "passes.cuh"
#include "tma.cuh"
#include "wfft.cuh"

namespace nlos {

namespace {

constexpr int kWarpThreads = 256;  // 8 warps: 8 column pairs, 16 columns per CTA
constexpr int kWarpCols = 16;

template <int V>
struct WP {
  static constexpr int N = 32 * V;                        // time bins
  static constexpr int G = 32 / V;                        // lanes per length-32 sequence
  static constexpr int XP = 32 + G;                       // scratch row pitch of the exchange (float2)
  static constexpr int SCR = V * XP > N + 16 ? V * XP : N + 16;  // scratch per warp (float2)
  static constexpr int BOX2 = N / 2 < 256 ? N / 2 : 256;  // rows of one parity per TMA box, padded spectrum
  static constexpr int BOXP = N / 2 < 256 ? N / 2 : 256;  // rows per TMA box, periodic spectrum
  static constexpr int TILE = ((N + 1) * 128 + 1023) / 1024 * 1024;
  static constexpr int OFF_TW1 = TILE;                    // [k1][l] w_N^(l k1)
  static constexpr int OFF_TWC = OFF_TW1 + 8 * N;         // [n] w_2N^n, n < N
  static constexpr int OFF_SCR = OFF_TWC + 8 * N;
  static constexpr int OFF_BAR = OFF_SCR + 8 * 8 * SCR;
  static constexpr int SMEM = OFF_BAR + 64 + 1024;        // + slack to align the base to 1024
  // R_z^T rows of the tadj pass, staged into the tile region behind the
  // output rows [0, N/2) once the input tile has been read
  static constexpr int OFF_RPTR = (N / 2) * 128;
  static constexpr int OFF_RENT = OFF_RPTR + ((N + 1) * 4 + 15) / 16 * 16;
  static_assert(OFF_RENT + 2 * N * 8 <= TILE, "R_z^T rows must fit behind the output rows");
};

// Byte offset of 16-byte chunk c of row r in a swizzled tile.
__device__ __forceinline__ int tile_off(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }
// Tile row of padded-spectrum bin kt: the even bins in rows [0, N/2), the odd
// bins in rows [N/2, N) (each half loaded or stored as one run of rows, so
// the bins 2k of consecutive k sit in consecutive rows), bin N in row N.
template <int N>
__device__ __forceinline__ int prow(int kt) {
  return kt == N ? N : (kt & 1) * (N / 2) + (kt >> 1);
}
// Scratch position of frequency k when a transform's output (the header's
// order) is written out in natural order: padded so that the 16 lanes of a
// half-warp, which hold frequencies k1 + V^2 rev(g), fall in distinct banks.
template <int V>
__device__ __forceinline__ int natp(int k) {
  constexpr int G = 32 / V;
  return k + ((k / (V * V)) % G) * (16 / G);
}

// Streaming load: read once, not kept in L1 (the tables read through L1 stay there).
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
// Asynchronous global -> shared copies (no registers); completed by cp_async_wait.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}
// Pulls a contiguous range (16-byte aligned, a multiple of 16 bytes) into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bin kt in [0, 2N) of the padded spectrum of the pair in chunk c of the
// tile (rows prow(0..N)), packed z = X_a + i X_b; bins above N by Hermitian
// symmetry of the real columns.
template <int N>
__device__ __forceinline__ float2 padded_bin(const unsigned char* tile, int kt, int c) {
  const bool mir = kt > N;
  const int r = prow<N>(mir ? 2 * N - kt : kt);
  const float4 v = *reinterpret_cast<const float4*>(tile + tile_off(r, c));
  const float ay = mir ? -v.y : v.y, by = mir ? -v.w : v.w;
  return make_float2(v.x - by, ay + v.z);
}
// Bin k in [0, N) of the periodic spectrum (rows 0..N/2), packed likewise.
template <int N>
__device__ __forceinline__ float2 periodic_bin(const unsigned char* tile, int k, int c) {
  const bool mir = k > N / 2;
  const int r = mir ? N - k : k;
  const float4 v = *reinterpret_cast<const float4*>(tile + tile_off(r, c));
  const float ay = mir ? -v.y : v.y, by = mir ? -v.w : v.w;
  return make_float2(v.x - by, ay + v.z);
}
// The bins of both real columns from the packed transform at k (za) and at
// the mirrored bin (zb): X_a = (za + conj zb) / 2, X_b = (za - conj zb) / 2i.
__device__ __forceinline__ float4 hermitian_split(float2 za, float2 zb) {
  return make_float4(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y), 0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
}

// Stage the twiddle tables of one CTA from the 2N roots w_2N^j (j < 2N).
template <int V>
__device__ __forceinline__ void stage_wtw(float2* tw1, float2* twc, const float2* __restrict__ tw2g, int tid) {
  constexpr int N = WP<V>::N;
  for (int i = tid; i < N; i += kWarpThreads) {
    tw1[i] = __ldg(tw2g + ((2 * (i & 31) * (i >> 5)) & (2 * N - 1)));
    twc[i] = __ldg(tw2g + i);
  }
}

// ---------------------------------------------------------------------------
// Stages shared by the kernels below.  Every one is called by all threads of
// the CTA (warp w: the pair in chunk w of the tiles, columns ca = col0 + 2 w
// and ca + 1), with the twiddle tables staged.
// ---------------------------------------------------------------------------
// Tile start: thread 0 initialises the load mbarrier and issues the TMA loads
// of `bytes` (the boxes are issued by `issue`); prefetches of the CTA's real
// columns into L2 may follow in `issue`.
template <typename Issue>
__device__ __forceinline__ void tile_load_start(uint32_t bar, uint32_t bytes, volatile int* fail, Issue issue) {
  if (threadIdx.x == 0) {
    *fail = 0;
    mbar_init(bar, 1);
    mbar_expect_tx(bar, bytes);
    issue();
  }
}
// The padded spectrum tile (rows prow(0..N-1) by TMA as two runs of row
// pairs, row N by plain loads).
template <int V>
__device__ __forceinline__ void padded_tile_load(uint32_t tile, uint32_t bar, const CUtensorMap* tm,
                                                 const float2* __restrict__ S, int pitch, int col0,
                                                 unsigned char* sm, volatile int* fail) {
  constexpr int N = WP<V>::N;
  tile_load_start(bar, N * 128, fail, [&] {
#pragma unroll 1
    for (int par = 0; par < 2; ++par)
      for (int r0 = 0; r0 < N / 2; r0 += WP<V>::BOX2)
        tma_load_3d(tile + (par * (N / 2) + r0) * 128, tm, 2 * col0, par, r0, bar);
  });
  if (threadIdx.x < 8) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(S + (size_t)N * pitch + col0) + threadIdx.x);
    *reinterpret_cast<float4*>(sm + tile_off(N, threadIdx.x)) = v;
  }
}
// Stores the CTA's output tile (padded spectrum: rows prow(0..N-1); periodic:
// rows 0..N/2-1) by TMA once every thread has written its rows, then waits.
template <int V, bool PADDED>
__device__ __forceinline__ void tile_store(uint32_t tile, const CUtensorMap* tm, int col0) {
  constexpr int N = WP<V>::N;
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (PADDED) {
#pragma unroll 1
      for (int par = 0; par < 2; ++par)
        for (int r0 = 0; r0 < N / 2; r0 += WP<V>::BOX2)
          tma_store_3d(tm, 2 * col0, par, r0, tile + (par * (N / 2) + r0) * 128);
    } else {
#pragma unroll 1
      for (int r0 = 0; r0 < N / 2; r0 += WP<V>::BOXP) tma_store_2d(tm, 2 * col0, r0, tile + r0 * 128);
    }
    bulk_commit();
  }
}
__device__ __forceinline__ void tile_store_wait() {
  if (threadIdx.x == 0) bulk_wait_all();
}

// Padded inverse of the pair's spectrum in the tile: the first N samples of
// the length-2N real inverse of both columns, c[n] = (even[n] + conj(w_2N^n)
// odd[n]) / 2N, left in natural order in the warp's scratch (scr[n], n < N).
// Ends with every warp past a CTA barrier after its tile reads (the tile
// region is free from there) and, when stage is given, with stage() issued
// right after that barrier.
template <int V, typename Stage>
__device__ __forceinline__ void padded_inverse_to_scratch(const unsigned char* sm, int warp, int lane, float2* scr,
                                                          const float2* tw1, const float2* twc, Stage stage) {
  constexpr int N = WP<V>::N, G = WP<V>::G;
  const int k1 = lane / G, gr = rev_bits<G>(lane % G);
  float2 e[V], o[V];
#pragma unroll
  for (int a = 0; a < V; ++a) {
    const int k = k1 + V * a + V * V * gr;
    e[a] = padded_bin<N>(sm, 2 * k, warp);
    o[a] = padded_bin<N>(sm, 2 * k + 1, warp);
  }
  __syncthreads();  // every pair is read: the tile region is free
  stage();
  wfft_inv<V>(e, scr, tw1, twc, lane);
  wfft_inv<V>(o, scr, tw1, twc, lane);
  const float scale = 1.0f / (2.0f * N);
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int n = lane + 32 * m;
    scr[n] = cscale(cadd(e[m], cmulc(o[m], twc[n])), scale);
  }
}

// Periodic forward transform of the pair r (natural order) and the bins
// k <= N/2 of both columns: rows k < N/2 of the tile (chunk warp), row N/2
// straight to Sp.
template <int V>
__device__ __forceinline__ void periodic_forward_to_tile(float2 (&r)[V], unsigned char* sm, int warp, int lane,
                                                         float2* scr, const float2* tw1, const float2* twc,
                                                         float2* __restrict__ Sp, int pitch, int ca) {
  constexpr int N = WP<V>::N, G = WP<V>::G;
  const int k1 = lane / G, gr = rev_bits<G>(lane % G);
  wfft_fwd<V>(r, scr, tw1, twc, lane);
#pragma unroll
  for (int a = 0; a < V; ++a) scr[natp<V>(k1 + V * a + V * V * gr)] = r[a];
  __syncwarp();
#pragma unroll
  for (int j = 0; j <= N / 64; ++j) {
    const int k = lane + 32 * j;
    if (k <= N / 2) {
      const float4 x = hermitian_split(scr[natp<V>(k)], scr[natp<V>((N - k) & (N - 1))]);
      if (k < N / 2)
        *reinterpret_cast<float4*>(sm + tile_off(k, warp)) = x;
      else
        *reinterpret_cast<float4*>(Sp + (size_t)k * pitch + ca) = x;
    }
  }
}

// Padded forward transform of the pair z (natural order, the first N samples
// of the zero-padded length-2N columns): even bins kt = 2k (k <= N/2) and odd
// bins kt = 2k + 1 (k < N/2) of both columns into tile rows prow(kt), bin N
// straight to S.
template <int V>
__device__ __forceinline__ void padded_forward_to_tile(float2 (&z)[V], unsigned char* sm, int warp, int lane,
                                                       float2* scr, const float2* tw1, const float2* twc,
                                                       float2* __restrict__ S, int pitch, int ca) {
  constexpr int N = WP<V>::N, G = WP<V>::G;
  const int k1 = lane / G, gr = rev_bits<G>(lane % G);
  float2 zo[V];
#pragma unroll
  for (int m = 0; m < V; ++m) zo[m] = cmul(z[m], twc[lane + 32 * m]);
  wfft_fwd<V>(z, scr, tw1, twc, lane);
#pragma unroll
  for (int a = 0; a < V; ++a) scr[natp<V>(k1 + V * a + V * V * gr)] = z[a];
  __syncwarp();
#pragma unroll
  for (int j = 0; j <= N / 64; ++j) {
    const int k = lane + 32 * j;
    if (k <= N / 2) {
      const float4 v = hermitian_split(scr[natp<V>(k)], scr[natp<V>((N - k) & (N - 1))]);
      if (k < N / 2)
        *reinterpret_cast<float4*>(sm + tile_off(k, warp)) = v;  // bin 2k
      else
        *reinterpret_cast<float4*>(S + (size_t)N * pitch + ca) = v;
    }
  }
  __syncwarp();
  wfft_fwd<V>(zo, scr, tw1, twc, lane);
#pragma unroll
  for (int a = 0; a < V; ++a) scr[natp<V>(k1 + V * a + V * V * gr)] = zo[a];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < N / 64; ++j) {
    const int k = lane + 32 * j;
    const float4 v = hermitian_split(scr[natp<V>(k)], scr[natp<V>(N - 1 - k)]);
    *reinterpret_cast<float4*>(sm + tile_off(N / 2 + k, warp)) = v;  // bin 2k + 1
  }
}

// ---------------------------------------------------------------------------
// tadj pass: S (padded spectrum of A^T's lateral output, full grid) ->
// rhs = c0 u-bar - R_z^T F^{-1} S + reg -> Sp (periodic spectrum of rhs).
// ---------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(kWarpThreads, 2)
    k_tadj_w(const __grid_constant__ CUtensorMap tm_s, const float2* __restrict__ S,
             const __grid_constant__ CUtensorMap tm_sp, float2* __restrict__ Sp, int pitch, SolveRhs sr,
             const int32_t* __restrict__ rptr, const float2* __restrict__ rent, const float2* __restrict__ tw2g,
             int32_t* status) {
  using W = WP<V>;
  constexpr int N = W::N;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int fail;
  unsigned char* sm = align1024(smem_raw);
  float2* tw1 = reinterpret_cast<float2*>(sm + W::OFF_TW1);
  float2* twc = reinterpret_cast<float2*>(sm + W::OFF_TWC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* scr = reinterpret_cast<float2*>(sm + W::OFF_SCR) + warp * W::SCR;
  const int col0 = blockIdx.x * kWarpCols;
  const uint32_t tile = smem_u32(sm), bar = smem_u32(sm + W::OFF_BAR);
  padded_tile_load<V>(tile, bar, &tm_s, S, pitch, col0, sm, &fail);
  if (tid == 0) {  // the CTA's u-bar and reg columns are read after the inverse transforms
    prefetch_l2(sr.ubar + (size_t)col0 * N, kWarpCols * N * 4);
    prefetch_l2(sr.reg + (size_t)col0 * N, kWarpCols * N * 4);
  }
  stage_wtw<V>(tw1, twc, tw2g, tid);
  const int ca = col0 + 2 * warp, cb = ca + 1;
  __syncthreads();
  mbar_wait_bounded(bar, 0, &fail, status);

  // c = first N samples of the padded inverse; meanwhile the R_z^T rows are
  // staged into the tile region behind the output rows [0, N/2)
  int* s_rptr = reinterpret_cast<int*>(sm + W::OFF_RPTR);
  float2* s_rent = reinterpret_cast<float2*>(sm + W::OFF_RENT);
  padded_inverse_to_scratch<V>(sm, warp, lane, scr, tw1, twc, [&] {
    for (int i = tid; i <= N; i += kWarpThreads) cp_async4(s_rptr + i, rptr + i);
    for (int i = tid; i < N; i += kWarpThreads) cp_async16(s_rent + 2 * i, rent + 2 * i);
  });
  cp_async_wait();
  __syncthreads();  // the R_z^T rows are staged; every warp's c is in its scratch

  // g = R_z^T c (CSR rows, the order of the rows' entries), rhs = c0 u-bar - g + reg
  const float c0 = sr.sc ? (float)sr.sc->L : (float)sr.c0_host;
  float2 r[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int i = lane + 32 * m;
    r[m] = make_float2(c0 * ld_stream(sr.ubar + (size_t)ca * N + i) + ld_stream(sr.reg + (size_t)ca * N + i),
                       c0 * ld_stream(sr.ubar + (size_t)cb * N + i) + ld_stream(sr.reg + (size_t)cb * N + i));
  }
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int i = lane + 32 * m;
    const int q0 = s_rptr[i], q1 = s_rptr[i + 1];
    float ga = 0.f, gb = 0.f;
    for (int q = q0; q < q1; ++q) {
      const float2 w = s_rent[q];
      const float2 c = scr[__float_as_int(w.y)];
      ga += w.x * c.x;
      gb += w.x * c.y;
    }
    r[m].x -= ga;
    r[m].y -= gb;
  }
  __syncwarp();
  periodic_forward_to_tile<V>(r, sm, warp, lane, scr, tw1, twc, Sp, pitch, ca);
  tile_store<V, false>(tile, &tm_sp, col0);
  tile_store_wait();
}

// ---------------------------------------------------------------------------
// Periodic inverse pass: Sp (periodic spectrum of a solution, full grid) ->
// x = F^{-1} Sp (stored; partial sums of (x - ref)^2).  RZ: then R_z x and
// its padded t-FFT into S (the forward start of A x; the sinv_rz pass).
// ---------------------------------------------------------------------------
template <int V, bool RZ>
__global__ void __launch_bounds__(kWarpThreads, 2)
    k_sinv_rz_w(const __grid_constant__ CUtensorMap tm_sp, const float2* __restrict__ Sp,
                const __grid_constant__ CUtensorMap tm_s, float2* __restrict__ S, int pitch, float* __restrict__ x,
                const float* __restrict__ ref, double* __restrict__ partials, const float4* __restrict__ ftab,
                const float2* __restrict__ tw2g, int32_t* status) {
  using W = WP<V>;
  constexpr int N = W::N, G = W::G;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int fail;
  unsigned char* sm = align1024(smem_raw);
  float2* tw1 = reinterpret_cast<float2*>(sm + W::OFF_TW1);
  float2* twc = reinterpret_cast<float2*>(sm + W::OFF_TWC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* scr = reinterpret_cast<float2*>(sm + W::OFF_SCR) + warp * W::SCR;
  const int col0 = blockIdx.x * kWarpCols;
  const uint32_t tile = smem_u32(sm), bar = smem_u32(sm + W::OFF_BAR);
  tile_load_start(bar, (N / 2) * 128, &fail, [&] {
#pragma unroll 1
    for (int r0 = 0; r0 < N / 2; r0 += W::BOXP) tma_load_2d(tile + r0 * 128, &tm_sp, 2 * col0, r0, bar);
    if (ref) prefetch_l2(ref + (size_t)col0 * N, kWarpCols * N * 4);
  });
  if (tid < 8) {  // row N/2 (the Nyquist bin)
    const float4 v = __ldg(reinterpret_cast<const float4*>(Sp + (size_t)(N / 2) * pitch + col0) + tid);
    *reinterpret_cast<float4*>(sm + tile_off(N / 2, tid)) = v;
  }
  stage_wtw<V>(tw1, twc, tw2g, tid);
  const int ca = col0 + 2 * warp, cb = ca + 1;
  __syncthreads();
  mbar_wait_bounded(bar, 0, &fail, status);

  const int k1 = lane / G, gr = rev_bits<G>(lane % G);
  float2 z[V];
#pragma unroll
  for (int a = 0; a < V; ++a) z[a] = periodic_bin<N>(sm, k1 + V * a + V * V * gr, warp);
  __syncthreads();  // every pair is read: the tile region now takes the output rows
  wfft_inv<V>(z, scr, tw1, twc, lane);

  // x of both columns, n = lane + 32 m: stored, summed against ref, and (RZ)
  // kept in the scratch for the R_z taps
  const float scale = 1.0f / N;
  SumAcc<1> acc;
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int n = lane + 32 * m;
    const float2 v = cscale(z[m], scale);
    x[(size_t)ca * N + n] = v.x;
    x[(size_t)cb * N + n] = v.y;
    if (ref) {
      const float da = v.x - ld_stream(ref + (size_t)ca * N + n), db = v.y - ld_stream(ref + (size_t)cb * N + n);
      acc.add(0, da * da);
      acc.add(0, db * db);
    }
    if (RZ) scr[n] = v;
  }
  if constexpr (RZ) {
    if (lane == 0) scr[N] = make_float2(0.f, 0.f);  // read with weight 0 by a last tap at i0 = N - 1
    __syncwarp();
    // u~_n = (w0 g)_n x[i0_n] + (w1 g)_n x[i0_n + 1]
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const float4 t = __ldg(ftab + lane + 32 * m);
      const int i0 = __float_as_int(t.z);
      const float2 u0 = scr[i0], u1 = scr[i0 + 1];
      z[m] = make_float2(t.x * u0.x + t.y * u1.x, t.x * u0.y + t.y * u1.y);
    }
    __syncwarp();
    padded_forward_to_tile<V>(z, sm, warp, lane, scr, tw1, twc, S, pitch, ca);
    tile_store<V, true>(tile, &tm_s, col0);
  }
  if (partials) block_reduce_acc(acc, partials);
  if (RZ) tile_store_wait();
}

// ---------------------------------------------------------------------------
// Fit pass (full grid): S (padded spectrum of A's lateral output) -> tau =
// R_t^{-1} F^{-1} S stored to out (A u), partial sums 0 = sum (tau - data)^2
// and (need_d) 1 = sum (tau - A u-bar)^2 with A u-bar = (1 + beta') A u^k -
// beta' A u^{k-1}; SPX: also the periodic spectrum of tau + x2 into Sp (the
// tau-solve right-hand side of Algorithm 2).
// ---------------------------------------------------------------------------
template <int V, bool SPX>
__global__ void __launch_bounds__(kWarpThreads, 2)
    k_tinv_fit_w(const __grid_constant__ CUtensorMap tm_s, const float2* __restrict__ S,
                 const __grid_constant__ CUtensorMap tm_sp, int pitch, float* __restrict__ out, FitArgs fa,
                 const float4* __restrict__ ftab, const float2* __restrict__ tw2g, int32_t* status) {
  using W = WP<V>;
  constexpr int N = W::N;
  extern __shared__ unsigned char smem_raw[];
  __shared__ int fail;
  unsigned char* sm = align1024(smem_raw);
  float2* tw1 = reinterpret_cast<float2*>(sm + W::OFF_TW1);
  float2* twc = reinterpret_cast<float2*>(sm + W::OFF_TWC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* scr = reinterpret_cast<float2*>(sm + W::OFF_SCR) + warp * W::SCR;
  const int col0 = blockIdx.x * kWarpCols;
  const uint32_t tile = smem_u32(sm), bar = smem_u32(sm + W::OFF_BAR);
  padded_tile_load<V>(tile, bar, &tm_s, S, pitch, col0, sm, &fail);
  if (tid == 0) {  // the CTA's columns of the fit inputs, read after the inverse transforms
    const size_t o = (size_t)col0 * N;
    prefetch_l2(fa.data + o, kWarpCols * N * 4);
    if (fa.need_d) {
      prefetch_l2(fa.auk + o, kWarpCols * N * 4);
      prefetch_l2(fa.aukm1 + o, kWarpCols * N * 4);
    }
    if (SPX) prefetch_l2(fa.x2 + o, kWarpCols * N * 4);
  }
  stage_wtw<V>(tw1, twc, tw2g, tid);
  const int ca = col0 + 2 * warp, cb = ca + 1;
  __syncthreads();
  mbar_wait_bounded(bar, 0, &fail, status);

  padded_inverse_to_scratch<V>(sm, warp, lane, scr, tw1, twc, [] {});
  if (lane == 0) scr[N] = make_float2(0.f, 0.f);  // read with weight 0 by a last tap at k0 = N - 1
  __syncwarp();
  // tau_n = (v0 wt)_n c[k0_n] + (v1 wt)_n c[k0_n + 1] of both columns
  const float bp = (float)fa.sc->beta_prev;
  SumAcc<2> acc;
  float2 z[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int n = lane + 32 * m;
    const float4 t = __ldg(ftab + n);
    const int k0 = __float_as_int(t.z);
    const float2 u0 = scr[k0], u1 = scr[k0 + 1];
    const float2 tau = make_float2(t.x * u0.x + t.y * u1.x, t.x * u0.y + t.y * u1.y);
    const size_t ga = (size_t)ca * N + n, gb = (size_t)cb * N + n;
    out[ga] = tau.x;
    out[gb] = tau.y;
    const float ra = tau.x - ld_stream(fa.data + ga), rb = tau.y - ld_stream(fa.data + gb);
    acc.add(0, ra * ra);
    acc.add(0, rb * rb);
    if (fa.need_d) {
      const float da = tau.x - ((1.0f + bp) * ld_stream(fa.auk + ga) - bp * ld_stream(fa.aukm1 + ga));
      const float db = tau.y - ((1.0f + bp) * ld_stream(fa.auk + gb) - bp * ld_stream(fa.aukm1 + gb));
      acc.add(1, da * da);
      acc.add(1, db * db);
    }
    if (SPX) z[m] = make_float2(tau.x + ld_stream(fa.x2 + ga), tau.y + ld_stream(fa.x2 + gb));
  }
  if constexpr (SPX) {
    __syncwarp();
    periodic_forward_to_tile<V>(z, sm, warp, lane, scr, tw1, twc, fa.Sp, pitch, ca);
    tile_store<V, false>(tile, &tm_sp, col0);
  }
  block_reduce_acc(acc, fa.partials);
  if (SPX) tile_store_wait();
}

// ---------------------------------------------------------------------------
// Residual pass (full grid): r = the Lin3 combination of up to three fields
// -> R_t^{-T} r (CSR rows) -> its padded t-FFT into S (the start of A^T r).
// ---------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(kWarpThreads, 2)
    k_tfwd_rtt_w(Lin3 src, const __grid_constant__ CUtensorMap tm_s, float2* __restrict__ S, int pitch,
                 const int32_t* __restrict__ tptr, const float2* __restrict__ tent,
                 const float2* __restrict__ tw2g) {
  using W = WP<V>;
  constexpr int N = W::N;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = align1024(smem_raw);
  float2* tw1 = reinterpret_cast<float2*>(sm + W::OFF_TW1);
  float2* twc = reinterpret_cast<float2*>(sm + W::OFF_TWC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* scr = reinterpret_cast<float2*>(sm + W::OFF_SCR) + warp * W::SCR;
  const int col0 = blockIdx.x * kWarpCols;
  const uint32_t tile = smem_u32(sm);
  // the R_t^{-T} rows go to the start of the (not yet used) tile region
  int* s_tptr = reinterpret_cast<int*>(sm);
  float2* s_tent = reinterpret_cast<float2*>(sm + ((N + 1) * 4 + 15) / 16 * 16);
  for (int i = tid; i <= N; i += kWarpThreads) cp_async4(s_tptr + i, tptr + i);
  for (int i = tid; i < N; i += kWarpThreads) cp_async16(s_tent + 2 * i, tent + 2 * i);
  stage_wtw<V>(tw1, twc, tw2g, tid);
  float c0 = src.c[0], c1 = src.c[1], c2 = src.c[2];
  if (src.sc) {
    const float b = (float)src.sc->beta_prev;
    c0 = 1.0f + b;
    c1 = -b;
    c2 = -1.0f;
  }
  const int ca = col0 + 2 * warp, cb = ca + 1;
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int n = lane + 32 * m;
    const size_t ga = (size_t)ca * N + n, gb = (size_t)cb * N + n;
    float2 v = make_float2(c0 * ld_stream(src.p[0] + ga), c0 * ld_stream(src.p[0] + gb));
    if (src.p[1]) {
      v.x += c1 * ld_stream(src.p[1] + ga);
      v.y += c1 * ld_stream(src.p[1] + gb);
    }
    if (src.p[2]) {
      v.x += c2 * ld_stream(src.p[2] + ga);
      v.y += c2 * ld_stream(src.p[2] + gb);
    }
    scr[n] = v;
  }
  cp_async_wait();
  __syncthreads();  // the R_t^{-T} rows and the twiddles are staged; every warp's r is in its scratch
  // c_n = sum over the t-bins k that interpolate v-bin n of (w wt)_k r_k
  float2 z[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int n = lane + 32 * m;
    const int q0 = s_tptr[n], q1 = s_tptr[n + 1];
    float a = 0.f, b = 0.f;
    for (int q = q0; q < q1; ++q) {
      const float2 w = s_tent[q];
      const float2 rv = scr[__float_as_int(w.y)];
      a += w.x * rv.x;
      b += w.x * rv.y;
    }
    z[m] = make_float2(a, b);
  }
  __syncthreads();  // every warp's rows are gathered: the tile region now takes the output rows
  padded_forward_to_tile<V>(z, sm, warp, lane, scr, tw1, twc, S, pitch, ca);
  tile_store<V, true>(tile, &tm_s, col0);
  tile_store_wait();
}

// Self-test of the bounded wait: an mbarrier that expects 128 transaction
// bytes which no copy delivers (nothing is issued, so nothing is in flight
// when the CTA exits); the wait gives up after limit_ns and records
// NLOS_ERR_TIMEOUT.
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int fail;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    fail = 0;
    *status = NLOS_OK;
    mbar_init(b, 1);
    mbar_expect_tx(b, 128);
  }
  __syncthreads();
  mbar_wait_bounded(b, 0, &fail, status, limit_ns);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

template <int V>
nlos_status tadj_solve_w(const Plan& P, const float2* S, int pitch, const SolveRhs& sr, float2* Sp,
                         cudaStream_t st) {
  using W = WP<V>;
  CUtensorMap ms, mp;
  NLOS_TRY(make_tmap_rowpairs(&ms, S, 2ull * pitch, W::N / 2, 8ull * pitch, 32, W::BOX2));
  NLOS_TRY(make_tmap_2d(&mp, Sp, 2ull * pitch, W::N / 2 + 1, 8ull * pitch, 32, W::BOXP));
  int32_t* status = sr.sc ? const_cast<int32_t*>(&sr.sc->status) : nullptr;
  KTimer kt_(P, KC_TADJ, st);
  k_tadj_w<V><<<pitch / kWarpCols, kWarpThreads, W::SMEM, st>>>(ms, S, mp, Sp, pitch, sr, P.d_rzT_ptr, P.d_rzT_ent,
                                                                 P.d_tw2t, status);
  NLOS_LAUNCH_CHECK("k_tadj_w");
  return NLOS_OK;
}

template <int V, bool RZ>
nlos_status sinv_rz_w(const Plan& P, const float2* Sp, int pitch, float* x, const float* ref, double* partials,
                      int* nblocks, float2* S, DevScalars* sc, cudaStream_t st) {
  using W = WP<V>;
  const int blocks = pitch / kWarpCols;
  if (partials && blocks > P.partial_blocks) return fail(NLOS_ERR_INVALID_ARG, "partials buffer too small");
  if (nblocks) *nblocks = blocks;
  CUtensorMap mp, ms;
  NLOS_TRY(make_tmap_2d(&mp, Sp, 2ull * pitch, W::N / 2 + 1, 8ull * pitch, 32, W::BOXP));
  if (RZ)
    NLOS_TRY(make_tmap_rowpairs(&ms, S, 2ull * pitch, W::N / 2, 8ull * pitch, 32, W::BOX2));
  else
    ms = mp;  // not read
  KTimer kt_(P, KC_SINV, st);
  k_sinv_rz_w<V, RZ><<<blocks, kWarpThreads, W::SMEM, st>>>(mp, Sp, ms, S, pitch, x, ref, partials, P.d_rz_f4,
                                                             P.d_tw2t, sc ? &sc->status : nullptr);
  NLOS_LAUNCH_CHECK("k_sinv_rz_w");
  return NLOS_OK;
}

template <int V>
nlos_status tinv_fit_w(const Plan& P, const float2* S, int pitch, float* out, const FitArgs& fa, int* nblocks,
                       cudaStream_t st) {
  using W = WP<V>;
  const int blocks = pitch / kWarpCols;
  if (blocks > P.partial_blocks) return fail(NLOS_ERR_INVALID_ARG, "partials buffer too small");
  *nblocks = blocks;
  CUtensorMap ms, mp;
  NLOS_TRY(make_tmap_rowpairs(&ms, S, 2ull * pitch, W::N / 2, 8ull * pitch, 32, W::BOX2));
  if (fa.Sp)
    NLOS_TRY(make_tmap_2d(&mp, fa.Sp, 2ull * pitch, W::N / 2 + 1, 8ull * pitch, 32, W::BOXP));
  else
    mp = ms;  // not read
  int32_t* status = fa.sc ? const_cast<int32_t*>(&fa.sc->status) : nullptr;
  KTimer kt_(P, KC_TINV, st);
  auto kern = fa.Sp ? k_tinv_fit_w<V, true> : k_tinv_fit_w<V, false>;
  kern<<<blocks, kWarpThreads, W::SMEM, st>>>(ms, S, mp, pitch, out, fa, P.d_rt_f4, P.d_tw2t, status);
  NLOS_LAUNCH_CHECK("k_tinv_fit_w");
  return NLOS_OK;
}

template <int V>
nlos_status tfwd_rtt_w(const Plan& P, const Lin3& r, float2* S, int pitch, cudaStream_t st) {
  using W = WP<V>;
  CUtensorMap ms;
  NLOS_TRY(make_tmap_rowpairs(&ms, S, 2ull * pitch, W::N / 2, 8ull * pitch, 32, W::BOX2));
  KTimer kt_(P, KC_TFWD, st);
  k_tfwd_rtt_w<V><<<pitch / kWarpCols, kWarpThreads, W::SMEM, st>>>(r, ms, S, pitch, P.d_rtT_ptr, P.d_rtT_ent,
                                                                     P.d_tw2t);
  NLOS_LAUNCH_CHECK("k_tfwd_rtt_w");
  return NLOS_OK;
}

template <int V>
nlos_status prepare_w() {
  NLOS_TRY(ensure_smem(k_tadj_w<V>, WP<V>::SMEM));
  NLOS_TRY(ensure_smem(k_sinv_rz_w<V, true>, WP<V>::SMEM));
  NLOS_TRY(ensure_smem(k_sinv_rz_w<V, false>, WP<V>::SMEM));
  NLOS_TRY(ensure_smem(k_tinv_fit_w<V, true>, WP<V>::SMEM));
  NLOS_TRY(ensure_smem(k_tinv_fit_w<V, false>, WP<V>::SMEM));
  NLOS_TRY(ensure_smem(k_tfwd_rtt_w<V>, WP<V>::SMEM));
  return NLOS_OK;
}

}  // namespace

nlos_status make_tmap_2d(CUtensorMap* map, const void* base, uint64_t row_floats, uint64_t rows,
                         uint64_t pitch_bytes, uint32_t box_x, uint32_t box_y) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn) return fail(NLOS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {row_floats, rows};
  const cuuint64_t strides[1] = {pitch_bytes};
  const cuuint32_t box[2] = {box_x, box_y};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(NLOS_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult " + std::to_string((int)r) + ")");
  return NLOS_OK;
}

nlos_status make_tmap_rowpairs(CUtensorMap* map, const void* base, uint64_t row_floats, uint64_t pairs,
                               uint64_t pitch_bytes, uint32_t box_x, uint32_t box_r) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn) return fail(NLOS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[3] = {row_floats, 2, pairs};
  const cuuint64_t strides[2] = {pitch_bytes, 2 * pitch_bytes};
  const cuuint32_t box[3] = {box_x, 1, box_r};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(NLOS_ERR_CUDA, "cuTensorMapEncodeTiled (row pairs) failed (CUresult " + std::to_string((int)r) + ")");
  return NLOS_OK;
}

bool tpass_warp_applies(const Plan& P, int ncols, int pitch) {
  return (P.nt == 128 || P.nt == 256 || P.nt == 512) && ncols == P.nx * P.ny && pitch == ncols &&
         ncols % kWarpCols == 0;
}

bool tpass_warp_applies_cols(const Plan& P, int ncols, int pitch) {
  return (P.nt == 128 || P.nt == 256 || P.nt == 512) && pitch == ncols && ncols % kWarpCols == 0;
}

nlos_status prepare_tpass_warp(int nt) {
  switch (nt) {
    case 128: return prepare_w<4>();
    case 256: return prepare_w<8>();
    case 512: return prepare_w<16>();
  }
  return NLOS_OK;
}

nlos_status launch_tadj_solve_warp(const Plan& P, const float2* S, int pitch, const SolveRhs& sr, float2* Sp,
                                   cudaStream_t st) {
  switch (P.nt) {
    case 128: return tadj_solve_w<4>(P, S, pitch, sr, Sp, st);
    case 256: return tadj_solve_w<8>(P, S, pitch, sr, Sp, st);
    case 512: return tadj_solve_w<16>(P, S, pitch, sr, Sp, st);
  }
  return fail(NLOS_ERR_INVALID_ARG, "warp t-pass: unsupported nt");
}

nlos_status launch_sinv_rz_warp(const Plan& P, const float2* Sp, int pitch, float* x, const float* ref,
                                double* partials, int* nblocks, float2* S, DevScalars* sc, cudaStream_t st) {
  switch (P.nt) {
    case 128: return sinv_rz_w<4, true>(P, Sp, pitch, x, ref, partials, nblocks, S, sc, st);
    case 256: return sinv_rz_w<8, true>(P, Sp, pitch, x, ref, partials, nblocks, S, sc, st);
    case 512: return sinv_rz_w<16, true>(P, Sp, pitch, x, ref, partials, nblocks, S, sc, st);
  }
  return fail(NLOS_ERR_INVALID_ARG, "warp t-pass: unsupported nt");
}

nlos_status launch_sinv_warp(const Plan& P, const float2* Sp, int pitch, float* x, const float* ref,
                             double* partials, int* nblocks, cudaStream_t st) {
  switch (P.nt) {
    case 128: return sinv_rz_w<4, false>(P, Sp, pitch, x, ref, partials, nblocks, nullptr, nullptr, st);
    case 256: return sinv_rz_w<8, false>(P, Sp, pitch, x, ref, partials, nblocks, nullptr, nullptr, st);
    case 512: return sinv_rz_w<16, false>(P, Sp, pitch, x, ref, partials, nblocks, nullptr, nullptr, st);
  }
  return fail(NLOS_ERR_INVALID_ARG, "warp t-pass: unsupported nt");
}

nlos_status launch_tinv_fit_warp(const Plan& P, const float2* S, int pitch, float* out, const FitArgs& fa,
                                 int* nblocks, cudaStream_t st) {
  switch (P.nt) {
    case 128: return tinv_fit_w<4>(P, S, pitch, out, fa, nblocks, st);
    case 256: return tinv_fit_w<8>(P, S, pitch, out, fa, nblocks, st);
    case 512: return tinv_fit_w<16>(P, S, pitch, out, fa, nblocks, st);
  }
  return fail(NLOS_ERR_INVALID_ARG, "warp t-pass: unsupported nt");
}

nlos_status launch_tfwd_rtt_warp(const Plan& P, const Lin3& r, float2* S, int pitch, cudaStream_t st) {
  switch (P.nt) {
    case 128: return tfwd_rtt_w<4>(P, r, S, pitch, st);
    case 256: return tfwd_rtt_w<8>(P, r, S, pitch, st);
    case 512: return tfwd_rtt_w<16>(P, r, S, pitch, st);
  }
  return fail(NLOS_ERR_INVALID_ARG, "warp t-pass: unsupported nt");
}

nlos_status selftest_wait_timeout(int32_t wait_ms, int32_t* status_dev, cudaStream_t st) {
  if (wait_ms < 1 || wait_ms > 5000 || !status_dev)
    return fail(NLOS_ERR_INVALID_ARG, "nlos_selftest_wait_timeout: wait_ms in [1, 5000] and a status pointer");
  k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)wait_ms * 1000000ull, status_dev);
  NLOS_LAUNCH_CHECK("k_wait_selftest");
  return NLOS_OK;
}

}  // namespace nlos
