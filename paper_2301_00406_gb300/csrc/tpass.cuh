// Per-column t-passes of the LCT operator and of the periodic solve (see
// lct.cu for the factorisation).  The kernels are templates on the number of
// time bins; TpassOps<NT> holds the launchers of one size and is explicitly
// instantiated in one translation unit per size so the build runs in parallel.
#pragma once

#include <type_traits>

#include "fft.cuh"
#include "passes.cuh"

namespace nlos {

template <int NT>
struct TpassOps {
  static nlos_status tfwd_rz(const Plan& P, const float* u, int ncols, float2* S, int pitch, cudaStream_t st);
  static nlos_status tfwd_rtt(const Plan& P, const Lin3& r, int ncols, float2* S, int pitch, cudaStream_t st);
  static nlos_status tinv_store(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                                const int32_t* outmap, cudaStream_t st);
  static nlos_status tinv_fit(const Plan& P, const float2* S, int pitch, int ncols, float* out, const FitArgs& fa,
                              int* nblocks, cudaStream_t st);
  static nlos_status tadj_store(const Plan& P, const float2* S, int pitch, int ncols, float* out, cudaStream_t st);
  static nlos_status tadj_solve(const Plan& P, const float2* S, int pitch, int ncols, const SolveRhs& sr, float2* Sp,
                                cudaStream_t st);
  static nlos_status sfwd(const Plan& P, const float* x, const float* x2, int ncols, float2* Sp, cudaStream_t st);
  static nlos_status sinv(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref, double* partials,
                          int* nblocks, cudaStream_t st);
  static nlos_status sinv_rz(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref,
                             double* partials, int* nblocks, float2* S, int pitch, cudaStream_t st);
  // Raise every t-pass kernel's shared-memory limit to its largest launch
  // shape (so no attribute call happens later, e.g. during a stream capture).
  static nlos_status prepare();
};

#ifdef NLOS_TPASS_IMPL

// ---------------------------------------------------------------------------
// t-pass geometry
// ---------------------------------------------------------------------------
template <int NT>
struct TP {
  static constexpr int COLS = NT >= 1024 ? 8 : 16;  // columns per CTA (heuristic default)
  static constexpr int PAIRS = COLS / 2;
};

// Shared-memory layout of the packed pair transforms ("work"): element e of
// transform p sits at p * pitch + swz(e), where swz XORs a linear function of
// e's bits 4 and up into its low four bits (the float2 bank slot) and the
// pitch NT + pad depends on the number of transforms per CTA.  The constants
// come from a bank model of the access patterns of the shared-memory FFT steps
// (lanes over transforms and over stride-R positions): with them a warp's
// accesses need at most two wavefronts per half-warp where the plain odd pitch
// needed up to eight.
template <int NT>
struct WLay;
#define NLOS_WLAY(NTV, NBV, C0, C1, C2, C3, C4, C5, P1V, P2V, P4V, P8V)                                          \
  template <>                                                                                                      \
  struct WLay<NTV> {                                                                                               \
    static constexpr int NB = NBV, P1 = P1V, P2 = P2V, P4 = P4V, P8 = P8V;                                        \
    __host__ __device__ static constexpr int L(int i) {                                                            \
      return i == 0 ? C0 : i == 1 ? C1 : i == 2 ? C2 : i == 3 ? C3 : i == 4 ? C4 : C5;                             \
    }                                                                                                              \
  };
NLOS_WLAY(16, 0, 0, 0, 0, 0, 0, 0, 2, 6, 5, 6)
NLOS_WLAY(32, 1, 1, 0, 0, 0, 0, 0, 1, 6, 3, 6)
NLOS_WLAY(64, 2, 2, 4, 0, 0, 0, 0, 1, 8, 12, 2)
NLOS_WLAY(128, 3, 7, 12, 6, 0, 0, 0, 0, 8, 2, 6)
NLOS_WLAY(256, 4, 3, 13, 11, 4, 0, 0, 12, 8, 3, 6)
NLOS_WLAY(512, 5, 13, 6, 10, 2, 3, 0, 2, 8, 4, 2)
NLOS_WLAY(1024, 6, 10, 13, 11, 12, 4, 9, 4, 8, 12, 6)
#undef NLOS_WLAY

template <int NT>
__host__ __device__ constexpr int work_pitch(int pairs) {
  return NT + (pairs >= 8 ? WLay<NT>::P8 : pairs == 4 ? WLay<NT>::P4 : pairs == 2 ? WLay<NT>::P2 : WLay<NT>::P1);
}
template <int NT>
__device__ __forceinline__ int work_swz(int e) {
  int v = e;
#pragma unroll
  for (int i = 0; i < WLay<NT>::NB; ++i)
    if ((e >> (4 + i)) & 1) v ^= WLay<NT>::L(i);
  return v;
}
template <int NT>
struct WorkAddr {
  int pitch;
  __device__ __forceinline__ int operator()(int p, int e) const { return p * pitch + work_swz<NT>(e); }
  // e = er + ec with disjoint bits: the swizzle is linear over GF(2) (an XOR
  // of fixed masks selected by e's bits), so swz(er | ec) = swz(er) ^ swz(ec)
  // and swz(ec) folds to a constant for a compile-time ec.
  __device__ __forceinline__ int operator()(int p, int er, int ec) const {
    return p * pitch + (work_swz<NT>(er) ^ work_swz<NT>(ec));
  }
  // Element n of transform p in a loop whose index advances by the thread
  // count (256): n's low eight bits stay those of the thread, whose part of
  // the swizzle (slo = swz_lo(tid)) is computed once; only n's higher bits
  // are swizzled per element.
  __device__ __forceinline__ int at(int p, int n, int slo) const {
    return p * pitch + (slo ^ work_swz<NT>(n & ~255));
  }
};
template <int NT>
__device__ __forceinline__ int swz_lo(int tid) {
  return work_swz<NT>(tid & ((NT < 256 ? NT : 256) - 1));
}
constexpr int kTpassThreads = 256;

// Shared-memory table region (float4 slots): forward taps use nt slots; a CSR
// transpose uses ceil((nt + 1) / 4) slots of row pointers then nt slots of
// {weight, index} pairs.
template <int NT>
struct TabLayout {
  static constexpr int PTR4 = (NT + 4) / 4;
  static constexpr int SLOTS = NT + PTR4;
};

// Table staging: n 16-byte words from global to shared memory, eight loads in
// flight per thread (a plain strided loop waits for each load in turn, which
// dominates the short launches over the sampled columns).
__device__ __forceinline__ void stage16(float4* dst, const float4* __restrict__ src, int n, int tid, int nthr) {
  batched_copy<8, float4>(
      n, tid, nthr, [&](int i) { return __ldg(src + i); }, [&](int i, float4 v) { dst[i] = v; });
}
// The 2 nt roots exp(-2 pi i j / 2nt) in shared memory, one pad slot after
// every 16: root j at j + j / 16.  The FFT steps read roots at strided
// indices (multiples of 2, 16, 32 ... with lanes over transforms and
// sub-sequences); unpadded, those fall into a few float2 bank slots (up to
// 8-way conflicts), padded they spread over all 16.
// After the roots, fp[k] = the swizzled work position of frequency k
// (work_swz(fpos(k))), k < nt: the spectrum loads and the Hermitian split
// read one table entry per element instead of recomputing the digit
// reversal and the swizzle (integer arithmetic was the busiest pipe).
struct Tw2 {
  const float2* t;
  const int* fp;
  __device__ __forceinline__ float2 operator[](int j) const { return t[j + (j >> 4)]; }
};
template <int NT>
__host__ __device__ constexpr int tw2_slots() {
  // roots with pads, then nt ints (nt / 2 float2); a multiple of 2 float2, so
  // the next region stays 16-byte aligned
  return 2 * NT + (2 * NT) / 16 + NT / 2;
}
template <int NT>
__device__ __forceinline__ Tw2 stage_twiddles(float2* tw2, const float2* __restrict__ g, int tid, int nthr) {
  batched_copy<8, float2>(
      2 * NT, tid, nthr, [&](int j) { return __ldg(g + j); }, [&](int j, float2 v) { tw2[j + (j >> 4)] = v; });
  int* fp = reinterpret_cast<int*>(tw2 + 2 * NT + (2 * NT) / 16);
  for (int k = tid; k < NT; k += nthr) fp[k] = work_swz<NT>(fpos<NT>(k));
  return Tw2{tw2, fp};
}
template <int NT>
__device__ __forceinline__ void stage_fwd_taps(float4* tab, const float4* __restrict__ g, int tid, int nthr) {
  stage16(tab, g, NT, tid, nthr);
}
template <int NT>
__device__ __forceinline__ void stage_csr(float4* tab, const int32_t* __restrict__ ptr, const float2* __restrict__ ent,
                                          int tid, int nthr) {
  int* p = reinterpret_cast<int*>(tab);
  batched_copy<4, int>(
      NT + 1, tid, nthr, [&](int i) { return __ldg(ptr + i); }, [&](int i, int v) { p[i] = v; });
  stage16(tab + TabLayout<NT>::PTR4, reinterpret_cast<const float4*>(ent), NT, tid, nthr);
}
// sum over the CSR row n of w * x[index]
template <int NT>
__device__ __forceinline__ float2 csr_row2(const float4* tab, int n, const float* xa, const float* xb) {
  const int* p = reinterpret_cast<const int*>(tab);
  const float2* e = reinterpret_cast<const float2*>(tab + TabLayout<NT>::PTR4);
  float a = 0.f, b = 0.f;
  for (int q = p[n]; q < p[n + 1]; ++q) {
    const float2 w = e[q];
    const int k = __float_as_int(w.y);
    a += w.x * xa[k];
    b += w.x * xb[k];
  }
  return make_float2(a, b);
}



// The two columns (ca, ca + 1) of a pair from spectrum row `row`: one
// 16-byte load when both exist and the pair is 16-byte aligned (even pitch
// and even ca, base from cudaMalloc), else one or two 8-byte loads.
__device__ __forceinline__ void load_pair(const float2* __restrict__ row, int ca, int ncols, bool even_pitch,
                                          float2& A, float2& B) {
  if (even_pitch && ca + 1 < ncols) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row + ca));
    A = make_float2(v.x, v.y);
    B = make_float2(v.z, v.w);
  } else {
    A = ca < ncols ? __ldg(row + ca) : make_float2(0.f, 0.f);
    B = ca + 1 < ncols ? __ldg(row + ca + 1) : make_float2(0.f, 0.f);
  }
}

// Hermitian split of a packed pair transform at one bin (za at k, zb at the
// mirrored bin) into the bins of its two columns ca, ca + 1 of a spectrum row:
// one 16-byte store when both exist and the row is 16-byte aligned.
__device__ __forceinline__ void store_pair(float2* __restrict__ row, int ca, int ncols, bool even_pitch, float2 za,
                                           float2 zb) {
  const float2 xa = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
  const float2 xb = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
  if (even_pitch && ca + 1 < ncols) {
    *reinterpret_cast<float4*>(row + ca) = make_float4(xa.x, xa.y, xb.x, xb.y);
  } else {
    if (ca < ncols) row[ca] = xa;
    if (ca + 1 < ncols) row[ca + 1] = xb;
  }
}

// Post-processing of the padded forward t-FFT of packed pairs: writes bins
// kt = 2 k' + half of both columns of every pair to S, for the halves
// [h0, h0 + nh); the transform of pair p and half h is h * PAIRS + p when both
// halves are in `work` (nh = 2), else p.  One item per (bin, pair).
template <int NT>
__device__ __forceinline__ void tfwd_post_store(const float2* work, const WorkAddr<NT>& wa, const int* fp, int h0,
                                                int nh, float2* S, int pitch, int col0, int ncols, int COLS, int tid,
                                                int nthr) {
  const int PAIRS = COLS >> 1, lp = __ffs(PAIRS) - 1;  // PAIRS is a power of two
  const int n0 = (NT / 2 + 1 - h0) * PAIRS;              // items of the first half
  const int total = nh == 2 ? (NT + 1) * PAIRS : n0;
  const bool even_pitch = (pitch & 1) == 0;
  for (int i = tid; i < total; i += nthr) {
    const int half = i < n0 ? h0 : 1;
    const int j = i < n0 ? i : i - n0;
    const int kp = j >> lp, p = j & (PAIRS - 1);
    const int ca = col0 + 2 * p;
    if (ca >= ncols) continue;
    const int q = nh == 2 ? half * PAIRS + p : p;
    const int m = half ? (NT - 1 - kp) : ((NT - kp) & (NT - 1));
    const float2 za = work[q * wa.pitch + fp[kp]];
    const float2 zb = work[q * wa.pitch + fp[m]];
    store_pair(S + (size_t)(2 * kp + half) * pitch, ca, ncols, even_pitch, za, zb);
  }
}

// Loads the padded spectrum bins kt = 2 k' + half (k' in [0, nt)) of the CTA's
// column pairs into `work` in the permuted input order of the inverse FFT,
// using Hermitian symmetry for kt > nt, packed as Z = X_a + i X_b.
template <int NT>
__device__ __forceinline__ void tinv_load(const float2* __restrict__ S, int pitch, int col0, int ncols, int half,
                                          float2* work, const WorkAddr<NT>& wa, const int* fp, int q0, int PAIRS,
                                          int tid, int nthr) {
  const int lp = __ffs(PAIRS) - 1;
  batched_copy<8, float2>(
      NT * PAIRS, tid, nthr,
      [&](int i) {
        const int kp = i >> lp, p = i & (PAIRS - 1);
        int kt = 2 * kp + half;
        const bool mir = kt > NT;
        if (mir) kt = 2 * NT - kt;
        const int ca = col0 + 2 * p;
        float2 A, B;
        load_pair(S + (size_t)kt * pitch, ca, ncols, (pitch & 1) == 0, A, B);
        if (mir) {
          A.y = -A.y;
          B.y = -B.y;
        }
        return make_float2(A.x - B.y, A.y + B.x);
      },
      [&](int i, float2 z) { work[(q0 + (i & (PAIRS - 1))) * wa.pitch + fp[i >> lp]] = z; });
}

// Inverse padded t-FFT of the CTA's pairs: cbuf[c][n] = (1/(2nt)) * real signal
// of column c at n in [0, nt).  The even and odd bins (halves) are two
// length-nt transforms; with hb both run in one batched FFT of 2 PAIRS
// transforms (twice the parallelism, half the steps), else one after the
// other.
template <int NT>
__device__ __forceinline__ void tinv_core(const float2* __restrict__ S, int pitch, int col0, int ncols,
                                          float2* work, float* cbuf, const Tw2& tw2, int PAIRS, bool hb, int tid,
                                          int nthr) {
  const float scale = 1.0f / (2.0f * NT);
  if (hb) {
    const WorkAddr<NT> wa{work_pitch<NT>(2 * PAIRS)};
    tinv_load<NT>(S, pitch, col0, ncols, 0, work, wa, tw2.fp, 0, PAIRS, tid, nthr);
    tinv_load<NT>(S, pitch, col0, ncols, 1, work, wa, tw2.fp, PAIRS, PAIRS, tid, nthr);
    __syncthreads();
    team_fft_a<NT, true>(work, 2 * PAIRS, wa, tw2, 2, tid, nthr);
    const int slo = swz_lo<NT>(tid);
    for (int i = tid; i < PAIRS * NT; i += nthr) {
      const int p = i / NT, n = i % NT;
      const float2 z0 = work[wa.at(p, n, slo)];
      const float2 z1 = cmulc(work[wa.at(PAIRS + p, n, slo)], tw2[n]);
      float* ca = cbuf + (2 * p) * NT;
      ca[n] = (z0.x + z1.x) * scale;
      ca[n + NT] = (z0.y + z1.y) * scale;
    }
    __syncthreads();
    return;
  }
  const WorkAddr<NT> wa{work_pitch<NT>(PAIRS)};
  for (int half = 0; half < 2; ++half) {
    tinv_load<NT>(S, pitch, col0, ncols, half, work, wa, tw2.fp, 0, PAIRS, tid, nthr);
    __syncthreads();
    team_fft_a<NT, true>(work, PAIRS, wa, tw2, 2, tid, nthr);
    const int slo = swz_lo<NT>(tid);
    for (int i = tid; i < PAIRS * NT; i += nthr) {
      const int p = i / NT, n = i % NT;
      float2 z = work[wa.at(p, n, slo)];
      if (half) z = cmulc(z, tw2[n]);
      float* ca = cbuf + (2 * p) * NT;
      float* cb = ca + NT;
      if (half) {
        ca[n] = (ca[n] + z.x) * scale;
        cb[n] = (cb[n] + z.y) * scale;
      } else {
        ca[n] = z.x;
        cb[n] = z.y;
      }
    }
    __syncthreads();
  }
}

// The resampling and padded forward t-FFT of the CTA's real columns staged in
// cbuf (COLS columns of nt values, zero past the last column): R_z taps
// (MODE 0) or the R_t^{-T} CSR rows (MODE 1) from tab, then both halves of
// the padded transform, stored to S.  Starts and ends with every thread past
// a barrier.
template <int NT, int MODE>
__device__ __forceinline__ void tfwd_from_cbuf(const float* cbuf, const float4* tab, float2* work, const Tw2& tw2,
                                               int COLS, int hb, float2* __restrict__ S, int pitch, int col0,
                                               int ncols, int tid, int nthr) {
  const int PAIRS = COLS >> 1;
  const int NB = hb ? 2 * PAIRS : PAIRS;  // transforms per FFT call (both halves at once with hb)
  const WorkAddr<NT> wa{work_pitch<NT>(NB)};
  // the even output bins (half 0) are the length-nt DFT of z, the odd ones
  // (half 1) that of z w^n
  const int slo = swz_lo<NT>(tid);
  for (int h0 = 0; h0 < 2; h0 += hb ? 2 : 1) {
    for (int i = tid; i < PAIRS * NT; i += nthr) {
      const int p = i / NT, n = i % NT;
      const float* ca = cbuf + (2 * p) * NT;
      const float* cb = ca + NT;
      float2 z;
      if (MODE == 0) {
        // u~_n = (w0 g)_n u[i0_n] + (w1 g)_n u[i0_n + 1]
        const float4 t = tab[n];
        const int i0 = __float_as_int(t.z);
        z = make_float2(t.x * ca[i0] + t.y * ca[i0 + 1], t.x * cb[i0] + t.y * cb[i0 + 1]);
      } else {
        // c_n = sum over the t-bins k that interpolate v-bin n of (w wt)_k r_k
        z = csr_row2<NT>(tab, n, ca, cb);
      }
      if (hb) {
        work[wa.at(p, n, slo)] = z;
        work[wa.at(PAIRS + p, n, slo)] = cmul(z, tw2[n]);
      } else {
        work[wa.at(p, n, slo)] = h0 ? cmul(z, tw2[n]) : z;
      }
    }
    __syncthreads();
    team_fft_a<NT, false>(work, NB, wa, tw2, 2, tid, nthr);
    tfwd_post_store<NT>(work, wa, tw2.fp, h0, hb ? 2 : 1, S, pitch, col0, ncols, COLS, tid, nthr);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Forward t-pass: R_z (MODE 0) or R_t^{-T} of a residual (MODE 1), then the
// padded real FFT.
// ---------------------------------------------------------------------------
template <int NT, int MODE>
__global__ void __launch_bounds__(kTpassThreads)
    k_tfwd(Lin3 src, int ncols, float2* __restrict__ S, int pitch, const float4* __restrict__ ftab,
           const int32_t* __restrict__ tptr, const float2* __restrict__ tent, const float2* __restrict__ tw2g,
           int cols, int hb) {
  const int COLS = cols, PAIRS = cols >> 1;
  const int NB = hb ? 2 * PAIRS : PAIRS;
  extern __shared__ float4 smem_f4[];
  float2* tw2s = reinterpret_cast<float2*>(smem_f4);
  float4* tab = reinterpret_cast<float4*>(tw2s + tw2_slots<NT>());
  float2* work = reinterpret_cast<float2*>(tab + TabLayout<NT>::SLOTS);
  float* cbuf = reinterpret_cast<float*>(work + ((NB * work_pitch<NT>(NB) + 1) & ~1));
  const int tid = threadIdx.x;
  constexpr int nthr = kTpassThreads;  // every launch: strides fold at compile time
  const int col0 = blockIdx.x * COLS;
  const Tw2 tw2 = stage_twiddles<NT>(tw2s, tw2g, tid, nthr);
  if (MODE == 0)
    stage_fwd_taps<NT>(tab, ftab, tid, nthr);
  else
    stage_csr<NT>(tab, tptr, tent, tid, nthr);

  // stage the CTA's input columns in shared memory
  float c0 = src.c[0], c1 = src.c[1], c2 = src.c[2];
  if (src.sc) {
    const float b = (float)src.sc->beta_prev;
    c0 = 1.0f + b;
    c1 = -b;
    c2 = -1.0f;
  }
  batched_copy<4, float4>(
      COLS * NT / 4, tid, nthr,
      [&](int i) {
        const int c = (i * 4) / NT;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (col0 + c < ncols) {
          const size_t off = (size_t)col0 * NT / 4 + i;
          const float4 a = __ldg(reinterpret_cast<const float4*>(src.p[0]) + off);
          v = make_float4(c0 * a.x, c0 * a.y, c0 * a.z, c0 * a.w);
          if (src.p[1]) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(src.p[1]) + off);
            v.x += c1 * q.x; v.y += c1 * q.y; v.z += c1 * q.z; v.w += c1 * q.w;
          }
          if (src.p[2]) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(src.p[2]) + off);
            v.x += c2 * q.x; v.y += c2 * q.y; v.z += c2 * q.z; v.w += c2 * q.w;
          }
        }
        return v;
      },
      [&](int i, float4 v) { reinterpret_cast<float4*>(cbuf)[i] = v; });
  __syncthreads();

  tfwd_from_cbuf<NT, MODE>(cbuf, tab, work, tw2, COLS, hb, S, pitch, col0, ncols, tid, nthr);
}

// Hermitian split of the periodic forward FFT of the CTA's packed pairs:
// bins k <= nt / 2 of both columns of every pair, stored to Sp [k][column].
template <int NT>
__device__ __forceinline__ void periodic_fwd_post(const float2* work, const int* fp, float2* Sp, int col0, int ncols,
                                                  int pitch, int COLS, int tid, int nthr) {
  const int PAIRS = COLS >> 1;
  const WorkAddr<NT> wa{work_pitch<NT>(PAIRS)};
  const int lp = __ffs(PAIRS) - 1;  // PAIRS is a power of two
  const bool even_pitch = (pitch & 1) == 0;
  for (int i = tid; i < (NT / 2 + 1) * PAIRS; i += nthr) {
    const int k = i >> lp, p = i & (PAIRS - 1);
    const int ca = col0 + 2 * p;
    if (ca >= ncols) continue;
    const float2 za = work[p * wa.pitch + fp[k]];
    const float2 zb = work[p * wa.pitch + fp[(NT - k) & (NT - 1)]];
    store_pair(Sp + (size_t)k * pitch, ca, ncols, even_pitch, za, zb);
  }
}

// ---------------------------------------------------------------------------
// Forward t-inverse: C2R, crop, R_t^{-1}; store (EPI 0) or fit epilogue
// (EPI 1).  EPI 2 is the fit epilogue that also forms A u + fa.x2 in the
// packed-pair layout and runs its periodic forward FFT into fa.Sp (the
// tau-solve rhs of Algorithm 2).
// ---------------------------------------------------------------------------
template <int NT, int EPI>
__global__ void __launch_bounds__(kTpassThreads)
    k_tinv(const float2* __restrict__ S, int pitch, int ncols, float* __restrict__ out,
           const int32_t* __restrict__ outmap, FitArgs fa, const float4* __restrict__ ftab,
           const float2* __restrict__ tw2g, int cols, int hb) {
  const int COLS = cols, PAIRS = cols >> 1;
  const int NB = hb ? 2 * PAIRS : PAIRS;
  extern __shared__ float4 smem_f4[];
  float2* tw2s = reinterpret_cast<float2*>(smem_f4);
  float4* tab = reinterpret_cast<float4*>(tw2s + tw2_slots<NT>());
  float2* work = reinterpret_cast<float2*>(tab + TabLayout<NT>::SLOTS);
  float* cbuf = reinterpret_cast<float*>(work + ((NB * work_pitch<NT>(NB) + 1) & ~1));
  const int tid = threadIdx.x;
  constexpr int nthr = kTpassThreads;  // every launch: strides fold at compile time
  const int col0 = blockIdx.x * COLS;
  const Tw2 tw2 = stage_twiddles<NT>(tw2s, tw2g, tid, nthr);
  stage_fwd_taps<NT>(tab, ftab, tid, nthr);
  __syncthreads();
  tinv_core<NT>(S, pitch, col0, ncols, work, cbuf, tw2, PAIRS, hb != 0, tid, nthr);

  SumAcc<2> ca;
  float bp = 0.f;
  if (EPI >= 1) bp = (float)fa.sc->beta_prev;
  const int total4 = min(COLS, ncols - col0) * (NT / 4);
  // four consecutive bins of one column per item (16-byte loads and store;
  // nt is a multiple of 4 and every array 16-byte aligned).  ld: the data,
  // A u^k and A u^{k-1} samples (fit epilogue only); st: resample, store and
  // accumulate
  struct In4 {
    float4 d, a, b, x2;
  };
  constexpr bool fuse = EPI == 2;  // tau-solve rhs spectrum as well
  const WorkAddr<NT> wp{work_pitch<NT>(PAIRS)};    // layout of that periodic FFT
  batched_copy<2, In4>(
      total4, tid, nthr,
      [&](int i) {
        In4 v;
        if (EPI >= 1) {
          const size_t g4 = (size_t)col0 * (NT / 4) + i;
          v.d = __ldg(reinterpret_cast<const float4*>(fa.data) + g4);
          if (fa.need_d) {
            v.a = __ldg(reinterpret_cast<const float4*>(fa.auk) + g4);
            v.b = __ldg(reinterpret_cast<const float4*>(fa.aukm1) + g4);
          }
          if (fuse) v.x2 = __ldg(reinterpret_cast<const float4*>(fa.x2) + g4);
        }
        return v;
      },
      [&](int i, const In4& in) {
        const int c = i / (NT / 4), k = 4 * (i % (NT / 4));
        const float* cc = cbuf + c * NT;
        float tau[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 t = tab[k + e];
          const int k0 = __float_as_int(t.z);
          tau[e] = t.x * cc[k0] + t.y * cc[k0 + 1];
        }
        const int oc = outmap ? __ldg(outmap + col0 + c) : col0 + c;
        *reinterpret_cast<float4*>(out + (size_t)oc * NT + k) = make_float4(tau[0], tau[1], tau[2], tau[3]);
        if (EPI >= 1) {
          const float dd[4] = {in.d.x, in.d.y, in.d.z, in.d.w};
          const float aa[4] = {in.a.x, in.a.y, in.a.z, in.a.w};
          const float bb[4] = {in.b.x, in.b.y, in.b.z, in.b.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float r = tau[e] - dd[e];
            ca.add(0, r * r);
            if (fa.need_d) {
              const float d = tau[e] - ((1.0f + bp) * aa[e] - bp * bb[e]);
              ca.add(1, d * d);
            }
          }
          if (fuse) {
            // A u + x2 of column c into its packed pair (column 2p real, 2p + 1 imaginary)
            const float xx[4] = {in.x2.x, in.x2.y, in.x2.z, in.x2.w};
            float* wf = reinterpret_cast<float*>(work);
#pragma unroll
            for (int e = 0; e < 4; ++e) wf[2 * wp(c >> 1, k + e) + (c & 1)] = tau[e] + xx[e];
          }
        }
      });
  if (EPI >= 1) {
    block_reduce_acc(ca, fa.partials);
  }
  if (fuse) {
    // a missing partner column (ragged last CTA) transforms as zero
    const int valid = min(COLS, ncols - col0);
    if (valid & 1) {
      float* wf = reinterpret_cast<float*>(work);
      for (int n = tid; n < NT; n += nthr) wf[2 * wp(valid >> 1, n) + 1] = 0.0f;
    }
    __syncthreads();
    team_fft_a<NT, false>(work, PAIRS, wp, tw2, 2, tid, nthr);
    periodic_fwd_post<NT>(work, tw2.fp, fa.Sp, col0, ncols, ncols, COLS, tid, nthr);
  }
}

// ---------------------------------------------------------------------------
// Adjoint end: C2R, crop, R_z^T.  MODE 0 stores g; MODE 1 forms the solve
// right-hand side rhs = L u-bar - g + reg and runs the periodic real FFT.
// ---------------------------------------------------------------------------
template <int NT, int MODE>
__global__ void __launch_bounds__(kTpassThreads)
    k_tadj(const float2* __restrict__ S, int pitch, int ncols, float* __restrict__ out, SolveRhs sr,
           float2* __restrict__ Sp, const int32_t* __restrict__ tptr, const float2* __restrict__ tent,
           const float2* __restrict__ tw2g, int cols, int hb) {
  const int COLS = cols, PAIRS = cols >> 1;
  const int NB = hb ? 2 * PAIRS : PAIRS;
  const WorkAddr<NT> wa{work_pitch<NT>(PAIRS)};  // layout of the periodic forward FFT (MODE 1)
  extern __shared__ float4 smem_f4[];
  float2* tw2s = reinterpret_cast<float2*>(smem_f4);
  float4* tab = reinterpret_cast<float4*>(tw2s + tw2_slots<NT>());
  float2* work = reinterpret_cast<float2*>(tab + TabLayout<NT>::SLOTS);
  float* cbuf = reinterpret_cast<float*>(work + ((NB * work_pitch<NT>(NB) + 1) & ~1));
  const int tid = threadIdx.x;
  constexpr int nthr = kTpassThreads;  // every launch: strides fold at compile time
  const int col0 = blockIdx.x * COLS;
  const Tw2 tw2 = stage_twiddles<NT>(tw2s, tw2g, tid, nthr);
  stage_csr<NT>(tab, tptr, tent, tid, nthr);
  __syncthreads();
  tinv_core<NT>(S, pitch, col0, ncols, work, cbuf, tw2, PAIRS, hb != 0, tid, nthr);

  // g_i = sum over the v-bins j whose R_z taps touch rho-bin i of (w g)_j c_j,
  // gathered straight into the output (MODE 0) or into the solve rhs (MODE 1)
  if (MODE == 0) {
    for (int idx = tid; idx < PAIRS * NT; idx += nthr) {
      const int p = idx / NT, i = idx % NT;
      const int ca = col0 + 2 * p, cb = ca + 1;
      const float2 v = csr_row2<NT>(tab, i, cbuf + (2 * p) * NT, cbuf + (2 * p + 1) * NT);
      if (ca < ncols) out[(size_t)ca * NT + i] = v.x;
      if (cb < ncols) out[(size_t)cb * NT + i] = v.y;
    }
    return;
  }
  const float L = sr.sc ? (float)sr.sc->L : (float)sr.c0_host;
  // ld: u-bar and reg of both columns of the pair; st: rhs = L u-bar - g + reg
  const int slo = swz_lo<NT>(tid);
  batched_copy<8, float4>(
      PAIRS * NT, tid, nthr,
      [&](int i) {
        const int p = i / NT, n = i % NT;
        const int ca = col0 + 2 * p, cb = ca + 1;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ca < ncols) {
          const size_t g = (size_t)ca * NT + n;
          v.x = __ldg(sr.ubar + g);
          v.y = __ldg(sr.reg + g);
        }
        if (cb < ncols) {
          const size_t g = (size_t)cb * NT + n;
          v.z = __ldg(sr.ubar + g);
          v.w = __ldg(sr.reg + g);
        }
        return v;
      },
      [&](int i, float4 v) {
        const int p = i / NT, n = i % NT;
        const int ca = col0 + 2 * p, cb = ca + 1;
        const float2 gv = csr_row2<NT>(tab, n, cbuf + (2 * p) * NT, cbuf + (2 * p + 1) * NT);
        const float a = ca < ncols ? L * v.x - gv.x + v.y : 0.f;
        const float b = cb < ncols ? L * v.z - gv.y + v.w : 0.f;
        work[wa.at(p, n, slo)] = make_float2(a, b);
      });
  __syncthreads();
  team_fft_a<NT, false>(work, PAIRS, wa, tw2, 2, tid, nthr);
  periodic_fwd_post<NT>(work, tw2.fp, Sp, col0, ncols, ncols, COLS, tid, nthr);
}

// Periodic real FFT of a field (rhs of a solve): of x, or of x + x2 when x2
// is given.
template <int NT>
__global__ void __launch_bounds__(kTpassThreads)
    k_sfwd(const float* __restrict__ x, const float* __restrict__ x2, int ncols, float2* __restrict__ Sp,
           const float2* __restrict__ tw2g, int cols) {
  const int COLS = cols, PAIRS = cols >> 1;
  const WorkAddr<NT> wa{work_pitch<NT>(PAIRS)};
  extern __shared__ float4 smem_f4[];
  float2* tw2s = reinterpret_cast<float2*>(smem_f4);
  float2* work = tw2s + tw2_slots<NT>();
  const int tid = threadIdx.x;
  constexpr int nthr = kTpassThreads;  // every launch: strides fold at compile time
  const int col0 = blockIdx.x * COLS;
  const Tw2 tw2 = stage_twiddles<NT>(tw2s, tw2g, tid, nthr);
  const int slo = swz_lo<NT>(tid);
  batched_copy<8, float2>(
      PAIRS * NT, tid, nthr,
      [&](int i) {
        const int p = i / NT, n = i % NT;
        const int ca = col0 + 2 * p, cb = ca + 1;
        float2 z = make_float2(ca < ncols ? __ldg(x + (size_t)ca * NT + n) : 0.f,
                               cb < ncols ? __ldg(x + (size_t)cb * NT + n) : 0.f);
        if (x2) {
          if (ca < ncols) z.x += __ldg(x2 + (size_t)ca * NT + n);
          if (cb < ncols) z.y += __ldg(x2 + (size_t)cb * NT + n);
        }
        return z;
      },
      [&](int i, float2 z) { work[wa.at(i / NT, i % NT, slo)] = z; });
  __syncthreads();
  team_fft_a<NT, false>(work, PAIRS, wa, tw2, 2, tid, nthr);
  periodic_fwd_post<NT>(work, tw2.fp, Sp, col0, ncols, ncols, COLS, tid, nthr);
}

// Periodic inverse real FFT to a field; optional partial sums of (x - ref)^2.
template <int NT>
__global__ void __launch_bounds__(kTpassThreads)
    k_sinv(const float2* __restrict__ Sp, int ncols, float* __restrict__ x, const float* __restrict__ ref,
           double* __restrict__ partials, const float2* __restrict__ tw2g, int cols) {
  const int COLS = cols, PAIRS = cols >> 1;
  const WorkAddr<NT> wa{work_pitch<NT>(PAIRS)};
  extern __shared__ float4 smem_f4[];
  float2* tw2s = reinterpret_cast<float2*>(smem_f4);
  float2* work = tw2s + tw2_slots<NT>();
  const int tid = threadIdx.x;
  constexpr int nthr = kTpassThreads;  // every launch: strides fold at compile time
  const int col0 = blockIdx.x * COLS;
  const Tw2 tw2 = stage_twiddles<NT>(tw2s, tw2g, tid, nthr);
  __syncthreads();  // the position table is read by the load below
  const int lp = __ffs(PAIRS) - 1;
  batched_copy<8, float2>(
      NT * PAIRS, tid, nthr,
      [&](int i) {
        const int k = i >> lp, p = i & (PAIRS - 1);
        int kk = k;
        const bool mir = k > NT / 2;
        if (mir) kk = NT - k;
        const int ca = col0 + 2 * p;
        float2 A, B;
        load_pair(Sp + (size_t)kk * ncols, ca, ncols, (ncols & 1) == 0, A, B);
        if (mir) {
          A.y = -A.y;
          B.y = -B.y;
        }
        return make_float2(A.x - B.y, A.y + B.x);
      },
      [&](int i, float2 z) { work[(i & (PAIRS - 1)) * wa.pitch + tw2.fp[i >> lp]] = z; });
  __syncthreads();
  team_fft_a<NT, true>(work, PAIRS, wa, tw2, 2, tid, nthr);
  const float scale = 1.0f / NT;
  const int slo = swz_lo<NT>(tid);
  SumAcc<1> ca;
  const int total = min(COLS, ncols - col0) * NT;
  batched_copy<8, float>(
      total, tid, nthr, [&](int i) { return ref ? __ldg(ref + (size_t)col0 * NT + i) : 0.f; },
      [&](int i, float rv) {
        const int c = i / NT, n = i % NT;
        const float2 z = work[wa.at(c >> 1, n, slo)];
        const float v = ((c & 1) ? z.y : z.x) * scale;
        x[(size_t)col0 * NT + i] = v;
        if (ref) {
          const float d = v - rv;
          ca.add(0, d * d);
        }
      });
  if (partials) {
    block_reduce_acc(ca, partials);
  }
}


// Periodic inverse t-FFT fused with the forward t-pass of its result: the
// columns x = F_t^{-1}(Sp) (u+ of the u-step, with the partial sums of
// (x - ref)^2 as k_sinv) are written out and kept in shared memory, and R_z
// and the padded forward t-FFT of the same columns (k_tfwd, MODE 0) follow
// from there, so x is not read back from global memory.  The stored x and S
// equal those of k_sinv followed by k_tfwd bit for bit.
template <int NT>
__global__ void __launch_bounds__(kTpassThreads)
    k_sinv_rz(const float2* __restrict__ Sp, int ncols, float* __restrict__ x, const float* __restrict__ ref,
              double* __restrict__ partials, float2* __restrict__ S, int pitch, const float4* __restrict__ ftab,
              const float2* __restrict__ tw2g, int cols, int hb) {
  const int COLS = cols, PAIRS = cols >> 1;
  const int NB = hb ? 2 * PAIRS : PAIRS;
  const WorkAddr<NT> wa{work_pitch<NT>(PAIRS)};  // layout of the periodic inverse FFT
  extern __shared__ float4 smem_f4[];
  float2* tw2s = reinterpret_cast<float2*>(smem_f4);
  float4* tab = reinterpret_cast<float4*>(tw2s + tw2_slots<NT>());
  float2* work = reinterpret_cast<float2*>(tab + TabLayout<NT>::SLOTS);
  float* cbuf = reinterpret_cast<float*>(work + ((NB * work_pitch<NT>(NB) + 1) & ~1));
  const int tid = threadIdx.x;
  constexpr int nthr = kTpassThreads;  // every launch: strides fold at compile time
  const int col0 = blockIdx.x * COLS;
  const Tw2 tw2 = stage_twiddles<NT>(tw2s, tw2g, tid, nthr);
  stage_fwd_taps<NT>(tab, ftab, tid, nthr);
  __syncthreads();  // the position table is read by the load below
  const int lp = __ffs(PAIRS) - 1;
  batched_copy<8, float2>(
      NT * PAIRS, tid, nthr,
      [&](int i) {
        const int k = i >> lp, p = i & (PAIRS - 1);
        int kk = k;
        const bool mir = k > NT / 2;
        if (mir) kk = NT - k;
        const int ca = col0 + 2 * p;
        float2 A, B;
        load_pair(Sp + (size_t)kk * ncols, ca, ncols, (ncols & 1) == 0, A, B);
        if (mir) {
          A.y = -A.y;
          B.y = -B.y;
        }
        return make_float2(A.x - B.y, A.y + B.x);
      },
      [&](int i, float2 z) { work[(i & (PAIRS - 1)) * wa.pitch + tw2.fp[i >> lp]] = z; });
  __syncthreads();
  team_fft_a<NT, true>(work, PAIRS, wa, tw2, 2, tid, nthr);
  const float scale = 1.0f / NT;
  const int slo = swz_lo<NT>(tid);
  SumAcc<1> ca;
  const int total = min(COLS, ncols - col0) * NT;
  batched_copy<8, float>(
      total, tid, nthr, [&](int i) { return ref ? __ldg(ref + (size_t)col0 * NT + i) : 0.f; },
      [&](int i, float rv) {
        const int c = i / NT, n = i % NT;
        const float2 z = work[wa.at(c >> 1, n, slo)];
        const float v = ((c & 1) ? z.y : z.x) * scale;
        x[(size_t)col0 * NT + i] = v;
        cbuf[i] = v;
        if (ref) {
          const float d = v - rv;
          ca.add(0, d * d);
        }
      });
  for (int i = total + tid; i < COLS * NT; i += nthr) cbuf[i] = 0.f;  // columns past the last
  if (partials) {
    block_reduce_acc(ca, partials);
  }
  __syncthreads();
  tfwd_from_cbuf<NT, 0>(cbuf, tab, work, tw2, COLS, hb, S, pitch, col0, ncols, tid, nthr);
}

template <typename K>
static nlos_status set_smem_tp(K kernel, size_t bytes) {
  return ensure_smem(kernel, bytes);
}

// Launch shape of a t-pass: columns per CTA (fewer when there are few
// columns, e.g. the sampled columns of A_D, so the grid still covers the
// GPU), threads per CTA and dynamic shared memory (twiddles, the packed pair
// transforms, `extra` real column buffers).
// hb: both halves (even and odd bins of the padded transform) in one batched
// FFT, for the kernels that have two halves.
struct TpShape {
  int cols, hb, threads, blocks;
  size_t smem;
};

// Dynamic shared memory of a t-pass launch: twiddles, the work region
// (padded to an even number of float2 so the real column buffers after it
// stay 16-byte aligned for float4 accesses), the tap table, `extra` real
// column buffers.
template <int NT>
static size_t tp_smem(int cols, int hb, int extra, bool tab) {
  const int nb = hb ? cols : cols / 2;
  return sizeof(float2) * (tw2_slots<NT>() + ((nb * work_pitch<NT>(nb) + 1) & ~1)) +
         (tab ? sizeof(float4) * TabLayout<NT>::SLOTS : 0) + sizeof(float) * extra * cols * NT;
}

// Launch shape: the tuned (columns per CTA, hb) of this kind and column count
// (encoded cols | hb << 8), else the default rule (enough CTAs to cover the
// GPU twice, halves one after the other).
template <int NT>
static TpShape tp_shape(int ncols, int extra, bool tab, int kind, bool halves) {
  TpShape sh;
  const int tuned = kind >= 0 ? tp_cols_for(kind, NT, ncols) : 0;
  const int tc = tuned & 0xff;
  if (tc >= 2 && tc <= TP<NT>::COLS) {
    sh.cols = tc;
    sh.hb = halves ? (tuned >> 8) & 1 : 0;
  } else {
    sh.cols = TP<NT>::COLS;
    sh.hb = 0;
    while (sh.cols > 2 && div_up(ncols, sh.cols) < 2 * device_sm_count()) sh.cols >>= 1;
  }
  sh.threads = kTpassThreads;  // the kernels' loops assume this count
  sh.blocks = div_up(ncols, sh.cols);
  sh.smem = tp_smem<NT>(sh.cols, sh.hb, extra, tab);
  return sh;
}

template <int NT>
nlos_status TpassOps<NT>::tfwd_rz(const Plan& P, const float* u, int ncols, float2* S, int pitch, cudaStream_t st) {
  KTimer kt_(P, KC_TFWD, st);
  auto kern = k_tfwd<NT, 0>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_TFWD_RZ, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  Lin3 src{{u, nullptr, nullptr}, {1.f, 0.f, 0.f}, nullptr};
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(src, ncols, S, pitch, P.d_rz_f4, nullptr, nullptr, P.d_tw2t,
                                               sh.cols, sh.hb);
  NLOS_LAUNCH_CHECK("k_tfwd<rz>");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::tfwd_rtt(const Plan& P, const Lin3& r, int ncols, float2* S, int pitch, cudaStream_t st) {
  KTimer kt_(P, KC_TFWD, st);
  auto kern = k_tfwd<NT, 1>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_TFWD_RTT, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(r, ncols, S, pitch, nullptr, P.d_rtT_ptr, P.d_rtT_ent, P.d_tw2t,
                                               sh.cols, sh.hb);
  NLOS_LAUNCH_CHECK("k_tfwd<rtt>");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::tinv_store(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                                     const int32_t* outmap, cudaStream_t st) {
  KTimer kt_(P, KC_TINV, st);
  auto kern = k_tinv<NT, 0>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_TINV_STORE, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  FitArgs fa{};
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(S, pitch, ncols, out, outmap, fa, P.d_rt_f4, P.d_tw2t, sh.cols,
                                               sh.hb);
  NLOS_LAUNCH_CHECK("k_tinv<store>");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::tinv_fit(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                                   const FitArgs& fa, int* nblocks, cudaStream_t st) {
  KTimer kt_(P, KC_TINV, st);
  auto kern = fa.Sp ? k_tinv<NT, 2> : k_tinv<NT, 1>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_TINV_FIT, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  if (sh.blocks > P.partial_blocks) return fail(NLOS_ERR_INVALID_ARG, "partials buffer too small");
  *nblocks = sh.blocks;
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(S, pitch, ncols, out, nullptr, fa, P.d_rt_f4, P.d_tw2t, sh.cols,
                                               sh.hb);
  NLOS_LAUNCH_CHECK("k_tinv<fit>");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::tadj_store(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                                     cudaStream_t st) {
  KTimer kt_(P, KC_TADJ, st);
  auto kern = k_tadj<NT, 0>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_TADJ_STORE, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  SolveRhs sr{};
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(S, pitch, ncols, out, sr, nullptr, P.d_rzT_ptr, P.d_rzT_ent,
                                               P.d_tw2t, sh.cols, sh.hb);
  NLOS_LAUNCH_CHECK("k_tadj<store>");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::tadj_solve(const Plan& P, const float2* S, int pitch, int ncols, const SolveRhs& sr,
                                     float2* Sp, cudaStream_t st) {
  KTimer kt_(P, KC_TADJ, st);
  auto kern = k_tadj<NT, 1>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_TADJ_SOLVE, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(S, pitch, ncols, nullptr, sr, Sp, P.d_rzT_ptr, P.d_rzT_ent,
                                               P.d_tw2t, sh.cols, sh.hb);
  NLOS_LAUNCH_CHECK("k_tadj<solve>");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::sfwd(const Plan& P, const float* x, const float* x2, int ncols, float2* Sp,
                              cudaStream_t st) {
  KTimer kt_(P, KC_SFWD, st);
  auto kern = k_sfwd<NT>;
  const TpShape sh = tp_shape<NT>(ncols, 0, false, TPK_SFWD, false);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(x, x2, ncols, Sp, P.d_tw2t, sh.cols);
  NLOS_LAUNCH_CHECK("k_sfwd");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::sinv(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref,
                               double* partials, int* nblocks, cudaStream_t st) {
  KTimer kt_(P, KC_SINV, st);
  auto kern = k_sinv<NT>;
  const TpShape sh = tp_shape<NT>(ncols, 0, false, TPK_SINV, false);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  if (partials && sh.blocks > P.partial_blocks) return fail(NLOS_ERR_INVALID_ARG, "partials buffer too small");
  if (nblocks) *nblocks = sh.blocks;
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(Sp, ncols, x, ref, partials, P.d_tw2t, sh.cols);
  NLOS_LAUNCH_CHECK("k_sinv");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::sinv_rz(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref,
                                  double* partials, int* nblocks, float2* S, int pitch, cudaStream_t st) {
  KTimer kt_(P, KC_SINV, st);
  auto kern = k_sinv_rz<NT>;
  const TpShape sh = tp_shape<NT>(ncols, 1, true, TPK_SINV_RZ, true);
  NLOS_TRY(set_smem_tp(kern, sh.smem));
  if (partials && sh.blocks > P.partial_blocks) return fail(NLOS_ERR_INVALID_ARG, "partials buffer too small");
  if (nblocks) *nblocks = sh.blocks;
  kern<<<sh.blocks, sh.threads, sh.smem, st>>>(Sp, ncols, x, ref, partials, S, pitch, P.d_rz_f4, P.d_tw2t, sh.cols,
                                               sh.hb);
  NLOS_LAUNCH_CHECK("k_sinv_rz");
  return NLOS_OK;
}

template <int NT>
nlos_status TpassOps<NT>::prepare() {
  // largest shapes: the most columns per CTA, both halves batched
  const size_t m1 = tp_smem<NT>(TP<NT>::COLS, 1, 1, true), m0 = tp_smem<NT>(TP<NT>::COLS, 0, 0, false);
  NLOS_TRY(set_smem_tp(k_tfwd<NT, 0>, m1));
  NLOS_TRY(set_smem_tp(k_tfwd<NT, 1>, m1));
  NLOS_TRY(set_smem_tp(k_tinv<NT, 0>, m1));
  NLOS_TRY(set_smem_tp(k_tinv<NT, 1>, m1));
  NLOS_TRY(set_smem_tp(k_tinv<NT, 2>, m1));
  NLOS_TRY(set_smem_tp(k_tadj<NT, 0>, m1));
  NLOS_TRY(set_smem_tp(k_tadj<NT, 1>, m1));
  NLOS_TRY(set_smem_tp(k_sfwd<NT>, m0));
  NLOS_TRY(set_smem_tp(k_sinv<NT>, m0));
  NLOS_TRY(set_smem_tp(k_sinv_rz<NT>, m1));
  return NLOS_OK;
}

#endif  // NLOS_TPASS_IMPL

}  // namespace nlos
