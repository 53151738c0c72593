// Lateral convolution of the light-cone transform (the H of Eq. 3 and its
// conjugate in A^T, applied to every kt plane of the t-transformed volume) as
// DFT-matrix products on the fifth-generation tensor cores: tcgen05.mma with
// split-BF16 operands (hi + lo terms, products hi hi + hi lo + lo hi) and FP32
// accumulation in tensor memory, for nx = ny = 128.
//
// Per kt plane X[x][y] (128 x 128 complex, zero-padded to 256 x 256 by the
// convolution) with w = exp(-2 pi i / 256) and F[f][n] = w^(4 f n), the
// 64-point DFT matrix (f, n < 64):
//   * the padded y bins ky = 4 j + q' (q' = ky mod 4) are 64-point DFTs of
//     the row folded once: sum_n F[j][n] w^(q' n) (X[n] + (-i)^q' X[n + 64]);
//   * the padded x bins kx = 4 m + p likewise along x.  Because the y
//     transform acts on each row separately, the x fold and its twist
//     w^(p x0) are applied to the input rows before it, so the x transform
//     of the result is a plain F product;
//   * after the multiply by H (conj H for the adjoint) the inverse x
//     transform per parity, I_p[x0] = sum_m conj F[x0][m] W_p[m], recombines
//     as out[x0 + 64 t] = sum_p i^(p t) w^(-p x0) I_p[x0], and the inverse y
//     transform the same way over the four ky parities.
// Every product is (128 rows of data) x F: a complex 128 x 64 by 64 x 64
// product as one real MMA chain M = 128, N = 128, K = 128 against the block
// constant
//     B[f][n] = Fr[f][n],  B[f][64 + n] = -Fi[f][n],
//     B[64 + f][n] = Fi[f][n],  B[64 + f][64 + n] = Fr[f][n],
// which turns a row [re x | im x] into [re (F x) | im (F x)].  The inverse
// uses conj(F) x = conj(F conj(x)): the data is written conjugated and read
// back conjugated, so one constant serves every stage.
//
// A cluster of two CTAs runs one kt plane; CTA q owns the ky parities q and
// q + 2 (sub-parity s: q' = q + 2 s).  The fourteen MMA groups of a plane
// (four y transforms, one per x parity p with rows (s, x0); four x
// transforms with rows (s, j); four inverse x transforms; two inverse y
// transforms with rows x) each fill a 128-column region of the CTA's 512
// tensor-memory columns.  Between groups the 256 threads read a region back
// (tcgen05.ld, one lane per thread), apply folds, twists, H and the split
// into BF16 hi / lo, and write the next group's A operand into one of two
// 64 KB shared-memory buffers, K-major (same rows) or MN-major (the
// transposing steps).  One thread issues the MMAs; commits to one mbarrier
// per group let the threads prepare group g + 1 while group g runs.  The two
// CTAs' partial results (their ky halves) are summed through distributed
// shared memory.
//
// Layouts (no swizzle, 16-bit elements): a K-major 128 x 128 tile keeps each
// 8-row by 8-element core matrix as 128 contiguous bytes, K chunks 128 bytes
// apart (leading byte offset) and 8-row groups 2048 bytes apart (stride byte
// offset); an MN-major tile keeps 8 consecutive rows of one K index in 16
// bytes, 8-row groups 128 bytes apart and 8-K groups 2048 bytes apart.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "passes.cuh"

namespace cg = cooperative_groups;

namespace nlos {

struct LateralTC {
  int mode = 0;                // 1 split BF16 (three products), 2 BF16 hi only
  uint4* d_B = nullptr;        // shared-memory image of the block constant: hi tile, lo tile
  float2* d_Hp = nullptr;      // H rearranged [kt][q][fold kx][row]
  int* d_status = nullptr;     // nonzero after a bounded wait gave up
};

namespace {

constexpr int kTcN = 128;
constexpr int kTcThreads = 512;
constexpr int kTcGroups = 14;
constexpr uint32_t kTile = 128 * 128 * 2;               // one 16-bit 128 x 128 operand tile
constexpr uint32_t kOffB = 0;                           // constant: hi, lo
constexpr uint32_t kOffA0 = 2 * kTile;                  // A buffer 0: hi, lo
constexpr uint32_t kOffA1 = 4 * kTile;                  // A buffer 1: hi, lo
constexpr int kExPitch = 130;                           // float2 per row of the staging buffers
constexpr uint32_t kStage = 64 * kExPitch * 8;          // 64 rows of a CTA's partial results
constexpr uint32_t kOffEx = kOffA0;                     // final stage: rows of the partner CTA
constexpr uint32_t kOffOwn = kOffEx + kStage;           //              this CTA's own rows
constexpr uint32_t kOffTw = kOffOwn + kStage;           // 256 twiddles w^e
constexpr uint32_t kOffBar = kOffTw + 256 * 8;          // one mbarrier per MMA group
constexpr uint32_t kOffMisc = kOffBar + 16 * 8;         // tensor-memory base, failure flag
constexpr uint32_t kTcSmem = kOffMisc + 16;
static_assert(kOffTw >= kOffA1 + 2 * kTile, "staging buffers must cover only the operand buffers");
static_assert(kTcSmem <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of the 16-byte chunk holding (row r, k .. k + 7), k % 8 == 0, K-major.
__device__ __forceinline__ uint32_t kmaj(int r, int k) {
  return (uint32_t)((r >> 3) * 2048 + (k >> 3) * 128 + (r & 7) * 16);
}
// ... holding (rows r .. r + 7, k), r % 8 == 0, MN-major.
__device__ __forceinline__ uint32_t mnmaj(int r, int k) {
  return (uint32_t)((k >> 3) * 2048 + (r >> 3) * 128 + (k & 7) * 16);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: D F32, A and B BF16, M = N = 128,
// A MN-major when transposed.
__host__ __device__ constexpr uint32_t tc_idesc(bool a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of an mbarrier with the given parity, giving up after
// one second: the failure is recorded (shared flag and the plan's status
// word) and every later wait of the CTA returns at once, so the kernel still
// runs to its end.
__device__ __forceinline__ void tc_wait(uint32_t bar, uint32_t parity, volatile int* fail, int* status) {
  if (!*fail) {
    const uint64_t t0 = global_ns();
    for (;;) {
      uint32_t done;
      asm volatile(
          "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}\n"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
      if (done) break;
      if (global_ns() - t0 > 1000000000ull) {
        *fail = 1;
        atomicOr(status, 1);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// All threads: make the generic-proxy writes of an operand visible to the
// tensor core and order this thread's tensor-memory reads before the sync.
__device__ __forceinline__ void tc_sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
}

// tcgen05.ld of 8 / 16 consecutive columns of this warp's lane quarter.
__device__ __forceinline__ void tld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// BF16 pair packing (element k in the low half) and the hi / lo split:
// hi = rn(v), lo = rn(v - hi), so hi + lo carries about 16 significand bits.
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <int TERMS>
__device__ __forceinline__ void store8(uint8_t* buf, uint32_t off, const float* v) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    hi[i] = pack_bf2(v[2 * i], v[2 * i + 1]);
    if (TERMS > 1) {
      const float h0 = __uint_as_float(hi[i] << 16), h1 = __uint_as_float(hi[i] & 0xFFFF0000u);
      lo[i] = pack_bf2(v[2 * i] - h0, v[2 * i + 1] - h1);
    }
  }
  *reinterpret_cast<uint4*>(buf + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  if (TERMS > 1) *reinterpret_cast<uint4*>(buf + kTile + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// One MMA group: D (128 columns at d) = A (buffer abuf) x B, the products of
// the split terms accumulated over K = 128 (eight K = 16 steps each).
template <int TERMS>
__device__ __forceinline__ void tc_issue(uint32_t sbase, uint32_t abuf, bool a_mn, uint32_t d, uint32_t bar) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t idesc = tc_idesc(a_mn);
  const uint32_t a_step = a_mn ? 4096 : 256;
  // the start address is the descriptor's low field (16-byte units, below
  // 256 KB here), so later K steps and the lo tiles are added to it
  const uint64_t a0 = umma_desc(sbase + abuf, a_mn ? 2048 : 128, a_mn ? 128 : 2048);
  const uint64_t b0 = umma_desc(sbase + kOffB, 128, 2048);
#pragma unroll
  for (int t = 0; t < TERMS; ++t) {
    const uint64_t at = a0 + ((t == 2 ? kTile : 0) >> 4), bt = b0 + ((t == 1 ? kTile : 0) >> 4);
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
      tc_mma(d, at + ((ks * a_step) >> 4), bt + ((ks * 256) >> 4), idesc, (t | ks) != 0 ? 1u : 0u);
  }
  tc_commit(bar);
}

__device__ __forceinline__ float2 rot_mi(float2 v, int p) {  // v (-i)^p
  const float2 r = (p & 1) ? make_float2(v.y, -v.x) : v;
  return (p & 2) ? make_float2(-r.x, -r.y) : r;
}
__device__ __forceinline__ float2 rot_i(float2 v, int p) {   // v i^p
  const float2 r = (p & 1) ? make_float2(-v.y, v.x) : v;
  return (p & 2) ? make_float2(-r.x, -r.y) : r;
}

// Eight consecutive values X[x][y0 .. y0 + 7] of the input plane: dense, or
// gathered through the column map of a compact plane (zero off the samples).
__device__ __forceinline__ void load8(const float2* __restrict__ src, const int32_t* __restrict__ pos, int x, int y0,
                                      float2 (&v)[8]) {
  if (pos == nullptr) {
    const float4* p = reinterpret_cast<const float4*>(src + x * kTcN + y0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 f = __ldg(p + i);
      v[2 * i] = make_float2(f.x, f.y);
      v[2 * i + 1] = make_float2(f.z, f.w);
    }
  } else {
    const int4* pp = reinterpret_cast<const int4*>(pos + x * kTcN + y0);
    const int4 a = __ldg(pp), b = __ldg(pp + 1);
    const int j[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = j[i] >= 0 ? __ldg(src + j[i]) : make_float2(0.f, 0.f);
  }
}

// The four values a thread folds for each of its eight rows: X[x][n],
// X[x][n + 64], X[x + 64][n], X[x + 64][n + 64] for x = xb + r.  Loaded once
// per plane and kept in registers for both operand passes.
struct YIn {
  float2 e0[8], o0[8], e1[8], o1[8];
};

// Thread (n, eight consecutive x0): the lanes of a warp read 32 consecutive
// values of a row.
__device__ __forceinline__ void tc_load_y(YIn& in, const float2* __restrict__ src, const int32_t* __restrict__ pos,
                                          int q, int tid) {
  const int n = tid & 63, xb = (tid >> 6) * 8;
  auto ld = [&](int x, int y) -> float2 {
    if (pos == nullptr) return __ldg(src + x * kTcN + y);
    const int j = __ldg(pos + x * kTcN + y);
    return j >= 0 ? __ldg(src + j) : make_float2(0.f, 0.f);
  };
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    in.e0[r] = ld(xb + r, n);
    in.o0[r] = ld(xb + r, 64 + n);
    in.e1[r] = ld(xb + r + 64, n);
    in.o1[r] = ld(xb + r + 64, 64 + n);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    in.o0[r] = rot_mi(in.o0[r], q);
    in.o1[r] = rot_mi(in.o1[r], q);
  }
}

// Operand of the y transform of x parity p (one buffer), MN-major: row 64 s + x0, K = n (real part) and 64 + n (imaginary part)
// holds
//   w^(q' n + p x0) [(X[x0][n] + (-i)^q' X[x0][n+64]) + (-i)^p (X[x0+64][n] + (-i)^q' X[x0+64][n+64])];
// each thread writes 16-byte runs of eight rows.
template <int TERMS>
__device__ __forceinline__ void tc_build_y(uint8_t* buf, const YIn& in, const float2* tw, int q, int p, int tid) {
  const int n = tid & 63, xb = (tid >> 6) * 8;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int qq = q + 2 * s;
    float re[8], im[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const float2 a = s ? csub(in.e0[r], in.o0[r]) : cadd(in.e0[r], in.o0[r]);
      const float2 b = s ? csub(in.e1[r], in.o1[r]) : cadd(in.e1[r], in.o1[r]);
      const float2 v = cmul(cadd(a, rot_mi(b, p)), tw[(qq * n + p * (xb + r)) & 255]);
      re[r] = v.x;
      im[r] = v.y;
    }
    const int r0 = 64 * s + xb;
    store8<TERMS>(buf, mnmaj(r0, n), re);
    store8<TERMS>(buf, mnmaj(r0, 64 + n), im);
  }
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

}  // namespace

// Persistent: each cluster of two CTAs runs the planes kt = cluster, cluster
// + clusters, ...; the constant, the twiddles, the barriers and the tensor
// memory are set up once.  Each of the 16 warps reads the tensor-memory
// lanes of quarter (warp mod 4) and a quarter of every region's columns.
template <int TERMS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTcThreads, 1)
    k_conv_tc(const float2* __restrict__ Sin, int in_pitch, const int32_t* __restrict__ in_pos,
              float2* __restrict__ Sout, int out_pitch, const int32_t* __restrict__ out_pos,
              const float2* __restrict__ Hq, const uint4* __restrict__ Bimg, const float2* __restrict__ twg,
              int planes, int adj, int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int cid = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qw = warp & 3, cq = warp >> 2;
  const int L = 32 * qw + lane;  // tensor-memory lane (matrix row) this thread reads
  float2* tw = reinterpret_cast<float2*>(smem + kOffTw);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kOffMisc);
  volatile int* fail = reinterpret_cast<volatile int*>(smem + kOffMisc + 4);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = sbase + kOffBar;

  // constant, twiddles, barriers, tensor memory (once)
  {
    const int nb = TERMS > 1 ? 2 * kTile / 16 : kTile / 16;
    uint4* bs = reinterpret_cast<uint4*>(smem + kOffB);
    for (int i = tid; i < nb; i += kTcThreads) bs[i] = __ldg(Bimg + i);
    for (int i = tid; i < 256; i += kTcThreads) tw[i] = __ldg(twg + i);
  }
  if (tid == 0) {
    *fail = 0;
    for (int g = 0; g < kTcGroups; ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * g));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_sync_for_mma();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  const uint32_t tl = tbase + ((uint32_t)(32 * qw) << 16);  // this warp's lane quarter
  const float scale = 1.0f / (4.0f * kTcN * kTcN);
  const bool own = (L >> 6) == q;

#pragma unroll 1
  for (int kt = cid, it = 0; kt < planes; kt += nclusters, ++it) {
    const uint32_t ph = (uint32_t)it & 1u;  // barrier phase of this plane
    const float2* src = Sin + (size_t)kt * in_pitch;

    // 1. y transforms (groups 0-3), operands built from the input plane (read
    // once per plane into registers), one buffer at a time: parity p into
    // buffer p mod 2 once the group that last read it (p - 2) is done
    YIn yin;
    tc_load_y(yin, src, in_pos, q, tid);
    if (it > 0) cluster_wait();  // the partner has read the previous plane's staging rows (buffers 0, 1)
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
      if (p >= 2) tc_wait(bar0 + 8 * (p - 2), ph, fail, status);
      tc_build_y<TERMS>(smem + ((p & 1) ? kOffA1 : kOffA0), yin, tw, q, p, tid);
      tc_sync_for_mma();
      if (tid == 0) tc_issue<TERMS>(sbase, (p & 1) ? kOffA1 : kOffA0, true, tbase + 128 * p, bar0 + 8 * p);
    }

    // 2. x transforms (groups 4-7): region p (rows (s, x0), columns j) ->
    // MN-major operand rows (s, j), K = x0
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
      tc_wait(bar0 + 8 * (2 + p), ph, fail, status);
      const int s = L >> 6, x0 = L & 63;
      float re[16], im[16];
      tld16(tl + 128 * p + 16 * cq, re);
      tld16(tl + 128 * p + 64 + 16 * cq, im);
      tld_wait();
      uint8_t* buf = smem + ((p & 1) ? kOffA1 : kOffA0);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int r0 = 64 * s + 16 * cq + 8 * g;
        store8<TERMS>(buf, mnmaj(r0, x0), re + 8 * g);
        store8<TERMS>(buf, mnmaj(r0, 64 + x0), im + 8 * g);
      }
      tc_sync_for_mma();
      if (tid == 0) tc_issue<TERMS>(sbase, (p & 1) ? kOffA1 : kOffA0, true, tbase + 128 * p, bar0 + 8 * (4 + p));
    }

    // 3. multiply by H (conj H for the adjoint), inverse x transforms (groups
    // 8-11): rows (s, j) stay; the operand is written conjugated
#pragma unroll 1
    for (int p = 0; p < 4; ++p) {
      // H(kx = 4 m + p, ky of row L) at Hq[kt][q][fold kx][L]: a warp reads 32 consecutive values
      const float2* hcol = Hq + ((size_t)kt * 2 + q) * (kTcN + 1) * 128 + L;
      float2 h[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int kx = 4 * (16 * cq + i) + p, fx = kx <= kTcN ? kx : 2 * kTcN - kx;
        h[i] = __ldg(hcol + fx * 128);
      }
      tc_wait(bar0 + 8 * (6 + p), ph, fail, status);
      float re[16], im[16];
      tld16(tl + 128 * p + 16 * cq, re);
      tld16(tl + 128 * p + 64 + 16 * cq, im);
      tld_wait();
      const float sg = adj ? -1.f : 1.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float hr = h[i].x, hi = sg * h[i].y;
        const float zr = re[i], zi = im[i];
        re[i] = zr * hr - zi * hi;
        im[i] = -(zr * hi + zi * hr);
      }
      uint8_t* buf = smem + ((p & 1) ? kOffA1 : kOffA0);
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int k0 = 16 * cq + 8 * g;
        store8<TERMS>(buf, kmaj(L, k0), re + 8 * g);
        store8<TERMS>(buf, kmaj(L, 64 + k0), im + 8 * g);
      }
      tc_sync_for_mma();
      if (tid == 0) tc_issue<TERMS>(sbase, (p & 1) ? kOffA1 : kOffA0, false, tbase + 128 * p, bar0 + 8 * (8 + p));
    }

    // 4. recombine the four x parities, out[x0 + 64 t] = sum_p i^(p t) w^(-p x0) I_p[x0]
    // with I_p = conj(region p), into the inverse y operands (buffer s, MN-major
    // rows x, K = j, conjugated)
    tc_wait(bar0 + 8 * 11, ph, fail, status);
    {
      const int s = L >> 6, j = L & 63;
      uint8_t* buf = smem + (s ? kOffA1 : kOffA0);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int xb = 16 * cq + 8 * c;
        float ur[4][8], ui[4][8];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          tld8(tl + 128 * p + xb, ur[p]);
          tld8(tl + 128 * p + 64 + xb, ui[p]);
        }
        tld_wait();
        float v0r[8], v0i[8], v1r[8], v1i[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float2 u[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            u[p] = make_float2(ur[p][i], -ui[p][i]);
            if (p) u[p] = cmulc(u[p], tw[(p * (xb + i)) & 255]);
          }
          const float2 e02 = cadd(u[0], u[2]), d02 = csub(u[0], u[2]);
          const float2 e13 = cadd(u[1], u[3]), d13 = csub(u[1], u[3]);
          v0r[i] = e02.x + e13.x;
          v0i[i] = -(e02.y + e13.y);
          v1r[i] = d02.x - d13.y;
          v1i[i] = -(d02.y + d13.x);
        }
        store8<TERMS>(buf, mnmaj(xb, j), v0r);
        store8<TERMS>(buf, mnmaj(xb, 64 + j), v0i);
        store8<TERMS>(buf, mnmaj(64 + xb, j), v1r);
        store8<TERMS>(buf, mnmaj(64 + xb, 64 + j), v1i);
      }
    }
    tc_sync_for_mma();
    if (tid == 0) {
      tc_issue<TERMS>(sbase, kOffA0, true, tbase + 0, bar0 + 8 * 12);
      tc_issue<TERMS>(sbase, kOffA1, true, tbase + 128, bar0 + 8 * 13);
    }

    // 5. recombine the two ky sub-parities: this CTA's part
    //   P[x][y0 + 64 t] = sum_s i^(q' t) w^(-q' y0) conj(region s)[x][y0],
    // and sum the two CTAs' parts; CTA q writes rows [64 q, 64 q + 64)
    tc_wait(bar0 + 8 * 13, ph, fail, status);
    if (tid == 0 && kt + nclusters < planes) {  // the next plane's input and spectrum into L2
      if (in_pos == nullptr) prefetch_l2(Sin + (size_t)(kt + nclusters) * in_pitch, kTcN * kTcN * 8);
      prefetch_l2(Hq + ((size_t)(kt + nclusters) * 2 + q) * (kTcN + 1) * 128, (kTcN + 1) * 128 * 8);
    }
    auto part = [&](int c, float2 (&o0)[8], float2 (&o1)[8]) {
      const int yb = 16 * cq + 8 * c;
      float r0[8], i0[8], r1[8], i1[8];
      tld8(tl + yb, r0);
      tld8(tl + 64 + yb, i0);
      tld8(tl + 128 + yb, r1);
      tld8(tl + 192 + yb, i1);
      tld_wait();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int y0 = yb + i;
        const float2 u0 = cmulc(make_float2(r0[i], -i0[i]), tw[(q * y0) & 255]);
        const float2 u1 = cmulc(make_float2(r1[i], -i1[i]), tw[((q + 2) * y0) & 255]);
        o0[i] = cscale(cadd(u0, u1), scale);
        o1[i] = cscale(rot_i(csub(u0, u1), q), scale);
      }
    };
    {
      // every row's partial into shared memory: own rows to the own buffer,
      // the partner's rows to the exchange buffer it reads
      float2* row = reinterpret_cast<float2*>(smem + (own ? kOffOwn : kOffEx)) + (L & 63) * kExPitch;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float2 o0[8], o1[8];
        part(c, o0, o1);
        const int yb = 16 * cq + 8 * c;
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          *reinterpret_cast<float4*>(row + yb + i) = make_float4(o0[i].x, o0[i].y, o0[i + 1].x, o0[i + 1].y);
          *reinterpret_cast<float4*>(row + 64 + yb + i) = make_float4(o1[i].x, o1[i].y, o1[i + 1].x, o1[i + 1].y);
        }
      }
    }
    cluster.sync();
    {
      // rows [64 q, 64 q + 64): own part + the partner's, a warp per 32
      // consecutive y of a row
      const float2* mine = reinterpret_cast<const float2*>(smem + kOffOwn);
      const float2* theirs = cluster.map_shared_rank(reinterpret_cast<const float2*>(smem + kOffEx), 1 - q);
      float2* dst = Sout + (size_t)kt * out_pitch;
      // two consecutive y per thread (16-byte accesses), 8 rows per pass
      const int y = 2 * (tid & 63), r0 = tid >> 6;
      constexpr int RS = kTcThreads / 64, R = 64 / RS;
      float4 a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int r = r0 + i * RS;
        a[i] = *reinterpret_cast<const float4*>(mine + r * kExPitch + y);
        b[i] = *reinterpret_cast<const float4*>(theirs + r * kExPitch + y);
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const float2 v0 = cadd(make_float2(a[i].x, a[i].y), make_float2(b[i].x, b[i].y));
        const float2 v1 = cadd(make_float2(a[i].z, a[i].w), make_float2(b[i].z, b[i].w));
        const int x = 64 * q + r0 + i * RS;
        if (out_pos == nullptr) {
          *reinterpret_cast<float4*>(dst + x * kTcN + y) = make_float4(v0.x, v0.y, v1.x, v1.y);
        } else {
          const int2 j = __ldg(reinterpret_cast<const int2*>(out_pos + x * kTcN + y));
          if (j.x >= 0) dst[j.x] = v0;
          if (j.y >= 0) dst[j.y] = v1;
        }
      }
    }
    // done reading the partner's staging rows; the matching wait comes before
    // the next plane writes buffers 0 and 1 (or before the exit), so the
    // next plane's input loads overlap the partner's last reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cluster_arrive();
  }
  if (cid < planes) cluster_wait();
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

// Shared-memory image of the block constant from its FP32 values Bf[n][k]
// (128 x 128): hi tile then lo tile, K-major core matrices.
__global__ void k_tc_bimage(const float* __restrict__ Bf, uint16_t* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 128 * 128) return;
  const int n = i >> 7, k = i & 127;
  const float v = Bf[i];
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  const int off = ((n >> 3) * 2048 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
  img[off] = *reinterpret_cast<const uint16_t*>(&hi);
  img[kTile / 2 + off] = *reinterpret_cast<const uint16_t*>(&lo);
}

// H rearranged for the kernel's reads: Hq[kt][q][fx][L] = H(kx, ky) for
// every kx with fold(kx) = fx and the ky of row L = 64 s + j of CTA q,
// ky = 4 j + q + 2 s; the plan stores H[kt][fold kx][fold ky], fold(k) =
// min(k, 2N - k).  A warp's 32 rows are then 32 consecutive values.
__global__ void k_tc_hperm(const float2* __restrict__ H, float2* __restrict__ Hq, int planes) {
  const size_t total = (size_t)planes * 2 * (kTcN + 1) * 128;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int L = (int)(i & 127);
    const size_t r = i >> 7;
    const int fx = (int)(r % (kTcN + 1));
    const int q = (int)((r / (kTcN + 1)) & 1);
    const size_t kt = r / (2 * (kTcN + 1));
    const int ky = 4 * (L & 63) + q + 2 * (L >> 6), fy = ky <= kTcN ? ky : 2 * kTcN - ky;
    Hq[i] = H[(kt * (kTcN + 1) + fx) * (kTcN + 1) + fy];
  }
}

void free_lateral_tc(Plan* P) {
  LateralTC* L = P->lateral;
  if (!L) return;
  cudaFree(L->d_B);
  cudaFree(L->d_Hp);
  cudaFree(L->d_status);
  delete L;
  P->lateral = nullptr;
}

nlos_status lateral_status(const Plan& P) {
  if (!P.lateral) return NLOS_OK;
  int v = 0;
  NLOS_CUDA(cudaMemcpy(&v, P.lateral->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v == 0) return NLOS_OK;
  NLOS_CUDA(cudaMemset(P.lateral->d_status, 0, sizeof(int)));
  return fail(NLOS_ERR_TIMEOUT, "tensor-core lateral stage: an MMA completion wait gave up");
}

nlos_status set_lateral_mode(Plan& P, int mode, cudaStream_t st) {
  if (mode < 0 || mode > 2) return fail(NLOS_ERR_INVALID_ARG, "lateral mode must be 0, 1 or 2");
  if (P.lateral) NLOS_TRY(lateral_status(P));
  if (mode == 0) {
    free_lateral_tc(&P);
    return NLOS_OK;
  }
  if (P.nx != kTcN || P.ny != kTcN)
    return fail(NLOS_ERR_INVALID_ARG, "the tensor-core lateral stage needs nx = ny = 128");
  if (P.lateral) {
    P.lateral->mode = mode;
    return NLOS_OK;
  }
  NLOS_TRY(ensure_smem(k_conv_tc<3>, kTcSmem));
  NLOS_TRY(ensure_smem(k_conv_tc<1>, kTcSmem));
  LateralTC* L = new LateralTC();
  P.lateral = L;
  const int planes = P.nt + 1;
  const size_t hp = (size_t)planes * 2 * (kTcN + 1) * 128;
  float* d_Bf = nullptr;
  auto cleanup = [&](nlos_status s) {
    cudaFree(d_Bf);
    free_lateral_tc(&P);
    return s;
  };
  if (cudaMalloc(&L->d_B, 2 * kTile) != cudaSuccess || cudaMalloc(&L->d_Hp, hp * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(&L->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&d_Bf, 128 * 128 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(NLOS_ERR_OOM, "tensor-core lateral stage: device memory"));
  }
  // block constant from FP64: F[f][n] = exp(-2 pi i f n / 64)
  std::vector<float> Bf(128 * 128);
  const double pi = 3.14159265358979323846;
  for (int f = 0; f < 64; ++f)
    for (int n = 0; n < 64; ++n) {
      const double a = -2.0 * pi * (double)((f * n) % 64) / 64.0;
      const float fr = (float)std::cos(a), fi = (float)std::sin(a);
      Bf[f * 128 + n] = fr;
      Bf[f * 128 + 64 + n] = -fi;
      Bf[(64 + f) * 128 + n] = fi;
      Bf[(64 + f) * 128 + 64 + n] = fr;
    }
  if (cudaMemcpyAsync(d_Bf, Bf.data(), Bf.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(L->d_status, 0, sizeof(int), st) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "tensor-core lateral stage: constants"));
  k_tc_bimage<<<64, 256, 0, st>>>(d_Bf, reinterpret_cast<uint16_t*>(L->d_B));
  k_tc_hperm<<<device_sm_count() * 8, 256, 0, st>>>(P.d_H, L->d_Hp, planes);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return cleanup(cuda_fail(cudaGetLastError(), "tensor-core lateral stage: set-up kernels"));
  cudaFree(d_Bf);
  d_Bf = nullptr;
  L->mode = mode;
  return NLOS_OK;
}

nlos_status launch_conv_tc(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact,
                           bool adj, cudaStream_t st) {
  const LateralTC* L = P.lateral;
  const int full = P.nx * P.ny;
  if ((reinterpret_cast<uintptr_t>(Sin) & 15) != 0 || (reinterpret_cast<uintptr_t>(Sout) & 15) != 0)
    return fail(NLOS_ERR_INVALID_ARG, "tensor-core lateral stage: spectra must be 16-byte aligned");
  auto kern = L->mode == 2 ? k_conv_tc<1> : k_conv_tc<3>;
  NLOS_TRY(ensure_smem(kern, kTcSmem));
  const int planes = P.nt + 1;
  const int clusters = std::min(planes, std::max(1, device_sm_count() / 2));
  kern<<<2 * clusters, kTcThreads, kTcSmem, st>>>(
      Sin, in_compact ? P.ncols : full, in_compact ? P.d_colpos : nullptr, Sout, out_compact ? P.ncols : full,
      out_compact ? P.d_colpos : nullptr, L->d_Hp, L->d_B, P.d_twx, planes, adj ? 1 : 0, L->d_status);
  NLOS_LAUNCH_CHECK("k_conv_tc");
  return NLOS_OK;
}

}  // namespace nlos
