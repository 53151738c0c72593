// Lateral convolution of the light-cone transform (the H of Eq. 3 applied to
// every kt plane) as dense DFT-matrix products on the tensor cores: the
// optional GEMM variant of the lateral stage, for the precision comparison
// of the FP32 FFT kernels with a split-BF16 GEMM (FP32 accumulate).
//
// Per kt plane X[x][y] (N x N), with w = exp(-2 pi i / 2N) and the
// zero-padding to 2N x 2N folded into rectangular DFT matrices:
//   Y(ky, x)  = sum_y  F1(ky, y) X(y, x)      F1 = w^(y ky)      (2N x N)
//   Z(ky, kx) = sum_x  Y(ky, x)  F2(x, kx)    F2 = w^(x kx)      (N x 2N)
//   W         = H(kx, ky) Z  (conj H for the adjoint)
//   V(ky, x)  = sum_kx W(ky, kx) G1(kx, x)    G1 = w^(-x kx)     (2N x N)
//   O(y, x)   = s sum_ky G2(y, ky) V(ky, x)   G2 = w^(-ky y), s = 1 / (4 N^2)
// (column-major matrices: a plane stored [x][y], y contiguous, is X(y, x)).
// Complex products run as real BF16 GEMMs (FP32 accumulate and output) on
// planar operands: a constant on the left enters as the real 2x2 block
// matrix [[Ar, -Ai], [Ai, Ar]] against the row-stacked data [Br; Bi]; data on
// the left enters as Br * [Cr | Ci] + Bi * [-Ci | Cr] against the constant C.
// Mode 1 splits every operand into hi + lo BF16 terms and sums the products
// hi hi + hi lo + lo hi (about 16 significand bits each); mode 2 keeps hi.
// Each product is one strided-batched cuBLAS GEMM over the nt + 1 planes.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <cmath>
#include <type_traits>
#include <vector>

#include "passes.cuh"

namespace nlos {

typedef __nv_bfloat16 bf16;

struct LateralGemm {
  cublasHandle_t h = nullptr;
  int mode = 0;
  // constants, hi and lo terms (index 0 / 1), column-major
  bf16* A1[2] = {};   // (4N x 2N) [[F1r, -F1i], [F1i, F1r]]
  bf16* B2a[2] = {};  // (N x 4N)  [F2r | F2i]
  bf16* B2b[2] = {};  // (N x 4N)  [-F2i | F2r]
  bf16* B4a[2] = {};  // (2N x 2N) [G1r | G1i]
  bf16* B4b[2] = {};  // (2N x 2N) [-G1i | G1r]
  bf16* A5[2] = {};   // (2N x 4N) [[G2r, -G2i], [G2i, G2r]]
  // per-plane data
  bf16* Xs[2] = {};   // (2N x N)  [Xr; Xi]
  float* Ys = nullptr;  // (4N x N)  [Yr; Yi]
  bf16* Yb[2] = {};     // (4N x N)  the same in BF16
  float* Zc = nullptr;  // (2N x 4N) [Zr | Zi]
  bf16* Wb[2] = {};     // (2N x 4N) [Wr | Wi]
  float* Vc = nullptr;  // (2N x 2N) [Vr | Vi]
  bf16* Vs[2] = {};     // (4N x N)  [Vr; Vi]
  float* Os = nullptr;  // (2N x N)  [Or; Oi]
  std::vector<void*> allocs;
};

__device__ __forceinline__ void split_bf16(float v, bf16& hi, bf16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Input plane (interleaved complex X(y, x) at y + N x, planes at stride
// pitch; compact: sampled columns j at col = cols[j], zero elsewhere) ->
// row-stacked [Xr; Xi] (2N x N) hi / lo.
__global__ void k_gemm_load_x(const float2* __restrict__ S, int pitch, const int32_t* __restrict__ colpos, int n,
                              int planes, bf16* __restrict__ xh, bf16* __restrict__ xl) {
  const size_t per = (size_t)n * n, total = per * planes;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kt = (int)(i / per), col = (int)(i % per), y = col % n, x = col / n;
    float2 v = make_float2(0.f, 0.f);
    if (colpos) {
      const int j = __ldg(colpos + col);
      if (j >= 0) v = S[(size_t)kt * pitch + j];
    } else {
      v = S[(size_t)kt * pitch + col];
    }
    const size_t o = (size_t)kt * 2 * per + y + (size_t)2 * n * x;
    split_bf16(v.x, xh[o], xl[o]);
    split_bf16(v.y, xh[o + n], xl[o + n]);
  }
}

// FP32 -> BF16 hi / lo, same layout.
__global__ void k_gemm_split(const float* __restrict__ a, size_t count, bf16* __restrict__ hi, bf16* __restrict__ lo) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    split_bf16(a[i], hi[i], lo[i]);
}

// W = H Z (conj H for the adjoint) on [Zr | Zi] (2N x 4N per plane), element
// (ky, kx) of Zr at ky + 2N kx, of Zi 4N^2 further; H[kt][fold kx][fold ky].
__global__ void k_gemm_hmul(const float* __restrict__ Zc, const float2* __restrict__ H, int n, int planes, int adj,
                            bf16* __restrict__ wh, bf16* __restrict__ wl) {
  const int n2 = 2 * n;
  const size_t per = (size_t)n2 * n2, total = per * planes;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kt = (int)(i / per);
    const int r = (int)(i % per), ky = r % n2, kx = r / n2;
    const int fx = kx <= n ? kx : n2 - kx, fy = ky <= n ? ky : n2 - ky;
    float2 hv = __ldg(H + ((size_t)kt * (n + 1) + fx) * (n + 1) + fy);
    if (adj) hv.y = -hv.y;
    const size_t o = (size_t)kt * 2 * per + r;
    const float zr = Zc[o], zi = Zc[o + per];
    split_bf16(zr * hv.x - zi * hv.y, wh[o], wl[o]);
    split_bf16(zr * hv.y + zi * hv.x, wh[o + per], wl[o + per]);
  }
}

// [Vr | Vi] (2N x 2N, FP32) -> row-stacked [Vr; Vi] (4N x N) hi / lo.
__global__ void k_gemm_restack(const float* __restrict__ Vc, int n, int planes, bf16* __restrict__ vh,
                               bf16* __restrict__ vl) {
  const int n2 = 2 * n;
  const size_t per = (size_t)n2 * n, total = per * planes;  // complex elements (ky, x)
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kt = (int)(i / per);
    const int r = (int)(i % per), ky = r % n2, x = r / n2;
    const size_t src = (size_t)kt * 2 * per + ky + (size_t)n2 * x;
    const size_t dst = (size_t)kt * 2 * per + ky + (size_t)2 * n2 * x;
    split_bf16(Vc[src], vh[dst], vl[dst]);
    split_bf16(Vc[src + per], vh[dst + n2], vl[dst + n2]);
  }
}

// [Or; Oi] (2N x N) -> output plane (interleaved, O(y, x) at y + N x), or
// its sampled columns.
__global__ void k_gemm_store(const float* __restrict__ Os, int n, int planes, const int32_t* __restrict__ cols,
                             int ncols, float2* __restrict__ S, int pitch) {
  const size_t per = (size_t)n * n;
  const size_t count = cols ? (size_t)ncols : per, total = count * planes;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kt = (int)(i / count), j = (int)(i % count);
    const int col = cols ? __ldg(cols + j) : j, y = col % n, x = col / n;
    const size_t src = (size_t)kt * 2 * per + y + (size_t)2 * n * x;
    S[(size_t)kt * pitch + j] = make_float2(Os[src], Os[src + n]);
  }
}

static int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)152 * 16); }

static nlos_status cublas_ok(cublasStatus_t s, const char* what) {
  if (s == CUBLAS_STATUS_SUCCESS) return NLOS_OK;
  return fail(NLOS_ERR_CUDA, std::string(what) + ": cuBLAS status " + std::to_string((int)s));
}

void free_lateral_gemm(Plan* P) {
  LateralGemm* L = P->lateral;
  if (!L) return;
  if (L->h) cublasDestroy(L->h);
  for (void* p : L->allocs) cudaFree(p);
  delete L;
  P->lateral = nullptr;
}

nlos_status set_lateral_mode(Plan& P, int mode, cudaStream_t st) {
  (void)st;
  if (mode < 0 || mode > 2) return fail(NLOS_ERR_INVALID_ARG, "lateral mode must be 0, 1 or 2");
  if (mode == 0) {
    free_lateral_gemm(&P);
    return NLOS_OK;
  }
  if (P.nx != P.ny) return fail(NLOS_ERR_INVALID_ARG, "the GEMM lateral stage needs nx = ny");
  if (P.lateral) {
    P.lateral->mode = mode;
    return NLOS_OK;
  }
  LateralGemm* L = new LateralGemm();
  P.lateral = L;
  const int n = P.nx, n2 = 2 * n;
  const size_t planes = (size_t)P.nt + 1, nn = (size_t)n * n;
  nlos_status s = NLOS_OK;
  auto dal = [&](auto** p, size_t count) {
    if (s != NLOS_OK) return;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(**p)) != cudaSuccess) {
      cudaGetLastError();
      s = fail(NLOS_ERR_OOM, "GEMM lateral stage: device memory");
      return;
    }
    L->allocs.push_back(q);
    *p = reinterpret_cast<std::remove_reference_t<decltype(*p)>>(q);
  };
  for (int t = 0; t < 2; ++t) {
    dal(&L->A1[t], 8 * nn);
    dal(&L->B2a[t], 4 * nn);
    dal(&L->B2b[t], 4 * nn);
    dal(&L->B4a[t], 4 * nn);
    dal(&L->B4b[t], 4 * nn);
    dal(&L->A5[t], 8 * nn);
    dal(&L->Xs[t], planes * 2 * nn);
    dal(&L->Yb[t], planes * 4 * nn);
    dal(&L->Wb[t], planes * 8 * nn);
    dal(&L->Vs[t], planes * 4 * nn);
  }
  dal(&L->Ys, planes * 4 * nn);
  dal(&L->Zc, planes * 8 * nn);
  dal(&L->Vc, planes * 4 * nn);
  dal(&L->Os, planes * 2 * nn);
  if (s == NLOS_OK) s = cublas_ok(cublasCreate(&L->h), "cublasCreate");
  if (s != NLOS_OK) {
    free_lateral_gemm(&P);
    return s;
  }
  // constants from FP64, split into hi / lo BF16 on the host
  const double pi = 3.14159265358979323846;
  auto root = [&](long long e, double& c, double& sn) {  // w^e, w = exp(-2 pi i / 2N)
    const long long m = ((e % n2) + n2) % n2;
    const double a = -2.0 * pi * (double)m / (double)n2;
    c = std::cos(a);
    sn = std::sin(a);
  };
  auto split = [](double v, bf16& hi, bf16& lo) {
    hi = __float2bfloat16_rn((float)v);
    lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
  };
  std::vector<bf16> a1h(8 * nn), a1l(8 * nn), b2ah(4 * nn), b2al(4 * nn), b2bh(4 * nn), b2bl(4 * nn);
  std::vector<bf16> b4ah(4 * nn), b4al(4 * nn), b4bh(4 * nn), b4bl(4 * nn), a5h(8 * nn), a5l(8 * nn);
  for (int a = 0; a < n2; ++a)
    for (int b = 0; b < n; ++b) {
      double c, sn;
      // F1(ky = a, y = b) = w^(ab): A1 (4N x 2N), rows [re(ky); im(ky)], cols [y re; y im]
      root((long long)a * b, c, sn);
      split(c, a1h[a + (size_t)4 * n * b], a1l[a + (size_t)4 * n * b]);                   // (a, b): F1r
      split(-sn, a1h[a + (size_t)4 * n * (n + b)], a1l[a + (size_t)4 * n * (n + b)]);     // (a, N + b): -F1i
      split(sn, a1h[n2 + a + (size_t)4 * n * b], a1l[n2 + a + (size_t)4 * n * b]);        // (2N + a, b): F1i
      split(c, a1h[n2 + a + (size_t)4 * n * (n + b)], a1l[n2 + a + (size_t)4 * n * (n + b)]);
      // F2(x = b, kx = a) = w^(ab): B2a = [F2r | F2i], B2b = [-F2i | F2r] (N x 4N)
      split(c, b2ah[b + (size_t)n * a], b2al[b + (size_t)n * a]);
      split(sn, b2ah[b + (size_t)n * (n2 + a)], b2al[b + (size_t)n * (n2 + a)]);
      split(-sn, b2bh[b + (size_t)n * a], b2bl[b + (size_t)n * a]);
      split(c, b2bh[b + (size_t)n * (n2 + a)], b2bl[b + (size_t)n * (n2 + a)]);
      // G1(kx = a, x = b) = w^(-ab): B4a = [G1r | G1i], B4b = [-G1i | G1r] (2N x 2N)
      root(-(long long)a * b, c, sn);
      split(c, b4ah[a + (size_t)n2 * b], b4al[a + (size_t)n2 * b]);
      split(sn, b4ah[a + (size_t)n2 * (n + b)], b4al[a + (size_t)n2 * (n + b)]);
      split(-sn, b4bh[a + (size_t)n2 * b], b4bl[a + (size_t)n2 * b]);
      split(c, b4bh[a + (size_t)n2 * (n + b)], b4bl[a + (size_t)n2 * (n + b)]);
      // G2(y = b, ky = a) = w^(-ab): A5 (2N x 4N), rows [re(y); im(y)], cols [ky re; ky im]
      split(c, a5h[b + (size_t)n2 * a], a5l[b + (size_t)n2 * a]);
      split(-sn, a5h[b + (size_t)n2 * (n2 + a)], a5l[b + (size_t)n2 * (n2 + a)]);
      split(sn, a5h[n + b + (size_t)n2 * a], a5l[n + b + (size_t)n2 * a]);
      split(c, a5h[n + b + (size_t)n2 * (n2 + a)], a5l[n + b + (size_t)n2 * (n2 + a)]);
    }
  auto up = [&](bf16* d, const std::vector<bf16>& v) {
    if (s == NLOS_OK && cudaMemcpy(d, v.data(), v.size() * sizeof(bf16), cudaMemcpyHostToDevice) != cudaSuccess)
      s = cuda_fail(cudaGetLastError(), "GEMM lateral stage: DFT matrices");
  };
  up(L->A1[0], a1h); up(L->A1[1], a1l);
  up(L->B2a[0], b2ah); up(L->B2a[1], b2al);
  up(L->B2b[0], b2bh); up(L->B2b[1], b2bl);
  up(L->B4a[0], b4ah); up(L->B4a[1], b4al);
  up(L->B4b[0], b4bh); up(L->B4b[1], b4bl);
  up(L->A5[0], a5h); up(L->A5[1], a5l);
  if (s != NLOS_OK) {
    free_lateral_gemm(&P);
    return s;
  }
  L->mode = mode;
  return NLOS_OK;
}

nlos_status launch_conv_gemm(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact,
                             bool adj, cudaStream_t st) {
  const LateralGemm* L = P.lateral;
  const int n = P.nx, n2 = 2 * n, planes = P.nt + 1;
  const size_t nn = (size_t)n * n;
  const int full = (int)nn;
  NLOS_TRY(cublas_ok(cublasSetStream(L->h, st), "cublasSetStream"));
  // hi hi (+ hi lo + lo hi for the split mode) into C, FP32 accumulate
  const int terms = L->mode == 1 ? 3 : 1;
  auto gemm = [&](int m, int nc, int k, float alpha, float beta0, bf16* const (&A)[2], size_t aoff, int lda,
                  long long sa, bf16* const (&B)[2], size_t boff, int ldb, long long sb, float* C, int ldc,
                  long long sc) -> nlos_status {
    const int ia[3] = {0, 0, 1}, ib[3] = {0, 1, 0};
    for (int t = 0; t < terms; ++t) {
      const float beta = t == 0 ? beta0 : 1.0f;
      NLOS_TRY(cublas_ok(cublasGemmStridedBatchedEx(L->h, CUBLAS_OP_N, CUBLAS_OP_N, m, nc, k, &alpha,
                                                    A[ia[t]] + aoff, CUDA_R_16BF, lda, sa, B[ib[t]] + boff,
                                                    CUDA_R_16BF, ldb, sb, &beta, C, CUDA_R_32F, ldc, sc, planes,
                                                    CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT),
                         "cublasGemmStridedBatchedEx"));
    }
    return NLOS_OK;
  };
  // [Xr; Xi] hi / lo
  const int in_pitch = in_compact ? P.ncols : full;
  k_gemm_load_x<<<grid_for(nn * planes), 256, 0, st>>>(Sin, in_pitch, in_compact ? P.d_colpos : nullptr, n, planes,
                                                        L->Xs[0], L->Xs[1]);
  NLOS_LAUNCH_CHECK("k_gemm_load_x");
  // [Yr; Yi] (4N x N) = A1 (4N x 2N) [Xr; Xi] (2N x N)
  NLOS_TRY(gemm(2 * n2, n, n2, 1.f, 0.f, L->A1, 0, 2 * n2, 0, L->Xs, 0, n2, 2 * nn, L->Ys, 2 * n2, 4 * nn));
  k_gemm_split<<<grid_for(4 * nn * planes), 256, 0, st>>>(L->Ys, 4 * nn * planes, L->Yb[0], L->Yb[1]);
  NLOS_LAUNCH_CHECK("k_gemm_split");
  // [Zr | Zi] (2N x 4N) = Yr (2N x N) [F2r | F2i] + Yi (2N x N) [-F2i | F2r]
  NLOS_TRY(gemm(n2, 2 * n2, n, 1.f, 0.f, L->Yb, 0, 2 * n2, 4 * nn, L->B2a, 0, n, 0, L->Zc, n2, 8 * nn));
  NLOS_TRY(gemm(n2, 2 * n2, n, 1.f, 1.f, L->Yb, n2, 2 * n2, 4 * nn, L->B2b, 0, n, 0, L->Zc, n2, 8 * nn));
  k_gemm_hmul<<<grid_for(4 * nn * planes), 256, 0, st>>>(L->Zc, P.d_H, n, planes, adj ? 1 : 0, L->Wb[0], L->Wb[1]);
  NLOS_LAUNCH_CHECK("k_gemm_hmul");
  // [Vr | Vi] (2N x 2N) = Wr (2N x 2N) [G1r | G1i] + Wi (2N x 2N) [-G1i | G1r]
  NLOS_TRY(gemm(n2, n2, n2, 1.f, 0.f, L->Wb, 0, n2, 8 * nn, L->B4a, 0, n2, 0, L->Vc, n2, 4 * nn));
  NLOS_TRY(gemm(n2, n2, n2, 1.f, 1.f, L->Wb, 4 * nn, n2, 8 * nn, L->B4b, 0, n2, 0, L->Vc, n2, 4 * nn));
  k_gemm_restack<<<grid_for(2 * nn * planes), 256, 0, st>>>(L->Vc, n, planes, L->Vs[0], L->Vs[1]);
  NLOS_LAUNCH_CHECK("k_gemm_restack");
  // [Or; Oi] (2N x N) = s A5 (2N x 4N) [Vr; Vi] (4N x N)
  NLOS_TRY(gemm(n2, n, 2 * n2, 1.0f / (4.0f * n * n), 0.f, L->A5, 0, n2, 0, L->Vs, 0, 2 * n2, 4 * nn, L->Os, n2,
                2 * nn));
  const int out_pitch = out_compact ? P.ncols : full;
  k_gemm_store<<<grid_for((out_compact ? (size_t)P.ncols : nn) * planes), 256, 0, st>>>(
      L->Os, n, planes, out_compact ? P.d_cols : nullptr, P.ncols, Sout, out_pitch);
  NLOS_LAUNCH_CHECK("k_gemm_store");
  return NLOS_OK;
}

}  // namespace nlos
