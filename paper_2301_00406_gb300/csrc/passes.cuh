// Declarations of the FFT-pass launchers implemented in lct.cu and the
// stencil/reduction launchers implemented in admm.cu.
#pragma once

#include "common.cuh"

namespace nlos {

// A linear combination of up to three [cols][nt] sources, with coefficients
// either fixed or taken from the device scalars (extrapolated residual
// r = (1 + beta) P0 - beta P1 - P2, beta = sc->beta_prev).
struct Lin3 {
  const float* p[3];
  float c[3];
  const DevScalars* sc;  // non-null: c = {1 + beta_prev, -beta_prev, -1}
};

// Epilogue of the forward t-inverse pass.
struct FitArgs {
  const float* data;   // [cols][nt] data the fit is measured against (tau0 or tau-bar)
  const float* auk;    // [cols][nt] A u^k (cache)
  const float* aukm1;  // [cols][nt] A u^{k-1} (cache)
  const DevScalars* sc;
  double* partials;    // [gridDim][kMaxTerms]: 0 = sum (A u - data)^2, 1 = sum (A u - A u-bar)^2
  // optional (full columns only): Sp receives the periodic t-spectrum of
  // A u + x2, the right-hand side of Algorithm 2's tau solve
  const float* x2 = nullptr;
  float2* Sp = nullptr;
  // false when the backtracking test cannot reject (its A d term is then
  // neither loaded nor summed; partial 1 stays 0)
  bool need_d = true;
};

// Solve-mode arguments of the adjoint end pass: rhs = c0 * ubar - grad f + reg.
struct SolveRhs {
  const float* ubar;
  const float* reg;
  const DevScalars* sc;  // c0 = sc->L when non-null, else c0_host
  double c0_host;
};

// Forward t-pass of A: u~ = R_z u, zero-pad to 2 nt, real FFT -> S[kt][col],
// kt in [0, nt].  u: [ncols][nt] (column col at u + col*nt).
nlos_status launch_tfwd_rz(const Plan& P, const float* u, int ncols, float2* S, int pitch, cudaStream_t st);
// Adjoint start: c = R_t^{-T} r with r from Lin3, then the same padded FFT.
nlos_status launch_tfwd_rtt(const Plan& P, const Lin3& r, int ncols, float2* S, int pitch, cudaStream_t st);
// Forward t-inverse: C2R of length 2 nt, keep [0, nt), tau = R_t^{-1} c.
// outmap (nullable) maps column j to the output column index.
nlos_status launch_tinv_store(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                              const int32_t* outmap, cudaStream_t st);
nlos_status launch_tinv_fit(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                            const FitArgs& fa, int* nblocks, cudaStream_t st);
// Adjoint end: C2R, crop, R_z^T -> g.  Store g, or form the solve rhs and
// run the periodic real FFT into Sp[k][col], k in [0, nt/2].
nlos_status launch_tadj_store(const Plan& P, const float2* S, int pitch, int ncols, float* out, cudaStream_t st);
nlos_status launch_tadj_solve(const Plan& P, const float2* S, int pitch, int ncols, const SolveRhs& sr,
                              float2* Sp, cudaStream_t st);
// Periodic real FFT of a field (of x + x2 when x2 is given), and its inverse
// (optionally with partial sums of (x - ref)^2 into partials[block][0]).
nlos_status launch_sfwd(const Plan& P, const float* x, int ncols, float2* Sp, cudaStream_t st,
                        const float* x2 = nullptr);
nlos_status launch_sinv(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref,
                        double* partials, int* nblocks, cudaStream_t st);
// launch_sinv followed by launch_tfwd_rz(x -> S) in one pass (x kept on chip).
// sc (nullable): the solver's scalars, whose status a timed-out wait of the
// full-grid kernel sets to NLOS_ERR_TIMEOUT.
nlos_status launch_sinv_rz(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref,
                           double* partials, int* nblocks, float2* S, int pitch, cudaStream_t st,
                           DevScalars* sc = nullptr);
// Full-grid tadj (solve mode) and sinv_rz passes with one warp per column
// pair and TMA tile transfers (tpass_warp.cu), for nt in {128, 256, 512};
// launch_tadj_solve and launch_sinv_rz dispatch to them when
// tpass_warp_applies (the column count and pitch are the full grid).
bool tpass_warp_applies(const Plan& P, int ncols, int pitch);
// The fit pass also runs on compact columns (the sampled columns of A_D)
// when their count is a multiple of 16.
bool tpass_warp_applies_cols(const Plan& P, int ncols, int pitch);
nlos_status prepare_tpass_warp(int nt);
nlos_status launch_tadj_solve_warp(const Plan& P, const float2* S, int pitch, const SolveRhs& sr, float2* Sp,
                                   cudaStream_t st);
nlos_status launch_sinv_rz_warp(const Plan& P, const float2* Sp, int pitch, float* x, const float* ref,
                                double* partials, int* nblocks, float2* S, DevScalars* sc, cudaStream_t st);
// ... and the full-grid sinv, tinv (fit) and tfwd (R_t^{-T}) passes, to which
// launch_sinv, launch_tinv_fit and launch_tfwd_rtt dispatch likewise.
nlos_status launch_sinv_warp(const Plan& P, const float2* Sp, int pitch, float* x, const float* ref,
                             double* partials, int* nblocks, cudaStream_t st);
nlos_status launch_tinv_fit_warp(const Plan& P, const float2* S, int pitch, float* out, const FitArgs& fa,
                                 int* nblocks, cudaStream_t st);
nlos_status launch_tfwd_rtt_warp(const Plan& P, const Lin3& r, float2* S, int pitch, cudaStream_t st);
// nlos_selftest_wait_timeout (tpass_warp.cu).
nlos_status selftest_wait_timeout(int32_t wait_ms, int32_t* status_dev, cudaStream_t st);
// Lateral 2-D zero-padded convolution of each kt plane with H (adj: conj H).
// in_cols/out_cols: nullptr = full plane [nx][ny]; else compact column lists
// (the plan's sampled columns) with plane pitch ncols.
nlos_status launch_conv(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact,
                        bool adj, cudaStream_t st);
// The same on the tensor cores (plans with P.lateral set; conv_tc.cu).
nlos_status launch_conv_tc(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact,
                           bool adj, cudaStream_t st);
// Select the lateral stage: 0 FFT kernels, 1 tcgen05 MMAs on split-BF16
// operands (three products), 2 the same with the hi terms only.  Builds the
// block DFT constant and the rearranged kernel spectrum on the first non-zero
// mode (synchronises st).
nlos_status set_lateral_mode(Plan& P, int mode, cudaStream_t st);
void free_lateral_tc(Plan* P);
// NLOS_ERR_TIMEOUT (and the flag cleared) if a wait of the tensor-core
// lateral kernel gave up since the last check; synchronous.
nlos_status lateral_status(const Plan& P);
// Four-CTA-cluster lateral convolution for nx in {32, 64, 128} (conv4.cu);
// launch_conv dispatches to it.
nlos_status launch_conv4(const Plan& P, const float2* Sin, bool in_compact, float2* Sout, bool out_compact,
                         bool adj, cudaStream_t st);
nlos_status prepare_conv4(int n);
// Periodic lateral solve per kt plane: divide by c0 + c1 (lx + ly + lt).
nlos_status launch_sxy(const Plan& P, float2* Sp, const DevScalars* sc, double c0_host, double c1,
                       cudaStream_t st);
// Cone-kernel spectrum of the plan (plan time).
nlos_status launch_kernel_spectrum(const Plan& P, const int32_t* m0, const float2* hw, cudaStream_t st);

// Launch-shape tuning of the t-passes.  Every t-pass kind picks its columns
// per CTA (16, 8, 4 or 2) and, where the kernel has two halves (even and odd
// bins of the padded transform), whether they run as one batched FFT, by
// timing at plan creation (autotune_tpass, on the plan's own scratch
// buffers); the choice is cached for the whole process per (kind, nt, launch
// column count), so all plans of a geometry launch the same shapes and their
// block-partial reductions sum in the same order.  TPK_SXY is not a t-pass:
// for the lateral periodic solve of N x N planes (N >= 32) it picks the
// kernel, keyed by (TPK_SXY, nt, N): kSxyPasses (the transform steps as
// CTA-wide passes over the plane in shared memory, k_sxy) or kSxyHalfWarp
// (every transform in the registers of a half-warp, k_sxy_w).
enum TpKind {
  TPK_TFWD_RZ, TPK_TFWD_RTT, TPK_TINV_STORE, TPK_TINV_FIT, TPK_TADJ_STORE, TPK_TADJ_SOLVE, TPK_SFWD, TPK_SINV,
  TPK_SINV_RZ, TPK_SXY
};
constexpr int kSxyPasses = 1, kSxyHalfWarp = 2;
// Tuned shape of a launch, cols | hb << 8, or 0 (use the default rule).
int tp_cols_for(int kind, int nt, int ncols);
nlos_status autotune_tpass(Plan& P, cudaStream_t st);

// Pre-set the shared-memory attributes of every kernel for these sizes.
nlos_status prepare_tpass(int nt);
nlos_status prepare_xy(int n);

}  // namespace nlos
