// Runtime dispatch of the t-pass launchers to their per-size instances
// (tpass_*.cu).
#include <type_traits>

#include "tpass.cuh"

namespace nlos {

extern template struct TpassOps<16>;
extern template struct TpassOps<32>;
extern template struct TpassOps<64>;
extern template struct TpassOps<128>;
extern template struct TpassOps<256>;
extern template struct TpassOps<512>;
extern template struct TpassOps<1024>;

#define NLOS_DISPATCH_NT(nt, call)                                  \
  switch (nt) {                                                      \
    case 16: return TpassOps<16>::call;                              \
    case 32: return TpassOps<32>::call;                              \
    case 64: return TpassOps<64>::call;                              \
    case 128: return TpassOps<128>::call;                            \
    case 256: return TpassOps<256>::call;                            \
    case 512: return TpassOps<512>::call;                            \
    case 1024: return TpassOps<1024>::call;                          \
  }                                                                  \
  return fail(NLOS_ERR_INVALID_ARG, "unsupported nt")

nlos_status prepare_tpass(int nt) { NLOS_DISPATCH_NT(nt, prepare()); }

nlos_status launch_tfwd_rz(const Plan& P, const float* u, int ncols, float2* S, int pitch, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tfwd_rz(P, u, ncols, S, pitch, st));
}
nlos_status launch_tfwd_rtt(const Plan& P, const Lin3& r, int ncols, float2* S, int pitch, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tfwd_rtt(P, r, ncols, S, pitch, st));
}
nlos_status launch_tinv_store(const Plan& P, const float2* S, int pitch, int ncols, float* out,
                              const int32_t* outmap, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tinv_store(P, S, pitch, ncols, out, outmap, st));
}
nlos_status launch_tinv_fit(const Plan& P, const float2* S, int pitch, int ncols, float* out, const FitArgs& fa,
                            int* nblocks, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tinv_fit(P, S, pitch, ncols, out, fa, nblocks, st));
}
nlos_status launch_tadj_store(const Plan& P, const float2* S, int pitch, int ncols, float* out, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tadj_store(P, S, pitch, ncols, out, st));
}
nlos_status launch_tadj_solve(const Plan& P, const float2* S, int pitch, int ncols, const SolveRhs& sr, float2* Sp,
                              cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, tadj_solve(P, S, pitch, ncols, sr, Sp, st));
}
nlos_status launch_sfwd(const Plan& P, const float* x, int ncols, float2* Sp, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, sfwd(P, x, ncols, Sp, st));
}
nlos_status launch_sinv(const Plan& P, const float2* Sp, int ncols, float* x, const float* ref, double* partials,
                        int* nblocks, cudaStream_t st) {
  NLOS_DISPATCH_NT(P.nt, sinv(P, Sp, ncols, x, ref, partials, nblocks, st));
}

}  // namespace nlos
