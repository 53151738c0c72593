// Instantiation of the t-pass launchers for nt in {16, 32, 64, 128}.
#define NLOS_TPASS_IMPL
#include "tpass.cuh"

namespace nlos {
template struct TpassOps<16>;
template struct TpassOps<32>;
template struct TpassOps<64>;
template struct TpassOps<128>;
}  // namespace nlos
