// Instantiation of the t-pass launchers for nt in {512}.
#define NLOS_TPASS_IMPL
#include "tpass.cuh"

namespace nlos {
template struct TpassOps<512>;
}  // namespace nlos
