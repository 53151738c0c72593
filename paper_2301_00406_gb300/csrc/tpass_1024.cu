// Instantiation of the t-pass launchers for nt in {1024}.
#define NLOS_TPASS_IMPL
#include "tpass.cuh"

namespace nlos {
template struct TpassOps<1024>;
}  // namespace nlos
