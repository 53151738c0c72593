// Instantiation of the t-pass launchers for nt in {256}.
#define NLOS_TPASS_IMPL
#include "tpass.cuh"

namespace nlos {
template struct TpassOps<256>;
}  // namespace nlos
