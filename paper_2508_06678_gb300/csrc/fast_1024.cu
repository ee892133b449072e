// Specialised passes for N = 1024 (power of two); see fast_kernels.cuh.
#include "fast_kernels.cuh"

namespace qg {
QG_INSTANTIATE_FAST(1024)
}  // namespace qg
