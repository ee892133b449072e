// Specialised passes for N = 2048 (power of two); see fast_kernels.cuh.
#include "fast_kernels.cuh"

namespace qg {
QG_INSTANTIATE_FAST(2048)
}  // namespace qg
