// Specialised passes for N = 256 (power of two); see fast_kernels.cuh.
#include "fast_kernels.cuh"

namespace qg {
QG_INSTANTIATE_FAST(256)
}  // namespace qg
