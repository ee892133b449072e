// Specialised passes for N = 4096 (power of two); see fast_kernels.cuh.
#include "fast_kernels.cuh"

namespace qg {
QG_INSTANTIATE_FAST(4096)
}  // namespace qg
