// Specialised passes for N = 512 (power of two); see fast_kernels.cuh.
#include "fast_kernels.cuh"

namespace qg {
QG_INSTANTIATE_FAST(512)
}  // namespace qg
