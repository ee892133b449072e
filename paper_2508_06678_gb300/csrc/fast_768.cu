// Specialised passes for N = 768 (3 * 2^p, engine E12); see fast_kernels.cuh.
#include "fast_kernels.cuh"

namespace qg {
QG_INSTANTIATE_FAST(768)
}  // namespace qg
