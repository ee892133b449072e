// Host-side declarations of the kernel launchers of libqg.
#pragma once

#include "fft.cuh"

namespace qg {

template <typename T>
cudaError_t launch_row(const Geom& g, const FftPlan& plan, const RowDesc& d, const void* tw, int threads,
                       size_t smem, cudaStream_t st);

template <typename T>
cudaError_t launch_col(const Geom& g, const FftPlan& plan, const ColDesc& d, const void* tw, int W, int threads,
                       size_t smem, cudaStream_t st);

// Spectral diagnostics: out[0] = sum w |k|^2 |psi|^2, out[1] = sum w |w|^2 over the stored half spectrum
// (w = 1 on the k_x = 0 column, else 2), FP64, deterministic two-level reduction.
template <typename T>
cudaError_t launch_spectral_sums(const Geom& g, const void* w0, double* partials, int nblk, double* out,
                                 cudaStream_t st);

// Physical max |f| and finiteness: out[0] = max |f|, out[1] = 1 if all finite else 0.
template <typename T>
cudaError_t launch_phys_maxabs(const Geom& g, const void* f, double* partials, int nblk, double* out,
                               cudaStream_t st);

// Sets the thread-local message returned by qg_last_error().
void set_last_error(const char* msg);

// Element-wise precision conversion between device buffers.
cudaError_t launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, size_t count, cudaStream_t st);

}  // namespace qg
