// Diagnostics reductions and precision conversion.
//
// Energy and enstrophy of the state by Parseval over the stored half
// spectrum, in FP64 (E = sum w |k|^2 |psi|^2 / (2 N^4), Z = sum w |w|^2 /
// (2 N^4), w = 1 on the k_x = 0 column and 2 elsewhere).  Reductions are
// two-level and deterministic: fixed per-block partials, then one block sums
// them in a fixed order.
#include "qg_kernels.h"

namespace qg {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// blockDim.x must be 256
template <typename T>
__global__ void spectral_sums_kernel(Geom g, const cplx_t<T>* __restrict__ w, double* partials) {
  __shared__ double s[2][8];
  const int tid = threadIdx.x;
  const double ks2 = g.kscale * g.kscale;
  const size_t total = (size_t)g.Kc * g.Ny;
  double e = 0.0, z = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + tid; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / g.Ny), r = (int)(i - (size_t)c * g.Ny);
    const int my = my_of_r(g, r);
    const cplx_t<T> v = w[(size_t)c * g.SP + r];
    const double a2 = double(v.x) * double(v.x) + double(v.y) * double(v.y);
    const double wt = c == 0 ? 1.0 : 2.0;
    const double k2 = ks2 * double(c * c + my * my);
    z += wt * a2;
    if (k2 > 0.0) e += wt * a2 / k2;
  }
  e = warp_sum(e);
  z = warp_sum(z);
  if ((tid & 31) == 0) {
    s[0][tid >> 5] = e;
    s[1][tid >> 5] = z;
  }
  __syncthreads();
  if (tid < 32) {
    e = tid < 8 ? s[0][tid] : 0.0;
    z = tid < 8 ? s[1][tid] : 0.0;
    e = warp_sum(e);
    z = warp_sum(z);
    if (tid == 0) {
      partials[2 * blockIdx.x] = e;
      partials[2 * blockIdx.x + 1] = z;
    }
  }
}

__global__ void finish_sums_kernel(const double* partials, int nblk, double n4, double* out) {
  const int tid = threadIdx.x;
  double e = 0.0, z = 0.0;
  for (int i = tid; i < nblk; i += 32) {
    e += partials[2 * i];
    z += partials[2 * i + 1];
  }
  e = warp_sum(e);
  z = warp_sum(z);
  if (tid == 0) {
    out[0] = e / (2.0 * n4);
    out[1] = z / (2.0 * n4);
  }
}

template <typename T>
cudaError_t launch_spectral_sums(const Geom& g, const void* w0, double* partials, int nblk, double* out,
                                 cudaStream_t st) {
  spectral_sums_kernel<T><<<nblk, 256, 0, st>>>(g, reinterpret_cast<const cplx_t<T>*>(w0), partials);
  const double n2 = double(g.n) * double(g.n);
  finish_sums_kernel<<<1, 32, 0, st>>>(partials, nblk, n2 * n2, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void maxabs_kernel(const T* __restrict__ f, size_t count, double* partials) {
  __shared__ double s[2][8];
  const int tid = threadIdx.x;
  double m = 0.0, bad = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + tid; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double v = double(f[i]);
    if (!isfinite(v)) bad = 1.0;
    else m = fmax(m, fabs(v));
  }
  m = warp_max(m);
  bad = warp_max(bad);
  if ((tid & 31) == 0) {
    s[0][tid >> 5] = m;
    s[1][tid >> 5] = bad;
  }
  __syncthreads();
  if (tid < 32) {
    m = tid < 8 ? s[0][tid] : 0.0;
    bad = tid < 8 ? s[1][tid] : 0.0;
    m = warp_max(m);
    bad = warp_max(bad);
    if (tid == 0) {
      partials[2 * blockIdx.x] = m;
      partials[2 * blockIdx.x + 1] = bad;
    }
  }
}

__global__ void finish_max_kernel(const double* partials, int nblk, double* out) {
  const int tid = threadIdx.x;
  double m = 0.0, bad = 0.0;
  for (int i = tid; i < nblk; i += 32) {
    m = fmax(m, partials[2 * i]);
    bad = fmax(bad, partials[2 * i + 1]);
  }
  m = warp_max(m);
  bad = warp_max(bad);
  if (tid == 0) {
    out[0] = m;
    out[1] = bad > 0.0 ? 0.0 : 1.0;
  }
}

template <typename T>
cudaError_t launch_phys_maxabs(const Geom& g, const void* f, double* partials, int nblk, double* out,
                               cudaStream_t st) {
  maxabs_kernel<T><<<nblk, 256, 0, st>>>(reinterpret_cast<const T*>(f), (size_t)g.n * g.n, partials);
  finish_max_kernel<<<1, 32, 0, st>>>(partials, nblk, out);
  return cudaGetLastError();
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = D(src[i]);
}

cudaError_t launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, size_t count, cudaStream_t st) {
  const int blocks = 1216;
  if (src_fp32 && !dst_fp32)
    convert_kernel<float, double><<<blocks, 256, 0, st>>>((const float*)src, (double*)dst, count);
  else if (!src_fp32 && dst_fp32)
    convert_kernel<double, float><<<blocks, 256, 0, st>>>((const double*)src, (float*)dst, count);
  else if (src_fp32)
    convert_kernel<float, float><<<blocks, 256, 0, st>>>((const float*)src, (float*)dst, count);
  else
    convert_kernel<double, double><<<blocks, 256, 0, st>>>((const double*)src, (double*)dst, count);
  return cudaGetLastError();
}

template cudaError_t launch_spectral_sums<float>(const Geom&, const void*, double*, int, double*, cudaStream_t);
template cudaError_t launch_spectral_sums<double>(const Geom&, const void*, double*, int, double*, cudaStream_t);
template cudaError_t launch_phys_maxabs<float>(const Geom&, const void*, double*, int, double*, cudaStream_t);
template cudaError_t launch_phys_maxabs<double>(const Geom&, const void*, double*, int, double*, cudaStream_t);

}  // namespace qg
