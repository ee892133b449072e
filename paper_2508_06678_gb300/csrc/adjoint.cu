// Kernels of the discrete adjoint of the RK3 step (the step's vector-Jacobian
// product, qg_step_vjp) and of the step's unfused recomputation from w_n.
//
// With the inner product sum over grid points, the transpose of a spectral
// multiplier m(k) is its complex conjugate, the 2/3 truncation and the mean
// removal are their own transposes, and a pointwise product by a field is its
// own transpose.  The adjoint therefore needs three kinds of kernels besides
// the library's transform passes:
//   adj_combine   out = [out] + sum_j c_j m_j(k) in_j(k) over the stored band,
//                 m_j one of the multipliers below (conjugated where the
//                 adjoint needs it);
//   adj_products  pointwise products of the forward fields (J, g w_x, g w_y)
//                 and of the adjoint field with them (Eq. 1, 10, 13 linearised);
//   adj_dot       FP64 inner products: spectral (Parseval, exact for real
//                 fields) and physical (three-factor) sums, deterministic.
#include <cmath>

#include "qg_kernels.h"

namespace qg {

namespace {

template <typename T>
__device__ __forceinline__ cplx_t<T> ld(const void* p, size_t i) {
  return reinterpret_cast<const cplx_t<T>*>(p)[i];
}

constexpr int kThreads = 256;

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kThreads) adj_combine_kernel(Geom g, AdjCombine a) {
  pdl_enter();
  using C = cplx_t<T>;
  const size_t total = (size_t)g.Kcp * g.SP;
  C* out = reinterpret_cast<C*>(a.out);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / g.SP), r = (int)(e - (size_t)c * g.SP);
    if (c >= g.Kc || r >= g.Ny) {
      if (!a.accumulate) out[e] = mk<C>(T(0), T(0));
      continue;
    }
    const int my = my_of_r(g, r);
    const double kx = g.kscale * c, ky = g.kscale * my;
    const double k2 = kx * kx + ky * ky;
    const double ik2 = k2 > 0.0 ? 1.0 / k2 : 0.0;
    double re = 0.0, im = 0.0;
    if (a.accumulate) {
      const C o = out[e];
      re = double(o.x);
      im = double(o.y);
    }
    const bool in_test = (long)c * c + (long)my * my <= (long)a.test_m2max;
    for (int j = 0; j < a.nterm; ++j) {
      const int code = a.term[j].code;
      if ((code & AM_TESTF) && !in_test) continue;
      const C x = ld<T>(a.term[j].in, e);
      const double xr = double(x.x), xi = double(x.y);
      const double cf = a.term[j].cptr ? a.term[j].coef * a.term[j].cptr[0] : a.term[j].coef;
      double mr = 0.0, mi = 0.0;  // multiplier m = mr + i mi
      switch (code & 0xff) {
        case AM_ONE: mr = 1.0; break;
        case AM_CU: mi = -ky * ik2; break;  // conj(i k_y / |k|^2): transpose of w -> u
        case AM_CV: mi = kx * ik2; break;   // conj(-i k_x / |k|^2): transpose of w -> v
        case AM_CX: mi = -kx; break;        // conj(i k_x)
        case AM_CY: mi = -ky; break;        // conj(i k_y)
        case AM_IX: mi = kx; break;
        case AM_IY: mi = ky; break;
        case AM_XY: mr = kx * ky * ik2; break;              // w -> psi_xy (real)
        case AM_DD: mr = (kx * kx - ky * ky) * ik2; break;  // w -> psi_xx - psi_yy (real)
        case AM_VISC: mr = exp(-(a.nu * k2 + a.mu) * a.dt); break;
        default: break;
      }
      re += cf * (mr * xr - mi * xi);
      im += cf * (mr * xi + mi * xr);
    }
    if (a.zero_mean && c == 0 && my == 0) re = im = 0.0;
    out[e] = mk<C>(T(re), T(im));
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) adj_products_kernel(size_t count, AdjProducts a) {
  pdl_enter();
  auto L = [](const void* p, size_t i) { return reinterpret_cast<const T*>(p)[i]; };
  auto S = [&](int k, size_t i, T v) { reinterpret_cast<T*>(a.out[k])[i] = v; };
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const T wx = L(a.wx, i), wy = L(a.wy, i);
    T g = T(0), pxy = T(0), pd = T(0);
    if (a.kind == AK_LEITH) {
      g = sqrt(wx * wx + wy * wy);  // |grad w| (Eq. 13)
    } else if (a.kind == AK_SMAG) {
      pxy = L(a.pxy, i);
      pd = L(a.pd, i);
      g = sqrt(T(4) * pxy * pxy + pd * pd);  // |S| (Eq. 10)
    }
    if (a.mode == AP_FORWARD) {
      const T u = L(a.u, i), v = L(a.v, i);
      S(0, i, u * wx + v * wy);  // J (Eq. 1)
      if (a.kind != AK_NONE) {
        S(1, i, g * wx);
        S(2, i, g * wy);
      }
    } else {
      const T u = L(a.u, i), v = L(a.v, i), lam = L(a.lam, i);
      S(0, i, lam * wx);
      S(1, i, lam * wy);
      S(2, i, lam * u);
      S(3, i, lam * v);
      if (a.kind != AK_NONE) {
        // p, q: the transposed derivatives of lam; s multiplies the variation of g
        const T p = -L(a.lx, i), q = -L(a.ly, i);
        const T s = p * wx + q * wy;
        const T ig = g > T(0) ? T(1) / g : T(0);
        if (a.kind == AK_LEITH) {
          S(4, i, g * p + s * wx * ig);
          S(5, i, g * q + s * wy * ig);
        } else {
          S(4, i, g * p);
          S(5, i, g * q);
          S(6, i, T(4) * s * pxy * ig);
          S(7, i, s * pd * ig);
        }
      }
    }
  }
}

// out0 = s0 f x0, out1 = s1 f x1 (out1 skipped when x1 is null)
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_scale_kernel(size_t count, const void* f, const void* x0, T s0,
                                                             void* out0, const void* x1, T s1, void* out1) {
  pdl_enter();
  const T* F = reinterpret_cast<const T*>(f);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    reinterpret_cast<T*>(out0)[i] = s0 * F[i] * reinterpret_cast<const T*>(x0)[i];
    if (x1) reinterpret_cast<T*>(out1)[i] = s1 * F[i] * reinterpret_cast<const T*>(x1)[i];
  }
}

__device__ double adj_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// per-block partial of sum_k w_k Re(A conj B) over the stored band (w = 1 on the k_x = 0 column, else 2)
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_spec_dot_kernel(Geom g, const void* A, const void* B,
                                                                double* partials) {
  pdl_enter();
  __shared__ double red[kThreads / 32];
  const size_t total = (size_t)g.Kcp * g.SP;
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / g.SP), r = (int)(e - (size_t)c * g.SP);
    if (c >= g.Kc || r >= g.Ny) continue;
    const cplx_t<T> a = ld<T>(A, e), b = ld<T>(B, e);
    s += (c == 0 ? 1.0 : 2.0) * (double(a.x) * double(b.x) + double(a.y) * double(b.y));
  }
  s = adj_block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// per-block partial of sum_i x_i y_i z_i over physical points
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_phys_dot_kernel(size_t count, const void* X, const void* Y,
                                                                const void* Z, double* partials) {
  pdl_enter();
  __shared__ double red[kThreads / 32];
  const T* x = reinterpret_cast<const T*>(X);
  const T* y = reinterpret_cast<const T*>(Y);
  const T* z = reinterpret_cast<const T*>(Z);
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    s += double(x[i]) * double(y[i]) * double(z[i]);
  s = adj_block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void adj_scalar_kernel(int op, const double* x0, const double* x1, const double* x2, double n2,
                                  double* out) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  if (op == AS_COEFF) {
    out[0] = x1[0] > 0.0 ? fmax(0.0, x0[0] / x1[0]) : 0.0;
  } else {
    out[0] = (x0[0] > 0.0 && x1[0] > 0.0) ? x2[0] / (n2 * x1[0]) : 0.0;
  }
}

cudaError_t launch_adj_scalar(int op, const double* x0, const double* x1, const double* x2, double n2, double* out,
                              cudaStream_t st) {
  return launch_pdl(true, adj_scalar_kernel, dim3(1), dim3(32), 0, st, op, x0, x1, x2, n2, out);
}

// out[0] = scale * sum of the partials, in a fixed order
__global__ void adj_finish_kernel(const double* partials, int n, double scale, double* out) {
  pdl_enter();
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += partials[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[0] = scale * s;
}

namespace {
unsigned grid_for(size_t count) {
  const size_t b = (count + kThreads - 1) / kThreads;
  return (unsigned)(b < 1024 ? (b ? b : 1) : 1024);
}
}  // namespace

template <typename T>
cudaError_t launch_adj_combine(const Geom& g, const AdjCombine& a, cudaStream_t st) {
  return launch_pdl(true, adj_combine_kernel<T>, dim3(grid_for((size_t)g.Kcp * g.SP)), dim3(kThreads), 0, st, g, a);
}

template <typename T>
cudaError_t launch_adj_products(size_t count, const AdjProducts& a, cudaStream_t st) {
  return launch_pdl(true, adj_products_kernel<T>, dim3(grid_for(count)), dim3(kThreads), 0, st, count, a);
}

template <typename T>
cudaError_t launch_adj_scale(size_t count, const void* f, const void* x0, double s0, void* out0, const void* x1,
                             double s1, void* out1, cudaStream_t st) {
  return launch_pdl(true, adj_scale_kernel<T>, dim3(grid_for(count)), dim3(kThreads), 0, st, count, f, x0, T(s0), out0, x1,
                    T(s1), out1);
}

template <typename T>
cudaError_t launch_adj_spec_dot(const Geom& g, const void* A, const void* B, double scale, double* partials,
                                double* out, cudaStream_t st) {
  const cudaError_t e = launch_pdl(true, adj_spec_dot_kernel<T>, dim3(kAdjDotBlocks), dim3(kThreads), 0, st, g, A, B,
                                   partials);
  if (e != cudaSuccess) return e;
  return launch_pdl(true, adj_finish_kernel, dim3(1), dim3(32), 0, st, (const double*)partials, (int)kAdjDotBlocks, scale,
                    out);
}

template <typename T>
cudaError_t launch_adj_phys_dot(size_t count, const void* X, const void* Y, const void* Z, double scale,
                                double* partials, double* out, cudaStream_t st) {
  const cudaError_t e = launch_pdl(true, adj_phys_dot_kernel<T>, dim3(kAdjDotBlocks), dim3(kThreads), 0, st, count, X, Y,
                                   Z, partials);
  if (e != cudaSuccess) return e;
  return launch_pdl(true, adj_finish_kernel, dim3(1), dim3(32), 0, st, (const double*)partials, (int)kAdjDotBlocks, scale,
                    out);
}

#define QG_ADJ_INST(T)                                                                                         \
  template cudaError_t launch_adj_combine<T>(const Geom&, const AdjCombine&, cudaStream_t);                    \
  template cudaError_t launch_adj_products<T>(size_t, const AdjProducts&, cudaStream_t);                       \
  template cudaError_t launch_adj_scale<T>(size_t, const void*, const void*, double, void*, const void*,       \
                                           double, void*, cudaStream_t);                                       \
  template cudaError_t launch_adj_spec_dot<T>(const Geom&, const void*, const void*, double, double*, double*, \
                                              cudaStream_t);                                                   \
  template cudaError_t launch_adj_phys_dot<T>(size_t, const void*, const void*, const void*, double, double*,  \
                                              double*, cudaStream_t);
QG_ADJ_INST(float)
QG_ADJ_INST(double)
#undef QG_ADJ_INST

}  // namespace qg
