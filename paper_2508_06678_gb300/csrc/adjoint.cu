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

// The block that counts itself in last: every block's thread 0 has stored its partial; after a fence it adds
// one to the counter, and the block that sees kAdjDotBlocks - 1 there finds every partial stored.
__device__ bool adj_last_block(unsigned* counter) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// sum of n partials in a fixed order (lane i takes i, i + 32, ..., then a shuffle tree); lane 0 holds it
__device__ double adj_partials_sum(const double* partials, int n) {
  const volatile double* p = partials;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += p[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return s;
}

// the last block's share of a single sum: out = scale * sum, then kappa if asked, and the counter reset
__device__ void adj_dot_finish(const AdjDotOut& o) {
  if (!adj_last_block(o.counter) || threadIdx.x >= 32) return;
  const double s = adj_partials_sum(o.partials, gridDim.x);
  if (threadIdx.x == 0) {
    const double v = o.scale * s;
    o.out[0] = v;
    if (o.kappa) o.kappa[0] = (o.C[0] > 0.0 && o.mm[0] > 0.0) ? v / (o.n2 * o.mm[0]) : 0.0;
    *o.counter = 0u;
  }
}

__device__ __forceinline__ double spec_weight(const Geom& g, size_t e, int& ok) {
  const int c = (int)(e / g.SP), r = (int)(e - (size_t)c * g.SP);
  ok = c < g.Kc && r < g.Ny;
  return c == 0 ? 1.0 : 2.0;
}

// sum_k w_k Re(A conj B) over the stored band (w = 1 on the k_x = 0 column, else 2)
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_spec_dot_kernel(Geom g, const void* A, const void* B, AdjDotOut o) {
  pdl_enter();
  __shared__ double red[kThreads / 32];
  const size_t total = (size_t)g.Kcp * g.SP;
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int ok;
    const double w = spec_weight(g, e, ok);
    if (!ok) continue;
    const cplx_t<T> a = ld<T>(A, e), b = ld<T>(B, e);
    s += w * (double(a.x) * double(b.x) + double(a.y) * double(b.y));
  }
  s = adj_block_sum(s, red);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = s;
  adj_dot_finish(o);
}

// <H M> and <M M> in one pass (the two sums the separate dots would form, term by term); the last block adds
// C = max(0, <HM> / <MM>)
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_germano_dots_kernel(Geom g, const void* H, const void* M,
                                                                    AdjDotOut o) {
  pdl_enter();
  __shared__ double red[kThreads / 32];
  const size_t total = (size_t)g.Kcp * g.SP;
  double hm = 0.0, mm = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int ok;
    const double w = spec_weight(g, e, ok);
    if (!ok) continue;
    const cplx_t<T> a = ld<T>(H, e), b = ld<T>(M, e);
    hm += w * (double(a.x) * double(b.x) + double(a.y) * double(b.y));
    mm += w * (double(b.x) * double(b.x) + double(b.y) * double(b.y));
  }
  hm = adj_block_sum(hm, red);
  __syncthreads();  // red is reused
  mm = adj_block_sum(mm, red);
  if (threadIdx.x == 0) {
    o.partials[blockIdx.x] = hm;
    o.partials2[blockIdx.x] = mm;
  }
  if (!adj_last_block(o.counter) || threadIdx.x >= 32) return;
  const double shm = adj_partials_sum(o.partials, gridDim.x);
  const double smm = adj_partials_sum(o.partials2, gridDim.x);
  if (threadIdx.x == 0) {
    const double a = o.scale * shm, b = o.scale * smm;
    o.out[0] = a;
    o.out[1] = b;
    o.out[2] = b > 0.0 ? fmax(0.0, a / b) : 0.0;
    *o.counter = 0u;
  }
}

// sum_i x_i y_i z_i over physical points
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_phys_dot_kernel(size_t count, const void* X, const void* Y,
                                                                const void* Z, AdjDotOut o) {
  pdl_enter();
  __shared__ double red[kThreads / 32];
  const T* x = reinterpret_cast<const T*>(X);
  const T* y = reinterpret_cast<const T*>(Y);
  const T* z = reinterpret_cast<const T*>(Z);
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    s += double(x[i]) * double(y[i]) * double(z[i]);
  s = adj_block_sum(s, red);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = s;
  adj_dot_finish(o);
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
cudaError_t launch_adj_spec_dot(const Geom& g, const void* A, const void* B, const AdjDotOut& o, cudaStream_t st) {
  return launch_pdl(true, adj_spec_dot_kernel<T>, dim3(kAdjDotBlocks), dim3(kThreads), 0, st, g, A, B, o);
}

template <typename T>
cudaError_t launch_adj_germano_dots(const Geom& g, const void* H, const void* M, const AdjDotOut& o,
                                    cudaStream_t st) {
  return launch_pdl(true, adj_germano_dots_kernel<T>, dim3(kAdjDotBlocks), dim3(kThreads), 0, st, g, H, M, o);
}

template <typename T>
cudaError_t launch_adj_phys_dot(size_t count, const void* X, const void* Y, const void* Z, const AdjDotOut& o,
                                cudaStream_t st) {
  return launch_pdl(true, adj_phys_dot_kernel<T>, dim3(kAdjDotBlocks), dim3(kThreads), 0, st, count, X, Y, Z, o);
}

#define QG_ADJ_INST(T)                                                                                         \
  template cudaError_t launch_adj_combine<T>(const Geom&, const AdjCombine&, cudaStream_t);                    \
  template cudaError_t launch_adj_products<T>(size_t, const AdjProducts&, cudaStream_t);                       \
  template cudaError_t launch_adj_scale<T>(size_t, const void*, const void*, double, void*, const void*,       \
                                           double, void*, cudaStream_t);                                       \
  template cudaError_t launch_adj_spec_dot<T>(const Geom&, const void*, const void*, const AdjDotOut&,         \
                                              cudaStream_t);                                                   \
  template cudaError_t launch_adj_germano_dots<T>(const Geom&, const void*, const void*, const AdjDotOut&,     \
                                                  cudaStream_t);                                               \
  template cudaError_t launch_adj_phys_dot<T>(size_t, const void*, const void*, const void*, const AdjDotOut&, \
                                              cudaStream_t);
QG_ADJ_INST(float)
QG_ADJ_INST(double)
#undef QG_ADJ_INST

}  // namespace qg
