// Row pass: for one physical row y, inverse x-transform every incoming field,
// form the pointwise products of the step in physical space (collocation,
// Sec. II-C), and forward x-transform the products.
//
// Two real fields share one complex N-point FFT: inputs are packed as
// Z = A + i B with the Hermitian extension of the two half spectra, outputs
// are split with A = (Z_k + conj Z_{N-k}) / 2, B = (Z_k - conj Z_{N-k}) / 2i.
// Only the kept columns m_x <= K are read or written (2/3 rule).
//
// Products (per grid point, working precision):
//   J  = u_total w_x + v w_y                             (Eq. 1)
//   g  = |grad w| = sqrt(w_x^2 + w_y^2)                  (Eq. 13)
//   g  = |S| = sqrt(4 psi_xy^2 + (psi_xx - psi_yy)^2)    (Eq. 10)
//   P  = g w_x (times i k_x after the transform),  Q = g w_y   (Eq. 9)
//   Brinkman / sponge: f <- f * exp(-rate chi dt)        (Eq. 2, 3; exact)
#include "fft.cuh"
#include "qg_kernels.h"

namespace qg {

template <typename T>
__device__ __forceinline__ void leith3(T u, T v, T wx, T wy, T& J, T& P, T& Q) {
  J = u * wx + v * wy;
  const T g = sqrt(wx * wx + wy * wy);
  P = g * wx;
  Q = g * wy;
}

template <typename T>
__device__ __forceinline__ void smag3(T u, T v, T wx, T wy, T pxy, T pd, T& J, T& P, T& Q) {
  J = u * wx + v * wy;
  const T g = sqrt(T(4) * pxy * pxy + pd * pd);
  P = g * wx;
  Q = g * wy;
}

template <typename T>
__global__ void __launch_bounds__(512) row_kernel(Geom g, FftPlan plan, RowDesc d, const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.n;
  C* work = reinterpret_cast<C*>(smem_raw);
  T* slots = reinterpret_cast<T*>(work + N);
  const int y = blockIdx.x;
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  // extents for the bounds-checked debug build: shared work row, physical slots, global arrays
  int* const st = d.err;
  unsigned dyn_smem = 0;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
  const long long nslot_el = ((long long)dyn_smem - (long long)N * (long long)sizeof(C)) / (long long)sizeof(T);
  const long long n_mixed = (long long)N * g.IP, n_phys = (long long)N * N;
  (void)nslot_el; (void)n_mixed; (void)n_phys; (void)st;

  if (d.flag) {
    const int stop = __syncthreads_or(*reinterpret_cast<volatile int*>(d.flag) != 0);
    if (stop) return;
  }

  // ---- inputs -> physical rows in slots
  if (d.in_phys) {
    const T* src = reinterpret_cast<const T*>(d.phys_in);
    for (int x = tid; x < N; x += nt) QG_ST(slots, x, nslot_el, st, QG_LD(src, (long long)y * N + x, n_phys, st));
    if (d.phys_in2) {
      const T* src2 = reinterpret_cast<const T*>(d.phys_in2);
      for (int x = tid; x < N; x += nt)
        QG_ST(slots, N + x, nslot_el, st, QG_LD(src2, (long long)y * N + x, n_phys, st));
    }
  } else {
    for (int p = 0; p < d.nin; p += 2) {
      const C* A = reinterpret_cast<const C*>(d.in[p]);
      const C* B = (p + 1 < d.nin) ? reinterpret_cast<const C*>(d.in[p + 1]) : nullptr;
      const long long row0 = (long long)y * g.IP;
      for (int k = tid; k < N; k += nt) {
        C z = mk<C>(T(0), T(0));
        if (k <= g.K) {
          C a = QG_LD(A, row0 + k, n_mixed, st);
          C b = B ? QG_LD(B, row0 + k, n_mixed, st) : mk<C>(T(0), T(0));
          if (k == 0) {
            a.y = T(0);
            b.y = T(0);
          }
          z = mk<C>(a.x - b.y, a.y + b.x);
        } else if (k >= N - g.K) {
          const C a = QG_LD(A, row0 + N - k, n_mixed, st);
          const C b = B ? QG_LD(B, row0 + N - k, n_mixed, st) : mk<C>(T(0), T(0));
          z = mk<C>(a.x + b.y, b.x - a.y);
        }
        QG_ST(work, k, N, st, z);
      }
      fft_batched<C>(work, plan, 1, tw, +1, st);
      for (int x = tid; x < N; x += nt) {
        const C z = QG_LD(work, x, N, st);
        QG_ST(slots, (long long)p * N + x, nslot_el, st, z.x);
        if (B) QG_ST(slots, (long long)(p + 1) * N + x, nslot_el, st, z.y);
      }
      __syncthreads();
    }
  }
  __syncthreads();

  // ---- pointwise products, in place in the slots
  int bad = 0;
  const T* fac = d.factor ? reinterpret_cast<const T*>(d.factor) : nullptr;
  for (int x = tid; x < N; x += nt) {
#ifdef QG_CHECKED
    // every slot this point's program touches lies inside the dynamic shared memory
    const int used = d.nin > d.nout ? d.nin : d.nout;
    if (!QG_INB((long long)(used - 1) * N + x, nslot_el, st)) continue;
#endif
    T* s = slots + x;
#define S(i) s[(size_t)(i) * N]
    switch (d.prog) {
      case RP_NONE: {
        const T J = S(0) * S(2) + S(1) * S(3);
        S(0) = J;
        break;
      }
      case RP_LEITH: {
        T J, P, Q;
        leith3<T>(S(0), S(1), S(2), S(3), J, P, Q);
        S(0) = J; S(1) = P; S(2) = Q;
        break;
      }
      case RP_SMAG: {
        T J, P, Q;
        smag3<T>(S(0), S(1), S(2), S(3), S(4), S(5), J, P, Q);
        S(0) = J; S(1) = P; S(2) = Q;
        break;
      }
      case RP_DLEITH: {
        T J, P, Q, Jt, Pt, Qt;
        leith3<T>(S(0), S(1), S(2), S(3), J, P, Q);
        leith3<T>(S(4), S(5), S(6), S(7), Jt, Pt, Qt);
        S(0) = J; S(1) = P; S(2) = Q; S(3) = Jt; S(4) = Pt; S(5) = Qt;
        break;
      }
      case RP_DSMAG: {
        T J, P, Q, Jt, Pt, Qt;
        smag3<T>(S(0), S(1), S(2), S(3), S(4), S(5), J, P, Q);
        smag3<T>(S(6), S(7), S(8), S(9), S(10), S(11), Jt, Pt, Qt);
        S(0) = J; S(1) = P; S(2) = Q; S(3) = Jt; S(4) = Pt; S(5) = Qt;
        break;
      }
      case RP_SCALE: {
        const T f = QG_LD(fac, (long long)y * N + x, n_phys, st);
        for (int i = 0; i < d.nin; ++i) S(i) = S(i) * f;
        break;
      }
      default:
        break;
    }
    if (d.check_finite) {
      for (int i = 0; i < d.nout; ++i) bad |= !isfinite(S(i));
    }
#undef S
  }
  if (d.check_finite && d.flag) {
    if (__syncthreads_or(bad) && tid == 0) atomicOr(d.flag, 1);
  }

  // ---- physical rows -> forward x-transform -> mixed arrays
  if (d.out_phys) {
    __syncthreads();
    T* dst = reinterpret_cast<T*>(d.phys_out);
    for (int x = tid; x < N; x += nt) QG_ST(dst, (long long)y * N + x, n_phys, st, QG_LD(slots, x, nslot_el, st));
    if (d.phys_out2) {
      T* dst2 = reinterpret_cast<T*>(d.phys_out2);
      for (int x = tid; x < N; x += nt)
        QG_ST(dst2, (long long)y * N + x, n_phys, st, QG_LD(slots, N + x, nslot_el, st));
    }
    return;
  }
  const T ks = T(g.kscale);
  for (int p = 0; p < d.nout; p += 2) {
    __syncthreads();
    const bool two = p + 1 < d.nout;
    for (int x = tid; x < N; x += nt)
      QG_ST(work, x, N, st,
            mk<C>(QG_LD(slots, (long long)p * N + x, nslot_el, st),
                  two ? QG_LD(slots, (long long)(p + 1) * N + x, nslot_el, st) : T(0)));
    fft_batched<C>(work, plan, 1, tw, -1, st);
    C* A = reinterpret_cast<C*>(d.out[p]);
    C* B = two ? reinterpret_cast<C*>(d.out[p + 1]) : nullptr;
    const long long row0 = (long long)y * g.IP;
    const bool dxa = (d.dx_mask >> p) & 1u;
    const bool dxb = (d.dx_mask >> (p + 1)) & 1u;
    for (int k = tid; k < g.Kcp; k += nt) {
      C a = mk<C>(T(0), T(0)), b = mk<C>(T(0), T(0));
      if (k < g.Kc) {
        const C z = QG_LD(work, k, N, st);
        const C zm = QG_LD(work, (N - k) % N, N, st);
        a = mk<C>(T(0.5) * (z.x + zm.x), T(0.5) * (z.y - zm.y));
        b = mk<C>(T(0.5) * (z.y + zm.y), T(-0.5) * (z.x - zm.x));
        const T kx = ks * T(k);
        if (dxa) a = cmul_ik(a, kx);
        if (dxb) b = cmul_ik(b, kx);
      }
      QG_ST(A, row0 + k, n_mixed, st, a);
      if (two) QG_ST(B, row0 + k, n_mixed, st, b);
    }
  }
}

template <typename T>
cudaError_t launch_row(const Geom& g, const FftPlan& plan, const RowDesc& d, const void* tw, int threads,
                       size_t smem, cudaStream_t st) {
  auto k = row_kernel<T>;
  cudaError_t e = raise_smem_limit<row_kernel<T>>(smem);
  if (e != cudaSuccess) return e;
  k<<<g.n, threads, smem, st>>>(g, plan, d, reinterpret_cast<const cplx_t<T>*>(tw));
  return cudaGetLastError();
}

template cudaError_t launch_row<float>(const Geom&, const FftPlan&, const RowDesc&, const void*, int, size_t, cudaStream_t);
template cudaError_t launch_row<double>(const Geom&, const FftPlan&, const RowDesc&, const void*, int, size_t, cudaStream_t);

}  // namespace qg
