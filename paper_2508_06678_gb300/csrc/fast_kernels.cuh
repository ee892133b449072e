// Specialised row / column passes on the register-resident engines (E16 for N = 2^p, E12 for N = 3 * 2^p).
// Same arithmetic and data layouts as row.cu / column.cu (see there for the
// equations); only the FFT organisation differs.  Included by fast_<N>.cu,
// one translation unit per grid size.
#pragma once

#include <atomic>

#include "fast.cuh"
#include "qg_kernels.h"
#include "tma.cuh"

#ifndef QG_ROW_MINB
#define QG_ROW_MINB 4
#endif
#ifndef QG_COL_MINB
#define QG_COL_MINB 2
#endif
#ifndef QG_COL_MINB_REDUCE
#define QG_COL_MINB_REDUCE 2
#endif
#ifndef QG_LEAN_BATCH
#define QG_LEAN_BATCH 4
#endif
#ifndef QG_COL_MINB_FWD
#define QG_COL_MINB_FWD 1
#endif
#ifndef QG_COL_MINB_CURL
#define QG_COL_MINB_CURL 2
#endif

namespace qg {
namespace fast {

template <int N> struct RowCfg {
  static constexpr int TT = N / elems_per_thread(N);
  static constexpr int ROWS = TT >= QG_ROW_CTA_THREADS ? 1 : QG_ROW_CTA_THREADS / TT;
  static constexpr int THREADS = TT * ROWS;
};
// resident CTAs per SM requested from the register allocator (FP32; FP64 takes 1)
template <typename T, int OP = -1> struct Occ {
  static constexpr int row = QG_ROW_MINB * 128 / QG_ROW_CTA_THREADS > 0 ? QG_ROW_MINB * 128 / QG_ROW_CTA_THREADS : 1;
  static constexpr int col = OP == CO_DYN_REDUCE ? QG_COL_MINB_REDUCE
                             : (OP == CO_FORWARD || OP == CO_FORWARD2 || OP == CO_FORWARD_N ||
                                OP == CO_AB2CN_FINAL) ? QG_COL_MINB_FWD
                             : OP == CO_CURL    ? QG_COL_MINB_CURL
                                                : QG_COL_MINB;
};
template <int OP> struct Occ<double, OP> { static constexpr int row = 1, col = 1; };

#ifndef QG_COL_W
#define QG_COL_W 2
#endif
template <int N> struct ColCfg {
  static constexpr int W = QG_COL_W;  // k_x columns per CTA
  static constexpr int TT = N / elems_per_thread(N);
  static constexpr int THREADS = W * TT;
  // column stride in shared memory (complex elements): 16 / W mod 16 keeps the exchanges conflict-free
  static constexpr int CP = N + N / 16 + 16 / W;
  static constexpr int BR = fast_box_rows(N);  // rows per TMA box
  static constexpr int NBOX = N / BR;
};
// bytes of one shared-memory stage: a dense W x N tile for TMA, or W padded exchange columns
template <typename T, int N> __host__ __device__ constexpr int col_stage_bytes() {
  constexpr int dense = N * ColCfg<N>::W * 2 * (int)sizeof(T);
  constexpr int padded = ColCfg<N>::W * ColCfg<N>::CP * 2 * (int)sizeof(T);
  return ((dense > padded ? dense : padded) + 1023) / 1024 * 1024;
}
// three lean Germano-reduction CTAs (exchange buffer + one stage + alignment slack each) fit in shared memory
template <typename T, int N> constexpr bool lean_fits() {
  return sizeof(T) == 4 && 3 * (2 * col_stage_bytes<T, N>() + 2048) <= 227 * 1024;
}
// column ops whose FFTs use the packed FP32 butterflies (bit op set): all but the dynamic combine and the final
// passes (CO_DYN_COMBINE, CO_FORWARD, CO_AB2CN_FINAL), which measured 0.3-1.1 us faster per launch in the scalar
// form at 2048^2 (the row passes and the Germano reduction gain 7% and 6% from packing)
#ifndef QG_PACKED_COL_MASK
#define QG_PACKED_COL_MASK 0xFED7
#endif
template <int OP> constexpr bool col_packed() { return (QG_PACKED_COL_MASK >> OP) & 1; }
// bounded device waits: about one second of SM clocks
constexpr long long kWaitCycles = 2000000000LL;

template <typename T>
__device__ __forceinline__ void leith_p(T u, T v, T wx, T wy, T& J, T& P, T& Q) {
  J = u * wx + v * wy;
  const T g = sqrt(wx * wx + wy * wy);
  P = g * wx;
  Q = g * wy;
}

template <typename T>
__device__ __forceinline__ void smag_p(T u, T v, T wx, T wy, T pxy, T pd, T& J, T& P, T& Q) {
  J = u * wx + v * wy;
  const T g = sqrt(T(4) * pxy * pxy + pd * pd);
  P = g * wx;
  Q = g * wy;
}

// ---------------------------------------------------------------------------
// Row pass
// ---------------------------------------------------------------------------
template <typename T, int N>
struct RowCtx {
  using E = Eng<T, N>;
  using C = cplx_t<T>;
  static constexpr int TT = E::TT;
  int t, y;
  C* b0;
  C* b1;
  int ph;
  const C* tw;  // per-pass twiddle table
  const Geom* g;
  int bad;

  // inverse x-transform of the pair (A + i B) of half-spectrum rows; B may be null
  __device__ __forceinline__ void inv_pair(C* x, const void* Av, const void* Bv) {
    const C* A = reinterpret_cast<const C*>(Av) + (size_t)y * g->IP;
    const C* B = Bv ? reinterpret_cast<const C*>(Bv) + (size_t)y * g->IP : nullptr;
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      const int k = t + TT * m;
      C z = mk<C>(T(0), T(0));
      if (k <= E::K) {
        C a = A[k];
        C b = B ? B[k] : mk<C>(T(0), T(0));
        if (k == 0) {
          a.y = T(0);
          b.y = T(0);
        }
        z = mk<C>(a.x - b.y, a.y + b.x);
      } else if (k >= N - E::K) {
        const C a = A[N - k];
        const C b = B ? B[N - k] : mk<C>(T(0), T(0));
        z = mk<C>(a.x + b.y, b.x - a.y);
      }
      x[m] = z;
    }
    E::run(x, t, b0, b1, ph, tw, +1);
  }

  // forward x-transform of (re, im) = two real rows, split, optional i k_x, store kept columns
  __device__ __forceinline__ void fwd_store(C* x, void* Av, void* Bv, bool dxa, bool dxb) {
    E::run(x, t, b0, b1, ph, tw, -1);
    split_store(x, Av, Bv, dxa, dxb);
  }

  // split the forward transform of two real rows (re, im) into their half spectra, optional i k_x, store the
  // kept columns
  __device__ __forceinline__ void split_store(C* x, void* Av, void* Bv, bool dxa, bool dxb) {
    C* ub = ph ? b1 : b0;
    ph ^= 1;
#pragma unroll
    for (int m = 0; m < E::EL; ++m) ub[E::pad(t + TT * m)] = x[m];
    __syncthreads();
    C* A = reinterpret_cast<C*>(Av) + (size_t)y * g->IP;
    C* B = Bv ? reinterpret_cast<C*>(Bv) + (size_t)y * g->IP : nullptr;
    const T ks = T(g->kscale);
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      const int k = t + TT * m;
      if (k < g->Kcp) {
        C a = mk<C>(T(0), T(0)), b = mk<C>(T(0), T(0));
        if (k < E::Kc) {
          const C z = x[m];
          const C zm = ub[E::pad(k == 0 ? 0 : N - k)];
          a = mk<C>(T(0.5) * (z.x + zm.x), T(0.5) * (z.y - zm.y));
          b = mk<C>(T(0.5) * (z.y + zm.y), T(-0.5) * (z.x - zm.x));
          const T kx = ks * T(k);
          if (dxa) a = cmul_ik(a, kx);
          if (dxb) b = cmul_ik(b, kx);
        }
        A[k] = a;
        if (B) B[k] = b;
      }
    }
  }

  __device__ __forceinline__ void check(const T* v) {
#pragma unroll
    for (int m = 0; m < E::EL; ++m) bad |= !isfinite(v[m]);
  }
};

// One level of the stage products: inverse-transform (u, v), (w_x, w_y)
// [and (psi_xy, psi_xx - psi_yy)] and form J = u w_x + v w_y, P = g w_x,
// Q = g w_y with g = |grad w| (Leith) or |S| (Smagorinsky); NONE forms J only.
template <typename T, int N, bool SMAG, bool NONE>
__device__ __forceinline__ void level_products(RowCtx<T, N>& cx, cplx_t<T>* x, const void* const* in, T* J, T* P,
                                               T* Q) {
  using C = cplx_t<T>;
  using E = Eng<T, N>;
  cx.inv_pair(x, in[0], in[1]);
#pragma unroll
  for (int m = 0; m < E::EL; ++m) {
    J[m] = x[m].x;  // u_total
    P[m] = x[m].y;  // v
  }
  cx.inv_pair(x, in[2], in[3]);  // (w_x, w_y)
  if constexpr (SMAG) {
    C s[E::EL];
    cx.inv_pair(s, in[4], in[5]);
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      T j, p, q;
      smag_p<T>(J[m], P[m], x[m].x, x[m].y, s[m].x, s[m].y, j, p, q);
      J[m] = j;
      P[m] = p;
      Q[m] = q;
    }
  } else if constexpr (NONE) {
#pragma unroll
    for (int m = 0; m < E::EL; ++m) J[m] = J[m] * x[m].x + P[m] * x[m].y;
  } else {
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      T j, p, q;
      leith_p<T>(J[m], P[m], x[m].x, x[m].y, j, p, q);
      J[m] = j;
      P[m] = p;
      Q[m] = q;
    }
  }
  cx.check(J);
  if constexpr (!NONE) {
    cx.check(P);
    cx.check(Q);
  }
}

template <typename T, int N, int PROG>
__global__ void __launch_bounds__(RowCfg<N>::THREADS, Occ<T>::row) row_fast_kernel(Geom g, RowDesc d,
                                                                       const cplx_t<T>* __restrict__ tw) {
  pdl_enter();
  using E = Eng<T, N>;
  using C = cplx_t<T>;
  constexpr int TT = E::TT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int lr = threadIdx.x / TT;
  RowCtx<T, N> cx;
  cx.t = threadIdx.x % TT;
  cx.y = blockIdx.x * RowCfg<N>::ROWS + lr;
  cx.b0 = sm + (size_t)(2 * lr) * E::BUF;
  cx.b1 = cx.b0 + E::BUF;
  cx.ph = 0;
  cx.tw = tw;
  cx.g = &g;
  cx.bad = 0;
  if (d.flag) {
    if (__syncthreads_or(*reinterpret_cast<volatile int*>(d.flag) != 0)) return;
  }
  const int t = cx.t;
  const size_t yN = (size_t)cx.y * N;
  C x[E::EL];

  if constexpr (PROG == RP_NONE || PROG == RP_LEITH || PROG == RP_SMAG || PROG == RP_DLEITH || PROG == RP_DSMAG) {
    constexpr bool smag = PROG == RP_SMAG || PROG == RP_DSMAG;
    constexpr bool dyn = PROG == RP_DLEITH || PROG == RP_DSMAG;
    constexpr bool none = PROG == RP_NONE;
    constexpr int per = smag ? 6 : 4;  // inputs per level
    T J[E::EL], P[E::EL], Q[E::EL];
    level_products<T, N, smag, none>(cx, x, d.in + 0, J, P, Q);
    if constexpr (none) {
#pragma unroll
      for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(J[m], T(0));
      cx.fwd_store(x, d.out[0], nullptr, false, false);
    } else {
      // outputs: 0 J, 1 P (times i k_x), 2 Q [, 3 J~, 4 P~ (times i k_x), 5 Q~]
#pragma unroll
      for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(J[m], P[m]);
      cx.fwd_store(x, d.out[0], d.out[1], false, true);
      if constexpr (!dyn) {
#pragma unroll
        for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(Q[m], T(0));
        cx.fwd_store(x, d.out[2], nullptr, false, false);
      } else {
        T Qk[E::EL];
#pragma unroll
        for (int m = 0; m < E::EL; ++m) Qk[m] = Q[m];
        level_products<T, N, smag, false>(cx, x, d.in + per, J, P, Q);
#pragma unroll
        for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(Qk[m], Q[m]);
        cx.fwd_store(x, d.out[2], d.out[5], false, false);
#pragma unroll
        for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(J[m], P[m]);
        cx.fwd_store(x, d.out[3], d.out[4], false, true);
      }
    }
  } else if constexpr (PROG == RP_SCALE) {
    // Brinkman (2 fields) or sponge (1 field): multiply by the exact factor field
    const T* fac = reinterpret_cast<const T*>(d.factor) + yN;
    cx.inv_pair(x, d.in[0], d.nin > 1 ? d.in[1] : nullptr);
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      const T f = fac[t + TT * m];
      x[m] = mk<C>(x[m].x * f, x[m].y * f);
      cx.bad |= !isfinite(x[m].x) | !isfinite(x[m].y);
    }
    cx.fwd_store(x, d.out[0], d.nout > 1 ? d.out[1] : nullptr, false, false);
  } else if constexpr (PROG == RP_ADJ_FWD) {
    // one stage of the step recomputed for its adjoint: inverse transforms of (u_total, v), (w_x, w_y)
    // [, (psi_xy, psi_d)], which are kept as physical fields, then J, g w_x, g w_y (Eq. 1, 9, 10, 13) forward
    // transformed without the i k_x factor (the adjoint's spectral combine applies it)
    const int kind = d.adj_kind;
    T U[E::EL], V[E::EL];
    cx.inv_pair(x, d.in[0], d.in[1]);
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      U[m] = x[m].x;
      V[m] = x[m].y;
      reinterpret_cast<T*>(d.pf[0])[yN + t + TT * m] = U[m];
      reinterpret_cast<T*>(d.pf[1])[yN + t + TT * m] = V[m];
    }
    cx.inv_pair(x, d.in[2], d.in[3]);
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      reinterpret_cast<T*>(d.pf[2])[yN + t + TT * m] = x[m].x;
      reinterpret_cast<T*>(d.pf[3])[yN + t + TT * m] = x[m].y;
    }
    T G[E::EL];
    if (kind == 1) {
      C sv[E::EL];
      cx.inv_pair(sv, d.in[4], d.in[5]);
#pragma unroll
      for (int m = 0; m < E::EL; ++m) {
        reinterpret_cast<T*>(d.pf[4])[yN + t + TT * m] = sv[m].x;
        reinterpret_cast<T*>(d.pf[5])[yN + t + TT * m] = sv[m].y;
        G[m] = sqrt(T(4) * sv[m].x * sv[m].x + sv[m].y * sv[m].y);
      }
    } else {
#pragma unroll
      for (int m = 0; m < E::EL; ++m) G[m] = sqrt(x[m].x * x[m].x + x[m].y * x[m].y);
    }
    T Q[E::EL];
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      const T wx = x[m].x, wy = x[m].y;
      const T J = U[m] * wx + V[m] * wy;
      Q[m] = G[m] * wy;
      x[m] = mk<C>(J, kind == 0 ? T(0) : G[m] * wx);
    }
    cx.fwd_store(x, d.out[0], kind == 0 ? nullptr : d.out[1], false, false);
    if (kind != 0) {
#pragma unroll
      for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(Q[m], T(0));
      cx.fwd_store(x, d.out[2], nullptr, false, false);
    }
  } else if constexpr (PROG == RP_ADJ_REV) {
    // transposed products of one stage (the linearisation of Eq. 1, 9, 10, 13): the adjoint field lam and the
    // transposed derivatives p = -lam_x, q = -lam_y against the kept fields u_total, v, w_x, w_y [, psi_xy,
    // psi_d]: lam w_x, lam w_y, lam u, lam v, then g p + s w_x / g, g q + s w_y / g (Leith) or g p, g q,
    // 4 s psi_xy / g, s psi_d / g (Smagorinsky), s = p w_x + q w_y; pairs forward transformed
    const int kind = d.adj_kind;
    T LM[E::EL], P[E::EL];
    cx.inv_pair(x, d.in[0], d.in[1]);  // (lam, lam_x)
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      LM[m] = x[m].x;
      P[m] = -x[m].y;
    }
    cx.inv_pair(x, d.in[2], nullptr);  // lam_y
    T Qv[E::EL];
#pragma unroll
    for (int m = 0; m < E::EL; ++m) Qv[m] = -x[m].x;
    const T* fu = reinterpret_cast<const T*>(d.pf[0]) + yN;
    const T* fv = reinterpret_cast<const T*>(d.pf[1]) + yN;
    const T* fwx = reinterpret_cast<const T*>(d.pf[2]) + yN;
    const T* fwy = reinterpret_cast<const T*>(d.pf[3]) + yN;
#pragma unroll
    for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(LM[m] * fwx[t + TT * m], LM[m] * fwy[t + TT * m]);
    cx.fwd_store(x, d.out[0], d.out[1], false, false);
#pragma unroll
    for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(LM[m] * fu[t + TT * m], LM[m] * fv[t + TT * m]);
    cx.fwd_store(x, d.out[2], d.out[3], false, false);
    if (kind != 0) {
      T S6[E::EL], S7[E::EL];
#pragma unroll
      for (int m = 0; m < E::EL; ++m) {
        const T wx = fwx[t + TT * m], wy = fwy[t + TT * m];
        const T s = P[m] * wx + Qv[m] * wy;
        T g, a, b;
        if (kind == 1) {
          const T pxy = reinterpret_cast<const T*>(d.pf[4])[yN + t + TT * m];
          const T pd = reinterpret_cast<const T*>(d.pf[5])[yN + t + TT * m];
          g = sqrt(T(4) * pxy * pxy + pd * pd);
          const T ig = g > T(0) ? T(1) / g : T(0);
          a = g * P[m];
          b = g * Qv[m];
          S6[m] = T(4) * s * pxy * ig;
          S7[m] = s * pd * ig;
        } else {
          g = sqrt(wx * wx + wy * wy);
          const T ig = g > T(0) ? T(1) / g : T(0);
          a = g * P[m] + s * wx * ig;
          b = g * Qv[m] + s * wy * ig;
          S6[m] = T(0);
          S7[m] = T(0);
        }
        x[m] = mk<C>(a, b);
      }
      cx.fwd_store(x, d.out[4], d.out[5], false, false);
      if (kind == 1) {
#pragma unroll
        for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(S6[m], S7[m]);
        cx.fwd_store(x, d.out[6], d.out[7], false, false);
      }
    }
  } else if (d.npair > 0) {  // RP_COPY of npair pairs in one launch (one FFT code copy, a runtime loop)
#pragma unroll 1
    for (int p = 0; p < d.npair; ++p) {
      if (d.in_phys) {
        const T* src = reinterpret_cast<const T*>(d.pin[2 * p]) + yN;
        const T* src2 = d.pin[2 * p + 1] ? reinterpret_cast<const T*>(d.pin[2 * p + 1]) + yN : nullptr;
#pragma unroll
        for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(src[t + TT * m], src2 ? src2[t + TT * m] : T(0));
        cx.fwd_store(x, d.out[2 * p], src2 ? d.out[2 * p + 1] : nullptr, false, false);
      } else {
        void* dst2v = d.pout[2 * p + 1];
        cx.inv_pair(x, d.in[2 * p], dst2v ? d.in[2 * p + 1] : nullptr);
        T* dst = reinterpret_cast<T*>(d.pout[2 * p]) + yN;
#pragma unroll
        for (int m = 0; m < E::EL; ++m) dst[t + TT * m] = x[m].x;
        if (dst2v) {
          T* dst2 = reinterpret_cast<T*>(dst2v) + yN;
#pragma unroll
          for (int m = 0; m < E::EL; ++m) dst2[t + TT * m] = x[m].y;
        }
      }
    }
  } else {  // RP_COPY: one or two physical rows in or out (two as the real and imaginary parts of one FFT)
    if (d.in_phys) {
      const T* src = reinterpret_cast<const T*>(d.phys_in) + yN;
      const T* src2 = d.phys_in2 ? reinterpret_cast<const T*>(d.phys_in2) + yN : nullptr;
#pragma unroll
      for (int m = 0; m < E::EL; ++m) x[m] = mk<C>(src[t + TT * m], src2 ? src2[t + TT * m] : T(0));
      cx.fwd_store(x, d.out[0], src2 ? d.out[1] : nullptr, false, false);
    } else {
      cx.inv_pair(x, d.in[0], d.phys_out2 ? d.in[1] : nullptr);
      T* dst = reinterpret_cast<T*>(d.phys_out) + yN;
#pragma unroll
      for (int m = 0; m < E::EL; ++m) dst[t + TT * m] = x[m].x;
      if (d.phys_out2) {
        T* dst2 = reinterpret_cast<T*>(d.phys_out2) + yN;
#pragma unroll
        for (int m = 0; m < E::EL; ++m) dst2[t + TT * m] = x[m].y;
      }
    }
  }
  if (d.check_finite && d.flag) {
    if (__syncthreads_or(cx.bad) && threadIdx.x == 0) atomicOr(d.flag, 1);
  }
}

// ---------------------------------------------------------------------------
// Column pass
// ---------------------------------------------------------------------------
template <typename T> struct FInvK2;
template <> struct FInvK2<double> {
  __device__ static double get(double ks2, int m2) { return m2 == 0 ? 0.0 : 1.0 / (ks2 * double(m2)); }
};
template <> struct FInvK2<float> {
  __device__ static float get(double ks2, int m2) {
    if (m2 == 0) return 0.f;
    if (m2 <= 16) return float(1.0 / (ks2 * double(m2)));
    return 1.f / (float(ks2) * float(m2));
  }
};

// modes per batch in the column pass's state update (loads of a batch precede its stores)
#ifndef QG_STATE_BATCH
#define QG_STATE_BATCH 8
#endif
constexpr int kStateBatch = QG_STATE_BATCH;

// LEAN (the FP32 Germano reduction only): the cross-field values go to global scratch rather than registers
// and the tiles come through one TMA stage, so three CTAs fit on an SM.  The launcher picks it when that turns
// a partial second wave of column CTAs into one wave.
template <typename T, int N, int OP, bool LEAN = false>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, LEAN ? 3 : Occ<T, OP>::col) col_fast_kernel(
    Geom g, ColDesc d, const cplx_t<T>* __restrict__ tw, const __grid_constant__ TmaSet tm) {
  pdl_enter();
  using E = Eng<T, N>;
  using C = cplx_t<T>;
  constexpr int W = ColCfg<N>::W;
  constexpr int TT = E::TT;
  constexpr int CP = ColCfg<N>::CP;
  constexpr int K = E::K;
  constexpr int Ny = 2 * K + 1;
  constexpr int BR = ColCfg<N>::BR;
  constexpr int NBOX = ColCfg<N>::NBOX;
  constexpr int SB = col_stage_bytes<T, N>();
  constexpr uint32_t FIELD_BYTES = (uint32_t)N * W * 2 * sizeof(T);
  // shared memory: exchange buffer | stage 0 | stage 1.  A stage receives a
  // field's dense W x N tile by TMA, then serves as the FFT's second exchange
  // buffer, and in the inverse phase holds the dense output tile for the TMA store.
  extern __shared__ __align__(1024) unsigned char smem_col[];
  __shared__ double red[2][32];
  __shared__ __align__(8) uint64_t mbar[2];
  // TMA tiles need 128-byte aligned shared addresses: align the base explicitly (1 KB slack is allocated)
  unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_col) + 1023) & ~uintptr_t(1023));
  constexpr int NSTG = LEAN ? 1 : 2;  // TMA stages of the forward fields
  C* xbuf = reinterpret_cast<C*>(sbase);
  C* stage[2] = {reinterpret_cast<C*>(sbase + SB), reinterpret_cast<C*>(sbase + (NSTG == 2 ? 2 : 1) * SB)};
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int mx = blockIdx.x * W + c;
  const int c0 = blockIdx.x * W;
  const bool col_ok = mx < E::Kc;
  const bool lead = threadIdx.x == 0;
  int ph = 0;
  const C* twb = tw;
  if (d.flag) {
    if (__syncthreads_or(*reinterpret_cast<volatile int*>(d.flag) != 0)) return;
  }
  // thread 0 starts the first NSTG forward fields' tiles
  if (lead) {
    tma::mbar_init(&mbar[0], 1);
    tma::mbar_init(&mbar[1], 1);
    tma::fence_mbar_init();
    if constexpr (OP != CO_DERIVE && OP != CO_DYN_COMBINE && OP != CO_AB2CN_COMBINE) {
      const bool stall = (int)blockIdx.x + 1 == d.stall_cta1;
      if (stall && d.nfwd > 0) {
        // injected stall (failure-handling test): the first tile is expected but never requested
        tma::mbar_expect_tx(&mbar[0], FIELD_BYTES);
      }
      for (int f = 0; f < d.nfwd && f < NSTG && !stall; ++f) {
        tma::mbar_expect_tx(&mbar[f], FIELD_BYTES);
        for (int bx = 0; bx < NBOX; ++bx)
          tma::load_2d(reinterpret_cast<unsigned char*>(stage[f]) + (size_t)bx * BR * W * sizeof(C), &tm.in[f],
                       2 * c0, bx * BR, &mbar[f]);
      }
    }
  }
  __syncthreads();
  const double ks2 = g.kscale * g.kscale;
  const double n2 = double(N) * double(N);
  const T kxv = T(g.kscale) * T(mx);
  C* w0 = reinterpret_cast<C*>(d.w0);
  C* ws = reinterpret_cast<C*>(d.ws);
  C* jh = reinterpret_cast<C*>(d.jh);
  C* dh = reinterpret_cast<C*>(d.dh);
  const size_t colbase = (size_t)mx * g.SP;

  C x[E::EL], A[E::EL], B[E::EL];
  GermanoAcc<T> acc_hm, acc_mm;

  // ---- forward y-transforms (k values land in natural ownership: k = t + TT m)
  if constexpr (OP != CO_DERIVE && OP != CO_DYN_COMBINE && OP != CO_AB2CN_COMBINE) {
#pragma unroll 1
    for (int f = 0; f < d.nfwd; ++f) {
      const int sidx = f % NSTG;
      const uint32_t par = (f / NSTG) & 1;
      C* st = stage[sidx];
      const bool ok = tma::mbar_wait(&mbar[sidx], par, kWaitCycles);
      if (__syncthreads_or(!ok)) {
        // a tile never arrived: report, give the copy one more bounded wait, leave together
        if (lead) {
          if (d.err) atomicOr(d.err, kFlagTimeout);
          tma::mbar_wait(&mbar[sidx], par, kWaitCycles);
        }
        __syncthreads();
        return;
      }
#pragma unroll
      for (int m = 0; m < E::EL; ++m) x[m] = st[(t + TT * m) * W + c];
      ph = 0;
      E::template run<col_packed<OP>()>(x, t, xbuf + c * CP, st + c * CP, ph, twb, -1);
      // every thread is done with this stage: hand it to the TMA for field f + NSTG
      tma::fence_proxy_async();
      __syncthreads();
      if (lead && f + NSTG < d.nfwd) {
        tma::mbar_expect_tx(&mbar[sidx], FIELD_BYTES);
        for (int bx = 0; bx < NBOX; ++bx)
          tma::load_2d(reinterpret_cast<unsigned char*>(st) + (size_t)bx * BR * W * sizeof(C), &tm.in[f + NSTG],
                       2 * c0, bx * BR, &mbar[sidx]);
      }
      if constexpr (LEAN) {
        // The Germano reduction with its cross-field values in scratch (s0 = P, then the Brinkman
        // partial; s1 = -D, then r^p P~ - D; s2 = H): the same operations as the register form below.
        // Each thread reads back only what it wrote; a batch's loads are issued before its stores, since
        // the arrays may alias as far as the compiler can tell.
        C* s0 = reinterpret_cast<C*>(d.scr[0]);
        C* s1 = reinterpret_cast<C*>(d.scr[1]);
        C* s2 = reinterpret_cast<C*>(d.scr[2]);
        constexpr int LB = QG_LEAN_BATCH;
        static_assert(E::EL % LB == 0, "the load batch must divide the thread's elements");
#pragma unroll
        for (int m0 = 0; m0 < E::EL; m0 += LB) {
          C la[LB], lb[LB];
#pragma unroll
          for (int q = 0; q < LB; ++q) {
            const int k = t + TT * (m0 + q);
            const size_t gi = colbase + (k <= K ? k : k - N + Ny);
            la[q] = mk<C>(T(0), T(0));
            lb[q] = la[q];
            if (k <= K || k >= N - K) {
              if (f == 2 || f == 7) la[q] = s0[gi];
              else if (f == 3) la[q] = jh[gi];
              else if (f == 4 || f == 5) la[q] = s1[gi];
              if (f == 5) lb[q] = s2[gi];
            }
          }
#pragma unroll
          for (int q = 0; q < LB; ++q) {
            const int m = m0 + q;
            const int k = t + TT * m;
            if (!(k <= K || k >= N - K)) continue;
            const int my = k <= K ? k : k - N;
            const T ky = T(g.kscale) * T(my);
            const size_t gi = colbase + (k <= K ? k : k - N + Ny);
            const bool in_test = mx * mx + my * my <= d.test_m2max;
            const C X = col_ok ? x[m] : mk<C>(T(0), T(0));
            if (f == 0) {
              jh[gi] = X;
            } else if (f == 1) {
              s0[gi] = X;
            } else if (f == 2) {
              const C D = cadd(la[q], cmul_ik(X, ky));
              dh[gi] = D;
              s1[gi] = in_test ? mk<C>(-D.x, -D.y) : mk<C>(T(0), T(0));
            } else if (f == 3) {
              s2[gi] = in_test ? csub(X, la[q]) : X;
            } else if (f == 4) {
              s1[gi] = cadd(la[q], cscale(X, T(d.rpow)));
            } else if (f == 6) {
              s0[gi] = cscale(cmul_ik(X, ky), T(d.inv_eta));
            } else if (f == 7) {
              reinterpret_cast<C*>(d.bh)[gi] = csub(la[q], cscale(cmul_ik(X, kxv), T(d.inv_eta)));
            } else if (col_ok) {
              const C M = cadd(la[q], cscale(cmul_ik(X, ky), T(d.rpow)));
              const C H = lb[q];
              const T wgt = mx == 0 ? T(1) : T(2);
              acc_hm.add_prod(wgt * H.x, M.x);
              acc_hm.add_prod(wgt * H.y, M.y);
              acc_mm.add_prod(wgt * M.x, M.x);
              acc_mm.add_prod(wgt * M.y, M.y);
            }
          }
        }
      }
#pragma unroll
      for (int m = 0; m < E::EL && !LEAN; ++m) {
        const int k = t + TT * m;
        const int my = k <= K ? k : k - N;
        const T ky = T(g.kscale) * T(my);
        C X = col_ok ? x[m] : mk<C>(T(0), T(0));
        if constexpr (OP == CO_STAGE_STATIC) {
          if (f == 0) A[m] = mk<C>(-X.x, -X.y);
          else if (f == 1) B[m] = X;
          else B[m] = cadd(B[m], cmul_ik(X, ky));
        } else if constexpr (OP == CO_DYN_REDUCE) {
          const bool kept = k <= K || k >= N - K;
          const int r = k <= K ? k : k - N + Ny;
          const bool in_test = mx * mx + my * my <= d.test_m2max;
          if (f == 0) {
            A[m] = X;
            if (kept) jh[colbase + r] = X;
          } else if (f == 1) {
            B[m] = X;
          } else if (f == 2) {
            const C D = cadd(B[m], cmul_ik(X, ky));
            if (kept) dh[colbase + r] = D;
            B[m] = in_test ? mk<C>(-D.x, -D.y) : mk<C>(T(0), T(0));
          } else if (f == 3) {
            A[m] = in_test ? csub(X, A[m]) : X;
          } else if (f == 4) {
            B[m] = cadd(B[m], cscale(X, T(d.rpow)));
          } else if (f == 6) {  // Brinkman pair (paper's scheme): F_obs = (i ky F[chi u] - i kx F[chi v]) / eta
            A[m] = cscale(cmul_ik(X, ky), T(d.inv_eta));
          } else if (f == 7) {
            A[m] = csub(A[m], cscale(cmul_ik(X, kxv), T(d.inv_eta)));
            if (kept) reinterpret_cast<C*>(d.bh)[colbase + r] = A[m];
          } else {
            const C M = cadd(B[m], cscale(cmul_ik(X, ky), T(d.rpow)));
            const C H = A[m];
            if (kept && col_ok) {
              // weight 2 for k_x > 0 (the conjugate half), applied exactly
              const T wgt = mx == 0 ? T(1) : T(2);
              acc_hm.add_prod(wgt * H.x, M.x);
              acc_hm.add_prod(wgt * H.y, M.y);
              acc_mm.add_prod(wgt * M.x, M.x);
              acc_mm.add_prod(wgt * M.y, M.y);
            }
          }
        } else if constexpr (OP == CO_CURL) {
          if (f == 0) A[m] = X;
          else A[m] = csub(cmul_ik(X, kxv), cmul_ik(A[m], ky));
        } else if constexpr (OP == CO_AB2CN) {
          // E = -J + C D + F_obs: A collects -J + F_obs, B collects D
          if (f == 0) A[m] = mk<C>(-X.x, -X.y);
          else if (f < d.nst) B[m] = (f == 1) ? X : cadd(B[m], cmul_ik(X, ky));
          else if (f == d.nst) A[m] = cadd(A[m], cscale(cmul_ik(X, ky), T(d.inv_eta)));
          else A[m] = csub(A[m], cscale(cmul_ik(X, kxv), T(d.inv_eta)));
        } else if constexpr (OP == CO_FORWARD2) {
          if (f == 0) A[m] = X;
          else B[m] = X;
        } else if constexpr (OP == CO_FORWARD_N) {
          const bool kept = (k <= K || k >= N - K) && col_ok;
          if (kept) {
            const C v = (d.zero_mean && mx == 0 && my == 0) ? mk<C>(T(0), T(0)) : X;
            reinterpret_cast<C*>(d.fout[f])[colbase + (k <= K ? k : k - N + Ny)] = v;
          }
        } else {  // CO_FORWARD, CO_AB2CN_FINAL
          A[m] = X;
        }
      }
    }
  }

  if constexpr (OP == CO_FORWARD_N) {
    return;  // every field's band is stored; no state update, no derived fields, no bulk stores in flight
  } else if constexpr (OP == CO_DYN_REDUCE) {
    double hm = acc_hm.value(), mm = acc_mm.value();
    for (int o = 16; o > 0; o >>= 1) {
      hm += __shfl_down_sync(0xffffffffu, hm, o);
      mm += __shfl_down_sync(0xffffffffu, mm, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][wid] = hm;
      red[1][wid] = mm;
    }
    __syncthreads();
    if (wid == 0) {
      constexpr int nw = (ColCfg<N>::THREADS + 31) / 32;
      hm = lane < nw ? red[0][lane] : 0.0;
      mm = lane < nw ? red[1][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        hm += __shfl_down_sync(0xffffffffu, hm, o);
        mm += __shfl_down_sync(0xffffffffu, mm, o);
      }
      if (lane == 0) {
        d.partials[2 * blockIdx.x] = hm;
        d.partials[2 * blockIdx.x + 1] = mm;
      }
    }
    return;
  } else {
    T coeff = T(d.coeff);
    if constexpr (OP == CO_DYN_COMBINE || OP == CO_AB2CN_COMBINE) {
      if (threadIdx.x < 32) {
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < d.npartials; i += 32) {
          a += d.partials[2 * i];
          b += d.partials[2 * i + 1];
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_down_sync(0xffffffffu, a, o);
          b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (threadIdx.x == 0) {
          const double Cc = b > 0.0 ? fmax(0.0, a / b) : 0.0;
          red[0][0] = Cc;
          if (blockIdx.x == 0 && d.coeff_out) *d.coeff_out = Cc;
        }
      }
      __syncthreads();
      coeff = T(red[0][0]);
    }

    // ---- new state per owned mode (registers A).  The modes go in batches
    // of GB whose global loads are all issued before any of the batch's
    // stores: the state arrays may alias as far as the compiler can tell, so
    // a load placed after a store would wait for that store's round trip.
    const T dt = T(d.dt), a_rk = T(d.a), b_rk = T(d.b), beta = T(d.beta);
    const T* vx = reinterpret_cast<const T*>(d.visc_x);
    const T* vy = reinterpret_cast<const T*>(d.visc_y);
    const T vmu = T(d.visc_mu);
    const C* bhp = reinterpret_cast<const C*>(d.bh);
    C* ep = reinterpret_cast<C*>(d.eprev);
    C* wsp = reinterpret_cast<C*>(d.wss);
    constexpr int GB = E::EL % kStateBatch == 0 ? kStateBatch : 4;  // a divisor of the thread's elements
    static_assert(E::EL % GB == 0, "state batch must divide the elements per thread");
#pragma unroll
    for (int m0 = 0; m0 < E::EL; m0 += GB) {
      // per op: u0 = w^n (or w* in the AB2CN final), u1 = stage field or E_prev,
      // u2 = J, u3 = D, u4 = Brinkman forcing, u5 = previous w*; vf = viscous factor
      C u0[GB], u1[GB], u2[GB], u3[GB], u4[GB], u5[GB];
      T vf[GB];
#pragma unroll
      for (int q = 0; q < GB; ++q) {
        const int k = t + TT * (m0 + q);
        const bool kept = (k <= K || k >= N - K) && col_ok;
        const int r = k <= K ? k : k - N + Ny;
        const size_t gi = colbase + r;
        const C z = mk<C>(T(0), T(0));
        u0[q] = z; u1[q] = z; u2[q] = z; u3[q] = z; u4[q] = z; u5[q] = z;
        vf[q] = T(1);
        if (kept) {
          if constexpr (OP == CO_DERIVE) {
            u0[q] = w0[gi];
          } else if constexpr (OP == CO_STAGE_STATIC || OP == CO_DYN_COMBINE) {
            u0[q] = w0[gi];
            u1[q] = d.use_ws ? ws[gi] : u0[q];
            if constexpr (OP == CO_DYN_COMBINE) {
              u2[q] = jh[gi];
              u3[q] = dh[gi];
            }
          } else if constexpr (OP == CO_AB2CN || OP == CO_AB2CN_COMBINE) {
            u0[q] = w0[gi];
            if constexpr (OP == CO_AB2CN_COMBINE) {
              u2[q] = jh[gi];
              u3[q] = dh[gi];
              if (d.brink) u4[q] = bhp[gi];
            }
            if (!d.ab2_first) {
              u1[q] = ep[gi];
              if (d.sponge_next) u5[q] = wsp[gi];
            }
          } else if constexpr (OP == CO_AB2CN_FINAL) {
            u0[q] = wsp[gi];
          }
          if (d.viscous) vf[q] = vx[mx] * vy[r] * vmu;
        }
      }
#pragma unroll
      for (int q = 0; q < GB; ++q) {
        const int m = m0 + q;
        const int k = t + TT * m;
        const bool kept = (k <= K || k >= N - K) && col_ok;
        const int r = k <= K ? k : k - N + Ny;
        const int my = k <= K ? k : k - N;
        C wn = mk<C>(T(0), T(0));
        if (kept) {
          const size_t gi = colbase + r;
          if constexpr (OP == CO_DERIVE) {
            wn = u0[q];
          } else if constexpr (OP == CO_STAGE_STATIC || OP == CO_DYN_COMBINE) {
            const C wz = u0[q];
            const C wst = u1[q];
            const T ik2 = FInvK2<T>::get(ks2, mx * mx + my * my);
            const C psi = mk<C>(-wst.x * ik2, -wst.y * ik2);
            const C bv = cscale(cmul_ik(psi, kxv), beta);
            C L;
            if constexpr (OP == CO_STAGE_STATIC) {
              L = csub(A[m], bv);
              if (d.nfwd > 1) L = cadd(L, cscale(B[m], coeff));
            } else {
              L = csub(mk<C>(-u2[q].x, -u2[q].y), bv);
              L = cadd(L, cscale(u3[q], coeff));
            }
            const C inner = cadd(wst, cscale(L, dt));
            wn = cadd(cscale(wz, a_rk), cscale(inner, b_rk));
          } else if constexpr (OP == CO_AB2CN || OP == CO_AB2CN_COMBINE) {
            // Eq. 4: w* = ((1 + dt/2 lin) w^t + dt (3/2 E - 1/2 E_prev)) / (1 - dt/2 lin)
            C E;
            if constexpr (OP == CO_AB2CN) {
              E = (d.nst > 1) ? cadd(A[m], cscale(B[m], coeff)) : A[m];
            } else {
              E = cadd(mk<C>(-u2[q].x, -u2[q].y), cscale(u3[q], coeff));
              if (d.brink) E = cadd(E, u4[q]);
            }
            const C Ep = d.ab2_first ? E : u1[q];
            ep[gi] = E;
            const int m2 = mx * mx + my * my;
            const T k2 = T(ks2) * T(m2);
            const T ik2 = FInvK2<T>::get(ks2, m2);
            const T hdt = T(0.5) * dt;
            const T lre = -(T(d.nu) * k2 + T(d.mu));
            const T lim = beta * kxv * ik2;
            const C wz = u0[q];
            const C ab = mk<C>(T(1.5) * E.x - T(0.5) * Ep.x, T(1.5) * E.y - T(0.5) * Ep.y);
            const C num = cadd(cmul(mk<C>(T(1) + hdt * lre, hdt * lim), wz), cscale(ab, dt));
            const T dre = T(1) - hdt * lre, dim = -hdt * lim;
            const T den = dre * dre + dim * dim;
            const C wst = mk<C>((num.x * dre + num.y * dim) / den, (num.y * dre - num.x * dim) / den);
            if (d.sponge_next) {
              const C wss = d.ab2_first ? wst : u5[q];
              wsp[gi] = wst;
              wn = mk<C>(T(1.5) * wst.x - T(0.5) * wss.x, T(1.5) * wst.y - T(0.5) * wss.y);
            } else {
              wn = wst;
            }
          } else if constexpr (OP == CO_AB2CN_FINAL) {
            wn = csub(u0[q], A[m]);
          } else {
            wn = A[m];
          }
          if (d.viscous) wn = cscale(wn, vf[q]);
          if (d.zero_mean && mx == 0 && my == 0) wn = mk<C>(T(0), T(0));
          if (d.store_ws) reinterpret_cast<C*>(d.ws_out)[gi] = wn;
          if (d.store_w0) w0[gi] = wn;
          if constexpr (OP == CO_FORWARD2) {  // the second field, treated like the first
            C wb = B[m];
            if (d.viscous) wb = cscale(wb, vf[q]);
            if (d.zero_mean && mx == 0 && my == 0) wb = mk<C>(T(0), T(0));
            reinterpret_cast<C*>(d.w0b)[gi] = wb;
          }
        }
        A[m] = wn;
      }
    }

    // ---- derived fields, inverse y-transforms, mixed arrays out.
    // Per owned mode: the state scaled by 1/N^2 (so the two inverse passes
    // return physical values), 1/|k|^2, and masks of the kept 2/3 band and of
    // the test filter; each derived field then costs a few operations per mode.
    const T scale = T(1.0 / n2);
    T ik2[E::EL];
    unsigned keep = 0u, intest = 0u;
#pragma unroll
    for (int m = 0; m < E::EL; ++m) {
      const int k = t + TT * m;
      const int my = k <= K ? k : k - N;
      const int m2 = mx * mx + my * my;
      if ((k <= K || k >= N - K) && col_ok) keep |= 1u << m;
      if (m2 <= d.test_m2max) intest |= 1u << m;
      ik2[m] = FInvK2<T>::get(ks2, m2);
      A[m] = cscale(A[m], scale);
    }
    const T ksc = T(g.kscale);
    // Three shared buffers rotate between the transform's two exchange buffers and the output tile of the TMA
    // store: the tile goes to the exchange buffer the transform's last exchange did not use (so no barrier is
    // needed before it is written), and the next field avoids the buffer whose store may still be reading.
    // t1, t2: the buffers of the previous two fields' tiles (-1: none).  The first exchange buffer is never
    // either of them; the second may be t2, whose store the lead thread waits for before the first exchange's
    // barrier, which every thread passes before it writes the second exchange buffer.
    unsigned char* const bufs[3] = {sbase, sbase + SB, sbase + 2 * SB};
    int t1 = -1, t2 = -1;
#pragma unroll 1
    for (int q = 0; q < d.nder; ++q) {
      const int code = d.der[q];
      // test-filtered fields vanish for k_x beyond the test band: their arrays stay zero there
      if ((code & D_TEST) && c0 > d.test_kmax) continue;
      const unsigned on = (code & D_TEST) ? (keep & intest) : keep;
      C w[E::EL];
#pragma unroll
      for (int m = 0; m < E::EL; ++m) w[m] = ((on >> m) & 1u) ? A[m] : mk<C>(T(0), T(0));
#define QG_KY(m) (ksc * T((t + TT * (m)) <= K ? (t + TT * (m)) : (t + TT * (m)) - N))
      switch (code & 7) {
        case D_U:  // -i ky psi, psi = -w / |k|^2
#pragma unroll
          for (int m = 0; m < E::EL; ++m) x[m] = cmul_ik(cscale(w[m], ik2[m]), QG_KY(m));
          if (mx == 0 && t == 0) x[0] = mk<C>(T(d.U), T(0));
          break;
        case D_V:  // i kx psi
#pragma unroll
          for (int m = 0; m < E::EL; ++m) x[m] = cmul_ik(cscale(w[m], -ik2[m]), kxv);
          break;
        case D_WX:
#pragma unroll
          for (int m = 0; m < E::EL; ++m) x[m] = cmul_ik(w[m], kxv);
          break;
        case D_WY:
#pragma unroll
          for (int m = 0; m < E::EL; ++m) x[m] = cmul_ik(w[m], QG_KY(m));
          break;
        case D_PXY:  // -kx ky psi = kx ky w / |k|^2
#pragma unroll
          for (int m = 0; m < E::EL; ++m) x[m] = cscale(w[m], kxv * QG_KY(m) * ik2[m]);
          break;
        case D_PD:  // -(kx^2 - ky^2) psi = (kx^2 - ky^2) w / |k|^2
#pragma unroll
          for (int m = 0; m < E::EL; ++m) {
            const T ky = QG_KY(m);
            x[m] = cscale(w[m], (kxv * kxv - ky * ky) * ik2[m]);
          }
          break;
        default:
#pragma unroll
          for (int m = 0; m < E::EL; ++m) x[m] = w[m];
          break;
      }
#undef QG_KY
      int e2 = t2;
      if (e2 < 0 || e2 == t1) e2 = t1 == 1 ? 2 : 1;
      int e1 = 0;
      while (e1 == t1 || e1 == e2) ++e1;
      const int tb = (E::NEX % 2 == 0) ? e1 : e2;
      C* b0 = reinterpret_cast<C*>(bufs[e1]);
      C* b1 = reinterpret_cast<C*>(bufs[e2]);
      C* st = reinterpret_cast<C*>(bufs[tb]);
      // at most the previous field's store is still reading (its tile is in neither exchange buffer)
      if (lead) tma::wait_group_read<1>();
      ph = 0;
      E::template run<col_packed<OP>()>(x, t, b0 + c * CP, b1 + c * CP, ph, twb, +1);
      // the tile buffer's last reads in this transform came before its last exchange's barrier
#pragma unroll
      for (int m = 0; m < E::EL; ++m) st[(t + TT * m) * W + c] = x[m];
      tma::fence_proxy_async();
      __syncthreads();
      t2 = t1;
      t1 = tb;
      if (lead) {
        for (int bx = 0; bx < NBOX; ++bx)
          tma::store_2d(&tm.out[q], 2 * c0, bx * BR,
                        reinterpret_cast<const unsigned char*>(st) + (size_t)bx * BR * W * sizeof(C));
        tma::commit_group();
      }
    }
    if (lead) tma::wait_group_all();
  }
}

}  // namespace fast

template <typename T, int N>
cudaError_t launch_row_fast(const Geom& g, const RowDesc& d, const void* tw, cudaStream_t st) {
  using E = fast::Eng<T, N>;
  using Cfg = fast::RowCfg<N>;
  const size_t smem = (size_t)2 * Cfg::ROWS * E::BUF * sizeof(cplx_t<T>);
  const auto* twp = reinterpret_cast<const cplx_t<T>*>(tw);
  const int grid = N / Cfg::ROWS;
  cudaError_t e = cudaSuccess;
#define QG_ROW_CASE(P)                                                                                   \
  case P: {                                                                                              \
    auto k = fast::row_fast_kernel<T, N, P>;                                                            \
    e = raise_smem_limit<fast::row_fast_kernel<T, N, P>>(smem);                                          \
    if (e != cudaSuccess) return e;                                                                      \
    e = launch_pdl(d.pdl != 0, k, dim3(grid), dim3(Cfg::THREADS), smem, st, g, d, twp);                \
    if (e != cudaSuccess) return e;                                                                      \
    break;                                                                                               \
  }
  switch (d.prog) {
    QG_ROW_CASE(RP_NONE)
    QG_ROW_CASE(RP_LEITH)
    QG_ROW_CASE(RP_SMAG)
    QG_ROW_CASE(RP_DLEITH)
    QG_ROW_CASE(RP_DSMAG)
    QG_ROW_CASE(RP_SCALE)
    QG_ROW_CASE(RP_COPY)
    QG_ROW_CASE(RP_ADJ_FWD)
    QG_ROW_CASE(RP_ADJ_REV)
    default:
      return cudaErrorInvalidValue;
  }
#undef QG_ROW_CASE
  return cudaGetLastError();
}

template <typename T, int N, int P, bool LEAN>
cudaError_t launch_col_one(const Geom& g, const ColDesc& d, const cplx_t<T>* twp, const TmaSet& tm, int grid,
                           cudaStream_t st) {
  using Cfg = fast::ColCfg<N>;
  auto k = fast::col_fast_kernel<T, N, P, LEAN>;
  const size_t smem = (size_t)(LEAN ? 2 : 3) * fast::col_stage_bytes<T, N>() + 1024;
  const cudaError_t e = raise_smem_limit<fast::col_fast_kernel<T, N, P, LEAN>>(smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(d.pdl != 0, k, dim3(grid), dim3(Cfg::THREADS), smem, st, g, d, twp, tm);
}

// SMs of the current device, queried once per device (concurrent first calls store the same value)
inline int device_sms() {
  static std::atomic<int> sms[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  int n = sms[dev].load(std::memory_order_relaxed);
  if (!n) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    sms[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

template <typename T, int N>
cudaError_t launch_col_fast(const Geom& g, const ColDesc& d, const void* tw, const TmaSet& tm, cudaStream_t st) {
  using Cfg = fast::ColCfg<N>;
  const auto* twp = reinterpret_cast<const cplx_t<T>*>(tw);
  const int grid = g.Kcp / Cfg::W;
#define QG_COL_CASE(P) \
  case P:              \
    return launch_col_one<T, N, P, false>(g, d, twp, tm, grid, st);
  switch (d.op) {
    QG_COL_CASE(CO_DERIVE)
    QG_COL_CASE(CO_STAGE_STATIC)
    QG_COL_CASE(CO_DYN_COMBINE)
    QG_COL_CASE(CO_CURL)
    QG_COL_CASE(CO_FORWARD)
    QG_COL_CASE(CO_FORWARD2)
    QG_COL_CASE(CO_FORWARD_N)
    QG_COL_CASE(CO_AB2CN)
    QG_COL_CASE(CO_AB2CN_COMBINE)
    QG_COL_CASE(CO_AB2CN_FINAL)
    case CO_DYN_REDUCE:
      if constexpr (fast::lean_fits<T, N>()) {
        // the lean form when the columns need more than one wave at two CTAs per SM but one at three (or
        // whenever the caller asks for it)
        const bool one_wave = grid > 2 * device_sms() && grid <= 3 * device_sms();
        if (d.scr[0] && d.scr[1] && d.scr[2] && (d.lean == 1 || (d.lean == 0 && one_wave)))
          return launch_col_one<T, N, CO_DYN_REDUCE, true>(g, d, twp, tm, grid, st);
      }
      return launch_col_one<T, N, CO_DYN_REDUCE, false>(g, d, twp, tm, grid, st);
    default:
      return cudaErrorInvalidValue;
  }
#undef QG_COL_CASE
}

#define QG_INSTANTIATE_FAST(N)                                                                          \
  template <> int fast_col_width<N>() { return fast::ColCfg<N>::W; }                                    \
  template cudaError_t launch_row_fast<float, N>(const Geom&, const RowDesc&, const void*, cudaStream_t);  \
  template cudaError_t launch_row_fast<double, N>(const Geom&, const RowDesc&, const void*, cudaStream_t); \
  template cudaError_t launch_col_fast<float, N>(const Geom&, const ColDesc&, const void*, const TmaSet&,       \
                                                 cudaStream_t);                                             \
  template cudaError_t launch_col_fast<double, N>(const Geom&, const ColDesc&, const void*, const TmaSet&,      \
                                                  cudaStream_t);

}  // namespace qg
