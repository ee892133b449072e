// Register-resident FFT engines and the specialised row / column passes for
// grids N = 2^p (256 <= N <= 4096, engine E16) and N = 3 * 2^p (384 <= N <= 3072, engine E12).
//
// Engine (E16): a length-N sequence is owned by TT = N/16 threads; thread t
// holds the 16 elements at natural positions t + TT*m (m = 0..15).  A
// Stockham DIT pass of radix R with span Ns splits the 16 elements into
// 16/R butterflies (m = b + (16/R) r): butterfly j = t + TT b reads elements
// j + (N/R) r, which are exactly the thread's own elements.  Its outputs go to
// (j / Ns) Ns R + (j mod Ns) + Ns r; for every pass but the last that is a
// shared-memory exchange (one barrier, buffers alternate), while the last pass
// (Ns R = N) lands on t + TT m again.  Hence an inverse FFT, any pointwise
// work and a forward FFT chain with no shared-memory traffic between them, and
// every column-pass spectral operation happens in registers on the thread's
// own k values.  Shared memory is padded by one element every 16 so the
// exchanges are free of bank conflicts.
//
// Passes: radix 16 (as 4 x 4 with W16 twiddles) while possible, then one pass
// of radix 8, 4 or 2.  Twiddles come from per-pass tables computed on the host
// from exactly reduced angles (see pass()).
#pragma once

#include "fft.cuh"
#include "qg_common.cuh"

namespace qg {
namespace fast {

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

template <typename C> __device__ __forceinline__ C cmulk(C a, decltype(C::x) c, decltype(C::x) s) {
  return mk<C>(a.x * c - a.y * s, a.x * s + a.y * c);
}

// Complex sums and differences of the butterflies.  With QG_PACKED_F32 (the default) the FP32 forms use the
// packed pair instructions of the sm_100 family (add / sub .rn.f32x2): both parts in one instruction, each part
// rounded as the scalar operation rounds it.  The transforms then issue 14% fewer instructions; results differ
// from the scalar build only where the compiler had fused one of these sums into a neighbouring product (an FMA,
// one rounding fewer), at the level of FP32 rounding.
#ifndef QG_PACKED_F32
#define QG_PACKED_F32 1
#endif
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
template <typename C, bool PK> __device__ __forceinline__ C vadd(C a, C b) {
  if constexpr (QG_PACKED_F32 && PK && std::is_same<C, float2>::value) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
  } else {
    return cadd(a, b);
  }
}
template <typename C, bool PK> __device__ __forceinline__ C vsub(C a, C b) {
  if constexpr (QG_PACKED_F32 && PK && std::is_same<C, float2>::value) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
  } else {
    return csub(a, b);
  }
}
// plus = t + i s d, minus = t - i s d (s = +1 / -1) with the parts of d exchanged in place
template <typename C> __device__ __forceinline__ void rot_pm(C t, C d, int s, C& plus, C& minus) {
  if (s > 0) {
    plus = mk<C>(t.x - d.y, t.y + d.x);
    minus = mk<C>(t.x + d.y, t.y - d.x);
  } else {
    plus = mk<C>(t.x + d.y, t.y - d.x);
    minus = mk<C>(t.x - d.y, t.y + d.x);
  }
}

// 4-, 8- and 2-point DFTs with kernel exp(s 2 pi i n k / R) (the same operations as the generic kernels' forms)
template <typename C, bool PK> __device__ __forceinline__ void dft4v(C* v, int s) {
  const C t0 = vadd<C, PK>(v[0], v[2]);
  const C t1 = vsub<C, PK>(v[0], v[2]);
  const C t2 = vadd<C, PK>(v[1], v[3]);
  const C d = vsub<C, PK>(v[1], v[3]);
  v[0] = vadd<C, PK>(t0, t2);
  v[2] = vsub<C, PK>(t0, t2);
  rot_pm(t1, d, s, v[1], v[3]);
}
template <typename C, bool PK> __device__ __forceinline__ void dft8v(C* v, int s) {
  using T = decltype(C::x);
  const T h = T(0.70710678118654752440);
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  dft4v<C, PK>(e, s);
  dft4v<C, PK>(o, s);
  // o[m] *= w8^m, w8 = exp(s 2 pi i / 8) = (1 + s i) / sqrt 2
  const C o1 = mk<C>((o[1].x - s * o[1].y) * h, (o[1].y + s * o[1].x) * h);
  const C o3 = mk<C>((-o[3].x - s * o[3].y) * h, (-o[3].y + s * o[3].x) * h);
  v[0] = vadd<C, PK>(e[0], o[0]);
  v[4] = vsub<C, PK>(e[0], o[0]);
  v[1] = vadd<C, PK>(e[1], o1);
  v[5] = vsub<C, PK>(e[1], o1);
  rot_pm(e[2], o[2], s, v[2], v[6]);
  v[3] = vadd<C, PK>(e[3], o3);
  v[7] = vsub<C, PK>(e[3], o3);
}
template <typename C, bool PK> __device__ __forceinline__ void dft2v(C* v) {
  const C a = v[0], b = v[1];
  v[0] = vadd<C, PK>(a, b);
  v[1] = vsub<C, PK>(a, b);
}

template <typename C, bool PK> __device__ __forceinline__ void dft16(C* v, int s) {
  using T = decltype(C::x);
  const T c1 = T(0.92387953251128675613);  // cos(pi/8)
  const T s1 = T(0.38268343236508977173);  // sin(pi/8)
  const T h = T(0.70710678118654752440);
  C a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C q[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
    dft4v<C, PK>(q, s);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = q[k1];
  }
  // a[n2][k1] *= exp(s 2 pi i n2 k1 / 16)
  const T ss = T(s);
  a[1][1] = cmulk(a[1][1], c1, ss * s1);
  a[1][2] = cmulk(a[1][2], h, ss * h);
  a[1][3] = cmulk(a[1][3], s1, ss * c1);
  a[2][1] = cmulk(a[2][1], h, ss * h);
  a[2][2] = cmul_si(a[2][2], s);
  a[2][3] = cmulk(a[2][3], -h, ss * h);
  a[3][1] = cmulk(a[3][1], s1, ss * c1);
  a[3][2] = cmulk(a[3][2], -h, ss * h);
  a[3][3] = cmulk(a[3][3], -c1, -ss * s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C q[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4v<C, PK>(q, s);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = q[k2];
  }
}

// 3-point DFT with kernel exp(s 2 pi i n k / 3)
template <typename C, bool PK> __device__ __forceinline__ void dft3(C* v, int s) {
  using T = decltype(C::x);
  const T h = T(0.86602540378443864676);  // sin(pi/3)
  const C a = v[0];
  const C bc = vadd<C, PK>(v[1], v[2]);
  const C d = vsub<C, PK>(v[1], v[2]);
  const C m = mk<C>(a.x - T(0.5) * bc.x, a.y - T(0.5) * bc.y);
  v[0] = vadd<C, PK>(a, bc);
  rot_pm(m, cscale(d, h), s, v[1], v[2]);  // m +- i s sin(pi/3) (v1 - v2)
}

// 12-point DFT as 4 x 3: n = 3 n1 + n2, k = k1 + 4 k2; 4-point DFTs over n1, twiddles
// exp(s 2 pi i n2 k1 / 12), 3-point DFTs over n2
template <typename C, bool PK> __device__ __forceinline__ void dft12(C* v, int s) {
  using T = decltype(C::x);
  const T h = T(0.86602540378443864676);  // cos(pi/6) = sin(pi/3)
  const T ss = T(s);
  C a[3][4];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    C q[4] = {v[n2], v[3 + n2], v[6 + n2], v[9 + n2]};
    dft4v<C, PK>(q, s);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = q[k1];
  }
  a[1][1] = cmulk(a[1][1], h, ss * T(0.5));    // 30 degrees
  a[1][2] = cmulk(a[1][2], T(0.5), ss * h);    // 60
  a[1][3] = cmul_si(a[1][3], s);               // 90
  a[2][1] = cmulk(a[2][1], T(0.5), ss * h);    // 60
  a[2][2] = cmulk(a[2][2], T(-0.5), ss * h);   // 120
  a[2][3] = mk<C>(-a[2][3].x, -a[2][3].y);     // 180
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C q[3] = {a[0][k1], a[1][k1], a[2][k1]};
    dft3<C, PK>(q, s);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) v[k1 + 4 * k2] = q[k2];
  }
}

template <typename C, int R, bool PK> __device__ __forceinline__ void dftR(C* v, int s) {
  if constexpr (R == 16) dft16<C, PK>(v, s);
  else if constexpr (R == 12) dft12<C, PK>(v, s);
  else if constexpr (R == 8) dft8v<C, PK>(v, s);
  else if constexpr (R == 4) dft4v<C, PK>(v, s);
  else if constexpr (R == 3) dft3<C, PK>(v, s);
  else dft2v<C, PK>(v);
}

// grid sizes with register-resident kernels: 2^p (16 elements per thread) and 3 * 2^p (12)
constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
constexpr int elems_per_thread(int n) { return is_pow2(n) ? 16 : 12; }
constexpr bool fast_size(int n) {
  return (is_pow2(n) && n >= 256 && n <= 4096) || (n % 3 == 0 && is_pow2(n / 3) && n >= 384 && n <= 3072);
}

template <typename T, int N> struct E16 {
  using C = cplx_t<T>;
  static constexpr int EL = 16;
  static constexpr int TT = N / 16;
  static constexpr int LOG2N = ilog2(N);
  static constexpr int NP16 = LOG2N / 4;
  static constexpr int RLAST = 1 << (LOG2N % 4);
  static constexpr int BUF = N + N / 16;  // padded complex elements of one sequence
  static constexpr int K = (N - 1) / 3;
  static constexpr int Kc = K + 1;
  static_assert((N & (N - 1)) == 0 && N >= 256 && N <= 4096, "E16 engine: N must be 2^p, 256..4096");

  __device__ static __forceinline__ int pad(int i) { return i + (i >> 4); }

  // Twiddles of the non-first passes come from per-pass tables laid out
  // [r - 1][k] (k fastest): a pass of radix R and span NS multiplies element r
  // of butterfly j by W_N^(r k N / (NS R)), k = j mod NS, stored at
  // off + (r - 1) NS + k.  For fixed r the threads of a warp read consecutive
  // k, so every load touches one or two cache lines, and the values are the
  // correctly rounded table entries.
  static constexpr int OFF2 = 0;                                   // pass 2: NS = 16, R = 16
  static constexpr int OFF3 = NP16 >= 2 ? 15 * 16 : 0;             // pass 3: NS = 256, R = 16 (N = 4096)
  static constexpr int OFFL = OFF3 + (NP16 >= 3 ? 15 * 256 : 0);   // last pass: NS = N / RLAST, R = RLAST
  static constexpr int TABLE = OFFL + (RLAST > 1 ? (RLAST - 1) * (N / RLAST) : 0);
  static constexpr int NEX = NP16 + (RLAST > 1 ? 1 : 0) - 1;  // shared-memory exchanges of one transform

  // One Stockham pass; x in natural ownership on entry.  Non-last passes
  // exchange through buf (this sequence's padded slot area).
  template <int R, int NS, bool LAST, int OFF, bool PK>
  __device__ static __forceinline__ void pass(C* x, int t, C* buf, const C* __restrict__ ptw, int sign) {
    constexpr int NB = 16 / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + TT * b;
      const int k = j & (NS - 1);
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = x[b + NB * r];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = __ldg(&ptw[OFF + (r - 1) * NS + k]);
          if (sign > 0) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
      dftR<C, R, PK>(v, sign);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) x[b + NB * r] = v[r];
      } else {
        const int base_i = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad(base_i + NS * r)] = v[r];
      }
    }
    if constexpr (!LAST) {
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 16; ++m) x[m] = buf[pad(t + TT * m)];
    }
  }

  // Full transform.  b0, b1 alternate per exchange (ph toggles); callers
  // pass the same ph through every use of the two buffers.  PK: packed FP32 butterflies (QG_PACKED_F32).
  template <bool PK = true>
  __device__ static __forceinline__ void run(C* x, int t, C* b0, C* b1, int& ph, const C* __restrict__ ptw,
                                             int sign) {
    if constexpr (NP16 >= 1) {
      constexpr bool last = (NP16 == 1 && RLAST == 1);
      pass<16, 1, last, 0, PK>(x, t, ph ? b1 : b0, ptw, sign);
      if (!last) ph ^= 1;
    }
    if constexpr (NP16 >= 2) {
      constexpr bool last = (NP16 == 2 && RLAST == 1);
      pass<16, 16, last, OFF2, PK>(x, t, ph ? b1 : b0, ptw, sign);
      if (!last) ph ^= 1;
    }
    if constexpr (NP16 >= 3) {
      constexpr bool last = (NP16 == 3 && RLAST == 1);
      pass<16, 256, last, OFF3, PK>(x, t, ph ? b1 : b0, ptw, sign);
      if (!last) ph ^= 1;
    }
    if constexpr (RLAST > 1) {
      constexpr int NS = N / RLAST;
      pass<RLAST, NS, true, OFFL, PK>(x, t, ph ? b1 : b0, ptw, sign);
    }
  }
};

// Engine E12 for N = 3 * 2^j (384 <= N <= 3072): a length-N sequence is owned by TT = N/12 threads, thread t
// holding the 12 elements t + TT*m (m = 0..11).  The passes are Stockham DIT passes as in E16: radix 12
// first (as 4 x 3), then radix 4 while a factor 4 remains, then radix 2 for odd j.  A radix-R pass takes
// 12/R butterflies per thread, each reading the thread's own elements (N/R is a multiple of TT), and the
// last pass lands on natural ownership again.  Twiddle tables per pass as in E16: [r - 1][k], k = j mod NS.
template <typename T, int N> struct E12 {
  using C = cplx_t<T>;
  static constexpr int EL = 12;
  static constexpr int TT = N / 12;
  static constexpr int J = ilog2(N / 12);
  static constexpr int NP4 = J / 2;                 // radix-4 passes after the radix-12 one
  static constexpr int RLAST = (J % 2) ? 2 : 1;     // a final radix-2 pass for odd J
  static constexpr int BUF = N + N / 16;
  static constexpr int K = (N - 1) / 3;
  static constexpr int Kc = K + 1;
  static constexpr int NEX = NP4 + (RLAST == 2 ? 1 : 0);  // shared-memory exchanges: radix-12 pass + radix-4 passes
  static_assert(N % 12 == 0 && is_pow2(N / 12) && N >= 384 && N <= 3072, "E12 engine: N must be 3 * 2^p, 384..3072");

  __device__ static __forceinline__ int pad(int i) { return i + (i >> 4); }

  // span of radix-4 pass p (1-based) and its table offset; the radix-2 pass follows at span N / 2
  static constexpr int ns4(int p) { return p <= 1 ? 12 : 4 * ns4(p - 1); }
  static constexpr int off4(int p) { return p <= 1 ? 0 : off4(p - 1) + 3 * ns4(p - 1); }

  template <int R, int NS, bool LAST, int OFF, bool PK>
  __device__ static __forceinline__ void pass(C* x, int t, C* buf, const C* __restrict__ ptw, int sign) {
    constexpr int NB = 12 / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + TT * b;
      const int k = j % NS;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = x[b + NB * r];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = __ldg(&ptw[OFF + (r - 1) * NS + k]);
          if (sign > 0) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
      dftR<C, R, PK>(v, sign);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) x[b + NB * r] = v[r];
      } else {
        const int base_i = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad(base_i + NS * r)] = v[r];
      }
    }
    if constexpr (!LAST) {
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 12; ++m) x[m] = buf[pad(t + TT * m)];
    }
  }

  template <int P, bool PK>
  __device__ static __forceinline__ void run4(C* x, int t, C* b0, C* b1, int& ph, const C* __restrict__ ptw,
                                              int sign) {
    if constexpr (P <= NP4) {
      constexpr bool last = (P == NP4 && RLAST == 1);
      pass<4, ns4(P), last, off4(P), PK>(x, t, ph ? b1 : b0, ptw, sign);
      if (!last) ph ^= 1;
      run4<P + 1, PK>(x, t, b0, b1, ph, ptw, sign);
    }
  }

  template <bool PK = true>
  __device__ static __forceinline__ void run(C* x, int t, C* b0, C* b1, int& ph, const C* __restrict__ ptw,
                                             int sign) {
    pass<12, 1, false, 0, PK>(x, t, ph ? b1 : b0, ptw, sign);
    ph ^= 1;
    run4<1, PK>(x, t, b0, b1, ph, ptw, sign);
    if constexpr (RLAST == 2) pass<2, N / 2, true, off4(NP4 + 1), PK>(x, t, ph ? b1 : b0, ptw, sign);
  }
};

template <typename T, int N> struct EngineOf { using type = E16<T, N>; };
template <typename T> struct EngineOf<T, 384> { using type = E12<T, 384>; };
template <typename T> struct EngineOf<T, 768> { using type = E12<T, 768>; };
template <typename T> struct EngineOf<T, 1536> { using type = E12<T, 1536>; };
template <typename T> struct EngineOf<T, 3072> { using type = E12<T, 3072>; };
template <typename T, int N> using Eng = typename EngineOf<T, N>::type;

}  // namespace fast

// rows of one TMA box of the specialised column pass (a divisor of N)
constexpr int fast_box_rows(int n) { return n < 256 ? n : (n % 256 == 0 ? 256 : 128); }

// k_x columns per CTA of the specialised column pass
template <int N> int fast_col_width();
// complex entries of the per-pass twiddle table of the specialised kernels
int fast_pass_table_size(int n);
// fill the per-pass twiddle table (host doubles, interleaved re/im) from
// tw[j] = exp(-2 pi i j / n) given as cos/sin pairs
void fast_pass_table(int n, const double* tw_re_im, double* out_re_im);
template <typename T, int N>
cudaError_t launch_row_fast(const Geom& g, const RowDesc& d, const void* tw, cudaStream_t st);
struct TmaSet;
template <typename T, int N>
cudaError_t launch_col_fast(const Geom& g, const ColDesc& d, const void* tw, const TmaSet& tm, cudaStream_t st);

}  // namespace qg
