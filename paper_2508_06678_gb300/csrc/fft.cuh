// CTA-cooperative mixed-radix (2, 3, 4, 8) Stockham FFT in shared memory.
//
// A batch of B interleaved sequences of length N lives in shared memory with
// element (n, b) at d[n * B + b].  Each pass of radix R turns N/R groups of R
// elements (stride N/R) into radix-R butterflies with twiddles from a table
// tw[j] = exp(-2 pi i j / N); outputs go to stride Ns, so after all passes
// the sequence is in natural order (Stockham autosort).  The pass is done
// in place: every thread stages its butterflies in registers, the block
// synchronises, then writes.  sign = -1 computes the forward (unnormalised)
// DFT, +1 the inverse (unnormalised).
#pragma once

#include "qg_common.cuh"

namespace qg {

struct FftPlan {
  int n;
  int npass;
  int radix[16];
};

// butterflies a thread stages per pass: at most 8 complex values in registers
template <int R> struct MaxItems { static constexpr int value = 8 / R; };
template <> struct MaxItems<3> { static constexpr int value = 2; };

template <typename C> __device__ __forceinline__ void dft2(C* v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename C> __device__ __forceinline__ void dft4(C* v, int s) {
  C t0 = cadd(v[0], v[2]);
  C t1 = csub(v[0], v[2]);
  C t2 = cadd(v[1], v[3]);
  C t3 = cmul_si(csub(v[1], v[3]), s);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <typename C> __device__ __forceinline__ void dft8(C* v, int s) {
  using T = decltype(C::x);
  const T h = T(0.70710678118654752440);
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, s);
  dft4(o, s);
  // o[m] *= w8^m, w8 = exp(s 2 pi i / 8) = (1 + s i) / sqrt 2
  C o1 = mk<C>((o[1].x - s * o[1].y) * h, (o[1].y + s * o[1].x) * h);
  C o2 = cmul_si(o[2], s);
  C o3 = mk<C>((-o[3].x - s * o[3].y) * h, (-o[3].y + s * o[3].x) * h);
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

template <typename C> __device__ __forceinline__ void dft3(C* v, int s) {
  using T = decltype(C::x);
  const T c = T(0.86602540378443864676);  // sqrt(3) / 2
  C t1 = cadd(v[1], v[2]);
  C t2 = csub(v[1], v[2]);
  C m = mk<C>(v[0].x - T(0.5) * t1.x, v[0].y - T(0.5) * t1.y);
  C j = cmul_si(cscale(t2, c), s);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, j);
  v[2] = csub(m, j);
}

template <typename C, int R> __device__ __forceinline__ void dft(C* v, int s) {
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3(v, s);
  else if constexpr (R == 4) dft4(v, s);
  else dft8(v, s);
}

template <typename C, int R>
__device__ void stockham_pass(C* __restrict__ d, int N, int B, int Ns, const C* __restrict__ tw, int sign,
                              int* st) {
  constexpr int MI = MaxItems<R>::value;
  const int NR = N / R;
  const int items = NR * B;
  const int tws = N / (Ns * R);
  C v[MI][R];
  int ob[MI];
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    const int item = threadIdx.x + i * blockDim.x;
    ob[i] = -1;
    if (item < items) {
      const int b = item % B;
      const int j = item / B;
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = QG_LD(d, (j + r * NR) * B + b, N * B, st);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = QG_INB(r * k * tws, N, st) ? __ldg(&tw[r * k * tws]) : mk<C>(decltype(C::x)(1), decltype(C::x)(0));
          if (sign > 0) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      dft<C, R>(v[i], sign);
      ob[i] = ((j / Ns) * Ns * R + k) * B + b;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    if (ob[i] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) QG_ST(d, ob[i] + r * Ns * B, N * B, st, v[i][r]);
    }
  }
  __syncthreads();
}

// Full transform of B interleaved length-N sequences.  Synchronises on entry
// and exit.  Requires blockDim.x * MaxItems<R> >= (N / R) * B for every pass.
template <typename C>
__device__ void fft_batched(C* d, const FftPlan& p, int B, const C* __restrict__ tw, int sign, int* st = nullptr) {
  __syncthreads();
  int Ns = 1;
  for (int s = 0; s < p.npass; ++s) {
    const int R = p.radix[s];
    if (R == 8) stockham_pass<C, 8>(d, p.n, B, Ns, tw, sign, st);
    else if (R == 4) stockham_pass<C, 4>(d, p.n, B, Ns, tw, sign, st);
    else if (R == 2) stockham_pass<C, 2>(d, p.n, B, Ns, tw, sign, st);
    else stockham_pass<C, 3>(d, p.n, B, Ns, tw, sign, st);
    Ns *= R;
  }
}

}  // namespace qg
