// A posteriori comparison of two snapshot series (Sec. IV, Eq. 15-16).
//
// For every filtered snapshot t and lag phi the pair (les[t - phi], ff[t]) is
// reduced to two sums over the grid points: the squared L2 distance
// sum (a - b)^2 of Eq. 16 and the centred cross sum sum (a - a_mean)(b - b_mean)
// of the PCC of Eq. 15.  The lag of Eq. 16 minimises the mean distance over
// the snapshots for which the pair exists (ties: smallest |phi|, then the
// negative lag).
//
// Kernels (all reductions in a fixed order, so results are deterministic):
//   moments   (snapshot, slice) CTAs: each slice's sum, then its sum of
//             squares about its own mean (compensated per thread for FP32
//             fields); norm: the slices merged per snapshot in FP64 (mean,
//             1 / sqrt of the centred sum of squares)
//   pairs     a 16 x 16 tile of (t, phi) pairs per CTA of 64 threads, a 2 x 2
//             block of pairs per thread (two snapshots 8 apart, two lags 8
//             apart: three distinct les rows), over one chunk of the points;
//             the 16 ff rows and the 31 les rows the tile needs are staged
//             through shared memory and read 16 bytes at a time; sums run in
//             short FMA chains folded into compensated (TwoSum) totals for
//             FP32 series, FP64 partials per chunk
//   finish    the chunks' partials summed per pair (a warp per pair, fixed
//             order); PCC from the moments
//   phase     mean distance per lag (a warp per lag) and, in the last CTA to
//             finish, its argmin
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/qg.h"
#include "qg_kernels.h"

using namespace qg;

namespace {

constexpr int kTileT = 16;                   // ff snapshots per tile
constexpr int kTileL = 16;                   // lags per tile
constexpr int kRowsA = kTileT + kTileL - 1;  // les rows a tile touches
constexpr int kThreads = kTileT * kTileL;
constexpr int kMaxSnap = 1000000;  // keeps the pair grid (tiles x chunks) within the launch limits
constexpr int kMaxLag = 1 << 16;
constexpr size_t kMaxPairs = size_t(1) << 24;
constexpr size_t kPartialBytes = size_t(256) << 20;


__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// The 16-byte vector a thread reads from a staged row, and its lanes.
template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int W = 4; };
template <> struct Vec<double> { static constexpr int W = 2; };

template <typename T, int W>
__device__ __forceinline__ void load_lanes(const T* p, T (&x)[W]) {
  if constexpr (W == 4 && sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
  } else if constexpr (W == 2 && sizeof(T) == 8) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    x[0] = v.x, x[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < W; ++i) x[i] = p[i];
  }
}

template <typename T, int W>
__device__ __forceinline__ void store_lanes(T* p, const T (&x)[W]) {
  if constexpr (W == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else if constexpr (W == 2 && sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  } else {
#pragma unroll
    for (int i = 0; i < W; ++i) p[i] = x[i];
  }
}

// Per-snapshot moments over a grid of (snapshot, slice) CTAs, snapshots
// 0 .. n_a - 1 from series a and the rest from series b.  Each CTA reads its
// slice twice (the second time from L2: the resident slices fit in it): the
// slice's sum, then the sum of (x - m_s)^2 about the slice's own mean rounded
// to the working precision, m_s.  Per-thread sums are compensated for FP32
// fields.  The norm kernel then merges the slices exactly in FP64: the mean,
// and the centred sum of squares
//   M2 = sum_s [ sq_s - n_s (mu_s - m_s)^2 + n_s (mu_s - mean)^2 ],
// mu_s = sum_s / n_s (the pairwise-variance update of Chan, Golub and LeVeque).
struct MomArgs {
  int n_a, nsnap, nchunk;
  int64_t npts, chunk;
  double* sum_part;  // [snap][slice]: sum of the slice
  double* sq_part;   // [snap][slice]: sum of (x - m_s)^2 about the slice's mean in the working precision
  double* mean;      // [snap]
  double* rnorm;     // [snap]: 1 / sqrt(M2), 0 for a constant field
};

template <typename T>
__device__ const T* snapshot(const T* a, const T* b, const MomArgs& A, int s) {
  return s < A.n_a ? a + (size_t)s * (size_t)A.npts : b + (size_t)(s - A.n_a) * (size_t)A.npts;
}

template <typename T> struct SumAcc;
template <> struct SumAcc<double> {
  double s = 0.0;
  __device__ void add(double x) { s += x; }
  __device__ double value() const { return s; }
};
template <> struct SumAcc<float> {
  GermanoAcc<float> g;
  __device__ void add(float x) { g.add(x); }
  __device__ double value() const { return g.value(); }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) series_moments_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                                  MomArgs A) {
  __shared__ double red[kThreads / 32];
  __shared__ double m_sh;
  const int snap = blockIdx.x;
  const T* f = snapshot(a, b, A, snap);
  const int64_t p0 = (int64_t)blockIdx.y * A.chunk;
  const int64_t p1 = p0 + A.chunk < A.npts ? p0 + A.chunk : A.npts;
  SumAcc<T> acc;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) acc.add(f[p]);
  const double s = block_sum(acc.value(), red);
  if (threadIdx.x == 0) {
    A.sum_part[(size_t)snap * A.nchunk + blockIdx.y] = s;
    m_sh = s / double(p1 - p0);
  }
  __syncthreads();
  const T mc = T(m_sh);
  GermanoAcc<T> q;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {
    const T d = f[p] - mc;
    q.add_prod(d, d);
  }
  const double v = block_sum(q.value(), red);
  if (threadIdx.x == 0) A.sq_part[(size_t)snap * A.nchunk + blockIdx.y] = v;
}

// one warp per snapshot: the slices merged in a fixed order
constexpr int kNormThreads = 256;
__global__ void __launch_bounds__(kNormThreads) series_norm_kernel(MomArgs A, int fp32) {
  const int snap = blockIdx.x * (kNormThreads / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (snap >= A.nsnap) return;
  const double* sp = A.sum_part + (size_t)snap * A.nchunk;
  const double* qp = A.sq_part + (size_t)snap * A.nchunk;
  double s = 0.0;
  for (int c = lane; c < A.nchunk; c += 32) s += sp[c];
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  const double mean = s / double(A.npts);
  double q = 0.0;
  for (int c = lane; c < A.nchunk; c += 32) {
    const int64_t p0 = (int64_t)c * A.chunk;
    const double n = double((p0 + A.chunk < A.npts ? p0 + A.chunk : A.npts) - p0);
    const double mu = sp[c] / n;  // the moments kernel's slice mean, bit for bit
    const double m = fp32 ? double(float(mu)) : mu;
    q += qp[c] - n * (mu - m) * (mu - m) + n * (mu - mean) * (mu - mean);
  }
  for (int m = 16; m > 0; m >>= 1) q += __shfl_xor_sync(0xffffffffu, q, m);
  if (lane == 0) {
    A.mean[snap] = mean;
    A.rnorm[snap] = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  }
}

struct PairArgs {
  int n_les, n_ff, lag_min, nlag, tiles_l;
  int64_t npts, chunk;
  const double* mean_les;
  const double* mean_ff;
  double* part;  // [t][j][chunk][2]: sum (a - b)^2, sum (a - a_c)(b - b_c)
};

// One thread's four pairs at W consecutive points.  rows: les rows ra - 8, ra,
// ra + 8 and ff rows ti, ti + 8 of the tile; c: their centres.  Pair k = 2u + v
// (snapshot t + 8u, lag j + 8v) reads les row ra + 8(u - v) and ff row ti + 8u.
// cd / cc: per-lane chains of sum (a - b)^2 and sum (a - a_c)(b - b_c).
template <typename T, int W>
__device__ __forceinline__ void pair_terms(const T* const (&rows)[5], int p, const T (&c)[5], T (&cd)[4][W],
                                           T (&cc)[4][W]) {
  T x[5][W];
#pragma unroll
  for (int r = 0; r < 5; ++r) load_lanes<T, W>(rows[r] + p, x[r]);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const T a_m = x[0][w], a_0 = x[1][w], a_p = x[2][w], b_0 = x[3][w], b_8 = x[4][w];
    const T ca_m = a_m - c[0], ca_0 = a_0 - c[1], ca_p = a_p - c[2], cb_0 = b_0 - c[3], cb_8 = b_8 - c[4];
    T d = a_0 - b_0;
    cd[0][w] = fma(d, d, cd[0][w]);
    cc[0][w] = fma(ca_0, cb_0, cc[0][w]);
    d = a_m - b_0;
    cd[1][w] = fma(d, d, cd[1][w]);
    cc[1][w] = fma(ca_m, cb_0, cc[1][w]);
    d = a_p - b_8;
    cd[2][w] = fma(d, d, cd[2][w]);
    cc[2][w] = fma(ca_p, cb_8, cc[2][w]);
    d = a_0 - b_8;
    cd[3][w] = fma(d, d, cd[3][w]);
    cc[3][w] = fma(ca_0, cb_8, cc[3][w]);
  }
}

// the chains of one block summed as a balanced tree, added to the running totals
template <typename T, int W>
__device__ __forceinline__ void fold(T (&cd)[4][W], T (&cc)[4][W], SumAcc<T> (&td)[4], SumAcc<T> (&tc)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T sd, sc;
    if constexpr (W == 4) {
      sd = (cd[k][0] + cd[k][1]) + (cd[k][2] + cd[k][3]);
      sc = (cc[k][0] + cc[k][1]) + (cc[k][2] + cc[k][3]);
    } else if constexpr (W == 2) {
      sd = cd[k][0] + cd[k][1];
      sc = cc[k][0] + cc[k][1];
    } else {
      sd = cd[k][0];
      sc = cc[k][0];
    }
    td[k].add(sd);
    tc[k].add(sc);
#pragma unroll
    for (int w = 0; w < W; ++w) cd[k][w] = T(0), cc[k][w] = T(0);
  }
}

// A 16 x 16 tile of (t, phi) pairs per CTA of 64 threads; thread (ti, li)
// takes snapshots t0 + ti + {0, 8} and lags j0 + li + {0, 8}, whose four les
// snapshots are three rows of the staged tile.  Each round stages the 31 les
// rows and the 16 ff rows of P points (rows padded by 16 bytes: the 8 les rows
// a quarter warp reads with one 16-byte load each start 16 bytes apart modulo
// 128 bytes and fall in distinct banks), then each thread adds its pairs'
// terms in blocks of kFold vectors: plain FMA chains, one per vector lane,
// whose tree sum joins a compensated running total (TwoSum for FP32; a block
// sum carries at most (kFold + 2) u relative rounding of its terms).
// kVec (rows start on 16-byte boundaries): the rows are staged with 16-byte
// loads and stores; otherwise element by element.
constexpr int kPairW = 8;
constexpr int kPairThreads = kPairW * kPairW;
constexpr int kFold = 4;
constexpr int kRowsStaged = kRowsA + kTileT;  // les rows, then ff rows
constexpr int kStageBytes = 512;              // bytes of a staged row per round
static_assert(2 * kPairW == kTileT && 2 * kPairW == kTileL, "a thread takes two snapshots and two lags");

template <typename T, bool kVec>
__global__ void __launch_bounds__(kPairThreads) series_pairs_kernel(const T* __restrict__ les,
                                                                    const T* __restrict__ ff, PairArgs A) {
  constexpr int W = Vec<T>::W;
  constexpr int P = kStageBytes / int(sizeof(T));  // points per round
  constexpr int LD = P + W;                         // padded row length in elements
  constexpr int NQ = P / W;                         // vectors per staged row
  __shared__ __align__(16) T stage[kRowsStaged * LD];
  // grid: x = pair tile (lags fastest), y = point chunk, so the tiles that share a chunk's rows run together
  const int ti = threadIdx.x / kPairW, li = threadIdx.x % kPairW;
  const int by = int(blockIdx.x) / A.tiles_l, bz = int(blockIdx.x) - by * A.tiles_l;
  const int t0 = by * kTileT, j0 = bz * kTileL;
  const int s_row0 = t0 - A.lag_min - j0 - (kTileL - 1);  // les snapshot of staged row 0
  const int ra = ti - li + kTileL - 1;                     // les row of pairs (t, j) and (t + 8, j + 8)
  bool valid[4];
  bool any = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int t = t0 + ti + kPairW * (k >> 1), jl = j0 + li + kPairW * (k & 1);
    const int s = t - (A.lag_min + jl);
    valid[k] = t < A.n_ff && jl < A.nlag && s >= 0 && s < A.n_les;
    any = any || valid[k];
  }
  if (!__syncthreads_or(any)) return;  // no pair of this tile exists
  // centres in the working precision (the finish kernel corrects for their rounding)
  T c[5];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int sn = s_row0 + ra + kPairW * (r - 1);
    c[r] = (sn >= 0 && sn < A.n_les) ? T(A.mean_les[sn]) : T(0);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int tn = t0 + ti + kPairW * u;
    c[3 + u] = tn < A.n_ff ? T(A.mean_ff[tn]) : T(0);
  }
  const T* const rows[5] = {stage + (ra - kPairW) * LD, stage + ra * LD, stage + (ra + kPairW) * LD,
                            stage + (kRowsA + ti) * LD, stage + (kRowsA + ti + kPairW) * LD};
  SumAcc<T> td[4], tc[4];
  T cd[4][W] = {}, cc[4][W] = {};
  const int64_t p_begin = (int64_t)blockIdx.y * A.chunk;
  const int64_t p_end = p_begin + A.chunk < A.npts ? p_begin + A.chunk : A.npts;
  for (int64_t p0 = p_begin; p0 < p_end; p0 += P) {
    const int np = p_end - p0 < P ? int(p_end - p0) : P;
    __syncthreads();  // the previous round's reads are done
    if constexpr (kVec) {  // np is a whole number of vectors
      for (int e = threadIdx.x; e < kRowsStaged * NQ; e += kPairThreads) {
        const int r = e / NQ, q = e - r * NQ;
        const bool is_les = r < kRowsA;
        const int sn = is_les ? s_row0 + r : t0 + r - kRowsA;
        const bool in = q * W < np && sn >= 0 && sn < (is_les ? A.n_les : A.n_ff);
        T x[W] = {};
        if (in) load_lanes<T, W>((is_les ? les : ff) + (size_t)sn * (size_t)A.npts + (size_t)(p0 + q * W), x);
        store_lanes<T, W>(stage + r * LD + q * W, x);
      }
    } else {
      for (int e = threadIdx.x; e < kRowsStaged * P; e += kPairThreads) {
        const int r = e / P, p = e - r * P;
        const bool is_les = r < kRowsA;
        const int sn = is_les ? s_row0 + r : t0 + r - kRowsA;
        const bool in = p < np && sn >= 0 && sn < (is_les ? A.n_les : A.n_ff);
        stage[r * LD + p] = in ? (is_les ? les : ff)[(size_t)sn * (size_t)A.npts + (size_t)(p0 + p)] : T(0);
      }
    }
    __syncthreads();
    if (any) {
      const int nv = np / W;
      int q = 0;
      for (; q + kFold <= nv; q += kFold) {
#pragma unroll
        for (int i = 0; i < kFold; ++i) pair_terms<T, W>(rows, (q + i) * W, c, cd, cc);
        fold<T, W>(cd, cc, td, tc);
      }
      if (q < nv) {
        for (; q < nv; ++q) pair_terms<T, W>(rows, q * W, c, cd, cc);
        fold<T, W>(cd, cc, td, tc);
      }
      if (nv * W < np) {
        T ed[4][1] = {}, ec[4][1] = {};
        for (int p = nv * W; p < np; ++p) pair_terms<T, 1>(rows, p, c, ed, ec);
        fold<T, 1>(ed, ec, td, tc);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!valid[k]) continue;
    const int t = t0 + ti + kPairW * (k >> 1), jl = j0 + li + kPairW * (k & 1);
    double* o = A.part + 2 * (((size_t)t * A.nlag + jl) * gridDim.y + blockIdx.y);
    o[0] = td[k].value();
    o[1] = tc[k].value();
  }
}

struct FinishArgs {
  int n_les, n_ff, lag_min, nlag, nchunk, fp32;
  int64_t npts;
  const double* part;
  MomArgs mom;  // snapshots 0 .. n_les - 1 are les, then ff
  double* dist;
  double* pcc;
};

// one warp per pair: lane c sums chunks c, c + 32, ... and a fixed butterfly adds the lanes
constexpr int kFinishThreads = 256;
__global__ void __launch_bounds__(kFinishThreads) series_finish_kernel(FinishArgs A) {
  const size_t idx = (size_t)blockIdx.x * (kFinishThreads / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (idx >= (size_t)A.n_ff * A.nlag) return;
  const int t = int(idx / A.nlag), j = int(idx - (size_t)t * A.nlag);
  const int s = t - (A.lag_min + j);
  if (s < 0 || s >= A.n_les) {
    if (lane == 0) {
      A.dist[idx] = NAN;
      A.pcc[idx] = NAN;
    }
    return;
  }
  double d2 = 0.0, cr = 0.0;
  const double* o = A.part + 2 * idx * (size_t)A.nchunk;
  for (int c = lane; c < A.nchunk; c += 32) {
    d2 += o[2 * c];
    cr += o[2 * c + 1];
  }
  for (int m = 16; m > 0; m >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, m);
    cr += __shfl_xor_sync(0xffffffffu, cr, m);
  }
  if (lane != 0) return;
  // the pairs kernel centred on the means rounded to the working precision:
  // sum (a - a_c)(b - b_c) = sum (a - mean_a)(b - mean_b) + n (mean_a - a_c)(mean_b - b_c)
  const double ma = A.mom.mean[s], mb = A.mom.mean[A.n_les + t];
  const double ca = A.fp32 ? double(float(ma)) : ma, cb = A.fp32 ? double(float(mb)) : mb;
  cr -= double(A.npts) * (ma - ca) * (mb - cb);
  A.dist[idx] = d2;
  const double ra = A.mom.rnorm[s], rb = A.mom.rnorm[A.n_les + t];
  A.pcc[idx] = (ra > 0.0 && rb > 0.0) ? cr * ra * rb : NAN;
}

// Does lag phi with mean distance m come before lag pb with mean mb?  Smaller
// mean, then smaller |phi|, then the negative lag: a total order on the lags.
__device__ __forceinline__ bool lag_before(double m, int phi, double mb, int pb) {
  if (m != mb) return m < mb;
  const int aphi = phi < 0 ? -phi : phi, apb = pb < 0 ? -pb : pb;
  return aphi < apb || (aphi == apb && phi < pb);
}

// Mean distance per lag over the defined pairs (a warp per lag, lane-strided
// over the snapshots, fixed butterfly), then, in the last CTA to finish, its
// argmin (Eq. 16) by a block reduction; the order is total, so the argmin does
// not depend on the reduction's order.  phase: [lag, found, CTAs done] (the
// counter starts at zero).
constexpr int kPhaseThreads = 256;
__device__ __forceinline__ void argmin_step(int& best, double& mb, int ob, double om, int lag_min) {
  if (ob >= 0 && (best < 0 || lag_before(om, lag_min + ob, mb, lag_min + best))) best = ob, mb = om;
}

__global__ void __launch_bounds__(kPhaseThreads) series_phase_kernel(const double* dist, int n_ff, int nlag,
                                                                     int lag_min, double* mean_dist, int* phase) {
  constexpr int kWarps = kPhaseThreads / 32;
  __shared__ double wm[kWarps];
  __shared__ int wj[kWarps];
  __shared__ int is_last;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kWarps + warp;
  if (j < nlag) {
    double s = 0.0;
    int n = 0;
    for (int t = lane; t < n_ff; t += 32) {
      const double v = dist[(size_t)t * nlag + j];
      if (!isnan(v)) {
        s += v;
        ++n;
      }
    }
    for (int m = 16; m > 0; m >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, m);
      n += __shfl_xor_sync(0xffffffffu, n, m);
    }
    if (lane == 0) mean_dist[j] = n ? s / double(n) : NAN;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(&phase[2], 1) == int(gridDim.x) - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  int best = -1;
  double mb = 0.0;
  for (int k = threadIdx.x; k < nlag; k += kPhaseThreads) {
    const double m = __ldcg(mean_dist + k);
    if (!isnan(m)) argmin_step(best, mb, k, m, lag_min);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int ob = __shfl_xor_sync(0xffffffffu, best, o);
    const double om = __shfl_xor_sync(0xffffffffu, mb, o);
    argmin_step(best, mb, ob, om, lag_min);
  }
  if (lane == 0) wm[warp] = mb, wj[warp] = best;
  __syncthreads();
  if (warp == 0) {
    best = lane < kWarps ? wj[lane] : -1;
    mb = lane < kWarps ? wm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      const int ob = __shfl_xor_sync(0xffffffffu, best, o);
      const double om = __shfl_xor_sync(0xffffffffu, mb, o);
      argmin_step(best, mb, ob, om, lag_min);
    }
    if (lane == 0) {
      phase[0] = best < 0 ? 0 : lag_min + best;
      phase[1] = best >= 0;
    }
  }
}

int fail(int code, const char* msg) {
  qg::set_last_error(msg);
  return code;
}

// Device memory pool of the lag-table scratch, one per device, created on
// first use: blocks a call frees go back to the pool (release threshold
// unlimited), so a later call takes them again without a driver allocation and
// without the device-wide synchronisation of cudaFree.
cudaMemPool_t scratch_pool(int dev) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &pp) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return nullptr;
    }
    pools[dev] = p;
  }
  return pools[dev];
}

// One call's scratch, allocated and freed in the order of the call's stream.
struct Scratch {
  cudaStream_t st = nullptr;
  cudaMemPool_t pool = nullptr;
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  explicit Scratch(cudaStream_t s) : st(s) {
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess && !(pool = scratch_pool(dev))) err = cudaErrorMemoryAllocation;
  }
  void* get(size_t bytes) {
    void* p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, st);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
};

// Optional CUDA-event brackets around the call's kernels (moments, pairs, finish, phase).
struct Timer {
  cudaEvent_t ev[5] = {};
  bool on = false;
  cudaStream_t st = nullptr;
  void start(bool enable, cudaStream_t s) {
    st = s;
    on = enable;
    for (int i = 0; on && i < 5; ++i) on = cudaEventCreate(&ev[i]) == cudaSuccess;
  }
  void mark(int i) {
    if (on) cudaEventRecord(ev[i], st);
  }
  void read(double* ms) {
    for (int i = 0; i < 4; ++i) {
      float v = 0.f;
      ms[i] = (on && cudaEventElapsedTime(&v, ev[i], ev[i + 1]) == cudaSuccess) ? double(v) : -1.0;
    }
  }
  ~Timer() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// Per-device facts the launch configuration needs, queried once: the SM count and the resident
// CTAs per SM of each pairs-kernel variant ([FP64][16-byte staging]).
struct DevFacts {
  bool ready = false;
  int nsm = 1;
  int occ[2][2] = {{1, 1}, {1, 1}};
};

template <typename K>
int pair_occupancy(K kernel) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kPairThreads, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return occ;
}

const DevFacts& dev_facts(int dev) {
  static std::mutex mu;
  static std::vector<DevFacts> facts;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)facts.size() <= dev) facts.resize(dev + 1);
  DevFacts& f = facts[dev];
  if (!f.ready) {
    if (cudaDeviceGetAttribute(&f.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || f.nsm < 1) f.nsm = 1;
    f.occ[0][0] = pair_occupancy(series_pairs_kernel<float, false>);
    f.occ[0][1] = pair_occupancy(series_pairs_kernel<float, true>);
    f.occ[1][0] = pair_occupancy(series_pairs_kernel<double, false>);
    f.occ[1][1] = pair_occupancy(series_pairs_kernel<double, true>);
    f.ready = true;
  }
  return f;
}

template <typename T>
cudaError_t run_compare(const T* les, int n_les, const T* ff, int n_ff, int64_t npts, int lag_min, int nlag,
                        cudaStream_t st, Scratch& S, Timer& tm, double* d_dist, double* d_pcc, double* d_mean,
                        int* d_phase) {
  int dev = 0;
  cudaGetDevice(&dev);
  const DevFacts& facts = dev_facts(dev);
  const int nsm = facts.nsm;
  // moments: (snapshot, slice) CTAs, slices of at most 64 KB (the slices resident at once fit in L2, so
  // each CTA's second read of its slice hits it), at least four CTAs per SM, at least 1024 points a slice
  const int nsnap = n_les + n_ff;
  const int64_t slice_pts = 65536 / (int64_t)sizeof(T);
  int64_t mchunks = (npts + slice_pts - 1) / slice_pts;
  const int64_t min_mchunks = (4 * (int64_t)nsm + nsnap - 1) / nsnap;
  if (mchunks < min_mchunks) mchunks = min_mchunks;
  const int64_t max_mchunks = (npts + 1023) / 1024;
  if (mchunks > max_mchunks) mchunks = max_mchunks;
  if (mchunks > 65535) mchunks = 65535;
  if (mchunks < 1) mchunks = 1;
  const int64_t mchunk = (npts + mchunks - 1) / mchunks;
  mchunks = (npts + mchunk - 1) / mchunk;
  double* mbuf = static_cast<double*>(S.get(sizeof(double) * ((size_t)2 * nsnap * mchunks + 2 * (size_t)nsnap)));
  if (!mbuf) return S.err;
  double* mean = mbuf + (size_t)2 * nsnap * mchunks;
  MomArgs M{n_les, nsnap, (int)mchunks, npts, mchunk, mbuf, mbuf + (size_t)nsnap * mchunks, mean, mean + nsnap};
  const double* mean_les = M.mean;
  const double* mean_ff = M.mean + n_les;

  // split the points into chunks: a few waves of CTAs over the SMs, partials within budget
  const int tiles_t = (n_ff + kTileT - 1) / kTileT, tiles_l = (nlag + kTileL - 1) / kTileL;
  // 16-byte staging when every staged row starts on a 16-byte boundary
  const bool vec = npts % Vec<T>::W == 0 && reinterpret_cast<uintptr_t>(les) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(ff) % 16 == 0;
  void (*const pairs)(const T*, const T*, PairArgs) =
      vec ? series_pairs_kernel<T, true> : series_pairs_kernel<T, false>;
  const int64_t P = kStageBytes / sizeof(T);
  const int64_t rounds = (npts + P - 1) / P;
  const int64_t tiles = (int64_t)tiles_t * tiles_l;
  // about three waves of resident pair CTAs (tiles at the edges of the pair grid finish early)
  const int occ = facts.occ[sizeof(T) == 8][vec];
  int64_t nchunk = (3 * (int64_t)occ * nsm + tiles - 1) / tiles;
  const int64_t per_chunk_bytes = 16 * (int64_t)n_ff * nlag;
  const int64_t cap = (int64_t)kPartialBytes / per_chunk_bytes;
  if (nchunk > cap) nchunk = cap;
  if (nchunk > rounds) nchunk = rounds;
  if (nchunk > 65535) nchunk = 65535;
  if (nchunk < 1) nchunk = 1;
  const int64_t chunk = ((rounds + nchunk - 1) / nchunk) * P;
  nchunk = (npts + chunk - 1) / chunk;
  double* part = static_cast<double*>(S.get((size_t)per_chunk_bytes * nchunk));
  if (!part) return S.err;
  cudaError_t e = cudaMemsetAsync(d_phase, 0, 3 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  tm.mark(0);
  series_moments_kernel<T><<<dim3(nsnap, (unsigned)mchunks), kThreads, 0, st>>>(les, ff, M);
  const int per_norm = kNormThreads / 32;
  series_norm_kernel<<<(nsnap + per_norm - 1) / per_norm, kNormThreads, 0, st>>>(M, sizeof(T) == 4);
  tm.mark(1);
  PairArgs pa{n_les, n_ff, lag_min, nlag, tiles_l, npts, chunk, mean_les, mean_ff, part};
  pairs<<<dim3((unsigned)tiles, (unsigned)nchunk), kPairThreads, 0, st>>>(les, ff, pa);
  tm.mark(2);

  FinishArgs fa{n_les, n_ff, lag_min, nlag, (int)nchunk, sizeof(T) == 4, npts, part, M, d_dist, d_pcc};
  const size_t npair = (size_t)n_ff * nlag;
  const size_t per_cta = kFinishThreads / 32;
  series_finish_kernel<<<(unsigned)((npair + per_cta - 1) / per_cta), kFinishThreads, 0, st>>>(fa);
  tm.mark(3);
  const int per_phase = kPhaseThreads / 32;
  series_phase_kernel<<<(nlag + per_phase - 1) / per_phase, kPhaseThreads, 0, st>>>(d_dist, n_ff, nlag, lag_min,
                                                                                    d_mean, d_phase);
  tm.mark(4);
  return cudaGetLastError();
}

}  // namespace

extern "C" int qg_series_compare(const void* les, int32_t n_les_snap, const void* ff, int32_t n_ff_snap,
                                 int64_t npts, int32_t dtype, int32_t on_device, int32_t lag_min, int32_t lag_max,
                                 void* stream, double* dist, double* pcc, double* mean_dist, int32_t* phase,
                                 double* kernel_ms) {
  char msg[256];
  if (!les || !ff || !dist) return fail(QG_ERR_ARG, "qg_series_compare: NULL argument");
  if (dtype != QG_FP32 && dtype != QG_FP64) return fail(QG_ERR_ARG, "qg_series_compare: dtype must be QG_FP32 or QG_FP64");
  if (n_les_snap < 1 || n_ff_snap < 1 || n_les_snap > kMaxSnap || n_ff_snap > kMaxSnap || npts < 1) {
    snprintf(msg, sizeof(msg), "qg_series_compare: bad sizes n_les_snap=%d n_ff_snap=%d npts=%lld", n_les_snap,
             n_ff_snap, (long long)npts);
    return fail(QG_ERR_ARG, msg);
  }
  if (lag_max < lag_min || (int64_t)lag_max - lag_min + 1 > kMaxLag) {
    snprintf(msg, sizeof(msg), "qg_series_compare: bad lag range [%d, %d] (at most %d lags)", lag_min, lag_max,
             kMaxLag);
    return fail(QG_ERR_ARG, msg);
  }
  const int nlag = lag_max - lag_min + 1;
  if ((size_t)n_ff_snap * nlag > kMaxPairs) return fail(QG_ERR_ARG, "qg_series_compare: too many (t, lag) pairs");
  // a pair exists iff some t in [0, n_ff) has t - phi in [0, n_les) for some phi in the range
  if ((int64_t)lag_min > (int64_t)n_ff_snap - 1 || (int64_t)lag_max < -(int64_t)(n_les_snap - 1))
    return fail(QG_ERR_ARG, "qg_series_compare: no lag in the range pairs any two snapshots");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t esz = dtype == QG_FP32 ? 4 : 8;
  Scratch S(st);
  const void* dl = les;
  const void* df = ff;
  if (!on_device) {
    void* a = S.get(esz * (size_t)n_les_snap * (size_t)npts);
    void* b = S.get(esz * (size_t)n_ff_snap * (size_t)npts);
    if (!a || !b) return fail(QG_ERR_OOM, "qg_series_compare: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(a, les, esz * (size_t)n_les_snap * (size_t)npts, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b, ff, esz * (size_t)n_ff_snap * (size_t)npts, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      snprintf(msg, sizeof(msg), "qg_series_compare: %s", cudaGetErrorString(e));
      return fail(QG_ERR_CUDA, msg);
    }
    dl = a;
    df = b;
  }
  const size_t npair = (size_t)n_ff_snap * nlag;
  // results: dist, pcc, mean_dist (doubles), then phase, found and the phase kernel's CTA counter (ints)
  const size_t nres = 2 * npair + nlag;
  double* d_out = static_cast<double*>(S.get(sizeof(double) * nres + 4 * sizeof(int)));
  if (!d_out) return fail(QG_ERR_OOM, "qg_series_compare: device allocation failed");
  int* d_phase = reinterpret_cast<int*>(d_out + nres);
  Timer tm;
  tm.start(kernel_ms != nullptr, st);
  cudaError_t e = dtype == QG_FP32
                      ? run_compare<float>(static_cast<const float*>(dl), n_les_snap, static_cast<const float*>(df),
                                           n_ff_snap, npts, lag_min, nlag, st, S, tm, d_out, d_out + npair,
                                           d_out + 2 * npair, d_phase)
                      : run_compare<double>(static_cast<const double*>(dl), n_les_snap,
                                            static_cast<const double*>(df), n_ff_snap, npts, lag_min, nlag, st, S,
                                            tm, d_out, d_out + npair, d_out + 2 * npair, d_phase);
  if (e == cudaSuccess) e = S.err;
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "qg_series_compare: %s", cudaGetErrorString(e));
    return fail(e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA, msg);
  }
  // one copy back: the doubles and the two result ints behind them
  std::vector<unsigned char> hb(sizeof(double) * nres + 2 * sizeof(int));
  e = cudaMemcpyAsync(hb.data(), d_out, hb.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "qg_series_compare: %s", cudaGetErrorString(e));
    return fail(QG_ERR_CUDA, msg);
  }
  const double* h = reinterpret_cast<const double*>(hb.data());
  int hp[2];
  memcpy(hp, hb.data() + sizeof(double) * nres, sizeof(hp));
  std::copy(h, h + npair, dist);
  if (pcc) std::copy(h + npair, h + 2 * npair, pcc);
  if (mean_dist) std::copy(h + 2 * npair, h + nres, mean_dist);
  if (phase) *phase = hp[0];
  if (kernel_ms) tm.read(kernel_ms);
  if (!hp[1]) return fail(QG_ERR_ARG, "qg_series_compare: no lag in the range pairs any two snapshots");
  return QG_OK;
}
