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
//   moments   (chunk, snapshot) CTAs: chunk sums, then chunk sums of squares
//             about the mean (compensated per thread for FP32 fields)
//   pairs     a 16 x 16 tile of (t, phi) pairs per CTA, one pair per thread,
//             over one chunk of the points; the 16 ff rows and the 31 les
//             rows the tile needs are staged through shared memory (rows
//             padded by one element so the up to 17 distinct rows a warp
//             reads fall in distinct banks); FP32 series keep each thread's
//             sums compensated (TwoProduct / TwoSum), FP64 partials per chunk
//   finish    the chunks' partials summed per pair; PCC from the moments
//   phase     mean distance per lag and its argmin (one CTA)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/qg.h"
#include "qg_kernels.h"

using namespace qg;

namespace {

constexpr int kTileT = 16;                   // ff snapshots per tile
constexpr int kTileL = 16;                   // lags per tile
constexpr int kRowsA = kTileT + kTileL - 1;  // les rows a tile touches
constexpr int kThreads = kTileT * kTileL;
constexpr int kMaxSnap = 1000000;  // keeps the pair grid's y extent (snapshots / 16) within 65535
constexpr int kMaxLag = 1 << 16;
constexpr size_t kMaxPairs = size_t(1) << 24;
constexpr size_t kPartialBytes = size_t(256) << 20;

template <typename T> struct Stage { static constexpr int P = 128; };  // points staged per round
template <> struct Stage<double> { static constexpr int P = 64; };     // same shared-memory bytes

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

// Per-snapshot moments in two passes over a grid of (chunk, snapshot) CTAs,
// snapshots 0 .. n_a - 1 from series a and the rest from series b.
// Pass 1 writes each chunk's sum; pass 2 forms the mean from those sums (a
// fixed-order warp reduction, identical in every CTA of the snapshot) and
// writes each chunk's sum of (x - m_c)^2 about the mean rounded to the
// working precision, m_c.  Per-thread sums are compensated for FP32 fields.
struct MomArgs {
  int n_a, nsnap, nchunk;
  int64_t npts, chunk;
  double* sum_part;  // [snap][chunk]
  double* sq_part;   // [snap][chunk]
  double* mean;      // [snap]
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
__global__ void __launch_bounds__(kThreads) series_sum_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                              MomArgs A) {
  __shared__ double red[kThreads / 32];
  const int snap = blockIdx.x;
  const T* f = snapshot(a, b, A, snap);
  const int64_t p0 = (int64_t)blockIdx.y * A.chunk;
  const int64_t p1 = p0 + A.chunk < A.npts ? p0 + A.chunk : A.npts;
  SumAcc<T> acc;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) acc.add(f[p]);
  const double v = block_sum(acc.value(), red);
  if (threadIdx.x == 0) A.sum_part[(size_t)snap * A.nchunk + blockIdx.y] = v;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) series_sq_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                             MomArgs A) {
  __shared__ double red[kThreads / 32];
  __shared__ double m_sh;
  const int snap = blockIdx.x;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int c = threadIdx.x; c < A.nchunk; c += 32) s += A.sum_part[(size_t)snap * A.nchunk + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
      m_sh = s / double(A.npts);
      if (blockIdx.y == 0) A.mean[snap] = m_sh;
    }
  }
  __syncthreads();
  const T mc = T(m_sh);
  const T* f = snapshot(a, b, A, snap);
  const int64_t p0 = (int64_t)blockIdx.y * A.chunk;
  const int64_t p1 = p0 + A.chunk < A.npts ? p0 + A.chunk : A.npts;
  GermanoAcc<T> acc;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) {
    const T d = f[p] - mc;
    acc.add_prod(d, d);
  }
  const double v = block_sum(acc.value(), red);
  if (threadIdx.x == 0) A.sq_part[(size_t)snap * A.nchunk + blockIdx.y] = v;
}

// centred sum of squares of one snapshot: the chunks' sums about m_c, less n (m - m_c)^2
__device__ double snapshot_css(const MomArgs& M, int snap, int fp32) {
  double q = 0.0;
  for (int c = 0; c < M.nchunk; ++c) q += M.sq_part[(size_t)snap * M.nchunk + c];
  const double m = M.mean[snap];
  const double mc = fp32 ? double(float(m)) : m;
  return q - double(M.npts) * (m - mc) * (m - mc);
}

struct PairArgs {
  int n_les, n_ff, lag_min, nlag;
  int64_t npts, chunk;
  const double* mean_les;
  const double* mean_ff;
  double* part;  // [chunk][t][j][2]: sum (a - b)^2, sum (a - a_c)(b - b_c)
};

template <typename T>
__global__ void __launch_bounds__(kThreads) series_pairs_kernel(const T* __restrict__ les, const T* __restrict__ ff,
                                                                PairArgs A) {
  constexpr int P = Stage<T>::P;
  __shared__ T sa[kRowsA][P + 1];
  __shared__ T sb[kTileT][P + 1];
  const int i = threadIdx.x / kTileL, j = threadIdx.x % kTileL;
  const int t0 = blockIdx.y * kTileT, j0 = blockIdx.z * kTileL;
  const int t = t0 + i, jl = j0 + j;
  const int s = t - (A.lag_min + jl);                     // les snapshot of this pair
  const int s_row0 = t0 - A.lag_min - j0 - (kTileL - 1);  // les snapshot of staged row 0
  const bool valid = t < A.n_ff && jl < A.nlag && s >= 0 && s < A.n_les;
  if (!__syncthreads_or(valid)) return;  // no pair of this tile exists
  // centres of the cross sum in the working precision (the finish kernel corrects for their rounding)
  const T am = valid ? T(A.mean_les[s]) : T(0);
  const T bm = valid ? T(A.mean_ff[t]) : T(0);
  GermanoAcc<T> d2, cr;
  const int ra = i - j + kTileL - 1;
  const int64_t p_begin = (int64_t)blockIdx.x * A.chunk;
  const int64_t p_end = p_begin + A.chunk < A.npts ? p_begin + A.chunk : A.npts;
  for (int64_t p0 = p_begin; p0 < p_end; p0 += P) {
    const int np = p_end - p0 < P ? int(p_end - p0) : P;
    __syncthreads();  // the previous round's reads are done
    for (int e = threadIdx.x; e < kRowsA * P; e += kThreads) {
      const int r = e / P, p = e - r * P;
      const int sn = s_row0 + r;
      sa[r][p] = (p < np && sn >= 0 && sn < A.n_les) ? les[(size_t)sn * (size_t)A.npts + (size_t)(p0 + p)] : T(0);
    }
    for (int e = threadIdx.x; e < kTileT * P; e += kThreads) {
      const int r = e / P, p = e - r * P;
      const int tn = t0 + r;
      sb[r][p] = (p < np && tn < A.n_ff) ? ff[(size_t)tn * (size_t)A.npts + (size_t)(p0 + p)] : T(0);
    }
    __syncthreads();
    if (valid) {
      for (int p = 0; p < np; ++p) {
        const T a = sa[ra][p], b = sb[i][p];
        const T d = a - b;
        d2.add_prod(d, d);
        cr.add_prod(a - am, b - bm);
      }
    }
  }
  if (valid) {
    double* o = A.part + 2 * (((size_t)blockIdx.x * A.n_ff + t) * A.nlag + jl);
    o[0] = d2.value();
    o[1] = cr.value();
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

__global__ void series_finish_kernel(FinishArgs A) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)A.n_ff * A.nlag) return;
  const int t = int(idx / A.nlag), j = int(idx - (size_t)t * A.nlag);
  const int s = t - (A.lag_min + j);
  if (s < 0 || s >= A.n_les) {
    A.dist[idx] = NAN;
    A.pcc[idx] = NAN;
    return;
  }
  double d2 = 0.0, cr = 0.0;
  for (int c = 0; c < A.nchunk; ++c) {
    const double* o = A.part + 2 * ((size_t)c * A.n_ff * A.nlag + idx);
    d2 += o[0];
    cr += o[1];
  }
  // the pairs kernel centred on the means rounded to the working precision:
  // sum (a - a_c)(b - b_c) = sum (a - mean_a)(b - mean_b) + n (mean_a - a_c)(mean_b - b_c)
  const double ma = A.mom.mean[s], mb = A.mom.mean[A.n_les + t];
  const double ca = A.fp32 ? double(float(ma)) : ma, cb = A.fp32 ? double(float(mb)) : mb;
  cr -= double(A.npts) * (ma - ca) * (mb - cb);
  A.dist[idx] = d2;
  const double va = snapshot_css(A.mom, s, A.fp32), vb = snapshot_css(A.mom, A.n_les + t, A.fp32);
  A.pcc[idx] = (va > 0.0 && vb > 0.0) ? cr / (sqrt(va) * sqrt(vb)) : NAN;
}

// mean distance per lag over the defined pairs, and its argmin (Eq. 16)
__global__ void series_phase_kernel(const double* dist, int n_ff, int nlag, int lag_min, double* mean_dist,
                                    int* phase) {
  for (int j = threadIdx.x; j < nlag; j += blockDim.x) {
    double s = 0.0;
    int n = 0;
    for (int t = 0; t < n_ff; ++t) {
      const double v = dist[(size_t)t * nlag + j];
      if (!isnan(v)) {
        s += v;
        ++n;
      }
    }
    mean_dist[j] = n ? s / double(n) : NAN;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = -1;
    for (int j = 0; j < nlag; ++j) {
      const double m = mean_dist[j];
      if (isnan(m)) continue;
      if (best < 0) {
        best = j;
        continue;
      }
      const double mb = mean_dist[best];
      const int phi = lag_min + j, pb = lag_min + best;
      const int aphi = phi < 0 ? -phi : phi, apb = pb < 0 ? -pb : pb;
      if (m < mb || (m == mb && (aphi < apb || (aphi == apb && phi < pb)))) best = j;
    }
    phase[0] = best < 0 ? 0 : lag_min + best;
    phase[1] = best >= 0;
  }
}

int fail(int code, const char* msg) {
  qg::set_last_error(msg);
  return code;
}

struct Scratch {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = cudaMalloc(&p, bytes ? bytes : 16);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
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

template <typename T>
cudaError_t run_compare(const T* les, int n_les, const T* ff, int n_ff, int64_t npts, int lag_min, int nlag,
                        cudaStream_t st, Scratch& S, Timer& tm, double* d_dist, double* d_pcc, double* d_mean,
                        int* d_phase) {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // moments: a few waves of (chunk, snapshot) CTAs, at least 1024 points per CTA
  const int nsnap = n_les + n_ff;
  int64_t mchunks = (4 * (int64_t)nsm + nsnap - 1) / nsnap;
  const int64_t max_mchunks = (npts + 1023) / 1024;
  if (mchunks > max_mchunks) mchunks = max_mchunks;
  if (mchunks > 65535) mchunks = 65535;
  if (mchunks < 1) mchunks = 1;
  const int64_t mchunk = (npts + mchunks - 1) / mchunks;
  mchunks = (npts + mchunk - 1) / mchunk;
  double* mbuf = static_cast<double*>(S.get(sizeof(double) * ((size_t)2 * nsnap * mchunks + nsnap)));
  if (!mbuf) return S.err;
  MomArgs M{n_les, nsnap, (int)mchunks, npts, mchunk, mbuf, mbuf + (size_t)nsnap * mchunks,
            mbuf + (size_t)2 * nsnap * mchunks};
  const double* mean_les = M.mean;
  const double* mean_ff = M.mean + n_les;

  // split the points into chunks: a few waves of CTAs over the SMs, partials within budget
  const int tiles_t = (n_ff + kTileT - 1) / kTileT, tiles_l = (nlag + kTileL - 1) / kTileL;
  const int64_t P = Stage<T>::P;
  const int64_t rounds = (npts + P - 1) / P;
  const int64_t tiles = (int64_t)tiles_t * tiles_l;
  int64_t nchunk = (4 * (int64_t)nsm + tiles - 1) / tiles;
  const int64_t per_chunk_bytes = 16 * (int64_t)n_ff * nlag;
  const int64_t cap = (int64_t)kPartialBytes / per_chunk_bytes;
  if (nchunk > cap) nchunk = cap;
  if (nchunk > rounds) nchunk = rounds;
  if (nchunk < 1) nchunk = 1;
  const int64_t chunk = ((rounds + nchunk - 1) / nchunk) * P;
  nchunk = (npts + chunk - 1) / chunk;
  double* part = static_cast<double*>(S.get((size_t)per_chunk_bytes * nchunk));
  if (!part) return S.err;
  tm.mark(0);
  series_sum_kernel<T><<<dim3(nsnap, (unsigned)mchunks), kThreads, 0, st>>>(les, ff, M);
  series_sq_kernel<T><<<dim3(nsnap, (unsigned)mchunks), kThreads, 0, st>>>(les, ff, M);
  tm.mark(1);
  PairArgs pa{n_les, n_ff, lag_min, nlag, npts, chunk, mean_les, mean_ff, part};
  series_pairs_kernel<T><<<dim3((unsigned)nchunk, tiles_t, tiles_l), kThreads, 0, st>>>(les, ff, pa);
  tm.mark(2);

  FinishArgs fa{n_les, n_ff, lag_min, nlag, (int)nchunk, sizeof(T) == 4, npts, part, M, d_dist, d_pcc};
  const size_t npair = (size_t)n_ff * nlag;
  series_finish_kernel<<<(unsigned)((npair + 255) / 256), 256, 0, st>>>(fa);
  tm.mark(3);
  series_phase_kernel<<<1, 256, 0, st>>>(d_dist, n_ff, nlag, lag_min, d_mean, d_phase);
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
  Scratch S;
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
  double* d_out = static_cast<double*>(S.get(sizeof(double) * (2 * npair + nlag)));
  int* d_phase = static_cast<int*>(S.get(2 * sizeof(int)));
  if (!d_out || !d_phase) return fail(QG_ERR_OOM, "qg_series_compare: device allocation failed");
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
  std::vector<double> h(2 * npair + nlag);
  int hp[2] = {0, 0};
  e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp, d_phase, sizeof(hp), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "qg_series_compare: %s", cudaGetErrorString(e));
    return fail(QG_ERR_CUDA, msg);
  }
  std::copy(h.begin(), h.begin() + npair, dist);
  if (pcc) std::copy(h.begin() + npair, h.begin() + 2 * npair, pcc);
  if (mean_dist) std::copy(h.begin() + 2 * npair, h.end(), mean_dist);
  if (phase) *phase = hp[0];
  if (kernel_ms) tm.read(kernel_ms);
  if (!hp[1]) return fail(QG_ERR_ARG, "qg_series_compare: no lag in the range pairs any two snapshots");
  return QG_OK;
}
