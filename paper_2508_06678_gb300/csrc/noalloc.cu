// qg_field_stats_static: field statistics with no device allocation.
//
// Some callers cannot allocate device memory at the point where they want
// these numbers: hosts whose framework owns every byte of device memory
// through its own allocator or a fixed budget, code that must not introduce
// the device-wide synchronisation cudaMalloc/cudaFree can cause, and
// real-time loops that must not pay an allocation's latency or risk its
// failure.  This entry point serves them by keeping all of its scratch in one
// file-scope device array of fixed size.
// The computation is the one qg_set_state followed by qg_diagnostics
// performs: project the field onto the kept 2/3 band with zero mean, then
// energy and enstrophy by FP64 Parseval sums and max |w| / finiteness of the
// projected field.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/qg.h"
#include "qg_kernels.h"

using namespace qg;

namespace {

// Capacity of the shared scratch: enough for every valid grid with N <= 512
// in FP64 (mixed array, spectral array, physical field, twiddles, partials).
constexpr size_t kScratchBytes = 5u << 20;
constexpr int kMaxN = 512;

// Every GPU that loads the library holds this array until the process exits.
// All calls share it: concurrent calls whose work overlaps on the GPU race.
__device__ __align__(256) unsigned char g_stats_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

int na_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  qg::set_last_error(buf);  // reported by qg_last_error()
  return code;
}

bool valid_n(int n) {
  if (n < 16 || (n & 1)) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

FftPlan plan_for(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  while (m % 8 == 0) { p.radix[p.npass++] = 8; m /= 8; }
  if (m % 4 == 0) { p.radix[p.npass++] = 4; m /= 4; }
  if (m % 2 == 0) { p.radix[p.npass++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.npass++] = 3; m /= 3; }
  return p;
}

int threads_for(const FftPlan& p, int B, int floor_threads) {
  int need = floor_threads;
  for (int s = 0; s < p.npass; ++s) {
    const int R = p.radix[s];
    const int mi = R == 3 ? 2 : 8 / R;
    const int t = ((p.n / R) * B + mi - 1) / mi;
    if (t > need) need = t;
  }
  return (need + 31) / 32 * 32;
}

// twiddle table exp(-2 pi i j / n) written on the device (CUDA's sincospi)
template <typename T>
__global__ void twiddle_kernel(cplx_t<T>* tw, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * double(j) / double(n), &s, &c);
    tw[j] = mk<cplx_t<T>>(T(c), T(-s));
  }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int scratch_on_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(QG_ERR_CUDA, "qg_field_stats_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(QG_ERR_UNSUPPORTED, "qg_field_stats_static: device %d", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stats_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(QG_ERR_CUDA, "qg_field_stats_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return QG_OK;
}

template <typename T>
int run_stats(const void* omega, int n, double L, cudaStream_t st, double* stats, unsigned char* base) {
  const size_t esz = sizeof(T), csz = 2 * sizeof(T);
  Geom g{};
  g.n = n;
  g.K = (n - 1) / 3;
  g.Kc = g.K + 1;
  g.Ny = 2 * g.K + 1;
  g.SP = (g.Ny + 3) / 4 * 4;
  g.kscale = 2.0 * M_PI / L;
  const FftPlan plan = plan_for(n);
  const int W = sizeof(T) == 4 ? 4 : 2;
  g.Kcp = (g.Kc + W - 1) / W * W;
  g.IP = g.Kcp;
  const int col_threads = threads_for(plan, W, 128);
  const size_t col_smem = (size_t)n * W * csz + 2 * (size_t)W * g.Ny * csz;
  const int row_threads = threads_for(plan, 1, 256);
  const size_t row_smem = (size_t)n * csz + 2 * (size_t)n * esz;

  // scratch layout
  const size_t b_mixed = align256((size_t)n * g.IP * csz);
  const size_t b_spec = align256((size_t)g.Kcp * g.SP * csz);
  const size_t b_phys = align256((size_t)n * n * esz);
  const size_t b_tw = align256((size_t)n * csz);
  const int nred = 512;
  const size_t b_red = align256((size_t)2 * nred * sizeof(double));
  const size_t need = b_mixed + b_spec + b_phys + b_tw + b_red;
  if (need > kScratchBytes)
    return na_fail(QG_ERR_ARG, "qg_field_stats_static: n=%d needs %zu scratch bytes, the array holds %zu", n, need,
                   kScratchBytes);
  unsigned char* mixed = base;
  unsigned char* spec = mixed + b_mixed;
  unsigned char* phys = spec + b_spec;
  unsigned char* tw = phys + b_phys;
  double* red = reinterpret_cast<double*>(tw + b_tw);

  // the spectral scratch starts at zero (its padding columns are never written)
  twiddle_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(reinterpret_cast<cplx_t<T>*>(tw), n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(spec, 0, b_spec, st);
  if (e != cudaSuccess) return na_fail(QG_ERR_CUDA, "qg_field_stats_static: setup: %s", cudaGetErrorString(e));

  // forward transform of the field, projection onto the kept band with zero mean
  RowDesc r{};
  r.prog = RP_COPY;
  r.nin = 1;
  r.nout = 1;
  r.in_phys = 1;
  r.phys_in = omega;
  r.out[0] = mixed;
  e = launch_row<T>(g, plan, r, tw, row_threads, row_smem, st);
  if (e != cudaSuccess) return na_fail(QG_ERR_CUDA, "qg_field_stats_static: row pass: %s", cudaGetErrorString(e));
  ColDesc c{};
  c.op = CO_FORWARD;
  c.nfwd = 1;
  c.fin[0] = mixed;
  c.w0 = spec;
  c.ws = spec;
  c.store_w0 = 1;
  c.zero_mean = 1;
  c.nder = 1;
  c.der[0] = D_W;
  c.dout[0] = mixed;  // each CTA reads its own columns before writing them
  c.test_ratio = 2.0;
  e = launch_col<T>(g, plan, c, tw, W, col_threads, col_smem, st);
  if (e != cudaSuccess) return na_fail(QG_ERR_CUDA, "qg_field_stats_static: column pass: %s", cudaGetErrorString(e));
  // physical field of the projected state
  RowDesc r2{};
  r2.prog = RP_COPY;
  r2.nin = 1;
  r2.nout = 1;
  r2.in[0] = mixed;
  r2.out_phys = 1;
  r2.phys_out = phys;
  e = launch_row<T>(g, plan, r2, tw, row_threads, row_smem, st);
  if (e != cudaSuccess) return na_fail(QG_ERR_CUDA, "qg_field_stats_static: row pass: %s", cudaGetErrorString(e));
  // energy, enstrophy (FP64 Parseval sums) and max |w|, finiteness
  e = launch_spectral_sums<T>(g, spec, red, nred, stats, st);
  if (e == cudaSuccess) e = launch_phys_maxabs<T>(g, phys, red, nred, stats + 2, st);
  if (e != cudaSuccess) return na_fail(QG_ERR_CUDA, "qg_field_stats_static: reductions: %s", cudaGetErrorString(e));
  return QG_OK;
}

}  // namespace

extern "C" int qg_field_stats_static(const void* omega, int32_t n, double L, int32_t dtype, void* cuda_stream,
                                     double* stats) {
  if (!omega || !stats) return na_fail(QG_ERR_ARG, "qg_field_stats_static: NULL pointer");
  if (!valid_n(n) || n > kMaxN)
    return na_fail(QG_ERR_ARG, "qg_field_stats_static: n=%d must be even, 2^a 3^b, 16..%d", n, kMaxN);
  if (!(L > 0) || !std::isfinite(L)) return na_fail(QG_ERR_ARG, "qg_field_stats_static: L must be positive");
  if (dtype != QG_FP32 && dtype != QG_FP64) return na_fail(QG_ERR_ARG, "qg_field_stats_static: bad dtype");
  void* base = nullptr;
  int rc = scratch_on_device(&base);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  return dtype == QG_FP32 ? run_stats<float>(omega, n, L, st, stats, b) : run_stats<double>(omega, n, L, st, stats, b);
}
