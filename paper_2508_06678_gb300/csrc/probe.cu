// qg_probe_fma_rate: the device's measured fused multiply-add throughput in FP32 or FP64.
//
// The FP64 form of the step is bound by FP64 arithmetic rather than by HBM on this GPU, so its roofline needs an
// FP64 arithmetic peak; this entry point measures it (and the FP32 one for comparison) with a plain kernel of
// independent FMA chains timed by CUDA events.  It changes no clock or device setting.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../../include/qg.h"
#include "qg_kernels.h"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (hides the pipe latency)
constexpr int kUnroll = 16;  // FMAs per chain per loop iteration
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

int pr_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  qg::set_last_error(buf);
  return code;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == T(-1)) *sink = s;  // the chains converge to b / (1 - a) > 0: never taken, keeps them live
}

template <typename T>
int probe(double* flops_per_s, double* ms_out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return pr_fail(QG_ERR_CUDA, "qg_probe_fma_rate: %s", cudaGetErrorString(e));
  T* sink = nullptr;
  if ((e = cudaMalloc(&sink, sizeof(T))) != cudaSuccess)
    return pr_fail(QG_ERR_OOM, "qg_probe_fma_rate: cudaMalloc: %s", cudaGetErrorString(e));
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const dim3 grid(sms * kCtasPerSm), block(kThreads);
  const T a = T(0.999999), b = T(1e-6);
  auto run = [&](int iters, float* ms) -> cudaError_t {
    cudaEventRecord(t0);
    fma_probe_kernel<T><<<grid, block>>>(iters, a, b, sink);
    cudaEventRecord(t1);
    cudaError_t r = cudaEventSynchronize(t1);
    if (r == cudaSuccess) r = cudaGetLastError();
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, t0, t1);
    return r;
  };
  // calibrate to about 50 ms per launch, then keep the best of three
  float ms = 0.f;
  int iters = 64;
  e = run(iters, &ms);
  for (int k = 0; k < 12 && e == cudaSuccess && ms < 5.f; ++k) {
    iters *= 4;
    e = run(iters, &ms);
  }
  if (e == cudaSuccess && ms > 0.f) {
    const double scale = 50.0 / ms;
    iters = (int)std::fmin(2.0e9, std::fmax(1.0, iters * scale));
  }
  double best = 0.0, best_ms = 0.0;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = run(iters, &ms);
    const double flops = 2.0 * kChains * kUnroll * (double)iters * (double)grid.x * kThreads;
    if (e == cudaSuccess && ms > 0.f && flops / (ms * 1e-3) > best) {
      best = flops / (ms * 1e-3);
      best_ms = ms;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(sink);
  if (e != cudaSuccess) return pr_fail(QG_ERR_CUDA, "qg_probe_fma_rate: %s", cudaGetErrorString(e));
  *flops_per_s = best;
  if (ms_out) *ms_out = best_ms;
  return QG_OK;
}

}  // namespace

extern "C" int qg_probe_fma_rate(int32_t dtype, double* flops_per_s, double* ms) {
  if (!flops_per_s) return pr_fail(QG_ERR_ARG, "qg_probe_fma_rate: NULL output");
  if (dtype == QG_FP32) return probe<float>(flops_per_s, ms);
  if (dtype == QG_FP64) return probe<double>(flops_per_s, ms);
  return pr_fail(QG_ERR_ARG, "qg_probe_fma_rate: dtype must be QG_FP32 or QG_FP64");
}
