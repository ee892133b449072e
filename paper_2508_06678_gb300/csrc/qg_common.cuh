// Shared device types and layout descriptors of libqg.
//
// Layouts (all device-resident, owned by the handle):
//   spectral  S[c * SP + r] : truncated half spectrum, column-major in k_x.
//             c = m_x in [0, Kc), Kc = K + 1; r in [0, Ny), Ny = 2K + 1 with
//             m_y = r for r <= K and m_y = r - Ny otherwise.  Only the modes
//             the 2/3 rule keeps are stored (Sec. II-C); columns in
//             [Kc, Kcp) are zero padding.
//   mixed     I[y * IP + c]  : one field after the y-transform, rows y in
//             [0, N), columns m_x in [0, Kcp).  The column pass writes it in
//             W-wide tiles, the row pass reads whole rows.
//   physical  f[y * N + x]   : real field.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <atomic>
#include <mutex>
#include <type_traits>
#include <utility>

// threads per CTA of the register-resident row pass (whole rows of N / 16 or N / 12 threads each)
#ifndef QG_ROW_CTA_THREADS
#define QG_ROW_CTA_THREADS 128
#endif

namespace qg {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// (i s) * a for s = +1 / -1
template <typename C> __device__ __forceinline__ C cmul_si(C a, int s) {
  return s > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}
// (i k) * a for real k
template <typename C> __device__ __forceinline__ C cmul_ik(C a, decltype(C::x) k) { return mk<C>(-a.y * k, a.x * k); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }

// Grid geometry shared by every kernel.
struct Geom {
  int n;      // grid size N
  int K;      // 2/3-rule band limit floor((N-1)/3)
  int Kc;     // K + 1 kept k_x columns
  int Kcp;    // Kc rounded up to the column tile width
  int Ny;     // 2K + 1 kept k_y rows
  int SP;     // spectral column pitch (complex elements)
  int IP;     // mixed-array row pitch (complex elements) = Kcp
  double kscale;  // 2 pi / L
};

__host__ __device__ __forceinline__ int my_of_r(const Geom& g, int r) { return r <= g.K ? r : r - g.Ny; }
// row of an N-point k_y sequence (FFT order) holding spectral index r
__host__ __device__ __forceinline__ int row_of_r(const Geom& g, int r) { return r <= g.K ? r : g.n + r - g.Ny; }

constexpr int kMaxIn = 12;   // max fields entering one row pass
constexpr int kMaxOut = 8;   // max fields leaving one row pass
constexpr int kMaxDer = 12;  // max derived fields leaving one column pass
constexpr int kMaxFwd = 8;   // max fields entering one column pass
constexpr int kMaxY = 8;     // row-pass output arrays of a handle

// Codes of the spectral fields a column pass derives from a vorticity
// spectrum w (all scaled by 1/N^2 so that the two inverse passes return
// physical values).  The *_T codes apply the test filter first.
enum DerCode : int {
  D_U = 0,    // u_total = -d psi/dy + U
  D_V = 1,    // v = d psi/dx
  D_WX = 2,   // dw/dx
  D_WY = 3,   // dw/dy
  D_PXY = 4,  // d2 psi/dxdy
  D_PD = 5,   // d2 psi/dx2 - d2 psi/dy2
  D_W = 6,    // w itself
  D_TEST = 8  // flag: test-filtered version of the code in the low bits
};

// Row-pass product programs.
enum RowProg : int {
  RP_NONE = 0,    // (u, v, wx, wy) -> J
  RP_LEITH = 1,   // (u, v, wx, wy) -> J, g wx, g wy with g = |grad w|
  RP_SMAG = 2,    // (u, v, wx, wy, pxy, pd) -> J, g wx, g wy with g = |S|
  RP_DLEITH = 3,  // RP_LEITH at grid and test level
  RP_DSMAG = 4,   // RP_SMAG at grid and test level
  RP_SCALE = 5,   // f_i * factor(x, y) for each input (Brinkman, sponge)
  RP_COPY = 6,    // identity (forward transform of a physical field, or inverse to physical)
  // the adjoint's fused passes (register-resident kernels): the step's products of one stage with its physical
  // fields kept (RP_ADJ_FWD), and the transposed products of an adjoint field with kept fields (RP_ADJ_REV)
  RP_ADJ_FWD = 7,
  RP_ADJ_REV = 8,
};

// Column-pass operations.
enum ColOp : int {
  CO_DERIVE = 0,       // w <- stored state w0
  CO_STAGE_STATIC = 1, // forward J[, P, Q]; L = -J - beta v + C D; RK combine
  CO_DYN_REDUCE = 2,   // forward J, P, Q, J~, P~, Q~; store J, D; Germano partial sums
  CO_DYN_COMBINE = 3,  // L = -J - beta v + C D with C from the partial sums; RK combine
  CO_CURL = 4,         // forward u, v; w = i kx v - i ky u
  CO_FORWARD = 5,      // forward one field; w = that field
  // the paper's scheme (Eq. 4)
  CO_AB2CN = 6,          // forward J[, P, Q][, chi u, chi v]; CN / AB2 combine; sponge field or next state
  CO_AB2CN_COMBINE = 7,  // as CO_AB2CN from stored J, D, F_obs and the Germano partial sums
  CO_AB2CN_FINAL = 8,    // forward s = dt rate chi_s Z; w^{t+1} = w* - s
  CO_FORWARD2 = 9,       // forward two fields: the first to w0, the second to w0b (the adjoint's paired transforms)
  CO_FORWARD_N = 10,     // forward nfwd fields, field f's kept band to fout[f] (the adjoint's transform batches)
};

struct RowDesc {
  int prog;
  int nin, nout;
  int in_phys;   // inputs: 1 = physical rows from phys_in, 0 = mixed arrays in[]
  int out_phys;  // outputs: 1 = physical rows to phys_out, 0 = mixed arrays out[]
  unsigned dx_mask;  // bit f: multiply output f by i k_x after the forward transform
  const void* in[kMaxIn];
  void* out[kMaxOut];
  const void* phys_in;
  void* phys_out;
  const void* phys_in2;  // RP_COPY: a second physical field, transformed with the first (Hermitian pair)
  void* phys_out2;       // RP_COPY: the second field of an inverse pair
  int npair;             // RP_COPY, register-resident kernels: > 0 transforms npair pairs in one launch, pair p
                         // taking physical fields pin[2p], pin[2p + 1] to out[2p], out[2p + 1] (in_phys), or
                         // mixed in[2p], in[2p + 1] to pout[2p], pout[2p + 1]; a NULL second field is skipped
  const void* pin[kMaxOut];
  void* pout[kMaxOut];
  // RP_ADJ_FWD / RP_ADJ_REV: closure family (0 none, 1 Smagorinsky, 2 Leith) and the stage's physical fields
  // u_total, v, w_x, w_y [, psi_xy, psi_xx - psi_yy] (written by RP_ADJ_FWD, read by RP_ADJ_REV)
  int adj_kind;
  void* pf[6];
  const void* factor;  // RP_SCALE: physical factor field
  int check_finite;    // set *flag if a product is not finite
  int* flag;
  int* err;            // status bits of the bounds-checked debug build (NULL: not reported)
  int pdl;             // host side: launch with programmatic stream serialisation
};

struct ColDesc {
  int op;
  int nfwd;
  const void* fin[kMaxFwd];
  int nder;
  int der[kMaxDer];
  void* dout[kMaxDer];
  // spectral arrays
  void* w0;        // state w^n (read; written when store_w0)
  void* w0b;       // CO_FORWARD2: the second field's spectral band (written)
  void* fout[kMaxFwd];  // CO_FORWARD_N: field f's spectral band (written)
  void* ws;        // RK stage state read when use_ws
  void* ws_out;    // RK stage state written when store_ws (a different array, so split passes never race)
  void* jh;        // dynamic closures: stored J_hat
  void* dh;        // dynamic closures: stored D_hat
  void* scr[3];    // dynamic closures, FP32 register-resident kernels: the Germano reduction's cross-field
                   // values (spectral layout, kept modes only)
  int use_ws;      // the stage input is ws (else w0)
  int store_ws, store_w0;
  int zero_mean;   // set the (0,0) mode to zero before storing / deriving
  int viscous;     // multiply by exp(-(nu|k|^2 + mu) dt) after the combine
  // RK combine w_new = a w0 + b (w_s + dt L)
  double a, b, dt;
  double beta, U;
  double coeff;     // static closure coefficient C
  int closure_pow;  // p of r^p in the Germano M
  double test_ratio;
  int test_m2max;   // test filter keeps |m|^2 <= test_m2max (exact integer form of |m| <= N / (2 r))
  int test_kmax;    // largest k_x the test filter keeps; test-level fields vanish beyond it, and the
                    // column pass leaves those columns of their mixed arrays at the zeros set at creation
  double rpow;      // r^p
  // Germano partial sums: written by CO_DYN_REDUCE (2 doubles per block), read by CO_DYN_COMBINE
  double* partials;
  int npartials;
  double* coeff_out;  // CO_DYN_COMBINE: block 0 writes C here
  // the paper's scheme (Eq. 4)
  void* bh;          // dynamic closures: stored Brinkman forcing F_obs (CO_DYN_REDUCE fields 6, 7)
  void* eprev;       // explicit terms E of the previous step (read, then overwritten with this step's)
  void* wss;         // w** (read) / w* (written) of the sponge split
  int ab2_first;     // Euler start: E_prev = E, w** = w*
  int nst;           // forward fields of the closure products before the Brinkman pair
  int brink;         // the Brinkman pair chi u, chi v follows
  int sponge_next;   // derive Z = 3/2 w* - 1/2 w** for the sponge (else the next state)
  double inv_eta, nu, mu;
  const void* visc_x;  // exp(-nu kx^2 dt), per m_x
  const void* visc_y;  // exp(-nu ky^2 dt), per r
  double visc_mu;      // exp(-mu dt)
  int pdl;             // host side: launch with programmatic stream serialisation
  int lean;            // host side, FP32 Germano reduction: 0 = lean form where it makes one wave, 1 = lean form
                       // whenever it fits, 2 = never (the ensemble tuner's choice)
  int* flag;           // stop flag checked at entry (NULL: always run)
  int* err;            // status bits raised by bounded waits that give up (NULL: not reported)
  int stall_cta1;      // failure-handling test only (0 otherwise): CTA stall_cta1 - 1 arms its first tile's
                       // mbarrier but issues no copy at all, so its bounded wait runs out with nothing in flight
};

// Per-thread accumulator of the Germano sums.  FP64 fields accumulate in
// FP64; FP32 fields use error-free transformations (TwoProduct by FMA,
// TwoSum) so the per-thread partial carries about twice FP32 precision
// before it joins the FP64 cross-thread reduction.
// Programmatic dependent launch.  A kernel launched by launch_pdl may be scheduled while the kernel before
// it on the stream is still finishing: it first waits here, before any memory access, until that kernel has
// completed and its writes are visible, then lets the next kernel be scheduled.  Launched without the
// attribute, both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// programmatic launches are allowed unless QG_NO_PDL is set in the environment (read once)
inline bool pdl_enabled() {
  static const bool on = getenv("QG_NO_PDL") == nullptr;
  return on;
}

// k<<<grid, block, smem, st>>>(args...), with programmatic stream serialisation when pdl is set (k must call
// pdl_enter() first).  The adjoint's chains of small launches gain from it; the forward step's graph measured
// slower with it, so its launches leave it off.
template <typename... P, typename... A>
cudaError_t launch_pdl(bool pdl, void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl && pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Status bit of the bounds-checked debug build (-DQG_CHECKED): some kernel met an index outside its array.
constexpr int kFlagBounds = 4;

// Index checks of the debug build.  QG_INB(i, n, st) is true when 0 <= i < n; otherwise it sets kFlagBounds in
// *st (when st is not NULL) and is false, and the caller skips the access (a load yields zero).  In the release
// build it is the constant true and the check compiles away.
#ifdef QG_CHECKED
__device__ __forceinline__ bool qg_in_bounds(long long i, long long n, int* st) {
  if (i >= 0 && i < n) return true;
  if (st) atomicOr(st, kFlagBounds);
  return false;
}
#define QG_INB(i, n, st) ::qg::qg_in_bounds((long long)(i), (long long)(n), (st))
#else
#define QG_INB(i, n, st) true
#endif
// checked load p[i] of an array of n elements (zero when out of range in the debug build)
template <typename E>
__device__ __forceinline__ std::remove_cv_t<E> qg_load(E* p, long long i, long long n, int* st) {
#ifdef QG_CHECKED
  if (!qg_in_bounds(i, n, st)) return std::remove_cv_t<E>{};
#else
  (void)n;
  (void)st;
#endif
  return p[i];
}
#define QG_LD(p, i, n, st) ::qg::qg_load((p), (long long)(i), (long long)(n), (st))
// checked store p[i] = v
#define QG_ST(p, i, n, st, v)              \
  do {                                     \
    if (QG_INB((i), (n), (st))) (p)[(i)] = (v); \
  } while (0)

// Raise kernel KERNEL's dynamic shared-memory limit on the current device to at least `bytes`.  The limit only
// ever rises: each (kernel, device) keeps a high-water mark, raised under a lock, so one host thread can never
// lower the limit between another thread's raise and its launch (a launch with a larger request would then fail).
template <auto KERNEL>
cudaError_t raise_smem_limit(size_t bytes) {
  constexpr int kDev = 64;
  static std::atomic<int> high[kDev];
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int want = (int)bytes;
  if (dev < 0 || dev >= kDev) return cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (want <= high[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  if (want <= high[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (e == cudaSuccess) high[dev].store(want, std::memory_order_release);
  return e;
}

template <typename T> struct GermanoAcc;
template <> struct GermanoAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct GermanoAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float h = a * b;
    const float l = fmaf(a, b, -h);
    add(h);
    c += l;
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

}  // namespace qg
