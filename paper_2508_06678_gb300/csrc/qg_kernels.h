// Host-side declarations of the kernel launchers of libqg.
#pragma once

#include "fft.cuh"

namespace qg {

template <typename T>
cudaError_t launch_row(const Geom& g, const FftPlan& plan, const RowDesc& d, const void* tw, int threads,
                       size_t smem, cudaStream_t st);

template <typename T>
cudaError_t launch_col(const Geom& g, const FftPlan& plan, const ColDesc& d, const void* tw, int W, int threads,
                       size_t smem, cudaStream_t st);

// Spectral diagnostics: out[0] = sum w |k|^2 |psi|^2, out[1] = sum w |w|^2 over the stored half spectrum
// (w = 1 on the k_x = 0 column, else 2), FP64, deterministic two-level reduction.
template <typename T>
cudaError_t launch_spectral_sums(const Geom& g, const void* w0, double* partials, int nblk, double* out,
                                 cudaStream_t st);

// Physical max |f| and finiteness: out[0] = max |f|, out[1] = 1 if all finite else 0.
template <typename T>
cudaError_t launch_phys_maxabs(const Geom& g, const void* f, double* partials, int nblk, double* out,
                               cudaStream_t st);

// ---- discrete adjoint of the step (adjoint.cu)
// spectral multipliers of adj_combine (conjugates are the transposes the adjoint needs)
enum AdjMul : int {
  AM_ONE = 0,
  AM_CU,    // -i k_y / |k|^2   transpose of w -> u
  AM_CV,    // +i k_x / |k|^2   transpose of w -> v
  AM_CX,    // -i k_x           transpose of d/dx
  AM_CY,    // -i k_y           transpose of d/dy
  AM_IX,    // +i k_x
  AM_IY,    // +i k_y
  AM_XY,    // k_x k_y / |k|^2           w -> psi_xy
  AM_DD,    // (k_x^2 - k_y^2) / |k|^2   w -> psi_xx - psi_yy
  AM_VISC,  // exp(-(nu |k|^2 + mu) dt)
};
constexpr int AM_TESTF = 0x100;  // flag: also multiply by the test filter, |m|^2 (2r)^2 <= N^2
constexpr int kAdjTerms = 12;
struct AdjTerm {
  const void* in;        // spectral array (stored band layout)
  int code;              // AdjMul, optionally | AM_TESTF
  double coef;
  const double* cptr;    // if set, coef is multiplied by this device scalar
};
struct AdjCombine {
  void* out;
  int accumulate;  // out += sum (else out = sum)
  int zero_mean;   // set the (0, 0) mode to zero
  int nterm;
  AdjTerm term[kAdjTerms];
  double nu, mu, dt;  // AM_VISC
  int test_m2max;     // AM_TESTF
};
enum AdjKind : int { AK_NONE = 0, AK_SMAG = 1, AK_LEITH = 2 };
enum AdjProdMode : int { AP_FORWARD = 0, AP_ADJOINT = 1 };
// Pointwise products (physical arrays, working precision).
//   forward: out0 = u w_x + v w_y, out1 = g w_x, out2 = g w_y
//   adjoint: out0..3 = lam w_x, lam w_y, lam u, lam v; with a closure, p = -lam_x, q = -lam_y,
//            s = p w_x + q w_y: Leith out4,5 = g p + s w_x / g, g q + s w_y / g;
//            Smagorinsky out4,5 = g p, g q, out6,7 = 4 s psi_xy / g, s psi_d / g
struct AdjProducts {
  int kind, mode;
  const void *u, *v, *wx, *wy, *pxy, *pd;
  const void *lam, *lx, *ly;
  void* out[8];
};
constexpr int kAdjDotBlocks = 256;
// FP64 inner products, deterministic and in one launch: every block stores its partial sum, and the block that
// counts itself in last (an atomic counter, which it resets to zero) sums the partials in a fixed order.
struct AdjDotOut {
  double* partials;   // kAdjDotBlocks doubles
  double* partials2;  // kAdjDotBlocks more: the Germano pair's second sum
  unsigned* counter;  // zero between launches
  double scale;
  double* out;        // out[0] = scale * sum
  // then, if kappa is set: kappa[0] = out[0] / (n2 mm[0]) if C[0] > 0 and mm[0] > 0, else 0
  // (C_bar / (N^2 <MM>), the dynamic coefficient's share of a stage's transpose, Eq. 12, 14)
  const double* C;
  const double* mm;
  double* kappa;
  double n2;
};

template <typename T>
cudaError_t launch_adj_combine(const Geom& g, const AdjCombine& a, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_products(size_t count, const AdjProducts& a, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_scale(size_t count, const void* f, const void* x0, double s0, void* out0, const void* x1,
                             double s1, void* out1, cudaStream_t st);
// o.out[0] = o.scale * sum_k w_k Re(A conj B) over the stored band (w = 1 on the k_x = 0 column, else 2)
template <typename T>
cudaError_t launch_adj_spec_dot(const Geom& g, const void* A, const void* B, const AdjDotOut& o, cudaStream_t st);
// o.out[0] = o.scale * sum_i X_i Y_i Z_i
template <typename T>
cudaError_t launch_adj_phys_dot(size_t count, const void* X, const void* Y, const void* Z, const AdjDotOut& o,
                                cudaStream_t st);
// A stage's Germano sums in one pass over H and M (Eq. 12, 14): o.out[0] = o.scale <H M>, o.out[1] = o.scale
// <M M> (spectral, weighted as above), o.out[2] = C = max(0, out[0] / out[1]) if out[1] > 0, else 0
template <typename T>
cudaError_t launch_adj_germano_dots(const Geom& g, const void* H, const void* M, const AdjDotOut& o,
                                    cudaStream_t st);

// Sets the thread-local message returned by qg_last_error().
void set_last_error(const char* msg);

// Element-wise precision conversion between device buffers.
cudaError_t launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, size_t count, cudaStream_t st);

}  // namespace qg
