// Host side of libqg: the C-ABI declared in include/qg.h.
//
// One step (Sec. II-E split, sub-step integrators as documented in qg.h) is
// a chain of alternating row and column passes on the handle's stream:
//
//   for each of the 3 RK stages:
//     row pass   : inverse x-FFT of the stage's derived fields, products, forward x-FFT
//     column pass: forward y-FFT, L = -J - beta v + C D, RK combine, derived
//                  fields of the next stage (or of the Brinkman/sponge sub-step),
//                  inverse y-FFT
//     (dynamic closures split the column pass in two around the Germano sums)
//   Brinkman: row pass scales (u_total, v) by exp(-chi dt/eta); column pass curls
//   sponge  : row pass scales w by exp(-rate chi_s dt); column pass projects,
//             stores w^{n+1} and derives stage 1 of the next step.
//
// The column pass of one step therefore also prepares the next step, and a
// step costs 2 + 2 x 3 (+1 per stage for dynamic closures) launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <new>
#include <string>
#include <array>
#include <utility>
#include <algorithm>
#include <limits>
#include <map>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/qg.h"
#include "fast.cuh"
#include "qg_kernels.h"
#include "tma.cuh"

using namespace qg;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e),
              cudaGetErrorString(e));
}

#define CK(call, what)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

bool valid_n(int n) {
  if (n < 16 || n > 4096 || (n & 1)) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

FftPlan make_plan(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  while (m % 8 == 0) { p.radix[p.npass++] = 8; m /= 8; }
  if (m % 4 == 0) { p.radix[p.npass++] = 4; m /= 4; }
  if (m % 2 == 0) { p.radix[p.npass++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.npass++] = 3; m /= 3; }
  return p;
}

int max_items(int R) { return R == 3 ? 2 : 8 / R; }

int threads_for(const FftPlan& p, int B, int floor_threads) {
  int need = floor_threads;
  for (int s = 0; s < p.npass; ++s) {
    const int R = p.radix[s];
    const int items = (p.n / R) * B;
    const int t = (items + max_items(R) - 1) / max_items(R);
    if (t > need) need = t;
  }
  return (need + 31) / 32 * 32;
}

// cos and sin of 2 pi j / n with the argument reduced exactly to [0, pi/4].
void cos_sin_frac(long j, long n, double* c, double* s) {
  j %= n;
  if (j < 0) j += n;
  const long q4 = 4 * j;
  const long quad = q4 / n;
  const long rem = q4 - quad * n;  // angle within the quadrant = (pi/2) rem / n
  double cc, ss;
  if (2 * rem <= n) {
    const double phi = (M_PI / 2) * double(rem) / double(n);
    cc = std::cos(phi);
    ss = std::sin(phi);
  } else {
    const double phi = (M_PI / 2) * double(n - rem) / double(n);
    cc = std::sin(phi);
    ss = std::cos(phi);
  }
  switch (quad) {
    case 0: *c = cc; *s = ss; break;
    case 1: *c = -ss; *s = cc; break;
    case 2: *c = -cc; *s = -ss; break;
    default: *c = ss; *s = -cc; break;
  }
}

}  // namespace

namespace qg {
// Non-first passes of the specialised FFT in order (radix-16 passes, then the
// last pass of radix 2^(log2 n mod 4)); each contributes (R - 1) * NS entries
// [r - 1][k] = W_n^(r k n / (NS R)).
// The twiddled passes (every pass after the first) of the specialised engines, in order:
// N = 2^p: radix 16 while possible, then one radix-8/4/2 pass; N = 3 * 2^p: radix 4 after the first
// (radix-12) pass while a factor 4 remains, then one radix-2 pass for odd p.
static void for_each_pass(int n, void (*fn)(int, int, int, void*), void* ctx) {
  int off = 0;
  if (n % 3 == 0) {
    int m = n / 12, ns = 12;
    for (; m >= 4; m /= 4, ns *= 4) {
      fn(4, ns, off, ctx);
      off += 3 * ns;
    }
    if (m == 2) fn(2, ns, off, ctx);
    return;
  }
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  const int np16 = lg / 4, rlast = 1 << (lg % 4);
  int ns = 16;
  for (int p = 1; p < np16; ++p, ns *= 16) {
    fn(16, ns, off, ctx);
    off += 15 * ns;
  }
  if (rlast > 1) fn(rlast, n / rlast, off, ctx);
}

int fast_pass_table_size(int n) {
  int total = 0;
  for_each_pass(n, [](int R, int NS, int off, void* c) { *(int*)c = off + (R - 1) * NS; }, &total);
  return total;
}

void fast_pass_table(int n, const double* tw, double* out) {
  struct Ctx { int n; const double* tw; double* out; } cx{n, tw, out};
  for_each_pass(
      n,
      [](int R, int NS, int off, void* c) {
        Ctx& x = *(Ctx*)c;
        for (int r = 1; r < R; ++r)
          for (int k = 0; k < NS; ++k) {
            const long j = ((long)r * k * (x.n / (NS * R))) % x.n;
            const size_t e = (size_t)off + (size_t)(r - 1) * NS + k;
            x.out[2 * e] = x.tw[2 * j];
            x.out[2 * e + 1] = x.tw[2 * j + 1];
          }
      },
      &cx);
}

// Lets other translation units of the library report through qg_last_error().
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace qg

struct qg_handle {
  Geom g{};
  int fp32 = 0;
  size_t esz = 8;  // bytes per real
  double L = 0, beta = 0, U = 0;
  qg_closure cl{};
  qg_params par{};
  cudaStream_t stream = nullptr;
  FftPlan plan{};
  int W = 4, col_threads = 256, row_threads = 256;
  size_t col_smem = 0, row_smem = 0;
  int ncolblk = 0;
  bool fast = false;  // power-of-two grid served by the register-resident FFT kernels
  bool dynamic = false;
  double static_coeff = 0.0;
  int test_m2max = 0;  // largest |m|^2 the test filter keeps
  int test_kmax = 0;   // largest k_x the test filter keeps
  // stage program
  int row_prog = RP_NONE, nin = 4, nout = 1;
  unsigned dx_mask = 0;
  int nder = 4;
  int der[kMaxDer] = {};
  // device buffers
  void* w0 = nullptr;
  void* ws = nullptr;
  void* ws2 = nullptr;  // second stage-state array (stages alternate between ws and ws2)
  void* jh = nullptr;
  void* red_scr[3] = {nullptr, nullptr, nullptr};  // Germano reduction scratch (FP32 register-resident kernels)
  void* dh = nullptr;
  void* X[kMaxIn] = {};
  void* Y[kMaxY] = {};
  // the paper's scheme (Eq. 4): history of the explicit terms and of w*, stored F_obs
  int scheme = QG_SCHEME_RK3_EXACT;
  void* eprev = nullptr;
  void* wss = nullptr;
  void* bh = nullptr;
  bool ab2_hist = false;
  void* fac_b = nullptr;
  void* fac_s = nullptr;
  void* chi_s = nullptr;  // the sponge mask itself (the adjoint's sponge-rate derivative)
  // workspace of qg_step_vjp, allocated by its first call: spectral, physical and mixed arrays, dot results
  std::vector<void*> adj_S, adj_P, adj_M;
  double* adj_dots = nullptr;
  cudaGraphExec_t adj_graph = nullptr;  // one adjoint step, captured after its first eager run
  bool adj_graph_tried = false;
  // side branch of the adjoint step: a second stream, its fork event and join events (one per pending branch)
  cudaStream_t adj_side = nullptr;
  cudaEvent_t adj_fork_ev = nullptr;
  cudaEvent_t adj_join_ev[8] = {};
  int adj_njoin = 0;
  int32_t adj_graph_launches[QG_NUM_KCLASS] = {};
  void* tw = nullptr;
  void* ptw = nullptr;  // per-pass twiddle table of the power-of-two kernels
  void* visc_x = nullptr;
  void* visc_y = nullptr;
  void* phys = nullptr;
  double visc_mu = 1.0;
  double* partials = nullptr;  // Germano partial sums (2 per column block)
  double* red = nullptr;       // diagnostics partials
  double* dev_scalars = nullptr;  // [0..2] C per stage, [4..7] diagnostics
  int* flag = nullptr;
  int* flag_host = nullptr;
  // failure-handling test only: QG_INJECT_TMA_STALL=<cta> at creation makes that CTA of the first step's first
  // TMA column pass wait for a tile it never requested (one shot; 0 = off, else the CTA index + 1)
  int inject_stall = 0;
  // launch forms of the step chosen by an ensemble's tuner: programmatic dependent launch, the FP32 Germano
  // reduction's lean form (ColDesc::lean); both leave the arithmetic unchanged
  int step_pdl = 0;
  int lean_reduce = 0;
  cudaEvent_t flag_event = nullptr;
  bool flag_pending = false;
  int64_t step = 0;
  double t = 0;
  std::vector<void*> allocs;
  // TMA tensor maps of the mixed arrays (power-of-two kernels)
  std::vector<std::pair<const void*, CUtensorMap>> maps;
  // one step captured as a CUDA graph and replayed by qg_step (eager launches
  // while tracing, or where the stream cannot be captured)
  cudaGraphExec_t step_graph = nullptr;
  bool graph_tried = false;
  int64_t eager_steps = 0;
  int32_t graph_launches[QG_NUM_KCLASS] = {};
  // tracing
  bool prof = false;
  int32_t launches[QG_NUM_KCLASS] = {};
  double prof_ms[QG_NUM_KCLASS] = {};
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;

  ~qg_handle() {
    if (adj_side) cudaStreamSynchronize(adj_side);
    if (adj_side) cudaStreamDestroy(adj_side);
    if (adj_fork_ev) cudaEventDestroy(adj_fork_ev);
    for (cudaEvent_t ev : adj_join_ev)
      if (ev) cudaEventDestroy(ev);
    if (step_graph) cudaGraphExecDestroy(step_graph);
    if (adj_graph) cudaGraphExecDestroy(adj_graph);
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    if (flag_host) cudaFreeHost(flag_host);
    if (flag_event) cudaEventDestroy(flag_event);
  }
};

namespace {

int dalloc(qg_handle* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  h->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  return QG_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D map of one mixed array [y][k_x] (complex, IP columns, n rows); a box is
// W columns (2W reals, 16 or 32 bytes) by BR rows
int add_tensor_map(qg_handle* h, const void* base, int W, int BR) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(QG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * h->g.IP, (cuuint64_t)h->g.n};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * h->g.IP * h->esz};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * W), (cuuint32_t)BR};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = enc(&m, h->fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                   const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(QG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  h->maps.push_back({base, m});
  return QG_OK;
}

const CUtensorMap* find_map(const qg_handle* h, const void* base) {
  for (const auto& e : h->maps)
    if (e.first == base) return &e.second;
  return nullptr;
}

// upload host doubles as the handle's working precision
int upload_real(qg_handle* h, void* dst, const std::vector<double>& v) {
  if (h->fp32) {
    std::vector<float> f(v.begin(), v.end());
    CK(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->stream), "upload");
    CK(cudaStreamSynchronize(h->stream), "upload sync");
  } else {
    CK(cudaMemcpyAsync(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice, h->stream), "upload");
    CK(cudaStreamSynchronize(h->stream), "upload sync");
  }
  return QG_OK;
}

cudaEvent_t take_event(qg_handle* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// launch bracket: count, and with tracing on record an event pair around the launch
struct Bracket {
  qg_handle* h;
  int cls;
  cudaEvent_t a = nullptr;
  Bracket(qg_handle* h_, int c) : h(h_), cls(c) {
    h->launches[cls] += 1;
    if (h->prof) {
      a = take_event(h);
      if (a) cudaEventRecord(a, h->stream);
    }
  }
  void done() {
    if (!a) return;
    cudaEvent_t b = take_event(h);
    if (b) {
      cudaEventRecord(b, h->stream);
      h->recs.push_back({cls, a, b});
    } else {
      h->pool.push_back(a);
    }
  }
};

template <typename T>
cudaError_t row_fast_dispatch(qg_handle* h, const RowDesc& d) {
  switch (h->g.n) {
    case 256: return launch_row_fast<T, 256>(h->g, d, h->ptw, h->stream);
    case 512: return launch_row_fast<T, 512>(h->g, d, h->ptw, h->stream);
    case 1024: return launch_row_fast<T, 1024>(h->g, d, h->ptw, h->stream);
    case 2048: return launch_row_fast<T, 2048>(h->g, d, h->ptw, h->stream);
    case 4096: return launch_row_fast<T, 4096>(h->g, d, h->ptw, h->stream);
    case 384: return launch_row_fast<T, 384>(h->g, d, h->ptw, h->stream);
    case 768: return launch_row_fast<T, 768>(h->g, d, h->ptw, h->stream);
    case 1536: return launch_row_fast<T, 1536>(h->g, d, h->ptw, h->stream);
    case 3072: return launch_row_fast<T, 3072>(h->g, d, h->ptw, h->stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t col_fast_dispatch(qg_handle* h, const ColDesc& d) {
  TmaSet tm;
  memset(&tm, 0, sizeof(tm));
  for (int f = 0; f < d.nfwd; ++f) {
    const CUtensorMap* m = find_map(h, d.fin[f]);
    if (!m) return cudaErrorInvalidValue;
    tm.in[f] = *m;
  }
  for (int q = 0; q < d.nder; ++q) {
    const CUtensorMap* m = find_map(h, d.dout[q]);
    if (!m) return cudaErrorInvalidValue;
    tm.out[q] = *m;
  }
  switch (h->g.n) {
    case 256: return launch_col_fast<T, 256>(h->g, d, h->ptw, tm, h->stream);
    case 512: return launch_col_fast<T, 512>(h->g, d, h->ptw, tm, h->stream);
    case 1024: return launch_col_fast<T, 1024>(h->g, d, h->ptw, tm, h->stream);
    case 2048: return launch_col_fast<T, 2048>(h->g, d, h->ptw, tm, h->stream);
    case 4096: return launch_col_fast<T, 4096>(h->g, d, h->ptw, tm, h->stream);
    case 384: return launch_col_fast<T, 384>(h->g, d, h->ptw, tm, h->stream);
    case 768: return launch_col_fast<T, 768>(h->g, d, h->ptw, tm, h->stream);
    case 1536: return launch_col_fast<T, 1536>(h->g, d, h->ptw, tm, h->stream);
    case 3072: return launch_col_fast<T, 3072>(h->g, d, h->ptw, tm, h->stream);
    default: return cudaErrorInvalidValue;
  }
}

int run_row(qg_handle* h, RowDesc& d, int cls, bool use_flag = true) {
  d.flag = use_flag ? h->flag : nullptr;
  d.err = h->flag;
  if (h->step_pdl) d.pdl = 1;
  Bracket br(h, cls);
  cudaError_t e;
  if (h->fast)
    e = h->fp32 ? row_fast_dispatch<float>(h, d) : row_fast_dispatch<double>(h, d);
  else
    e = h->fp32 ? launch_row<float>(h->g, h->plan, d, h->tw, h->row_threads, h->row_smem, h->stream)
                : launch_row<double>(h->g, h->plan, d, h->tw, h->row_threads, h->row_smem, h->stream);
  br.done();
  if (e != cudaSuccess) return cuda_fail(e, "row pass launch");
  return QG_OK;
}

int run_col(qg_handle* h, ColDesc& d, int cls, bool use_flag = true) {
  d.flag = use_flag ? h->flag : nullptr;
  d.err = h->flag;
  if (h->step_pdl) d.pdl = 1;
  d.lean = h->lean_reduce;
  Bracket br(h, cls);
  cudaError_t e;
  if (h->fast)
    e = h->fp32 ? col_fast_dispatch<float>(h, d) : col_fast_dispatch<double>(h, d);
  else
    e = h->fp32 ? launch_col<float>(h->g, h->plan, d, h->tw, h->W, h->col_threads, h->col_smem, h->stream)
                : launch_col<double>(h->g, h->plan, d, h->tw, h->W, h->col_threads, h->col_smem, h->stream);
  br.done();
  if (e != cudaSuccess) return cuda_fail(e, "column pass launch");
  return QG_OK;
}

ColDesc col_base(qg_handle* h) {
  ColDesc d{};
  d.w0 = h->w0;
  d.ws = h->ws;
  d.ws_out = h->ws;
  d.jh = h->jh;
  for (int i = 0; i < 3; ++i) d.scr[i] = h->red_scr[i];
  d.dh = h->dh;
  d.dt = h->par.dt;
  d.beta = h->beta;
  d.U = h->U;
  d.coeff = h->static_coeff;
  d.test_ratio = h->cl.test_ratio;
  d.test_m2max = h->test_m2max;
  d.test_kmax = h->test_kmax;
  const int p = (h->cl.kind == QG_SMAG || h->cl.kind == QG_DSMAG) ? 2 : 3;
  d.closure_pow = p;
  d.rpow = std::pow(h->cl.test_ratio, p);
  d.partials = h->partials;
  d.npartials = h->ncolblk;
  d.visc_x = h->visc_x;
  d.visc_y = h->visc_y;
  d.visc_mu = h->visc_mu;
  d.eprev = h->eprev;
  d.wss = h->wss;
  d.bh = h->bh;
  d.ab2_first = h->ab2_hist ? 0 : 1;
  d.inv_eta = h->par.eta > 0 ? 1.0 / h->par.eta : 0.0;
  d.nu = h->par.nu;
  d.mu = h->par.mu;
  return d;
}


void set_stage_derived(qg_handle* h, ColDesc& d) {
  d.nder = h->nder;
  for (int i = 0; i < h->nder; ++i) {
    d.der[i] = h->der[i];
    d.dout[i] = h->X[i];
  }
}

void set_final(qg_handle* h, ColDesc& d) {
  d.zero_mean = 1;
  d.store_w0 = 1;
  set_stage_derived(h, d);
}

// after the RK combine of stage 3 (viscous factor applied): derive what the
// next sub-step needs
void set_after_rk(qg_handle* h, ColDesc& d) {
  if (h->fac_b) {
    d.nder = 2;
    d.der[0] = D_U;
    d.der[1] = D_V;
    d.dout[0] = h->X[0];
    d.dout[1] = h->X[1];
  } else if (h->fac_s) {
    d.nder = 1;
    d.der[0] = D_W;
    d.dout[0] = h->X[0];
  } else {
    set_final(h, d);
  }
}

const double kRK[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};

int enqueue_step(qg_handle* h) {
  int rc;
  for (int s = 0; s < 3; ++s) {
    RowDesc r{};
    r.prog = h->row_prog;
    r.nin = h->nin;
    r.nout = h->nout;
    r.dx_mask = h->dx_mask;
    r.check_finite = 1;
    for (int i = 0; i < h->nin; ++i) r.in[i] = h->X[i];
    for (int i = 0; i < h->nout; ++i) r.out[i] = h->Y[i];
    if ((rc = run_row(h, r, QG_K_ROW_STAGE))) return rc;

    ColDesc c = col_base(h);
    c.a = kRK[s][0];
    c.b = kRK[s][1];
    c.use_ws = s > 0;
    c.ws = s == 2 ? h->ws2 : h->ws;      // stage 1 state in ws, stage 2 state in ws2
    c.ws_out = s == 0 ? h->ws : h->ws2;
    if (h->dynamic) {
      ColDesc cr = c;
      cr.op = CO_DYN_REDUCE;
      cr.nfwd = 6;
      for (int i = 0; i < 6; ++i) cr.fin[i] = h->Y[i];
      cr.stall_cta1 = h->inject_stall;
      h->inject_stall = 0;
      if ((rc = run_col(h, cr, QG_K_COL_REDUCE))) return rc;
      c.op = CO_DYN_COMBINE;
      c.nfwd = 0;
      c.coeff_out = h->dev_scalars + s;
    } else {
      c.op = CO_STAGE_STATIC;
      c.nfwd = h->nout;
      for (int i = 0; i < h->nout; ++i) c.fin[i] = h->Y[i];
      c.stall_cta1 = h->inject_stall;
      h->inject_stall = 0;
    }
    if (s < 2) {
      c.store_ws = 1;
      set_stage_derived(h, c);
    } else {
      c.viscous = 1;
      set_after_rk(h, c);
    }
    if ((rc = run_col(h, c, (s == 2 && !h->fac_b && !h->fac_s) ? QG_K_COL_FINAL : QG_K_COL_STAGE))) return rc;
  }
  if (h->fac_b) {
    RowDesc r{};
    r.prog = RP_SCALE;
    r.nin = r.nout = 2;
    r.in[0] = h->X[0];
    r.in[1] = h->X[1];
    r.out[0] = h->Y[0];
    r.out[1] = h->Y[1];
    r.factor = h->fac_b;
    r.check_finite = 1;
    if ((rc = run_row(h, r, QG_K_ROW_BRINK))) return rc;
    ColDesc c = col_base(h);
    c.op = CO_CURL;
    c.nfwd = 2;
    c.fin[0] = h->Y[0];
    c.fin[1] = h->Y[1];
    if (h->fac_s) {
      c.nder = 1;
      c.der[0] = D_W;
      c.dout[0] = h->X[0];
    } else {
      set_final(h, c);
    }
    if ((rc = run_col(h, c, h->fac_s ? QG_K_COL_CURL : QG_K_COL_FINAL))) return rc;
  }
  if (h->fac_s) {
    RowDesc r{};
    r.prog = RP_SCALE;
    r.nin = r.nout = 1;
    r.in[0] = h->X[0];
    r.out[0] = h->Y[0];
    r.factor = h->fac_s;
    r.check_finite = 1;
    if ((rc = run_row(h, r, QG_K_ROW_SPONGE))) return rc;
    ColDesc c = col_base(h);
    c.op = CO_FORWARD;
    c.nfwd = 1;
    c.fin[0] = h->Y[0];
    set_final(h, c);
    if ((rc = run_col(h, c, QG_K_COL_FINAL))) return rc;
  }
  h->step += 1;
  h->t += h->par.dt;
  return QG_OK;
}

int enqueue_any_step(qg_handle* h);

// Capture one step on the handle's stream into a graph.  Needs a capturable
// (non-legacy) stream and one eager step first (kernel attributes set).
void try_build_graph(qg_handle* h) {
  h->graph_tried = true;
  if (!h->stream || getenv("QG_NO_GRAPH")) return;
  int32_t saved[QG_NUM_KCLASS];
  memcpy(saved, h->launches, sizeof(saved));
  const int64_t step = h->step;
  const double t = h->t;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const bool hist = h->ab2_hist;
  const int rc = enqueue_any_step(h);
  const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  h->ab2_hist = hist;
  for (int i = 0; i < QG_NUM_KCLASS; ++i) h->graph_launches[i] = h->launches[i] - saved[i];
  memcpy(h->launches, saved, sizeof(saved));
  h->step = step;
  h->t = t;
  if (rc != QG_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) h->step_graph = ex;
  cudaGraphDestroy(g);
  cudaGetLastError();
}

// One step of the paper's scheme (Sec. II-E, Eq. 4):
//   row pass     products of the closure (as an RK stage) [+ chi (u_total, v)]
//   column pass  E = -J + C D + F_obs, w* by Crank-Nicolson / AB2; then either
//                Z = 3/2 w* - 1/2 w** for the sponge or the next state
//   sponge       row pass s = dt rate chi_s Z; column pass w^{t+1} = w* - s
int enqueue_step_ab2(qg_handle* h) {
  int rc;
  RowDesc r{};
  r.prog = h->row_prog;
  r.nin = h->nin;
  r.nout = h->nout;
  r.dx_mask = h->dx_mask;
  r.check_finite = 1;
  for (int i = 0; i < h->nin; ++i) r.in[i] = h->X[i];
  for (int i = 0; i < h->nout; ++i) r.out[i] = h->Y[i];
  if ((rc = run_row(h, r, QG_K_ROW_STAGE))) return rc;
  if (h->fac_b) {  // chi (u_total, v): X[0], X[1] hold the stage's u_total and v
    RowDesc b{};
    b.prog = RP_SCALE;
    b.nin = b.nout = 2;
    b.in[0] = h->X[0];
    b.in[1] = h->X[1];
    b.out[0] = h->Y[6];
    b.out[1] = h->Y[7];
    b.factor = h->fac_b;
    b.check_finite = 1;
    if ((rc = run_row(h, b, QG_K_ROW_BRINK))) return rc;
  }
  ColDesc c = col_base(h);
  c.brink = h->fac_b ? 1 : 0;
  if (h->dynamic) {
    ColDesc cr = c;
    cr.op = CO_DYN_REDUCE;
    cr.nfwd = h->fac_b ? 8 : 6;
    for (int i = 0; i < 6; ++i) cr.fin[i] = h->Y[i];
    cr.fin[6] = h->Y[6];
    cr.fin[7] = h->Y[7];
    if ((rc = run_col(h, cr, QG_K_COL_REDUCE))) return rc;
    c.op = CO_AB2CN_COMBINE;
    c.nfwd = 0;
    c.coeff_out = h->dev_scalars + 2;
  } else {
    c.op = CO_AB2CN;
    c.nst = h->nout;
    c.nfwd = h->nout + (h->fac_b ? 2 : 0);
    for (int i = 0; i < h->nout; ++i) c.fin[i] = h->Y[i];
    if (h->fac_b) {
      c.fin[h->nout] = h->Y[6];
      c.fin[h->nout + 1] = h->Y[7];
    }
  }
  if (h->fac_s) {
    c.sponge_next = 1;
    c.nder = 1;
    c.der[0] = D_W;
    c.dout[0] = h->X[0];
  } else {
    set_final(h, c);
  }
  if ((rc = run_col(h, c, h->fac_s ? QG_K_COL_STAGE : QG_K_COL_FINAL))) return rc;
  if (h->fac_s) {
    RowDesc sp{};
    sp.prog = RP_SCALE;
    sp.nin = sp.nout = 1;
    sp.in[0] = h->X[0];
    sp.out[0] = h->Y[0];
    sp.factor = h->fac_s;
    sp.check_finite = 1;
    if ((rc = run_row(h, sp, QG_K_ROW_SPONGE))) return rc;
    ColDesc f = col_base(h);
    f.op = CO_AB2CN_FINAL;
    f.nfwd = 1;
    f.fin[0] = h->Y[0];
    set_final(h, f);
    if ((rc = run_col(h, f, QG_K_COL_FINAL))) return rc;
  }
  h->ab2_hist = true;
  h->step += 1;
  h->t += h->par.dt;
  return QG_OK;
}

int enqueue_any_step(qg_handle* h) { return h->scheme == QG_SCHEME_AB2CN ? enqueue_step_ab2(h) : enqueue_step(h); }


// ---------------------------------------------------------------------------
// Discrete adjoint of the RK3 step (qg_step_vjp).  The step's forward stages
// are recomputed from w_n with unfused operations (transform passes, the
// adjoint module's pointwise and multiplier kernels), then the transposes run
// in reverse order: final projection, sponge, Brinkman, viscous factor, the
// three Shu-Osher stages.  Each stage's transpose linearises L at that stage's
// state: conjugate multipliers for the spectral operators, pointwise products
// for the nonlinear terms (Eq. 1, 9, 10, 13).
// ---------------------------------------------------------------------------
constexpr int kAdjNS = 25;  // spectral: w0..w3, w5, lam, lam', acc, 11 product spectra, 3 x 2 stage SGS fluxes
constexpr int kAdjNP = 37;  // physical: 6 fields, 3 adjoint fields, 8 products, input, output, 3 x 6 stage fields
constexpr int kAdjNM = 8;   // mixed: the outputs of one derive pass, or one batch of forward transforms
constexpr int kAdjStageP = 19;  // first of the per-stage physical fields (u, v, w_x, w_y, psi_xy, psi_d)
constexpr int kAdjStageS = 19;  // first of the per-stage spectral SGS fluxes F[g w_x], F[g w_y]
// dynamic closures only: per stage the test-level state G w, H and M (spectral), G w's fields (physical),
// scratch spectra, one physical scratch field, and four device scalars <HM>, <MM>, C, kappa per stage
constexpr int kAdjDynS = 25;       // 3 x (G w, H, M)
constexpr int kAdjDynTmpS = 34;    // 5 scratch spectra
constexpr int kAdjNSDyn = 39;
constexpr int kAdjDynP = 37;       // 3 x 6 fields of G w
constexpr int kAdjDynMuP = 55;     // the field mu = M (or G M)
constexpr int kAdjNPDyn = 56;
constexpr int kAdjScalars = 8;     // offset of the per-stage scalars after the dot results

int adj_alloc(qg_handle* h) {
  if (!h->adj_S.empty()) return QG_OK;
  const size_t csz = 2 * h->esz;
  const size_t spec_bytes = (size_t)h->g.Kcp * h->g.SP * csz;
  const size_t mixed_bytes = (size_t)h->g.n * h->g.IP * csz;
  const size_t phys_bytes = (size_t)h->g.n * h->g.n * h->esz;
  const bool dyn = h->cl.kind == QG_DSMAG || h->cl.kind == QG_DLEITH;
  std::vector<void*> S(dyn ? kAdjNSDyn : kAdjNS), P(dyn ? kAdjNPDyn : kAdjNP), M(kAdjNM);
  int rc = QG_OK;
  for (auto& p : S) if (!rc) rc = dalloc(h, &p, spec_bytes);
  for (auto& p : P) if (!rc) rc = dalloc(h, &p, phys_bytes);
  for (auto& p : M) if (!rc) rc = dalloc(h, &p, mixed_bytes);
  void* dots = nullptr;
  // partials | dot results (kAdjScalars) | per-stage scalars (4 x 3) | second partials | counter (zeroed here)
  if (!rc) rc = dalloc(h, &dots, sizeof(double) * (2 * kAdjDotBlocks + kAdjScalars + 12 + 1));
  if (!rc && h->fast) {
    const int BR = fast_box_rows(h->g.n);
    for (void* m : M) if (!rc) rc = add_tensor_map(h, m, h->W, BR);
  }
  if (rc) return rc;
  h->adj_S = S;
  h->adj_P = P;
  h->adj_M = M;
  h->adj_dots = static_cast<double*>(dots);
  return QG_OK;
}

// Side branches.  Work enqueued between adj_fork and adj_unfork runs on the handle's second stream, after
// everything enqueued on the main stream before the fork; adj_unfork returns a join slot, and adj_join(slot) makes
// the main stream wait for that branch.  Branches among themselves run in order on the side stream.  Used for
// launches off the adjoint's critical path (the stages' coefficient derivatives, an accumulation, parts of the
// sponge transpose), so they overlap the main chain of dependent launches.
int adj_fork(qg_handle* h, cudaStream_t* saved) {
  if (!h->adj_side) {
    CK(cudaStreamCreateWithFlags(&h->adj_side, cudaStreamNonBlocking), "adjoint: side stream");
    CK(cudaEventCreateWithFlags(&h->adj_fork_ev, cudaEventDisableTiming), "adjoint: fork event");
    for (cudaEvent_t& ev : h->adj_join_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "adjoint: join");
  }
  CK(cudaEventRecord(h->adj_fork_ev, h->stream), "adjoint: fork");
  CK(cudaStreamWaitEvent(h->adj_side, h->adj_fork_ev, 0), "adjoint: fork wait");
  *saved = h->stream;
  h->stream = h->adj_side;
  return QG_OK;
}

int adj_unfork(qg_handle* h, cudaStream_t saved, int* slot) {
  h->stream = saved;
  if (h->adj_njoin >= 8) return fail(QG_ERR_ARG, "adjoint: too many pending branches");
  *slot = h->adj_njoin++;
  CK(cudaEventRecord(h->adj_join_ev[*slot], h->adj_side), "adjoint: join record");
  return QG_OK;
}

int adj_join(qg_handle* h, int slot) {
  CK(cudaStreamWaitEvent(h->stream, h->adj_join_ev[slot], 0), "adjoint: join");
  return QG_OK;
}

// spectral band (T F[f], mean removed if asked) of a physical field
int adj_to_spec(qg_handle* h, const void* P, void* S, bool zero_mean) {
  RowDesc r{};
  r.pdl = 1;  // the adjoint's chains of small launches overlap their launch latency
  r.prog = RP_COPY;
  r.nin = 1;
  r.nout = 1;
  r.in_phys = 1;
  r.phys_in = P;
  r.out[0] = h->adj_M[0];
  int rc = run_row(h, r, QG_K_ADJ_ROW, false);
  if (rc) return rc;
  ColDesc c = col_base(h);
  c.pdl = 1;
  c.op = CO_FORWARD;
  c.nfwd = 1;
  c.fin[0] = h->adj_M[0];
  c.w0 = S;
  c.store_w0 = 1;
  c.zero_mean = zero_mean ? 1 : 0;
  c.nder = 0;
  return run_col(h, c, QG_K_ADJ_COL, false);
}

// spectral bands of several physical fields (at most kAdjNM): the row passes take them in pairs (one complex FFT
// per pair; the register-resident kernels take every pair in one launch), then one column pass transforms them
// all, each to its own spectral array
int adj_to_spec_many(qg_handle* h, std::initializer_list<const void*> P, std::initializer_list<void*> S) {
  std::vector<const void*> p(P);
  std::vector<void*> s(S);
  const int n = (int)p.size();
  if (n < 1 || n > kAdjNM || (int)s.size() != n) return fail(QG_ERR_ARG, "adjoint: bad transform batch");
  int rc = QG_OK;
  if (h->fast && n > 2) {
    RowDesc r{};
    r.pdl = 1;  // the adjoint's chains of small launches overlap their launch latency
    r.prog = RP_COPY;
    r.nin = 1;
    r.nout = n;
    r.in_phys = 1;
    r.npair = (n + 1) / 2;
    for (int i = 0; i < n; ++i) {
      r.pin[i] = p[i];
      r.out[i] = h->adj_M[i];
    }
    rc = run_row(h, r, QG_K_ADJ_ROW, false);
  } else {
    for (int i = 0; i < n && !rc; i += 2) {
      const bool two = i + 1 < n;
      RowDesc r{};
      r.pdl = 1;
      r.prog = RP_COPY;
      r.nin = 1;
      r.nout = two ? 2 : 1;
      r.in_phys = 1;
      r.phys_in = p[i];
      r.phys_in2 = two ? p[i + 1] : nullptr;
      r.out[0] = h->adj_M[i];
      r.out[1] = two ? h->adj_M[i + 1] : nullptr;
      rc = run_row(h, r, QG_K_ADJ_ROW, false);
    }
  }
  if (rc) return rc;
  ColDesc c = col_base(h);
  c.pdl = 1;
  c.op = CO_FORWARD_N;
  c.nfwd = n;
  for (int i = 0; i < n; ++i) {
    c.fin[i] = h->adj_M[i];
    c.fout[i] = s[i];
  }
  c.nder = 0;
  return run_col(h, c, QG_K_ADJ_COL, false);
}

// physical fields of derived spectra (codes D_W, D_U (with U), D_V, D_WX, D_WY, D_PXY, D_PD) of a spectral
// state: one derive pass, then row passes in pairs
// m0: first of the mixed scratch arrays the passes use (a side branch takes ones the main chain leaves alone)
int adj_to_phys(qg_handle* h, const void* S, std::initializer_list<int> codes, std::initializer_list<void*> P,
                int m0 = 0) {
  ColDesc c = col_base(h);
  c.pdl = 1;
  c.op = CO_DERIVE;
  c.w0 = const_cast<void*>(S);
  c.nder = 0;
  for (int code : codes) {
    c.der[c.nder] = code;
    c.dout[c.nder] = h->adj_M[m0 + c.nder];
    ++c.nder;
  }
  int rc = run_col(h, c, QG_K_ADJ_COL, false);
  std::vector<void*> dst(P);
  if (!rc && h->fast && dst.size() > 2) {
    // every pair in one launch of the register-resident row pass
    RowDesc r{};
    r.pdl = 1;
    r.prog = RP_COPY;
    r.nin = (int)dst.size();
    r.nout = 1;
    r.out_phys = 1;
    r.npair = (int)(dst.size() + 1) / 2;
    for (size_t i = 0; i < dst.size(); ++i) {
      r.in[i] = h->adj_M[m0 + i];
      r.pout[i] = dst[i];
    }
    return run_row(h, r, QG_K_ADJ_ROW, false);
  }
  for (size_t i = 0; i < dst.size() && !rc; i += 2) {
    const bool two = i + 1 < dst.size();
    RowDesc r{};
    r.pdl = 1;  // the adjoint's chains of small launches overlap their launch latency
    r.prog = RP_COPY;
    r.nin = two ? 2 : 1;
    r.nout = 1;
    r.in[0] = h->adj_M[m0 + i];
    r.in[1] = two ? h->adj_M[m0 + i + 1] : nullptr;
    r.out_phys = 1;
    r.phys_out = dst[i];
    r.phys_out2 = two ? dst[i + 1] : nullptr;
    rc = run_row(h, r, QG_K_ADJ_ROW, false);
  }
  return rc;
}

int adj_combine(qg_handle* h, void* out, bool accumulate, bool zero_mean,
                std::initializer_list<AdjTerm> terms) {
  AdjCombine a{};
  a.out = out;
  a.accumulate = accumulate;
  a.zero_mean = zero_mean;
  for (const AdjTerm& t : terms) a.term[a.nterm++] = t;
  a.nu = h->par.nu;
  a.mu = h->par.mu;
  a.dt = h->par.dt;
  a.test_m2max = h->test_m2max;
  Bracket br(h, QG_K_ADJ_PW);
  const cudaError_t e =
      h->fp32 ? launch_adj_combine<float>(h->g, a, h->stream) : launch_adj_combine<double>(h->g, a, h->stream);
  br.done();
  CK(e, "adjoint: combine");
  return QG_OK;
}

int adj_products(qg_handle* h, AdjProducts a) {
  const size_t count = (size_t)h->g.n * h->g.n;
  Bracket br(h, QG_K_ADJ_PW);
  const cudaError_t e =
      h->fp32 ? launch_adj_products<float>(count, a, h->stream) : launch_adj_products<double>(count, a, h->stream);
  br.done();
  CK(e, "adjoint: products");
  return QG_OK;
}

int adj_scale(qg_handle* h, const void* f, const void* x0, double s0, void* out0, const void* x1, double s1,
              void* out1) {
  const size_t count = (size_t)h->g.n * h->g.n;
  Bracket br(h, QG_K_ADJ_PW);
  const cudaError_t e = h->fp32 ? launch_adj_scale<float>(count, f, x0, s0, out0, x1, s1, out1, h->stream)
                                : launch_adj_scale<double>(count, f, x0, s0, out0, x1, s1, out1, h->stream);
  br.done();
  CK(e, "adjoint: scale");
  return QG_OK;
}

// the physical fields u_total, v, w_x, w_y (and psi_xy, psi_d for Smagorinsky) of a stage state, kept per stage
// for the reverse sweep (first of six arrays at P[f0])
int adj_stage_fields(qg_handle* h, const void* Sw, int kind, int f0) {
  auto& P = h->adj_P;
  if (kind == AK_SMAG)
    return adj_to_phys(h, Sw, {D_U, D_V, D_WX, D_WY, D_PXY, D_PD},
                       {P[f0], P[f0 + 1], P[f0 + 2], P[f0 + 3], P[f0 + 4], P[f0 + 5]});
  return adj_to_phys(h, Sw, {D_U, D_V, D_WX, D_WY}, {P[f0], P[f0 + 1], P[f0 + 2], P[f0 + 3]});
}

AdjProducts adj_prod_desc(qg_handle* h, int kind, int mode, int f0, int lam = 6) {
  auto& P = h->adj_P;
  AdjProducts a{};
  a.kind = kind;
  a.mode = mode;
  a.u = P[f0];
  a.v = P[f0 + 1];
  a.wx = P[f0 + 2];
  a.wy = P[f0 + 3];
  a.pxy = P[f0 + 4];
  a.pd = P[f0 + 5];
  a.lam = P[lam];
  a.lx = P[7];
  a.ly = P[8];
  for (int k = 0; k < 8; ++k) a.out[k] = P[9 + k];
  return a;
}

// L(w) = -J - beta psi_x + C div(g grad w) of stage s's state Sw into spectral Sout scaled as
// Sout = a w0 + b (ws + dt L(ws)) (Shu-Osher stage); keeps the stage's fields and SGS flux spectra
// device scalars of stage s of a dynamic closure: <HM>, <MM>, C, kappa
double* adj_scalar(qg_handle* h, int s, int k) { return h->adj_dots + kAdjDotBlocks + kAdjScalars + 4 * s + k; }

// the partials and the counter of the one-launch dots (dots never run concurrently: those on the side branch are
// joined before the main chain's next dot)
AdjDotOut adj_dot_out(qg_handle* h, double scale, double* out) {
  AdjDotOut o{};
  o.partials = h->adj_dots;
  o.partials2 = h->adj_dots + kAdjDotBlocks + kAdjScalars + 12;
  o.counter = reinterpret_cast<unsigned*>(o.partials2 + kAdjDotBlocks);
  o.scale = scale;
  o.out = out;
  return o;
}

// Fused forms of the register-resident kernels.  Forward: the stage fields of Sw (one derive pass), one row pass
// that keeps them as physical fields P[f0..] and forms J, g w_x, g w_y in registers, one column pass to the
// spectral arrays o0 [, o1, o2].  Reverse: lam = D_W of Sl and the derivatives D_WX, D_WY of Sd (derive passes),
// one row pass of the transposed products against the fields at P[f0..], one column pass to S[8..].
int adj_fused_fwd(qg_handle* h, int kind, const void* Sw, int f0, void* o0, void* o1, void* o2) {
  auto& P = h->adj_P;
  auto& M = h->adj_M;
  static const int codes[6] = {D_U, D_V, D_WX, D_WY, D_PXY, D_PD};
  const int nf = kind == AK_SMAG ? 6 : 4;
  const int no = kind == AK_NONE ? 1 : 3;
  ColDesc c = col_base(h);
  c.pdl = 1;
  c.op = CO_DERIVE;
  c.w0 = const_cast<void*>(Sw);
  c.nder = nf;
  for (int i = 0; i < nf; ++i) {
    c.der[i] = codes[i];
    c.dout[i] = M[i];
  }
  int rc = run_col(h, c, QG_K_ADJ_COL, false);
  if (rc) return rc;
  RowDesc r{};
  r.pdl = 1;
  r.prog = RP_ADJ_FWD;
  r.adj_kind = kind;
  r.nin = nf;
  r.nout = no;
  for (int i = 0; i < nf; ++i) {
    r.in[i] = M[i];
    r.pf[i] = P[f0 + i];
  }
  for (int i = 0; i < no; ++i) r.out[i] = M[i];  // each row is read in full before it is written
  rc = run_row(h, r, QG_K_ADJ_ROW, false);
  if (rc) return rc;
  ColDesc f = col_base(h);
  f.pdl = 1;
  f.op = CO_FORWARD_N;
  f.nfwd = no;
  void* outs[3] = {o0, o1, o2};
  for (int i = 0; i < no; ++i) {
    f.fin[i] = M[i];
    f.fout[i] = outs[i];
  }
  return run_col(h, f, QG_K_ADJ_COL, false);
}

int adj_derive(qg_handle* h, const void* S, std::initializer_list<int> codes, int m0) {
  ColDesc c = col_base(h);
  c.pdl = 1;
  c.op = CO_DERIVE;
  c.w0 = const_cast<void*>(S);
  c.nder = 0;
  for (int code : codes) {
    c.der[c.nder] = code;
    c.dout[c.nder] = h->adj_M[m0 + c.nder];
    ++c.nder;
  }
  return run_col(h, c, QG_K_ADJ_COL, false);
}

// the exact Brinkman factor applied in one row pass to the pair adj_M[0], adj_M[1] (in place)
int adj_brinkman_row(qg_handle* h) {
  RowDesc r{};
  r.pdl = 1;
  r.prog = RP_SCALE;
  r.nin = r.nout = 2;
  r.in[0] = h->adj_M[0];
  r.in[1] = h->adj_M[1];
  r.out[0] = h->adj_M[0];  // each row is read in full before it is written
  r.out[1] = h->adj_M[1];
  r.factor = h->fac_b;
  return run_row(h, r, QG_K_ADJ_ROW, false);
}

// the row and column passes of the fused reverse products once adj_M[0..2] hold lam, lam_x, lam_y
int adj_fused_rev_tail(qg_handle* h, int kind, int f0) {
  auto& P = h->adj_P;
  auto& M = h->adj_M;
  auto& S = h->adj_S;
  const int no = kind == AK_SMAG ? 8 : kind == AK_LEITH ? 6 : 4;
  RowDesc r{};
  r.pdl = 1;
  r.prog = RP_ADJ_REV;
  r.adj_kind = kind;
  r.nin = 3;
  r.nout = no;
  for (int i = 0; i < 3; ++i) r.in[i] = M[i];
  for (int i = 0; i < 6; ++i) r.pf[i] = P[f0 + i];
  for (int i = 0; i < no; ++i) r.out[i] = M[i];  // lam, lam_x, lam_y of a row are read before any output row
  int rc = run_row(h, r, QG_K_ADJ_ROW, false);
  if (rc) return rc;
  ColDesc f = col_base(h);
  f.pdl = 1;
  f.op = CO_FORWARD_N;
  f.nfwd = no;
  for (int i = 0; i < no; ++i) {
    f.fin[i] = M[i];
    f.fout[i] = S[8 + i];
  }
  return run_col(h, f, QG_K_ADJ_COL, false);
}

// The dynamic coefficient of stage s (Eq. 11, 12, 14; R8) from its state Sw, recomputed with the stage:
// G w, its fields, H = J(G w) - G J(w), M = r^p D(G w) - G D(w), <HM>, <MM>, C = max(0, <HM>/<MM>).
// SJ holds J(w); the stage's SGS flux spectra hold F[g w_x], F[g w_y].
int adj_forward_germano(qg_handle* h, int kind, const void* Sw, const void* SJ, int s) {
  auto& S = h->adj_S;
  auto& P = h->adj_P;
  void* Swt = S[kAdjDynS + 3 * s];
  void* SH = S[kAdjDynS + 3 * s + 1];
  void* SM = S[kAdjDynS + 3 * s + 2];
  const void* Sgx = S[kAdjStageS + 2 * s];
  const void* Sgy = S[kAdjStageS + 2 * s + 1];
  void* T0 = S[kAdjDynTmpS];
  void* T1 = S[kAdjDynTmpS + 1];
  void* T2 = S[kAdjDynTmpS + 2];
  const int f0 = kAdjDynP + 6 * s;
  const double rp = std::pow(h->cl.test_ratio, kind == AK_SMAG ? 2 : 3);
  const double n4 = std::pow(double(h->g.n), 4);
  int rc = adj_combine(h, Swt, false, false, {{Sw, AM_ONE | AM_TESTF, 1.0}});
  if (h->fast) {
    if (!rc) rc = adj_fused_fwd(h, kind, Swt, f0, T0, T1, T2);
  } else {
    if (!rc) rc = adj_stage_fields(h, Swt, kind, f0);
    if (!rc) rc = adj_products(h, adj_prod_desc(h, kind, AP_FORWARD, f0));
    if (!rc) rc = adj_to_spec_many(h, {P[9], P[10], P[11]}, {T0, T1, T2});
  }
  if (!rc) rc = adj_combine(h, SH, false, false, {{T0, AM_ONE, 1.0}, {SJ, AM_ONE | AM_TESTF, -1.0}});
  if (!rc)
    rc = adj_combine(h, SM, false, false,
                     {{T1, AM_IX, rp}, {T2, AM_IY, rp}, {Sgx, AM_IX | AM_TESTF, -1.0}, {Sgy, AM_IY | AM_TESTF, -1.0}});
  if (rc) return rc;
  // <HM>, <MM> and C = max(0, <HM> / <MM>) to scalars 0, 1, 2 of stage s
  AdjDotOut o = adj_dot_out(h, 1.0 / n4, adj_scalar(h, s, 0));
  Bracket br(h, QG_K_ADJ_PW);
  const cudaError_t e = h->fp32 ? launch_adj_germano_dots<float>(h->g, SH, SM, o, h->stream)
                                : launch_adj_germano_dots<double>(h->g, SH, SM, o, h->stream);
  br.done();
  CK(e, "adjoint: Germano sums");
  return QG_OK;
}

int adj_forward_stage(qg_handle* h, int kind, bool dyn, double C, const void* S0, const void* Sw, void* Sout,
                      double a, double b, int s) {
  auto& S = h->adj_S;
  auto& P = h->adj_P;
  const double dt = h->par.dt;
  const int f0 = kAdjStageP + 6 * s;
  void* Sgx = S[kAdjStageS + 2 * s];
  void* Sgy = S[kAdjStageS + 2 * s + 1];
  int rc = QG_OK;
  if (h->fast) {
    rc = adj_fused_fwd(h, kind, Sw, f0, S[8], Sgx, Sgy);
  } else {
    rc = adj_stage_fields(h, Sw, kind, f0);
    if (!rc) rc = adj_products(h, adj_prod_desc(h, kind, AP_FORWARD, f0));
    if (!rc) rc = kind == AK_NONE ? adj_to_spec_many(h, {P[9]}, {S[8]})
                                   : adj_to_spec_many(h, {P[9], P[10], P[11]}, {S[8], Sgx, Sgy});
  }
  if (!rc && dyn) rc = adj_forward_germano(h, kind, Sw, S[8], s);
  if (rc) return rc;
  if (kind == AK_NONE)
    return adj_combine(h, Sout, false, false,
                       {{S0, AM_ONE, a}, {Sw, AM_ONE, b}, {S[8], AM_ONE, -b * dt}, {Sw, AM_CV, b * dt * h->beta}});
  const double* cp = dyn ? adj_scalar(h, s, 2) : nullptr;
  return adj_combine(h, Sout, false, false,
                     {{S0, AM_ONE, a}, {Sw, AM_ONE, b}, {S[8], AM_ONE, -b * dt}, {Sw, AM_CV, b * dt * h->beta},
                      {Sgx, AM_IX, b * dt * (dyn ? 1.0 : C), cp}, {Sgy, AM_IY, b * dt * (dyn ? 1.0 : C), cp}});
}

// The dynamic coefficient's share of stage s's transpose, kappa grad C (Eq. 12, 14) with kappa =
// C_bar / (N^2 <MM>), accumulated into Slam_out:
//   kappa [G J'(G w)^T M - J'(w)^T G M + r^p G D'(G w)^T nu - D'(w)^T G nu],  nu = H - 2 C M
int adj_reverse_germano(qg_handle* h, int kind, void* Slam_out, int s) {
  auto& S = h->adj_S;
  auto& P = h->adj_P;
  const void* SH = S[kAdjDynS + 3 * s + 1];
  const void* SM = S[kAdjDynS + 3 * s + 2];
  void* Snu = S[kAdjDynTmpS + 3];
  void* Sg = S[kAdjDynTmpS + 4];
  const double* C = adj_scalar(h, s, 2);
  double* kappa = adj_scalar(h, s, 3);  // set by the stage's C-derivative dot (adj_reverse_stage)
  const double rp = std::pow(h->cl.test_ratio, kind == AK_SMAG ? 2 : 3);
  const int mu = kAdjDynMuP;
  int rc = adj_combine(h, Snu, false, false, {{SH, AM_ONE, 1.0}, {SM, AM_ONE, -2.0, C}});
  // outer group, at the test-level state, filtered afterwards: mu = M, derivatives of nu
  if (h->fast) {
    if (!rc) rc = adj_derive(h, SM, {D_W}, 0);
    if (!rc) rc = adj_derive(h, Snu, {D_WX, D_WY}, 1);
  } else {
    if (!rc) rc = adj_to_phys(h, SM, {D_W}, {P[mu]});
    if (!rc) rc = adj_to_phys(h, Snu, {D_WX, D_WY}, {P[7], P[8]});
    if (!rc) rc = adj_products(h, adj_prod_desc(h, kind, AP_ADJOINT, kAdjDynP + 6 * s, mu));
  }
  for (int pass = 0; pass < 2 && !rc; ++pass) {
    if (pass == 1) {
      // inner group, at the stage state: mu = G M, derivatives of G nu
      rc = adj_combine(h, Sg, false, false, {{SM, AM_ONE | AM_TESTF, 1.0}});
      if (h->fast) {
        if (!rc) rc = adj_derive(h, Sg, {D_W}, 0);
      } else {
        if (!rc) rc = adj_to_phys(h, Sg, {D_W}, {P[mu]});
      }
      if (!rc) rc = adj_combine(h, Sg, false, false, {{Snu, AM_ONE | AM_TESTF, 1.0}});
      if (h->fast) {
        if (!rc) rc = adj_derive(h, Sg, {D_WX, D_WY}, 1);
      } else {
        if (!rc) rc = adj_to_phys(h, Sg, {D_WX, D_WY}, {P[7], P[8]});
        if (!rc) rc = adj_products(h, adj_prod_desc(h, kind, AP_ADJOINT, kAdjStageP + 6 * s, mu));
      }
    }
    if (!rc && h->fast)
      rc = adj_fused_rev_tail(h, kind, pass == 0 ? kAdjDynP + 6 * s : kAdjStageP + 6 * s);
    else if (!rc && kind == AK_SMAG)
      rc = adj_to_spec_many(h, {P[9], P[10], P[11], P[12], P[13], P[14], P[15], P[16]},
                            {S[8], S[9], S[10], S[11], S[12], S[13], S[14], S[15]});
    else if (!rc)
      rc = adj_to_spec_many(h, {P[9], P[10], P[11], P[12], P[13], P[14]}, {S[8], S[9], S[10], S[11], S[12], S[13]});
    if (rc) return rc;
    const int f = pass == 0 ? AM_TESTF : 0;
    const double sj = pass == 0 ? 1.0 : -1.0, sd = pass == 0 ? rp : -1.0;
    AdjCombine a{};
    a.out = Slam_out;
    a.accumulate = 1;
    a.test_m2max = h->test_m2max;
    auto add = [&](const void* in, int code, double coef) { a.term[a.nterm++] = AdjTerm{in, code | f, coef, kappa}; };
    add(S[8], AM_CU, sj);
    add(S[9], AM_CV, sj);
    add(S[10], AM_CX, sj);
    add(S[11], AM_CY, sj);
    add(S[12], AM_CX, sd);
    add(S[13], AM_CY, sd);
    if (kind == AK_SMAG) {
      add(S[14], AM_XY, sd);
      add(S[15], AM_DD, sd);
    }
    Bracket br(h, QG_K_ADJ_PW);
    const cudaError_t e =
        h->fp32 ? launch_adj_combine<float>(h->g, a, h->stream) : launch_adj_combine<double>(h->g, a, h->stream);
    br.done();
    CK(e, "adjoint: coefficient gradient");
  }
  return rc;
}

// Slam_out = b lam + L'(ws)^T (b dt lam) (one Shu-Osher stage in reverse); the derivative in C,
// b dt sum(lam * div(g grad ws)), goes to adj_dots[slot]
int adj_reverse_stage(qg_handle* h, int kind, bool dyn, double C, const void* Slam, void* Slam_out, double b,
                      int slot) {
  auto& S = h->adj_S;
  auto& P = h->adj_P;
  const double dt = h->par.dt, bd = b * dt;
  const int f0 = kAdjStageP + 6 * slot;  // the stage's fields, kept by the forward recomputation
  int rc = QG_OK;
  int cslot = -1;
  if (kind != AK_NONE) {
    // derivative in C, on a side branch: sum over points of lam * T div(g grad ws) (Parseval over the band)
    cudaStream_t main_st;
    rc = adj_fork(h, &main_st);
    if (!rc)
      rc = adj_combine(h, S[18], false, false,
                       {{S[kAdjStageS + 2 * slot], AM_IX, 1.0}, {S[kAdjStageS + 2 * slot + 1], AM_IY, 1.0}});
    if (!rc) {
      const double n2 = double(h->g.n) * double(h->g.n);
      AdjDotOut o = adj_dot_out(h, bd / n2, h->adj_dots + kAdjDotBlocks + slot);
      if (dyn) {
        // kappa = C_bar / (N^2 <MM>) for the dynamic coefficient's share of this stage's transpose
        o.C = adj_scalar(h, slot, 2);
        o.mm = adj_scalar(h, slot, 1);
        o.kappa = adj_scalar(h, slot, 3);
        o.n2 = n2;
      }
      Bracket br(h, QG_K_ADJ_PW);
      const cudaError_t e = h->fp32 ? launch_adj_spec_dot<float>(h->g, Slam, S[18], o, h->stream)
                                    : launch_adj_spec_dot<double>(h->g, Slam, S[18], o, h->stream);
      br.done();
      if (e != cudaSuccess) rc = cuda_fail(e, "adjoint: C derivative");
    }
    const int urc = adj_unfork(h, main_st, &cslot);
    if (rc) return rc;
    if (urc) return urc;
  }
  if (h->fast) {
    rc = adj_derive(h, Slam, {D_W, D_WX, D_WY}, 0);
    if (!rc) rc = adj_fused_rev_tail(h, kind, f0);
  } else {
    rc = adj_to_phys(h, Slam, {D_W, D_WX, D_WY}, {P[6], P[7], P[8]});
    if (!rc) rc = adj_products(h, adj_prod_desc(h, kind, AP_ADJOINT, f0));
  }
  if (!rc && h->fast) {
    // the fused passes wrote S[8..]
  } else if (!rc && kind == AK_SMAG)
    rc = adj_to_spec_many(h, {P[9], P[10], P[11], P[12], P[13], P[14], P[15], P[16]},
                          {S[8], S[9], S[10], S[11], S[12], S[13], S[14], S[15]});
  else if (!rc && kind != AK_NONE)
    rc = adj_to_spec_many(h, {P[9], P[10], P[11], P[12], P[13], P[14]}, {S[8], S[9], S[10], S[11], S[12], S[13]});
  else if (!rc)
    rc = adj_to_spec_many(h, {P[9], P[10], P[11], P[12]}, {S[8], S[9], S[10], S[11]});
  if (rc) return rc;
  AdjCombine a{};
  a.out = Slam_out;
  a.nu = h->par.nu;
  a.mu = h->par.mu;
  a.dt = dt;
  auto add = [&](const void* in, int code, double coef) { a.term[a.nterm++] = AdjTerm{in, code, coef}; };
  add(Slam, AM_ONE, b);
  // -J: each factor's transpose takes the other factor
  add(S[8], AM_CU, -bd);
  add(S[9], AM_CV, -bd);
  add(S[10], AM_CX, -bd);
  add(S[11], AM_CY, -bd);
  // -beta psi_x = (i beta k_x / |k|^2) w: transpose -i beta k_x / |k|^2
  add(Slam, AM_CV, -bd * h->beta);
  if (kind != AK_NONE) {
    const double* cp = dyn ? adj_scalar(h, slot, 2) : nullptr;
    const double cc = dyn ? bd : bd * C;
    a.term[a.nterm++] = AdjTerm{S[12], AM_CX, cc, cp};
    a.term[a.nterm++] = AdjTerm{S[13], AM_CY, cc, cp};
    if (kind == AK_SMAG) {
      a.term[a.nterm++] = AdjTerm{S[14], AM_XY, cc, cp};
      a.term[a.nterm++] = AdjTerm{S[15], AM_DD, cc, cp};
    }
  }
  {
    Bracket br(h, QG_K_ADJ_PW);
    const cudaError_t e =
        h->fp32 ? launch_adj_combine<float>(h->g, a, h->stream) : launch_adj_combine<double>(h->g, a, h->stream);
    br.done();
    CK(e, "adjoint: stage combine");
  }
  if (kind != AK_NONE) {
    if (cslot >= 0) {
      rc = adj_join(h, cslot);
      if (rc) return rc;
    }
    if (dyn) return adj_reverse_germano(h, kind, Slam_out, slot);
  }
  return QG_OK;
}

// in: physical w_n and lam_{n+1} in the working precision (P[17], P[18]); out: lam_n in P[18];
// adj_dots[kAdjDotBlocks + 0..2] = the stages' C derivatives, [+3] = the sponge-rate derivative
int adj_step(qg_handle* h) {
  auto& S = h->adj_S;
  auto& P = h->adj_P;
  const int kind = (h->cl.kind == QG_SMAG || h->cl.kind == QG_DSMAG)     ? AK_SMAG
                   : (h->cl.kind == QG_LEITH || h->cl.kind == QG_DLEITH) ? AK_LEITH
                                                                         : AK_NONE;
  const bool dyn = h->cl.kind == QG_DSMAG || h->cl.kind == QG_DLEITH;
  const double C = kind == AK_NONE || dyn ? 0.0 : h->static_coeff;
  const double dt = h->par.dt;
  double* dots = h->adj_dots + kAdjDotBlocks;
  h->adj_njoin = 0;
  CK(cudaMemsetAsync(dots, 0, (kAdjScalars + 12) * sizeof(double), h->stream), "adjoint: dots");
  static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, B[3] = {1.0, 0.25, 2.0 / 3.0};
  // forward: w0 -> w1 -> w2 -> w3 (S[0..3]), viscous factor, Brinkman -> S[4]
  int rc = adj_to_spec(h, P[17], S[0], true);
  for (int s = 0; s < 3 && !rc; ++s)
    rc = adj_forward_stage(h, kind, dyn, C, S[0], S[s], S[s + 1], A[s], B[s], s);
  if (!rc) rc = adj_combine(h, S[3], false, false, {{S[3], AM_VISC, 1.0}});
  if (rc) return rc;
  if (h->fac_b && h->fast) {
    // the forward step's own Brinkman passes: (u_total, v) derived, scaled by the exact factor in one row pass,
    // curl taken in the column pass that transforms them
    rc = adj_derive(h, S[3], {D_U, D_V}, 0);
    if (!rc) rc = adj_brinkman_row(h);
    if (!rc) {
      ColDesc c = col_base(h);
      c.pdl = 1;
      c.op = CO_CURL;
      c.nfwd = 2;
      c.fin[0] = h->adj_M[0];
      c.fin[1] = h->adj_M[1];
      c.w0 = S[4];
      c.store_w0 = 1;
      c.nder = 0;
      rc = run_col(h, c, QG_K_ADJ_COL, false);
    }
  } else if (h->fac_b) {
    rc = adj_to_phys(h, S[3], {D_U, D_V}, {P[0], P[1]});
    if (!rc) rc = adj_scale(h, h->fac_b, P[0], 1.0, P[9], P[1], 1.0, P[10]);  // chi-factor times (u_total, v)
    if (!rc) rc = adj_to_spec_many(h, {P[9], P[10]}, {S[8], S[9]});
    if (!rc) rc = adj_combine(h, S[4], false, false, {{S[9], AM_IX, 1.0}, {S[8], AM_IY, -1.0}});
  } else {
    rc = adj_combine(h, S[4], false, false, {{S[3], AM_ONE, 1.0}});
  }
  if (rc) return rc;

  // reverse: final projection (2/3 band, zero mean)
  void* lam = S[5];
  void* lam2 = S[6];
  // the sponge's forward field w5 in physical space (a side branch, beside the final projection's transpose)
  int w5slot = -1;
  if (h->fac_s) {
    cudaStream_t main_st;
    rc = adj_fork(h, &main_st);
    if (!rc) rc = adj_to_phys(h, S[4], {D_W}, {P[0]}, kAdjNM - 1);  // the last mixed array: the main chain's
                                                                     // transforms here use the first ones
    const int urc = adj_unfork(h, main_st, &w5slot);
    if (rc) return rc;
    if (urc) return urc;
  }
  rc = adj_to_spec(h, P[18], lam, true);
  int dotslot = -1;
  if (!rc && h->fac_s) {
    // w6 = T F[s w5]: d/drate = sum lam * (-chi_s dt s) * w5; lam <- T F[s lam]
    rc = adj_to_phys(h, lam, {D_W}, {P[6]});
    if (!rc) rc = adj_join(h, w5slot);
    if (!rc) rc = adj_scale(h, h->fac_s, P[0], 1.0, P[1], P[6], 1.0, P[2]);
    if (rc) return rc;
    if (h->chi_s) {
      // the sponge-rate derivative on a side branch (P[6] and P[1] are not written again in this step)
      cudaStream_t main_st;
      rc = adj_fork(h, &main_st);
      if (!rc) {
        Bracket br(h, QG_K_ADJ_PW);
        const AdjDotOut o = adj_dot_out(h, -dt, dots + 3);
        const cudaError_t e =
            h->fp32 ? launch_adj_phys_dot<float>((size_t)h->g.n * h->g.n, P[6], h->chi_s, P[1], o, h->stream)
                    : launch_adj_phys_dot<double>((size_t)h->g.n * h->g.n, P[6], h->chi_s, P[1], o, h->stream);
        br.done();
        if (e != cudaSuccess) rc = cuda_fail(e, "adjoint: sponge-rate derivative");
      }
      const int urc = adj_unfork(h, main_st, &dotslot);
      if (rc) return rc;
      if (urc) return urc;
    }
    rc = adj_to_spec(h, P[2], lam, false);
  }
  if (!rc && h->fac_b && h->fast) {
    // w5 = T (d_x (f v) - d_y (f u)): lam <- -conj(dv) F[f lam_x] + conj(du) F[f lam_y], the scaling in one row pass
    rc = adj_derive(h, lam, {D_WX, D_WY}, 0);
    if (!rc) rc = adj_brinkman_row(h);
    if (!rc) {
      ColDesc c = col_base(h);
      c.pdl = 1;
      c.op = CO_FORWARD_N;
      c.nfwd = 2;
      c.fin[0] = h->adj_M[0];
      c.fin[1] = h->adj_M[1];
      c.fout[0] = S[8];
      c.fout[1] = S[9];
      c.nder = 0;
      rc = run_col(h, c, QG_K_ADJ_COL, false);
    }
    if (!rc) rc = adj_combine(h, lam, false, false, {{S[8], AM_CV, -1.0}, {S[9], AM_CU, 1.0}});
  } else if (!rc && h->fac_b) {
    // w5 = T (d_x (f v) - d_y (f u)): lam <- conj(dv) F[f (-lam_x)] - conj(du) F[f (-lam_y)]
    rc = adj_to_phys(h, lam, {D_WX, D_WY}, {P[7], P[8]});
    if (!rc) rc = adj_scale(h, h->fac_b, P[7], -1.0, P[9], P[8], -1.0, P[10]);
    if (!rc) rc = adj_to_spec_many(h, {P[9], P[10]}, {S[8], S[9]});
    if (!rc) rc = adj_combine(h, lam, false, false, {{S[8], AM_CV, 1.0}, {S[9], AM_CU, -1.0}});
  }
  if (!rc) rc = adj_combine(h, lam, false, false, {{lam, AM_VISC, 1.0}});
  // the sponge-rate branch reads P[6], which the generic kernels' reverse stages overwrite
  if (!rc && dotslot >= 0) rc = adj_join(h, dotslot);
  dotslot = -1;
  // the three stages in reverse: w_{s+1} = a_s w0 + b_s (w_s + dt L(w_s)); the a_s lam share of w0's gradient
  // accumulates in S[7] on a side branch, joined before the next stage overwrites that lam
  bool s7_set = false;
  for (int s = 2; s >= 0 && !rc; --s) {
    int accslot = -1;
    if (A[s] != 0.0) {
      cudaStream_t main_st;
      rc = adj_fork(h, &main_st);
      if (!rc) rc = adj_combine(h, S[7], s7_set, false, {{lam, AM_ONE, A[s]}});
      const int urc = adj_unfork(h, main_st, &accslot);
      if (!rc) rc = urc;
      s7_set = true;
    }
    if (!rc) rc = adj_reverse_stage(h, kind, dyn, C, lam, lam2, B[s], s);
    if (!rc && accslot >= 0) rc = adj_join(h, accslot);
    std::swap(lam, lam2);
  }
  if (!rc) rc = adj_combine(h, S[7], s7_set, true, {{lam, AM_ONE, 1.0}});
  if (!rc) rc = adj_to_phys(h, S[7], {D_W}, {P[18]});
  if (!rc && dotslot >= 0) rc = adj_join(h, dotslot);
  return rc;
}

// Capture one adjoint step (fixed workspace, so every call replays the same graph).
void adj_build_graph(qg_handle* h) {
  h->adj_graph_tried = true;
  if (!h->stream || getenv("QG_NO_GRAPH")) return;
  if (h->adj_side) cudaStreamSynchronize(h->adj_side);  // the eager step's branches are done before capture
  int32_t saved[QG_NUM_KCLASS];
  memcpy(saved, h->launches, sizeof(saved));
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int rc = adj_step(h);
  const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  for (int i = 0; i < QG_NUM_KCLASS; ++i) h->adj_graph_launches[i] = h->launches[i] - saved[i];
  memcpy(h->launches, saved, sizeof(saved));
  if (rc != QG_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) h->adj_graph = ex;
  cudaGraphDestroy(g);
  cudaGetLastError();
}

// physical field of the state into h->phys (working precision)
int state_to_phys(qg_handle* h) {
  ColDesc c = col_base(h);
  c.op = CO_DERIVE;
  c.nder = 1;
  c.der[0] = D_W;
  c.dout[0] = h->Y[0];
  int rc = run_col(h, c, QG_K_OTHER, false);
  if (rc) return rc;
  RowDesc r{};
  r.prog = RP_COPY;
  r.nin = 1;
  r.nout = 1;
  r.in[0] = h->Y[0];
  r.out_phys = 1;
  r.phys_out = h->phys;
  return run_row(h, r, QG_K_OTHER, false);
}

}  // namespace


// ---------------------------------------------------------------------------
// Ensembles of independent members (different grids, closures, parameters).
// Each member is a full handle on a stream of its own.  A step of the
// ensemble is one CUDA graph in which the members' steps are parallel
// branches between a fork and a join on the ensemble's stream, so the GPU
// runs the members' kernels side by side: a single 256^2 - 768^2 member
// leaves most of the 152 SMs idle between its launches.
// ---------------------------------------------------------------------------
struct qg_ensemble {
  std::vector<qg_handle*> h;
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> ev;  // per member: tail of its stream before a step, its branch's end inside one
  std::vector<std::array<int32_t, QG_NUM_KCLASS>> graph_launches;
  cudaStream_t main = nullptr;
  bool own_main = false;
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  int64_t eager_steps = 0;
  // launch form of an ensemble step (chosen by the tuner at creation): members run in `lanes` chains (0: one
  // per member, all side by side), filled longest-first by estimated cost; programmatic dependent launch on or
  // off; the FP32 Germano reduction's lean form (ColDesc::lean).  None of them changes a member's arithmetic.
  int lanes = 0, pdl = 0, lean = 0;
  int tuned = 0;          // 0 default or forced by the environment, 1 timed at creation, 2 from the cache
  double tuned_ms = 0.0;  // the chosen form's time per ensemble step when timed
  std::vector<double> cost;  // estimated work per member step
  std::vector<int> order;    // members by decreasing cost
  ~qg_ensemble() {
    if (main) cudaStreamSynchronize(main);
    if (exec) cudaGraphExecDestroy(exec);
    for (qg_handle* x : h) qg_destroy(x);
    for (cudaStream_t s : st) cudaStreamDestroy(s);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (done) cudaEventDestroy(done);
    if (own_main && main) cudaStreamDestroy(main);
  }
};

namespace {

// fork on the ensemble stream, one step of every member on its stream, join.  Members are dealt to the lanes
// longest-first, each to the lane with the least work so far; a member waits for the one before it in its lane.
int ens_enqueue(qg_ensemble* e) {
  CK(cudaEventRecord(e->fork, e->main), "ensemble: fork");
  const int m = (int)e->h.size();
  const int nl = e->lanes > 0 && e->lanes < m ? e->lanes : m;
  std::vector<int> tail(nl, -1);
  std::vector<double> load(nl, 0.0);
  for (int k = 0; k < m; ++k) {
    const int i = e->order.empty() ? k : e->order[k];
    int l = 0;
    for (int j = 1; j < nl; ++j)
      if (load[j] < load[l]) l = j;
    load[l] += e->cost.empty() ? 1.0 : e->cost[i];
    CK(cudaStreamWaitEvent(e->st[i], tail[l] < 0 ? e->fork : e->ev[tail[l]], 0), "ensemble: fork wait");
    const int rc = enqueue_any_step(e->h[i]);
    if (rc) return rc;
    CK(cudaEventRecord(e->ev[i], e->st[i]), "ensemble: join");
    tail[l] = i;
  }
  for (int l = 0; l < nl; ++l)
    if (tail[l] >= 0) CK(cudaStreamWaitEvent(e->main, e->ev[tail[l]], 0), "ensemble: join wait");
  return QG_OK;
}

void ens_build_graph(qg_ensemble* e) {
  e->graph_tried = true;
  if (getenv("QG_NO_GRAPH")) return;
  const size_t m = e->h.size();
  std::vector<std::array<int32_t, QG_NUM_KCLASS>> saved(m);
  std::vector<int64_t> step(m);
  std::vector<double> t(m);
  std::vector<char> hist(m);
  for (size_t i = 0; i < m; ++i) {
    memcpy(saved[i].data(), e->h[i]->launches, sizeof(e->h[i]->launches));
    step[i] = e->h[i]->step;
    t[i] = e->h[i]->t;
    hist[i] = e->h[i]->ab2_hist;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(e->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int rc = ens_enqueue(e);
  const cudaError_t err = cudaStreamEndCapture(e->main, &g);
  e->graph_launches.assign(m, {});
  for (size_t i = 0; i < m; ++i) {
    qg_handle* x = e->h[i];
    for (int c = 0; c < QG_NUM_KCLASS; ++c) e->graph_launches[i][c] = x->launches[c] - saved[i][c];
    memcpy(x->launches, saved[i].data(), sizeof(x->launches));
    x->step = step[i];
    x->t = t[i];
    x->ab2_hist = hist[i];
  }
  if (rc != QG_OK || err != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) e->exec = ex;
  cudaGraphDestroy(g);
  cudaGetLastError();
}

// ---- the ensemble's tuner: the launch form of an ensemble step is chosen once per signature (the members'
// grids, precisions, closures, schemes and forcings, in order, on one device) by timing replays of each
// candidate's graph, and cached for later ensembles of the same signature in this process.
struct EnsChoice {
  int lanes, pdl, lean;
  double ms;
};
std::mutex g_tune_mu;
std::map<std::string, EnsChoice> g_tune_cache;

std::string ens_signature(const qg_ensemble* e) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::string sig = "dev" + std::to_string(dev);
  for (const qg_handle* x : e->h) {
    char b[96];
    snprintf(b, sizeof(b), "|%d:%d:%d:%d:%d:%d", x->g.n, x->fp32, x->cl.kind, x->scheme, x->fac_b ? 1 : 0,
             x->fac_s ? 1 : 0);
    sig += b;
  }
  return sig;
}

void ens_apply(qg_ensemble* e, int lanes, int pdl, int lean) {
  e->lanes = lanes;
  e->pdl = pdl;
  e->lean = lean;
  for (qg_handle* x : e->h) {
    x->step_pdl = pdl;
    x->lean_reduce = lean;
  }
  if (e->exec) cudaGraphExecDestroy(e->exec);
  e->exec = nullptr;
  e->graph_tried = false;
}

// one ensemble step in the current launch form, replayed `reps` times after one warm replay: ms per step, or
// +inf when the graph cannot be built
double ens_time_form(qg_ensemble* e, cudaEvent_t a, cudaEvent_t b, int reps) {
  ens_build_graph(e);
  if (!e->exec) return std::numeric_limits<double>::infinity();
  if (cudaGraphLaunch(e->exec, e->main) != cudaSuccess) return std::numeric_limits<double>::infinity();
  cudaEventRecord(a, e->main);
  for (int r = 0; r < reps; ++r) cudaGraphLaunch(e->exec, e->main);
  cudaEventRecord(b, e->main);
  float ms = 0.f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return std::numeric_limits<double>::infinity();
  }
  return ms / reps;
}

// Choose the launch form.  The environment can fix it (QG_ENSEMBLE_LANES, QG_ENSEMBLE_PDL, QG_ENSEMBLE_LEAN) or
// turn the timing off (QG_ENSEMBLE_TUNE=0: all members side by side, no PDL, automatic lean form).  Timing steps
// the members from their initial (zero) states; afterwards the states, step counters, histories and status flags
// are reset, so the ensemble starts exactly as an untuned one.
int ens_tune(qg_ensemble* e) {
  const int m = (int)e->h.size();
  e->cost.resize(m);
  for (int i = 0; i < m; ++i) {
    const qg_handle* x = e->h[i];
    const double n2 = (double)x->g.n * x->g.n;
    const double per = x->dynamic ? 2.0 : 1.0;  // the dynamic closures double the transforms
    e->cost[i] = per * n2 * std::log2(n2) * (x->fp32 ? 1.0 : 8.0);
  }
  e->order.resize(m);
  for (int i = 0; i < m; ++i) e->order[i] = i;
  std::stable_sort(e->order.begin(), e->order.end(), [&](int a, int b) { return e->cost[a] > e->cost[b]; });
  const char* fl = getenv("QG_ENSEMBLE_LANES");
  const char* fp = getenv("QG_ENSEMBLE_PDL");
  const char* fn = getenv("QG_ENSEMBLE_LEAN");
  const char* ft = getenv("QG_ENSEMBLE_TUNE");
  if (fl || fp || fn || (ft && atoi(ft) == 0) || getenv("QG_NO_GRAPH")) {
    ens_apply(e, fl ? std::max(0, atoi(fl)) : 0, fp ? (atoi(fp) != 0) : 0, fn ? std::max(0, std::min(2, atoi(fn))) : 0);
    return QG_OK;
  }
  const std::string sig = ens_signature(e);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      ens_apply(e, it->second.lanes, it->second.pdl, it->second.lean);
      e->tuned = 2;
      e->tuned_ms = it->second.ms;
      return QG_OK;
    }
  }
  // one eager step (kernel attributes, the AB2CN Euler start), then the candidates' graphs
  int rc = ens_enqueue(e);
  if (rc) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a), "ensemble tuner: event");
  CK(cudaEventCreate(&b), "ensemble tuner: event");
  const int reps = 3;
  EnsChoice best{0, 0, 0, std::numeric_limits<double>::infinity()};
  auto trial = [&](int lanes, int pdl, int lean) {
    ens_apply(e, lanes, pdl, lean);
    const double t = ens_time_form(e, a, b, reps);
    if (t < best.ms) best = {lanes, pdl, lean, t};
  };
  // lanes first (all side by side, then fewer chains), then PDL, then the lean reduction
  std::vector<int> lane_set = {0};
  for (int l : {48, 32, 24, 16, 12, 8, 6, 4, 2})
    if (l < m) lane_set.push_back(l);
  for (int l : lane_set) trial(l, 0, 0);
  trial(best.lanes, 1, best.lean);
  bool lean_possible = false;
  for (const qg_handle* x : e->h) lean_possible = lean_possible || (x->fast && x->fp32 && x->dynamic);
  if (lean_possible) trial(best.lanes, best.pdl, 1);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!(best.ms < std::numeric_limits<double>::infinity())) best = {0, 0, 0, 0.0};
  ens_apply(e, best.lanes, best.pdl, best.lean);
  e->tuned = 1;
  e->tuned_ms = best.ms;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[sig] = best;
  }
  // back to the initial state: zero states and stage fields (what a step reads first), counters, histories
  // and flags
  for (qg_handle* x : e->h) {
    const size_t spec_bytes = (size_t)x->g.Kcp * x->g.SP * 2 * x->esz;
    const size_t mixed_bytes = (size_t)x->g.n * x->g.IP * 2 * x->esz;
    CK(cudaMemsetAsync(x->w0, 0, spec_bytes, x->stream), "ensemble tuner: reset");
    for (int i = 0; i < kMaxIn; ++i)
      if (x->X[i]) CK(cudaMemsetAsync(x->X[i], 0, mixed_bytes, x->stream), "ensemble tuner: reset");
    CK(cudaMemsetAsync(x->flag, 0, sizeof(int), x->stream), "ensemble tuner: reset");
    CK(cudaStreamSynchronize(x->stream), "ensemble tuner: reset");
    *x->flag_host = 0;
    x->flag_pending = false;
    x->step = 0;
    x->t = 0.0;
    x->ab2_hist = false;
    memset(x->launches, 0, sizeof(x->launches));
  }
  CK(cudaStreamSynchronize(e->main), "ensemble tuner: sync");
  e->eager_steps = 1;
  return QG_OK;
}

}  // namespace

extern "C" {

const char* qg_last_error(void) { return g_err.c_str(); }

const char* qg_version(void) { return "libqg 0.1 (sm_103a)"; }

int qg_create(const qg_grid* grid, double beta, double U, const double* mask, const double* sponge,
              const qg_closure* closure, const qg_params* params, void* cuda_stream, qg_handle** out) {
  if (!grid || !closure || !params || !out) return fail(QG_ERR_ARG, "qg_create: NULL argument");
  *out = nullptr;
  const int n = grid->n;
  if (!valid_n(n)) return fail(QG_ERR_ARG, "qg_create: n=%d must be even, 2^a 3^b, 16..4096", n);
  if (!(grid->L > 0) || !std::isfinite(grid->L)) return fail(QG_ERR_ARG, "qg_create: L must be positive");
  if (grid->precision != QG_FP32 && grid->precision != QG_FP64)
    return fail(QG_ERR_ARG, "qg_create: precision must be QG_FP32 or QG_FP64");
  if (closure->kind < QG_NONE || closure->kind > QG_DLEITH) return fail(QG_ERR_ARG, "qg_create: bad closure kind");
  if ((closure->kind == QG_DSMAG || closure->kind == QG_DLEITH) && !(closure->test_ratio > 1.0))
    return fail(QG_ERR_ARG, "qg_create: test_ratio must exceed 1");
  if (!(params->dt > 0) || params->nu < 0 || params->mu < 0 || (mask && !(params->eta > 0)) ||
      (sponge && params->sponge_rate < 0))
    return fail(QG_ERR_ARG, "qg_create: bad time-step parameters");
  if (params->scheme != QG_SCHEME_RK3_EXACT && params->scheme != QG_SCHEME_AB2CN)
    return fail(QG_ERR_ARG, "qg_create: unknown time scheme %d", params->scheme);

  qg_handle* h = new qg_handle();
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->fp32 = grid->precision == QG_FP32;
  h->esz = h->fp32 ? 4 : 8;
  h->L = grid->L;
  h->beta = beta;
  h->U = U;
  h->cl = *closure;
  h->par = *params;
  h->scheme = params->scheme;
  h->dynamic = closure->kind == QG_DSMAG || closure->kind == QG_DLEITH;
  const double delta = grid->L / n;
  {
    // |m|^2 (2r)^2 <= N^2, evaluated in FP64 for every integer |m|^2 of the 2/3 band
    const double r2 = (2.0 * closure->test_ratio) * (2.0 * closure->test_ratio);
    const int kmax = (n - 1) / 3;
    int m2 = 0;
    while (m2 + 1 <= 2 * kmax * kmax && double(m2 + 1) * r2 <= double(n) * double(n)) ++m2;
    h->test_m2max = m2;
    int kx = 0;
    while ((kx + 1) * (kx + 1) <= m2) ++kx;
    h->test_kmax = kx;
  }
  if (closure->kind == QG_SMAG) h->static_coeff = std::pow(closure->c * delta, 2);
  if (closure->kind == QG_LEITH) h->static_coeff = std::pow(closure->c * delta, 3);

  Geom& g = h->g;
  g.n = n;
  g.K = (n - 1) / 3;
  g.Kc = g.K + 1;
  g.Ny = 2 * g.K + 1;
  g.SP = (g.Ny + 3) / 4 * 4;
  g.kscale = 2.0 * M_PI / grid->L;
  h->plan = make_plan(n);

  int dev = 0, smem_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "qg_create: device query");
  }
  const size_t csz = 2 * h->esz;
  const size_t smem_cap = (size_t)smem_optin - 1024;

  // stage program of the closure
  static const int base4[4] = {D_U, D_V, D_WX, D_WY};
  int nd = 0;
  for (int i = 0; i < 4; ++i) h->der[nd++] = base4[i];
  switch (closure->kind) {
    case QG_NONE: h->row_prog = RP_NONE; h->nout = 1; h->dx_mask = 0; break;
    case QG_LEITH: h->row_prog = RP_LEITH; h->nout = 3; h->dx_mask = 0x2; break;
    case QG_SMAG:
      h->row_prog = RP_SMAG; h->nout = 3; h->dx_mask = 0x2;
      h->der[nd++] = D_PXY; h->der[nd++] = D_PD;
      break;
    case QG_DLEITH:
      h->row_prog = RP_DLEITH; h->nout = 6; h->dx_mask = 0x12;
      for (int i = 0; i < 4; ++i) h->der[nd++] = base4[i] | D_TEST;
      break;
    case QG_DSMAG:
      h->row_prog = RP_DSMAG; h->nout = 6; h->dx_mask = 0x12;
      h->der[nd++] = D_PXY; h->der[nd++] = D_PD;
      for (int i = 0; i < 4; ++i) h->der[nd++] = base4[i] | D_TEST;
      h->der[nd++] = D_PXY | D_TEST; h->der[nd++] = D_PD | D_TEST;
      break;
  }
  h->nder = nd;
  h->nin = nd;

  // column tile width: 32-byte row segments, enough threads, shared memory fits
  int W = h->fp32 ? 4 : 2;
  const int col_max_threads = h->fp32 ? 1024 : 512;  // the kernels' launch bounds
  for (;; W /= 2) {
    const size_t sm = (size_t)n * W * csz + 2 * (size_t)W * g.Ny * csz;
    const int th = threads_for(h->plan, W, 128);
    if ((sm <= smem_cap && th <= col_max_threads) || W == 1) {
      h->W = W;
      h->col_smem = sm;
      h->col_threads = th;
      break;
    }
  }
  if (h->col_smem > smem_cap || h->col_threads > col_max_threads) {
    delete h;
    return fail(QG_ERR_UNSUPPORTED, "qg_create: column pass does not fit (n=%d)", n);
  }
  const int nslot = h->nin > 2 ? h->nin : 2;
  h->row_smem = (size_t)n * csz + (size_t)nslot * n * h->esz;
  h->row_threads = threads_for(h->plan, 1, 256);
  if (h->row_smem > smem_cap || h->row_threads > 512) {
    delete h;
    return fail(QG_ERR_UNSUPPORTED, "qg_create: row pass needs %zu B of shared memory (n=%d, closure %d)",
                h->row_smem, n, closure->kind);
  }
  // 2^p and 3 * 2^p grids use the register-resident kernels (two k_x columns per CTA)
  {
    const bool spec = fast::fast_size(n);
    int fw = 2;
    switch (n) {
      case 256: fw = fast_col_width<256>(); break;
      case 512: fw = fast_col_width<512>(); break;
      case 1024: fw = fast_col_width<1024>(); break;
      case 2048: fw = fast_col_width<2048>(); break;
      case 4096: fw = fast_col_width<4096>(); break;
      case 384: fw = fast_col_width<384>(); break;
      case 768: fw = fast_col_width<768>(); break;
      case 1536: fw = fast_col_width<1536>(); break;
      case 3072: fw = fast_col_width<3072>(); break;
    }
    const size_t dense = (size_t)n * fw * csz, padded = (size_t)fw * (n + n / 16 + 16 / fw) * csz;
    const size_t fast_col_smem = 3 * (((dense > padded ? dense : padded) + 1023) / 1024 * 1024) + 1024;
    const int tt = spec ? n / fast::elems_per_thread(n) : 1;
    const int rows = tt >= QG_ROW_CTA_THREADS ? 1 : QG_ROW_CTA_THREADS / tt;  // rows per CTA of the row pass
    const size_t fast_row_smem = (size_t)2 * rows * (n + n / 16) * csz;
    h->fast = spec && fast_col_smem <= smem_cap && fast_row_smem <= smem_cap;
    if (getenv("QG_FORCE_GENERIC")) h->fast = false;
    if (const char* inj = getenv("QG_INJECT_TMA_STALL")) h->inject_stall = h->fast ? atoi(inj) + 1 : 0;
    if (h->fast) h->W = fw;
  }
  g.Kcp = (g.Kc + h->W - 1) / h->W * h->W;
  g.IP = g.Kcp;
  h->ncolblk = g.Kcp / h->W;

  int rc = QG_OK;
  const size_t spec_bytes = (size_t)g.Kcp * g.SP * csz;
  const size_t mixed_bytes = (size_t)n * g.IP * csz;
  const size_t phys_bytes = (size_t)n * n * h->esz;
  if (!rc) rc = dalloc(h, &h->w0, spec_bytes);
  if (!rc) rc = dalloc(h, &h->ws, spec_bytes);
  if (!rc) rc = dalloc(h, &h->ws2, spec_bytes);
  if (!rc && h->dynamic) rc = dalloc(h, &h->jh, spec_bytes);
  if (!rc && h->dynamic) rc = dalloc(h, &h->dh, spec_bytes);
  for (int i = 0; i < 3 && !rc && h->dynamic && h->fast && h->fp32; ++i) rc = dalloc(h, &h->red_scr[i], spec_bytes);
  for (int i = 0; i < h->nin && !rc; ++i) rc = dalloc(h, &h->X[i], mixed_bytes);
  const int ny = h->nout > 2 ? h->nout : 2;
  for (int i = 0; i < ny && !rc; ++i) rc = dalloc(h, &h->Y[i], mixed_bytes);
  if (h->scheme == QG_SCHEME_AB2CN) {
    if (!rc && mask) rc = dalloc(h, &h->Y[6], mixed_bytes);
    if (!rc && mask) rc = dalloc(h, &h->Y[7], mixed_bytes);
    if (!rc) rc = dalloc(h, &h->eprev, spec_bytes);
    if (!rc) rc = dalloc(h, &h->wss, spec_bytes);
    if (!rc && mask && h->dynamic) rc = dalloc(h, &h->bh, spec_bytes);
  }
  if (!rc) rc = dalloc(h, &h->phys, phys_bytes);
  if (!rc) rc = dalloc(h, &h->tw, (size_t)n * csz);
  if (!rc) rc = dalloc(h, &h->visc_x, (size_t)g.Kcp * h->esz);
  if (!rc) rc = dalloc(h, &h->visc_y, (size_t)g.SP * h->esz);
  if (!rc) rc = dalloc(h, (void**)&h->partials, (size_t)2 * h->ncolblk * sizeof(double));
  if (!rc) rc = dalloc(h, (void**)&h->red, (size_t)2 * 1024 * sizeof(double));
  if (!rc) rc = dalloc(h, (void**)&h->dev_scalars, 16 * sizeof(double));
  if (!rc) rc = dalloc(h, (void**)&h->flag, sizeof(int));
  if (!rc && mask) rc = dalloc(h, &h->fac_b, phys_bytes);
  if (!rc && sponge) rc = dalloc(h, &h->fac_s, phys_bytes);
  if (rc) {
    delete h;
    return rc;
  }
  e = cudaMallocHost((void**)&h->flag_host, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->flag_event, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "qg_create: host flag");
  }
  *h->flag_host = 0;

  // twiddles exp(-2 pi i j / n)
  {
    std::vector<double> tw(2 * (size_t)n);
    for (int j = 0; j < n; ++j) {
      double c, s;
      cos_sin_frac(j, n, &c, &s);
      tw[2 * j] = c;
      tw[2 * j + 1] = -s;
    }
    if ((rc = upload_real(h, h->tw, tw))) { delete h; return rc; }
    if (h->fast) {
      const int nt = fast_pass_table_size(n);
      std::vector<double> pt(2 * (size_t)(nt > 0 ? nt : 1), 0.0);
      fast_pass_table(n, tw.data(), pt.data());
      if ((rc = dalloc(h, &h->ptw, pt.size() / 2 * csz)) || (rc = upload_real(h, h->ptw, pt))) {
        delete h;
        return rc;
      }
    }
  }
  // tensor maps of every mixed array for the TMA column pass
  if (h->fast) {
    const int BR = fast_box_rows(n);
    for (int i = 0; i < kMaxIn; ++i)
      if (h->X[i] && (rc = add_tensor_map(h, h->X[i], h->W, BR))) { delete h; return rc; }
    for (int i = 0; i < kMaxY; ++i)
      if (h->Y[i] && (rc = add_tensor_map(h, h->Y[i], h->W, BR))) { delete h; return rc; }
  }
  // exact viscous factors, separable in k_x and k_y
  {
    const double nu = params->nu, dt = params->dt;
    std::vector<double> vx(g.Kcp, 0.0), vy(g.SP, 0.0);
    for (int m = 0; m < g.Kcp; ++m) {
      const double k = g.kscale * m;
      vx[m] = std::exp(-nu * k * k * dt);
    }
    for (int r = 0; r < g.Ny; ++r) {
      const double k = g.kscale * my_of_r(g, r);
      vy[r] = std::exp(-nu * k * k * dt);
    }
    h->visc_mu = std::exp(-params->mu * dt);
    if ((rc = upload_real(h, h->visc_x, vx)) || (rc = upload_real(h, h->visc_y, vy))) { delete h; return rc; }
  }
  // exact penalisation factors
  // RK3 + exact sub-steps: exp(-chi dt / eta) and exp(-rate chi_s dt);
  // the paper's scheme: chi itself (explicit Brinkman forcing) and dt rate chi_s (AB2 sponge)
  const bool ab2 = h->scheme == QG_SCHEME_AB2CN;
  if (mask) {
    std::vector<double> f((size_t)n * n);
    for (size_t i = 0; i < f.size(); ++i) f[i] = ab2 ? mask[i] : std::exp(-mask[i] * params->dt / params->eta);
    if ((rc = upload_real(h, h->fac_b, f))) { delete h; return rc; }
  }
  if (sponge) {
    std::vector<double> f((size_t)n * n);
    for (size_t i = 0; i < f.size(); ++i)
      f[i] = ab2 ? params->dt * params->sponge_rate * sponge[i] : std::exp(-params->sponge_rate * sponge[i] * params->dt);
    if ((rc = upload_real(h, h->fac_s, f))) { delete h; return rc; }
    if (!ab2) {
      std::vector<double> cs(sponge, sponge + (size_t)n * n);
      if ((rc = dalloc(h, &h->chi_s, phys_bytes)) || (rc = upload_real(h, h->chi_s, cs))) { delete h; return rc; }
    }
  }
  // the zero state derives to zero fields: X already zeroed
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "qg_create: sync");
  }
  *out = h;
  return QG_OK;
}

void qg_destroy(qg_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h;
}

int qg_stream(qg_handle* h, void** stream) {
  if (!h || !stream) return fail(QG_ERR_ARG, "qg_stream: NULL argument");
  *stream = static_cast<void*>(h->stream);
  return QG_OK;
}

int qg_set_state(qg_handle* h, const void* omega, int32_t on_device, int32_t dtype) {
  if (!h || !omega) return fail(QG_ERR_ARG, "qg_set_state: NULL argument");
  if (dtype != QG_FP32 && dtype != QG_FP64) return fail(QG_ERR_ARG, "qg_set_state: bad dtype");
  const size_t count = (size_t)h->g.n * h->g.n;
  const int src32 = dtype == QG_FP32;
  if (on_device) {
    CK(launch_convert(omega, src32, h->phys, h->fp32, count, h->stream), "qg_set_state: convert");
  } else if (src32 == h->fp32) {
    CK(cudaMemcpyAsync(h->phys, omega, count * h->esz, cudaMemcpyHostToDevice, h->stream), "qg_set_state: copy");
    CK(cudaStreamSynchronize(h->stream), "qg_set_state: sync");
  } else {
    std::vector<double> v(count);
    if (src32) for (size_t i = 0; i < count; ++i) v[i] = ((const float*)omega)[i];
    else std::memcpy(v.data(), omega, count * 8);
    int rc = upload_real(h, h->phys, v);
    if (rc) return rc;
  }
  CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream), "qg_set_state: flag");
  h->flag_pending = false;
  h->ab2_hist = false;
  *h->flag_host = 0;
  RowDesc r{};
  r.prog = RP_COPY;
  r.nin = 1;
  r.nout = 1;
  r.in_phys = 1;
  r.phys_in = h->phys;
  r.out[0] = h->Y[0];
  int rc = run_row(h, r, QG_K_OTHER, false);
  if (rc) return rc;
  ColDesc c = col_base(h);
  c.op = CO_FORWARD;
  c.nfwd = 1;
  c.fin[0] = h->Y[0];
  set_final(h, c);
  return run_col(h, c, QG_K_OTHER, false);
}

int qg_get_state(qg_handle* h, void* omega, int32_t on_device, int32_t dtype) {
  if (!h || !omega) return fail(QG_ERR_ARG, "qg_get_state: NULL argument");
  if (dtype != QG_FP32 && dtype != QG_FP64) return fail(QG_ERR_ARG, "qg_get_state: bad dtype");
  int rc = state_to_phys(h);
  if (rc) return rc;
  const size_t count = (size_t)h->g.n * h->g.n;
  const int dst32 = dtype == QG_FP32;
  if (on_device) {
    CK(launch_convert(h->phys, h->fp32, omega, dst32, count, h->stream), "qg_get_state: convert");
    return QG_OK;
  }
  if (dst32 == h->fp32) {
    CK(cudaMemcpyAsync(omega, h->phys, count * h->esz, cudaMemcpyDeviceToHost, h->stream), "qg_get_state: copy");
    CK(cudaStreamSynchronize(h->stream), "qg_get_state: sync");
    return QG_OK;
  }
  std::vector<unsigned char> tmp(count * h->esz);
  CK(cudaMemcpyAsync(tmp.data(), h->phys, tmp.size(), cudaMemcpyDeviceToHost, h->stream), "qg_get_state: copy");
  CK(cudaStreamSynchronize(h->stream), "qg_get_state: sync");
  for (size_t i = 0; i < count; ++i) {
    const double v = h->fp32 ? (double)((const float*)tmp.data())[i] : ((const double*)tmp.data())[i];
    if (dst32) ((float*)omega)[i] = (float)v;
    else ((double*)omega)[i] = v;
  }
  return QG_OK;
}

int qg_step(qg_handle* h, int32_t nsteps) {
  if (!h) return fail(QG_ERR_ARG, "qg_step: NULL handle");
  if (nsteps < 0) return fail(QG_ERR_ARG, "qg_step: nsteps < 0");
  if (h->flag_pending && cudaEventQuery(h->flag_event) == cudaSuccess) h->flag_pending = false;
  if (!h->flag_pending && (*h->flag_host & kFlagBounds))
    return fail(QG_ERR_BOUNDS, "qg_step: a kernel met an index outside its array at an earlier step");
  if (!h->flag_pending && (*h->flag_host & kFlagTimeout))
    return fail(QG_ERR_TIMEOUT, "qg_step: a bounded device wait gave up at an earlier step; qg_set_state resets");
  if (!h->flag_pending && *h->flag_host)
    return fail(QG_ERR_NONFINITE, "qg_step: state became non-finite at an earlier step");
  for (int i = 0; i < nsteps; ++i) {
    // the Euler start of the paper's scheme differs from its later steps: always eager
    const bool start = h->scheme == QG_SCHEME_AB2CN && !h->ab2_hist;
    if (!h->prof && !start && h->eager_steps > 0 && !h->graph_tried) try_build_graph(h);
    if (!h->prof && !start && h->step_graph) {
      CK(cudaGraphLaunch(h->step_graph, h->stream), "qg_step: graph launch");
      for (int c = 0; c < QG_NUM_KCLASS; ++c) h->launches[c] += h->graph_launches[c];
      h->step += 1;
      h->t += h->par.dt;
    } else {
      int rc = enqueue_any_step(h);
      if (rc) return rc;
      h->eager_steps += 1;
    }
  }
  if (!h->flag_pending) {
    CK(cudaMemcpyAsync(h->flag_host, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "qg_step: flag");
    CK(cudaEventRecord(h->flag_event, h->stream), "qg_step: event");
    h->flag_pending = true;
  }
  return QG_OK;
}

int qg_sync(qg_handle* h) {
  if (!h) return fail(QG_ERR_ARG, "qg_sync: NULL handle");
  int f = 0;
  CK(cudaMemcpyAsync(h->flag_host, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "qg_sync: flag");
  CK(cudaStreamSynchronize(h->stream), "qg_sync");
  h->flag_pending = false;
  f = *h->flag_host;
  if (f & kFlagBounds) return fail(QG_ERR_BOUNDS, "qg_sync: a kernel met an index outside its array (checked build)");
  if (f & kFlagTimeout) return fail(QG_ERR_TIMEOUT, "qg_sync: a bounded device wait gave up (TMA tile never arrived)");
  if (f) return fail(QG_ERR_NONFINITE, "qg_sync: state became non-finite");
  return QG_OK;
}

int qg_diagnostics(qg_handle* h, qg_diag* out) {
  if (!h || !out) return fail(QG_ERR_ARG, "qg_diagnostics: NULL argument");
  int status = qg_sync(h);
  if (status != QG_OK && status != QG_ERR_NONFINITE) return status;
  const int nblk = 512;
  double* sc = h->dev_scalars;
  cudaError_t e = h->fp32 ? launch_spectral_sums<float>(h->g, h->w0, h->red, nblk, sc + 4, h->stream)
                          : launch_spectral_sums<double>(h->g, h->w0, h->red, nblk, sc + 4, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qg_diagnostics: sums");
  int rc = state_to_phys(h);
  if (rc) return rc;
  e = h->fp32 ? launch_phys_maxabs<float>(h->g, h->phys, h->red, nblk, sc + 6, h->stream)
              : launch_phys_maxabs<double>(h->g, h->phys, h->red, nblk, sc + 6, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qg_diagnostics: max");
  double host[16];
  CK(cudaMemcpyAsync(host, sc, sizeof(host), cudaMemcpyDeviceToHost, h->stream), "qg_diagnostics: copy");
  CK(cudaStreamSynchronize(h->stream), "qg_diagnostics: sync");
  out->t = h->t;
  out->step = h->step;
  out->energy = host[4];
  out->enstrophy = host[5];
  out->coeff = h->dynamic ? host[2] : h->static_coeff;
  out->max_abs_omega = host[6];
  out->finite = (host[7] > 0.5 && status == QG_OK) ? 1 : 0;
  out->reserved = 0;
  if (!out->finite) return fail(QG_ERR_NONFINITE, "qg_diagnostics: state is not finite");
  return QG_OK;
}

int qg_profile(qg_handle* h, int32_t enable) {
  if (!h) return fail(QG_ERR_ARG, "qg_profile: NULL handle");
  if (enable) {
    CK(cudaStreamSynchronize(h->stream), "qg_profile: sync");
    for (auto& r : h->recs) {
      h->pool.push_back(r.a);
      h->pool.push_back(r.b);
    }
    h->recs.clear();
    for (int i = 0; i < QG_NUM_KCLASS; ++i) {
      h->launches[i] = 0;
      h->prof_ms[i] = 0.0;
    }
  }
  h->prof = enable != 0;
  return QG_OK;
}

int qg_kernel_times(qg_handle* h, int32_t* counts, double* ms, int32_t nclass) {
  if (!h || nclass < 0 || nclass > QG_NUM_KCLASS) return fail(QG_ERR_ARG, "qg_kernel_times: bad argument");
  CK(cudaStreamSynchronize(h->stream), "qg_kernel_times: sync");
  for (auto& r : h->recs) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b), "qg_kernel_times: elapsed");
    h->prof_ms[r.cls] += t;
    h->pool.push_back(r.a);
    h->pool.push_back(r.b);
  }
  h->recs.clear();
  for (int i = 0; i < nclass; ++i) {
    if (counts) counts[i] = h->launches[i];
    if (ms) ms[i] = h->prof_ms[i];
  }
  return QG_OK;
}


int qg_ensemble_create(const qg_member* members, int32_t count, void* cuda_stream, qg_ensemble** out) {
  if (!members || !out || count < 1) return fail(QG_ERR_ARG, "qg_ensemble_create: NULL argument or count < 1");
  *out = nullptr;
  auto* e = new (std::nothrow) qg_ensemble();
  if (!e) return fail(QG_ERR_OOM, "qg_ensemble_create: out of host memory");
  e->main = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t ce = cudaSuccess;
  if (!e->main) {
    ce = cudaStreamCreateWithFlags(&e->main, cudaStreamNonBlocking);
    e->own_main = ce == cudaSuccess;
  }
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    if (!e->own_main) e->main = nullptr;
    delete e;
    return cuda_fail(ce, "qg_ensemble_create: stream/event");
  }
  for (int32_t i = 0; i < count; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce == cudaSuccess) e->st.push_back(s);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ce == cudaSuccess) e->ev.push_back(ev);
    if (ce != cudaSuccess) {
      delete e;
      return cuda_fail(ce, "qg_ensemble_create: member stream");
    }
    const qg_member& m = members[i];
    qg_handle* x = nullptr;
    const int rc = qg_create(&m.grid, m.beta, m.U, m.mask, m.sponge, &m.closure, &m.params, s, &x);
    if (rc != QG_OK) {
      const std::string why = g_err;
      delete e;
      return fail(rc, "qg_ensemble_create: member %d: %s", (int)i, why.c_str());
    }
    e->h.push_back(x);
  }
  const int rc = ens_tune(e);
  if (rc != QG_OK) {
    const std::string why = g_err;
    delete e;
    return fail(rc, "qg_ensemble_create: tuning: %s", why.c_str());
  }
  *out = e;
  return QG_OK;
}

int qg_ensemble_config(qg_ensemble* e, int32_t* form, double* ms_per_step) {
  if (!e || !form) return fail(QG_ERR_ARG, "qg_ensemble_config: NULL argument");
  form[0] = e->lanes > 0 && (size_t)e->lanes < e->h.size() ? e->lanes : (int32_t)e->h.size();
  form[1] = e->pdl;
  form[2] = e->lean;
  form[3] = e->tuned;
  if (ms_per_step) *ms_per_step = e->tuned_ms;
  return QG_OK;
}

int qg_ensemble_handle(qg_ensemble* e, int32_t i, qg_handle** out) {
  if (!e || !out || i < 0 || (size_t)i >= e->h.size()) return fail(QG_ERR_ARG, "qg_ensemble_handle: bad argument");
  *out = e->h[i];
  return QG_OK;
}

int qg_ensemble_step(qg_ensemble* e, int32_t nsteps) {
  if (!e) return fail(QG_ERR_ARG, "qg_ensemble_step: NULL ensemble");
  if (nsteps < 0) return fail(QG_ERR_ARG, "qg_ensemble_step: nsteps < 0");
  if (nsteps == 0) return QG_OK;
  const size_t m = e->h.size();
  // work already queued on a member's stream (set_state, ...) precedes the step
  for (size_t i = 0; i < m; ++i) {
    CK(cudaEventRecord(e->ev[i], e->st[i]), "qg_ensemble_step: member tail");
    CK(cudaStreamWaitEvent(e->main, e->ev[i], 0), "qg_ensemble_step: member tail wait");
  }
  for (int32_t k = 0; k < nsteps; ++k) {
    bool eager = false;  // the Euler start of the paper's scheme and tracing run eagerly
    for (qg_handle* x : e->h) eager = eager || x->prof || (x->scheme == QG_SCHEME_AB2CN && !x->ab2_hist);
    if (!eager && e->eager_steps > 0 && !e->graph_tried) ens_build_graph(e);
    if (!eager && e->exec) {
      CK(cudaGraphLaunch(e->exec, e->main), "qg_ensemble_step: graph launch");
      for (size_t i = 0; i < m; ++i) {
        qg_handle* x = e->h[i];
        for (int c = 0; c < QG_NUM_KCLASS; ++c) x->launches[c] += e->graph_launches[i][c];
        x->step += 1;
        x->t += x->par.dt;
        if (x->scheme == QG_SCHEME_AB2CN) x->ab2_hist = true;
      }
    } else {
      const int rc = ens_enqueue(e);
      if (rc) return rc;
      e->eager_steps += 1;
    }
  }
  // later work on a member's stream follows the step; each member's status flag comes back
  CK(cudaEventRecord(e->done, e->main), "qg_ensemble_step: done");
  for (size_t i = 0; i < m; ++i) {
    qg_handle* x = e->h[i];
    CK(cudaStreamWaitEvent(e->st[i], e->done, 0), "qg_ensemble_step: done wait");
    CK(cudaMemcpyAsync(x->flag_host, x->flag, sizeof(int), cudaMemcpyDeviceToHost, x->stream),
       "qg_ensemble_step: flag");
    CK(cudaEventRecord(x->flag_event, x->stream), "qg_ensemble_step: flag event");
    x->flag_pending = true;
  }
  return QG_OK;
}

int qg_ensemble_sync(qg_ensemble* e, int32_t* first_bad) {
  if (!e) return fail(QG_ERR_ARG, "qg_ensemble_sync: NULL ensemble");
  if (first_bad) *first_bad = -1;
  CK(cudaStreamSynchronize(e->main), "qg_ensemble_sync");
  int status = QG_OK;
  for (size_t i = 0; i < e->h.size(); ++i) {
    const int rc = qg_sync(e->h[i]);
    if (rc != QG_OK && status == QG_OK) {
      status = rc;
      if (first_bad) *first_bad = (int32_t)i;
    }
  }
  if (status != QG_OK) {
    const std::string why = g_err;
    return fail(status, "qg_ensemble_sync: member %d: %s", first_bad ? *first_bad : -1, why.c_str());
  }
  return QG_OK;
}

void qg_ensemble_destroy(qg_ensemble* e) { delete e; }

int qg_step_vjp(qg_handle* h, const void* omega_n, const void* lam_next, void* lam_n, int32_t on_device,
                int32_t dtype, double* grads) {
  if (!h || !omega_n || !lam_next || !lam_n) return fail(QG_ERR_ARG, "qg_step_vjp: NULL argument");
  if (dtype != QG_FP32 && dtype != QG_FP64) return fail(QG_ERR_ARG, "qg_step_vjp: bad dtype");
  if (h->scheme != QG_SCHEME_RK3_EXACT)
    return fail(QG_ERR_UNSUPPORTED, "qg_step_vjp: only the RK3 scheme has an adjoint");
  int rc = adj_alloc(h);
  if (rc) return rc;
  auto& P = h->adj_P;
  const size_t count = (size_t)h->g.n * h->g.n;
  const int src32 = dtype == QG_FP32;
  for (int k = 0; k < 2; ++k) {
    const void* src = k ? lam_next : omega_n;
    void* dst = P[17 + k];
    if (on_device) {
      CK(launch_convert(src, src32, dst, h->fp32, count, h->stream), "qg_step_vjp: convert");
    } else if (src32 == h->fp32) {
      CK(cudaMemcpyAsync(dst, src, count * h->esz, cudaMemcpyHostToDevice, h->stream), "qg_step_vjp: copy");
      CK(cudaStreamSynchronize(h->stream), "qg_step_vjp: sync");
    } else {
      std::vector<double> v(count);
      if (src32) for (size_t i = 0; i < count; ++i) v[i] = ((const float*)src)[i];
      else std::memcpy(v.data(), src, count * 8);
      if ((rc = upload_real(h, dst, v))) return rc;
    }
  }
  if (!h->prof && h->adj_graph) {
    CK(cudaGraphLaunch(h->adj_graph, h->stream), "qg_step_vjp: graph launch");
    for (int c = 0; c < QG_NUM_KCLASS; ++c) h->launches[c] += h->adj_graph_launches[c];
  } else {
    if ((rc = adj_step(h))) return rc;
    if (!h->prof && !h->adj_graph_tried) adj_build_graph(h);
  }
  double d[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(d, h->adj_dots + kAdjDotBlocks, sizeof(d), cudaMemcpyDeviceToHost, h->stream),
     "qg_step_vjp: derivatives");
  const int dst32 = src32;
  if (on_device) {
    CK(launch_convert(P[18], h->fp32, lam_n, dst32, count, h->stream), "qg_step_vjp: convert out");
    CK(cudaStreamSynchronize(h->stream), "qg_step_vjp: sync");
  } else {
    std::vector<unsigned char> tmp(count * h->esz);
    CK(cudaMemcpyAsync(tmp.data(), P[18], tmp.size(), cudaMemcpyDeviceToHost, h->stream), "qg_step_vjp: copy out");
    CK(cudaStreamSynchronize(h->stream), "qg_step_vjp: sync");
    for (size_t i = 0; i < count; ++i) {
      const double v = h->fp32 ? (double)((const float*)tmp.data())[i] : ((const double*)tmp.data())[i];
      if (dst32) ((float*)lam_n)[i] = (float)v;
      else ((double*)lam_n)[i] = v;
    }
  }
  if (grads) {
    const double dC = d[0] + d[1] + d[2];
    grads[0] = dC;
    grads[1] = 0.0;
    if (h->cl.kind == QG_SMAG || h->cl.kind == QG_LEITH) {
      const int p = h->cl.kind == QG_SMAG ? 2 : 3;
      const double delta = h->L / h->g.n;
      grads[1] = dC * p * std::pow(h->cl.c, p - 1) * std::pow(delta, p);
    }
    grads[2] = d[3];
  }
  return QG_OK;
}

}  // extern "C"
