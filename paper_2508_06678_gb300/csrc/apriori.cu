// A priori SGS analysis on the GPU (Sec. III, Eq. 5-8 and 15), FP64.
//
// From one fully resolved field w on the N_f grid:
//   fine grid    J = T F[u w_x + v w_y],  F_obs = -T curl(chi u)/eta,
//                F_sponge = -rate T F[chi_s w]                     (Eq. 1-3, 6)
//   grid filter  H = exp(-k^2 Delta^2 / 6) * [|m| <= N_c/2], spectral copy to
//                the N_c grid (coarse Nyquist lines dropped), Delta = L / N_c   (Eq. 5)
//   coarse grid  w~ = T_c H w, J(w~), F_obs(H chi, u~), F_sponge(H chi_s, w~)
//   ideal Pi     Pi = [J(w~) - H J] + [H F_obs - F_obs(H chi, u~)]
//                   + [H F_sponge - F_sponge(H chi_s, w~)]                  (Eq. 8)
//   model        C div(g grad w~), static (c Delta)^p or Germano/Lilly C    (Eq. 9-14)
//   PCC          of Pi and the model over the N_c^2 points                   (Eq. 15)
// Every transform and product runs in the generic row / column kernels of the
// time step on three grid descriptions: the fine 2/3 band, the coarse 2/3
// band, and the coarse band without its Nyquist lines for the filtered
// coefficient fields H chi and H chi_s (which are not truncated).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/qg.h"
#include "qg_kernels.h"

using namespace qg;

namespace {

using C2 = double2;

struct Grid {
  Geom g{};
  FftPlan plan{};
  int W = 2;
  int col_threads = 128, row_threads = 256;
  size_t col_smem = 0, row_smem = 0;
  void* tw = nullptr;
};

FftPlan plan_of(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  while (m % 8 == 0) { p.radix[p.npass++] = 8; m /= 8; }
  if (m % 4 == 0) { p.radix[p.npass++] = 4; m /= 4; }
  if (m % 2 == 0) { p.radix[p.npass++] = 2; m /= 2; }
  while (m % 3 == 0) { p.radix[p.npass++] = 3; m /= 3; }
  return p;
}

int threads_of(const FftPlan& p, int B, int floor_threads) {
  int need = floor_threads;
  for (int s = 0; s < p.npass; ++s) {
    const int R = p.radix[s];
    const int mi = R == 3 ? 2 : 8 / R;
    const int t = ((p.n / R) * B + mi - 1) / mi;
    if (t > need) need = t;
  }
  return (need + 31) / 32 * 32;
}

bool valid_n(int n) {
  if (n < 16 || n > 4096 || (n & 1)) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

// grid description with band limit K (2/3 rule: (n-1)/3; full band: n/2 - 1)
void make_grid(Grid& G, int n, int K, double L, int nslot) {
  Geom& g = G.g;
  g.n = n;
  g.K = K;
  g.Kc = K + 1;
  g.Ny = 2 * K + 1;
  g.SP = (g.Ny + 3) / 4 * 4;
  g.kscale = 2.0 * M_PI / L;
  G.plan = plan_of(n);
  G.W = 2;
  G.col_threads = threads_of(G.plan, G.W, 128);
  G.col_smem = (size_t)n * G.W * 16 + 2 * (size_t)G.W * g.Ny * 16;
  g.Kcp = (g.Kc + G.W - 1) / G.W * G.W;
  g.IP = g.Kcp;
  G.row_threads = threads_of(G.plan, 1, 256);
  G.row_smem = (size_t)n * 16 + (size_t)(nslot > 2 ? nslot : 2) * n * 8;
}

void cos_sin_frac(long j, long n, double* c, double* s) {
  j %= n;
  const long q4 = 4 * j, quad = q4 / n, rem = q4 - quad * n;
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

// Eq. 5: out(m) = scale * H(m) * in(m) on the output grid's stored modes,
// H = exp(-k^2 Delta^2 / 6) (optional) times the cut-off |m| <= N_c / 2.
__global__ void filter_copy_kernel(Geom gi, const C2* __restrict__ in, Geom go, C2* __restrict__ out, int n_c,
                                   double delta, int gaussian, double scale) {
  const size_t total = (size_t)go.Kcp * go.SP;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / go.SP), r = (int)(e - (size_t)c * go.SP);
    C2 v = make_double2(0.0, 0.0);
    if (c < go.Kc && r < go.Ny) {
      const int my = my_of_r(go, r);
      const long m2 = (long)c * c + (long)my * my;
      if (4 * m2 <= (long)n_c * n_c && c <= gi.K && my <= gi.K && -my <= gi.K) {
        const int ri = my >= 0 ? my : my + gi.Ny;
        const C2 x = in[(size_t)c * gi.SP + ri];
        double h = scale;
        if (gaussian) {
          const double k2 = gi.kscale * gi.kscale * double(m2);
          h *= exp(-k2 * delta * delta / 6.0);
        }
        v = make_double2(h * x.x, h * x.y);
      }
    }
    out[e] = v;
  }
}

// out = a A + b B (+ c Cc) elementwise over a spectral array; coef, when set,
// multiplies b (a device scalar, e.g. the Germano coefficient).
__global__ void lincomb_kernel(size_t count, double a, const C2* A, double b, const C2* B, double c, const C2* Cc,
                               const double* coef, C2* out) {
  const double bb = coef ? b * coef[0] : b;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    C2 v = make_double2(0.0, 0.0);
    if (A) v = make_double2(a * A[e].x, a * A[e].y);
    if (B) v = make_double2(v.x + bb * B[e].x, v.y + bb * B[e].y);
    if (Cc) v = make_double2(v.x + c * Cc[e].x, v.y + c * Cc[e].y);
    out[e] = v;
  }
}

// C = max(0, sum HM / sum MM) (0 if sum MM = 0), partial sums in a fixed order
__global__ void germano_finish_kernel(const double* partials, int n, double* coef) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (threadIdx.x == 0) coef[0] = b > 0.0 ? fmax(0.0, a / b) : 0.0;
}

// PCC moments sum x, y, xx, yy, xy (FP64), two-level deterministic: 256 threads per block
__global__ void moments_kernel(const double* X, const double* Y, size_t count, double* partials) {
  __shared__ double s[5][8];
  double m[5] = {0, 0, 0, 0, 0};
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double x = X[i], y = Y[i];
    m[0] += x;
    m[1] += y;
    m[2] += x * x;
    m[3] += y * y;
    m[4] += x * y;
  }
  for (int k = 0; k < 5; ++k)
    for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_down_sync(0xffffffffu, m[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 5; ++k) s[k][threadIdx.x >> 5] = m[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < 5; ++k) {
      double v = threadIdx.x < 8 ? s[k][threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) partials[5 * blockIdx.x + k] = v;
    }
  }
}

__global__ void moments_finish_kernel(const double* partials, int nblk, double* out) {
  for (int k = 0; k < 5; ++k) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nblk; i += 32) v += partials[5 * i + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[k] = v;
  }
}

struct Pool {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = cudaMalloc(&p, bytes);
    if (err != cudaSuccess) return nullptr;
    cudaMemset(p, 0, bytes);
    ptrs.push_back(p);
    return p;
  }
  ~Pool() {
    for (void* p : ptrs) cudaFree(p);
  }
};

struct Ctx {
  cudaStream_t st = nullptr;
  cudaError_t err = cudaSuccess;
  void row(const Grid& G, RowDesc d) {
    if (err == cudaSuccess) err = launch_row<double>(G.g, G.plan, d, G.tw, G.row_threads, G.row_smem, st);
  }
  void col(const Grid& G, ColDesc d) {
    if (err == cudaSuccess) err = launch_col<double>(G.g, G.plan, d, G.tw, G.W, G.col_threads, G.col_smem, st);
  }
};

ColDesc col_desc(double U, const qg_closure* cl, int test_m2max) {
  ColDesc d{};
  d.U = U;
  d.test_ratio = cl->test_ratio;
  d.test_m2max = test_m2max;
  const int p = (cl->kind == QG_SMAG || cl->kind == QG_DSMAG) ? 2 : 3;
  d.closure_pow = p;
  d.rpow = std::pow(cl->test_ratio, p);
  return d;
}

}  // namespace

extern "C" int qg_sgs_apriori(const double* omega_fr, int32_t n_fr, int32_t n_les, double L, const double* mask_fr,
                              const double* sponge_fr, const qg_closure* closure, const qg_params* params, double U,
                              double beta, int32_t flags, double* pi_exact, double* pi_model, double* pi_parts,
                              double* pcc) {
  (void)beta;  // the beta term is linear and commutes with the spectral filter: it does not enter Pi
  char msg[256];
  if (!omega_fr || !closure || !params || !pi_exact || !pi_model || !pcc) {
    qg::set_last_error("qg_sgs_apriori: NULL argument");
    return QG_ERR_ARG;
  }
  if (!valid_n(n_fr) || !valid_n(n_les) || n_les > n_fr || !(L > 0)) {
    snprintf(msg, sizeof(msg), "qg_sgs_apriori: bad grid sizes n_fr=%d n_les=%d", n_fr, n_les);
    qg::set_last_error(msg);
    return QG_ERR_ARG;
  }
  if (closure->kind < QG_NONE || closure->kind > QG_DLEITH || (mask_fr && !(params->eta > 0))) {
    qg::set_last_error("qg_sgs_apriori: bad closure or parameters");
    return QG_ERR_ARG;
  }
  const int Kf = (n_fr - 1) / 3;
  if (n_les / 2 - 1 > Kf) {
    snprintf(msg, sizeof(msg),
             "qg_sgs_apriori: the coarse band (n_les/2 - 1 = %d) exceeds the fine 2/3 band (%d); needs n_les <= %d",
             n_les / 2 - 1, Kf, 2 * Kf + 2);
    qg::set_last_error(msg);
    return QG_ERR_UNSUPPORTED;
  }
  const int kind = closure->kind;
  const bool dyn = kind == QG_DSMAG || kind == QG_DLEITH;
  const bool smag = kind == QG_SMAG || kind == QG_DSMAG;
  const int nslot_c = kind == QG_DSMAG ? 12 : (kind == QG_DLEITH ? 8 : 6);

  Grid F, Cg, Cf;
  make_grid(F, n_fr, Kf, L, 4);
  make_grid(Cg, n_les, (n_les - 1) / 3, L, nslot_c);
  make_grid(Cf, n_les, n_les / 2 - 1, L, 2);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (F.col_smem > (size_t)optin - 1024 || F.row_smem > (size_t)optin - 1024 || Cg.row_smem > (size_t)optin - 1024) {
    qg::set_last_error("qg_sgs_apriori: grid too large for the kernels' shared memory");
    return QG_ERR_UNSUPPORTED;
  }

  Pool pool;
  Ctx cx;
  auto mixed = [&](const Grid& G) { return pool.get((size_t)G.g.n * G.g.IP * 16); };
  auto spec = [&](const Grid& G) { return pool.get((size_t)G.g.Kcp * G.g.SP * 16); };
  auto phys = [&](int n) { return pool.get((size_t)n * n * 8); };
  // twiddles per grid size
  for (Grid* G : {&F, &Cg, &Cf}) {
    std::vector<double> tw(2 * (size_t)G->g.n);
    for (int j = 0; j < G->g.n; ++j) {
      double c, s;
      cos_sin_frac(j, G->g.n, &c, &s);
      tw[2 * j] = c;
      tw[2 * j + 1] = -s;
    }
    G->tw = pool.get(tw.size() * 8);
    if (G->tw) cudaMemcpy(G->tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
  }
  const size_t nf2 = (size_t)n_fr * n_fr, nc2 = (size_t)n_les * n_les;
  void* Pw = phys(n_fr);
  void* Pchi = mask_fr ? phys(n_fr) : nullptr;
  void* Pchis = sponge_fr ? phys(n_fr) : nullptr;
  void* M[10];
  for (int i = 0; i < 10; ++i) M[i] = mixed(F);
  void* Sw = spec(F);
  void* SJ = spec(F);
  void* Sobs = mask_fr ? spec(F) : nullptr;
  void* Ssp = sponge_fr ? spec(F) : nullptr;
  void* Schi = mask_fr ? spec(F) : nullptr;
  void* Schis = sponge_fr ? spec(F) : nullptr;
  void* Mc[18];  // up to 12 model inputs + 6 outputs
  for (int i = 0; i < 18; ++i) Mc[i] = mixed(Cg);
  void* Mcf = mixed(Cf);
  void* Cw = spec(Cg);
  void* CJ = spec(Cg);
  void* CJles = spec(Cg);
  void* Cobs = spec(Cg);
  void* Cobsl = spec(Cg);
  void* Csp = spec(Cg);
  void* Cspl = spec(Cg);
  void* Cpart[4];
  for (int i = 0; i < 4; ++i) Cpart[i] = spec(Cg);
  void* Cjh = spec(Cg);
  void* Cdh = spec(Cg);
  void* Cmodel = spec(Cg);
  void* Cchi = mask_fr ? spec(Cf) : nullptr;
  void* Cchis = sponge_fr ? spec(Cf) : nullptr;
  void* Pcchi = mask_fr ? phys(n_les) : nullptr;
  void* Pcchis = sponge_fr ? phys(n_les) : nullptr;
  void* Pout[5];
  for (int i = 0; i < 5; ++i) Pout[i] = phys(n_les);
  double* partials = (double*)pool.get(2 * 4096 * sizeof(double));
  double* coef = (double*)pool.get(8 * sizeof(double));
  double* mom = (double*)pool.get(5 * 1024 * sizeof(double));
  if (pool.err != cudaSuccess) {
    qg::set_last_error("qg_sgs_apriori: device allocation failed");
    return QG_ERR_OOM;
  }
  cudaMemcpy(Pw, omega_fr, nf2 * 8, cudaMemcpyHostToDevice);
  if (mask_fr) cudaMemcpy(Pchi, mask_fr, nf2 * 8, cudaMemcpyHostToDevice);
  if (sponge_fr) cudaMemcpy(Pchis, sponge_fr, nf2 * 8, cudaMemcpyHostToDevice);

  // test filter threshold of the coarse grid: |m|^2 (2r)^2 <= N_c^2
  int test_m2max = 0;
  {
    const double r2 = (2.0 * closure->test_ratio) * (2.0 * closure->test_ratio);
    const int kc = Cg.g.K;
    while (test_m2max + 1 <= 2 * kc * kc && double(test_m2max + 1) * r2 <= double(n_les) * double(n_les)) ++test_m2max;
  }
  const ColDesc base = col_desc(U, closure, test_m2max);

  // ---- fine grid: projected state and its velocity / gradient fields
  {
    RowDesc r{};
    r.prog = RP_COPY; r.nin = 1; r.nout = 1; r.in_phys = 1; r.phys_in = Pw; r.out[0] = M[0];
    cx.row(F, r);
    ColDesc c = base;
    c.op = CO_FORWARD; c.nfwd = 1; c.fin[0] = M[0]; c.w0 = Sw; c.store_w0 = 1; c.zero_mean = 1;
    c.nder = 4; c.der[0] = D_U; c.der[1] = D_V; c.der[2] = D_WX; c.der[3] = D_WY;
    for (int i = 0; i < 4; ++i) c.dout[i] = M[1 + i];
    cx.col(F, c);
  }
  // J = T F[u w_x + v w_y]
  {
    RowDesc r{};
    r.prog = RP_NONE; r.nin = 4; r.nout = 1;
    for (int i = 0; i < 4; ++i) r.in[i] = M[1 + i];
    r.out[0] = M[5];
    cx.row(F, r);
    ColDesc c = base;
    c.op = CO_FORWARD; c.nfwd = 1; c.fin[0] = M[5]; c.w0 = SJ; c.store_w0 = 1;
    cx.col(F, c);
  }
  // F_obs (unscaled): T curl(chi u); chi spectrum for its filtered coefficient field
  if (mask_fr) {
    RowDesc r{};
    r.prog = RP_SCALE; r.nin = 2; r.nout = 2; r.in[0] = M[1]; r.in[1] = M[2]; r.out[0] = M[6]; r.out[1] = M[7];
    r.factor = Pchi;
    cx.row(F, r);
    ColDesc c = base;
    c.op = CO_CURL; c.nfwd = 2; c.fin[0] = M[6]; c.fin[1] = M[7]; c.w0 = Sobs; c.store_w0 = 1;
    cx.col(F, c);
    RowDesc r2{};
    r2.prog = RP_COPY; r2.nin = 1; r2.nout = 1; r2.in_phys = 1; r2.phys_in = Pchi; r2.out[0] = M[8];
    cx.row(F, r2);
    ColDesc c2 = base;
    c2.op = CO_FORWARD; c2.nfwd = 1; c2.fin[0] = M[8]; c2.w0 = Schi; c2.store_w0 = 1;
    cx.col(F, c2);
  }
  // F_sponge (unscaled): T F[chi_s w]; chi_s spectrum
  if (sponge_fr) {
    ColDesc c = base;
    c.op = CO_DERIVE; c.w0 = Sw; c.nder = 1; c.der[0] = D_W; c.dout[0] = M[8];
    cx.col(F, c);
    RowDesc r{};
    r.prog = RP_SCALE; r.nin = 1; r.nout = 1; r.in[0] = M[8]; r.out[0] = M[9]; r.factor = Pchis;
    cx.row(F, r);
    ColDesc c2 = base;
    c2.op = CO_FORWARD; c2.nfwd = 1; c2.fin[0] = M[9]; c2.w0 = Ssp; c2.store_w0 = 1;
    cx.col(F, c2);
    RowDesc r2{};
    r2.prog = RP_COPY; r2.nin = 1; r2.nout = 1; r2.in_phys = 1; r2.phys_in = Pchis; r2.out[0] = M[8];
    cx.row(F, r2);
    ColDesc c3 = base;
    c3.op = CO_FORWARD; c3.nfwd = 1; c3.fin[0] = M[8]; c3.w0 = Schis; c3.store_w0 = 1;
    cx.col(F, c3);
  }

  // ---- grid filter (Eq. 5) onto the coarse grid
  const double delta = L / n_les;
  const int gauss = (flags & 1) ? 0 : 1;
  const double sc = (double(n_les) / double(n_fr)) * (double(n_les) / double(n_fr));
  auto filt = [&](const void* in, const Grid& Go, void* out, double s) {
    if (cx.err != cudaSuccess) return;
    filter_copy_kernel<<<256, 256, 0, cx.st>>>(F.g, (const C2*)in, Go.g, (C2*)out, n_les, delta, gauss, sc * s);
    cx.err = cudaGetLastError();
  };
  filt(Sw, Cg, Cw, 1.0);
  filt(SJ, Cg, CJ, 1.0);
  if (mask_fr) {
    filt(Sobs, Cg, Cobs, -1.0 / params->eta);
    filt(Schi, Cf, Cchi, 1.0);
  }
  if (sponge_fr) {
    filt(Ssp, Cg, Csp, -params->sponge_rate);
    filt(Schis, Cf, Cchis, 1.0);
  }

  // ---- filtered coefficient fields on the coarse grid (physical, not truncated)
  auto to_phys = [&](const Grid& G, void* S, void* Mtmp, void* P) {
    ColDesc c = base;
    c.op = CO_DERIVE; c.w0 = S; c.nder = 1; c.der[0] = D_W; c.dout[0] = Mtmp;
    cx.col(G, c);
    RowDesc r{};
    r.prog = RP_COPY; r.nin = 1; r.nout = 1; r.in[0] = Mtmp; r.out_phys = 1; r.phys_out = P;
    cx.row(G, r);
  };
  if (mask_fr) to_phys(Cf, Cchi, Mcf, Pcchi);
  if (sponge_fr) to_phys(Cf, Cchis, Mcf, Pcchis);

  // ---- coarse-grid operators on w~ (Eq. 7)
  {
    ColDesc c = base;
    c.op = CO_DERIVE; c.w0 = Cw; c.nder = 4; c.der[0] = D_U; c.der[1] = D_V; c.der[2] = D_WX; c.der[3] = D_WY;
    for (int i = 0; i < 4; ++i) c.dout[i] = Mc[i];
    cx.col(Cg, c);
    RowDesc r{};
    r.prog = RP_NONE; r.nin = 4; r.nout = 1;
    for (int i = 0; i < 4; ++i) r.in[i] = Mc[i];
    r.out[0] = Mc[4];
    cx.row(Cg, r);
    ColDesc c2 = base;
    c2.op = CO_FORWARD; c2.nfwd = 1; c2.fin[0] = Mc[4]; c2.w0 = CJles; c2.store_w0 = 1;
    cx.col(Cg, c2);
  }
  if (mask_fr) {
    RowDesc r{};
    r.prog = RP_SCALE; r.nin = 2; r.nout = 2; r.in[0] = Mc[0]; r.in[1] = Mc[1]; r.out[0] = Mc[5]; r.out[1] = Mc[6];
    r.factor = Pcchi;
    cx.row(Cg, r);
    ColDesc c = base;
    c.op = CO_CURL; c.nfwd = 2; c.fin[0] = Mc[5]; c.fin[1] = Mc[6]; c.w0 = Cobsl; c.store_w0 = 1;
    cx.col(Cg, c);
  }
  if (sponge_fr) {
    ColDesc c = base;
    c.op = CO_DERIVE; c.w0 = Cw; c.nder = 1; c.der[0] = D_W; c.dout[0] = Mc[7];
    cx.col(Cg, c);
    RowDesc r{};
    r.prog = RP_SCALE; r.nin = 1; r.nout = 1; r.in[0] = Mc[7]; r.out[0] = Mc[8]; r.factor = Pcchis;
    cx.row(Cg, r);
    ColDesc c2 = base;
    c2.op = CO_FORWARD; c2.nfwd = 1; c2.fin[0] = Mc[8]; c2.w0 = Cspl; c2.store_w0 = 1;
    cx.col(Cg, c2);
  }

  // ---- Eq. 8 components and their sum (spectral), then physical
  const size_t cnt = (size_t)Cg.g.Kcp * Cg.g.SP;
  auto lin = [&](double a, void* A, double b, void* B, double c, void* Cc, const double* cf, void* out) {
    if (cx.err != cudaSuccess) return;
    lincomb_kernel<<<256, 256, 0, cx.st>>>(cnt, a, (const C2*)A, b, (const C2*)B, c, (const C2*)Cc, cf, (C2*)out);
    cx.err = cudaGetLastError();
  };
  lin(1.0, CJles, -1.0, CJ, 0.0, nullptr, nullptr, Cpart[0]);                         // J(w~) - H J
  if (mask_fr) lin(1.0, Cobs, 1.0 / params->eta, Cobsl, 0.0, nullptr, nullptr, Cpart[1]);  // H F_obs - F_obs(~)
  if (sponge_fr) lin(1.0, Csp, params->sponge_rate, Cspl, 0.0, nullptr, nullptr, Cpart[2]);
  lin(1.0, Cpart[0], mask_fr ? 1.0 : 0.0, Cpart[1], sponge_fr ? 1.0 : 0.0, Cpart[2], nullptr, Cpart[3]);
  to_phys(Cg, Cpart[3], Mc[9], Pout[0]);
  for (int i = 0; i < 3; ++i) to_phys(Cg, Cpart[i], Mc[9], Pout[2 + i]);

  // ---- closure model on w~ (Eq. 9-14)
  bool have_model = false;
  if (kind != QG_NONE) {
    ColDesc c = base;
    c.op = CO_DERIVE; c.w0 = Cw;
    int nd = 0;
    const int b4[4] = {D_U, D_V, D_WX, D_WY};
    for (int i = 0; i < 4; ++i) c.der[nd++] = b4[i];
    if (smag) { c.der[nd++] = D_PXY; c.der[nd++] = D_PD; }
    if (dyn) {
      for (int i = 0; i < 4; ++i) c.der[nd++] = b4[i] | D_TEST;
      if (smag) { c.der[nd++] = D_PXY | D_TEST; c.der[nd++] = D_PD | D_TEST; }
    }
    c.nder = nd;
    for (int i = 0; i < nd; ++i) c.dout[i] = Mc[i];
    cx.col(Cg, c);
    RowDesc r{};
    r.prog = kind == QG_SMAG ? RP_SMAG : kind == QG_LEITH ? RP_LEITH : kind == QG_DSMAG ? RP_DSMAG : RP_DLEITH;
    r.nin = nd;
    r.nout = dyn ? 6 : 3;
    r.dx_mask = dyn ? 0x12u : 0x2u;
    for (int i = 0; i < nd; ++i) r.in[i] = Mc[i];
    for (int i = 0; i < r.nout; ++i) r.out[i] = Mc[nd + i];
    cx.row(Cg, r);
    ColDesc c2 = base;
    c2.op = CO_DYN_REDUCE;
    c2.nfwd = r.nout;
    for (int i = 0; i < r.nout; ++i) c2.fin[i] = r.out[i];
    c2.jh = Cjh;
    c2.dh = Cdh;
    c2.partials = partials;
    cx.col(Cg, c2);
    const int nblk = Cg.g.Kcp / Cg.W;
    if (dyn) {
      if (cx.err == cudaSuccess) {
        germano_finish_kernel<<<1, 32, 0, cx.st>>>(partials, nblk, coef);
        cx.err = cudaGetLastError();
      }
      lin(0.0, nullptr, 1.0, Cdh, 0.0, nullptr, coef, Cmodel);
    } else {
      const double p = smag ? 2.0 : 3.0;
      lin(0.0, nullptr, std::pow(closure->c * delta, p), Cdh, 0.0, nullptr, nullptr, Cmodel);
    }
    to_phys(Cg, Cmodel, Mc[9], Pout[1]);
    have_model = true;
  }

  // ---- PCC moments (Eq. 15)
  double moments[5] = {0, 0, 0, 0, 0};
  if (have_model && cx.err == cudaSuccess) {
    moments_kernel<<<256, 256, 0, cx.st>>>((const double*)Pout[0], (const double*)Pout[1], nc2, mom);
    moments_finish_kernel<<<1, 32, 0, cx.st>>>(mom, 256, mom + 5 * 512);
    cx.err = cudaGetLastError();
  }
  if (cx.err == cudaSuccess) cx.err = cudaDeviceSynchronize();
  if (cx.err != cudaSuccess) {
    snprintf(msg, sizeof(msg), "qg_sgs_apriori: %s", cudaGetErrorString(cx.err));
    qg::set_last_error(msg);
    return QG_ERR_CUDA;
  }
  cudaMemcpy(pi_exact, Pout[0], nc2 * 8, cudaMemcpyDeviceToHost);
  if (have_model) {
    cudaMemcpy(pi_model, Pout[1], nc2 * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(moments, mom + 5 * 512, 5 * 8, cudaMemcpyDeviceToHost);
  } else {
    memset(pi_model, 0, nc2 * 8);
  }
  if (pi_parts)
    for (int i = 0; i < 3; ++i) cudaMemcpy(pi_parts + i * nc2, Pout[2 + i], nc2 * 8, cudaMemcpyDeviceToHost);
  double r = NAN;
  if (have_model) {
    const double n = double(nc2);
    const double mx = moments[0] / n, my = moments[1] / n;
    const double vx = moments[2] / n - mx * mx, vy = moments[3] / n - my * my, cxy = moments[4] / n - mx * my;
    if (vx > 0.0 && vy > 0.0) r = cxy / (std::sqrt(vx) * std::sqrt(vy));
  }
  *pcc = r;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "qg_sgs_apriori: %s", cudaGetErrorString(e));
    qg::set_last_error(msg);
    return QG_ERR_CUDA;
  }
  return QG_OK;
}

// The grid filter of Eq. 5 alone, on a series of fields: project each fine
// field onto its 2/3 band (zero mean), filter and copy it to the coarse grid
// (the coarse 2/3 band), return the physical coarse field.  This is the
// filtered fully resolved field an LES is compared with a posteriori.
extern "C" int qg_grid_filter(const double* omega_fr, int32_t nsnap, int32_t n_fr, int32_t n_les, double L,
                              int32_t flags, double* omega_les) {
  char msg[256];
  if (!omega_fr || !omega_les) {
    qg::set_last_error("qg_grid_filter: NULL argument");
    return QG_ERR_ARG;
  }
  if (nsnap < 1 || !valid_n(n_fr) || !valid_n(n_les) || n_les > n_fr || !(L > 0)) {
    snprintf(msg, sizeof(msg), "qg_grid_filter: bad sizes nsnap=%d n_fr=%d n_les=%d", nsnap, n_fr, n_les);
    qg::set_last_error(msg);
    return QG_ERR_ARG;
  }
  const int Kf = (n_fr - 1) / 3;
  if (n_les / 2 - 1 > Kf) {
    snprintf(msg, sizeof(msg),
             "qg_grid_filter: the coarse band (n_les/2 - 1 = %d) exceeds the fine 2/3 band (%d); needs n_les <= %d",
             n_les / 2 - 1, Kf, 2 * Kf + 2);
    qg::set_last_error(msg);
    return QG_ERR_UNSUPPORTED;
  }
  Grid F, Cg;
  make_grid(F, n_fr, Kf, L, 2);
  make_grid(Cg, n_les, (n_les - 1) / 3, L, 2);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (F.col_smem > (size_t)optin - 1024 || F.row_smem > (size_t)optin - 1024) {
    qg::set_last_error("qg_grid_filter: grid too large for the kernels' shared memory");
    return QG_ERR_UNSUPPORTED;
  }
  Pool pool;
  Ctx cx;
  for (Grid* G : {&F, &Cg}) {
    std::vector<double> tw(2 * (size_t)G->g.n);
    for (int j = 0; j < G->g.n; ++j) {
      double c, s;
      cos_sin_frac(j, G->g.n, &c, &s);
      tw[2 * j] = c;
      tw[2 * j + 1] = -s;
    }
    G->tw = pool.get(tw.size() * 8);
    if (G->tw) cudaMemcpy(G->tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
  }
  const size_t nf2 = (size_t)n_fr * n_fr, nc2 = (size_t)n_les * n_les;
  void* Pw = pool.get(nf2 * 8);
  void* Mf = pool.get((size_t)F.g.n * F.g.IP * 16);
  void* Sw = pool.get((size_t)F.g.Kcp * F.g.SP * 16);
  void* Mc = pool.get((size_t)Cg.g.n * Cg.g.IP * 16);
  void* Cw = pool.get((size_t)Cg.g.Kcp * Cg.g.SP * 16);
  void* Pc = pool.get(nc2 * 8);
  if (pool.err != cudaSuccess) {
    qg::set_last_error("qg_grid_filter: device allocation failed");
    return QG_ERR_OOM;
  }
  qg_closure none{};
  none.test_ratio = 2.0;
  const ColDesc base = col_desc(0.0, &none, 0);
  const double sc = (double(n_les) / double(n_fr)) * (double(n_les) / double(n_fr));
  const int gauss = (flags & 1) ? 0 : 1;
  for (int k = 0; k < nsnap && cx.err == cudaSuccess; ++k) {
    cx.err = cudaMemcpy(Pw, omega_fr + (size_t)k * nf2, nf2 * 8, cudaMemcpyHostToDevice);
    RowDesc r{};
    r.prog = RP_COPY; r.nin = 1; r.nout = 1; r.in_phys = 1; r.phys_in = Pw; r.out[0] = Mf;
    cx.row(F, r);
    ColDesc c = base;
    c.op = CO_FORWARD; c.nfwd = 1; c.fin[0] = Mf; c.w0 = Sw; c.store_w0 = 1; c.zero_mean = 1;
    cx.col(F, c);
    if (cx.err == cudaSuccess) {
      filter_copy_kernel<<<256, 256, 0, cx.st>>>(F.g, (const C2*)Sw, Cg.g, (C2*)Cw, n_les, L / n_les, gauss, sc);
      cx.err = cudaGetLastError();
    }
    ColDesc c2 = base;
    c2.op = CO_DERIVE; c2.w0 = Cw; c2.nder = 1; c2.der[0] = D_W; c2.dout[0] = Mc;
    cx.col(Cg, c2);
    RowDesc r2{};
    r2.prog = RP_COPY; r2.nin = 1; r2.nout = 1; r2.in[0] = Mc; r2.out_phys = 1; r2.phys_out = Pc;
    cx.row(Cg, r2);
    if (cx.err == cudaSuccess) cx.err = cudaMemcpy(omega_les + (size_t)k * nc2, Pc, nc2 * 8, cudaMemcpyDeviceToHost);
  }
  if (cx.err != cudaSuccess) {
    snprintf(msg, sizeof(msg), "qg_grid_filter: %s", cudaGetErrorString(cx.err));
    qg::set_last_error(msg);
    return QG_ERR_CUDA;
  }
  return QG_OK;
}
