// Column pass: one CTA owns W adjacent k_x columns over the whole k_y / y
// range.  It forward y-transforms the mixed arrays produced by a row pass,
// does all spectral-space work of the step for its columns, and inverse
// y-transforms the fields the next row pass needs.
//
// Spectral-space work (Sec. II-A..E, III-A):
//   psi_hat = -w_hat / |k|^2, psi_hat(0) = 0                 (Eq. 1)
//   L = -J_hat - beta i k_x psi_hat + C D_hat                (Eq. 1, 9)
//   D_hat = i k_x F[g w_x] + i k_y F[g w_y]   (i k_x applied by the row pass)
//   SSP-RK3 stage  w_{s+1} = a w_0 + b (w_s + dt L)
//   Germano / Lilly (Eq. 12, 14): H = J~ - G J, M = r^p D~ - G D,
//     partial sums of sum_k w_k Re(H conj M) and w_k |M|^2 (w_k = 1 on k_x = 0,
//     else 2) in FP64 per CTA; C = max(0, <HM>/<MM>) (0 if <MM> = 0)
//   viscous/friction factor exp(-(nu|k|^2 + mu) dt) (exact)
//   Brinkman curl w = i k_x v_hat - i k_y u_hat (Eq. 2)
// Every output is confined to the 2/3 band by construction (only kept modes
// are stored).
#include "fft.cuh"
#include "qg_kernels.h"

namespace qg {

template <typename T> struct InvK2;
template <> struct InvK2<double> {
  __device__ static double get(double ks2, int m2) { return m2 == 0 ? 0.0 : 1.0 / (ks2 * double(m2)); }
};
template <> struct InvK2<float> {
  // the few smallest wavenumbers are inverted in FP64 before rounding
  __device__ static float get(double ks2, int m2) {
    if (m2 == 0) return 0.f;
    if (m2 <= 16) return float(1.0 / (ks2 * double(m2)));
    return 1.f / (float(ks2) * float(m2));
  }
};

template <typename T>
__device__ __forceinline__ cplx_t<T> derive(int code, cplx_t<T> w, int mx, int my, const Geom& g, double ks2,
                                            int test_m2max, T scale, T U) {
  using C = cplx_t<T>;
  const int m2 = mx * mx + my * my;
  if ((code & D_TEST) && m2 > test_m2max) w = mk<C>(T(0), T(0));
  const T kx = T(g.kscale) * T(mx);
  const T ky = T(g.kscale) * T(my);
  const T ik2 = InvK2<T>::get(ks2, m2);
  const C psi = mk<C>(-w.x * ik2, -w.y * ik2);
  C v;
  switch (code & 7) {
    case D_U: v = cmul_ik(psi, -ky); break;
    case D_V: v = cmul_ik(psi, kx); break;
    case D_WX: v = cmul_ik(w, kx); break;
    case D_WY: v = cmul_ik(w, ky); break;
    case D_PXY: v = cscale(psi, -(kx * ky)); break;
    case D_PD: v = cscale(psi, -(kx * kx - ky * ky)); break;
    default: v = w; break;
  }
  v = cscale(v, scale);
  if ((code & 7) == D_U && m2 == 0) v = mk<C>(U, T(0));
  return v;
}

template <typename T> struct ColBound { static constexpr int value = 1024; };
template <> struct ColBound<double> { static constexpr int value = 512; };

template <typename T>
__global__ void __launch_bounds__(ColBound<T>::value) col_kernel(Geom g, FftPlan plan, ColDesc d, const cplx_t<T>* __restrict__ tw, int W) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.n;
  const int Ny = g.Ny;
  C* tile = reinterpret_cast<C*>(smem_raw);  // [N][W]
  C* slotA = tile + (size_t)N * W;          // [W][Ny]
  C* slotB = slotA + (size_t)W * Ny;        // [W][Ny]
  __shared__ double red[2][32];
  const int c0 = blockIdx.x * W;
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  const int nspec = W * Ny;
  const double ks2 = g.kscale * g.kscale;
  // extents for the bounds-checked debug build
  int* const st = d.err;
  const long long n_tile = (long long)N * W, n_mixed = (long long)N * g.IP, n_spec = (long long)g.Kcp * g.SP;
  const long long n_part = 2LL * gridDim.x;  // Germano partial sums: two per column CTA
  (void)n_tile; (void)n_mixed; (void)n_spec; (void)n_part; (void)st;

  if (d.flag) {
    const int stop = __syncthreads_or(*reinterpret_cast<volatile int*>(d.flag) != 0);
    if (stop) return;
  }

  C* w0 = reinterpret_cast<C*>(d.w0);
  C* ws = reinterpret_cast<C*>(d.ws);
  C* jh = reinterpret_cast<C*>(d.jh);
  C* dh = reinterpret_cast<C*>(d.dh);
  const T rpow = T(d.rpow);
  GermanoAcc<T> acc_hm, acc_mm;

  // ---- Phase F: forward y-transforms of the incoming mixed arrays
  for (int f = 0; f < d.nfwd; ++f) {
    const C* src = reinterpret_cast<const C*>(d.fin[f]);
    for (int e = tid; e < N * W; e += nt) {
      const int y = e / W, c = e - y * W;
      QG_ST(tile, e, n_tile, st, QG_LD(src, (long long)y * g.IP + c0 + c, n_mixed, st));
    }
    fft_batched<C>(tile, plan, W, tw, -1, st);
    for (int e = tid; e < nspec; e += nt) {
      const int c = e / Ny, r = e - c * Ny;
      const int mx = c0 + c;
      const int my = my_of_r(g, r);
      C X = QG_LD(tile, (long long)row_of_r(g, r) * W + c, n_tile, st);
      if (mx >= g.Kc) X = mk<C>(T(0), T(0));
      const T ky = T(g.kscale) * T(my);
      const size_t gi = (size_t)mx * g.SP + r;
      switch (d.op) {
        case CO_STAGE_STATIC:
          if (f == 0) QG_ST(slotA, e, nspec, st, mk<C>(-X.x, -X.y));                  // -J
          else if (f == 1) QG_ST(slotB, e, nspec, st, X);                             // i kx F[g wx]
          else QG_ST(slotB, e, nspec, st, cadd(QG_LD(slotB, e, nspec, st), cmul_ik(X, ky)));            // + i ky F[g wy]
          break;
        case CO_DYN_REDUCE: {
          const bool in_test = mx * mx + my * my <= d.test_m2max;
          if (f == 0) {                                              // J
            QG_ST(slotA, e, nspec, st, X);
            QG_ST(jh, gi, n_spec, st, X);
          } else if (f == 1) {                                       // i kx F[g wx]
            QG_ST(slotB, e, nspec, st, X);
          } else if (f == 2) {                                       // D = .. + i ky F[g wy]
            const C D = cadd(QG_LD(slotB, e, nspec, st), cmul_ik(X, ky));
            QG_ST(dh, gi, n_spec, st, D);
            QG_ST(slotB, e, nspec, st, in_test ? mk<C>(-D.x, -D.y) : mk<C>(T(0), T(0)));   // -G D
          } else if (f == 3) {                                       // H = J~ - G J
            QG_ST(slotA, e, nspec, st, in_test ? csub(X, QG_LD(slotA, e, nspec, st)) : X);
          } else if (f == 4) {                                       // M = r^p D~ - G D
            QG_ST(slotB, e, nspec, st, cadd(QG_LD(slotB, e, nspec, st), cscale(X, rpow)));
          } else if (f == 6) {  // Brinkman pair of the paper's scheme: F_obs = (i ky F[chi u] - i kx F[chi v]) / eta
            QG_ST(slotA, e, nspec, st, cscale(cmul_ik(X, ky), T(d.inv_eta)));
          } else if (f == 7) {
            const T kx = T(g.kscale) * T(mx);
            QG_ST(slotA, e, nspec, st, csub(QG_LD(slotA, e, nspec, st), cscale(cmul_ik(X, kx), T(d.inv_eta))));
            QG_ST(reinterpret_cast<C*>(d.bh), gi, n_spec, st, QG_LD(slotA, e, nspec, st));
          } else {
            const C M = cadd(QG_LD(slotB, e, nspec, st), cscale(cmul_ik(X, ky), rpow));
            const C H = QG_LD(slotA, e, nspec, st);
            const T wgt = mx == 0 ? T(1) : T(2);
            if (mx < g.Kc) {
              acc_hm.add_prod(wgt * H.x, M.x);
              acc_hm.add_prod(wgt * H.y, M.y);
              acc_mm.add_prod(wgt * M.x, M.x);
              acc_mm.add_prod(wgt * M.y, M.y);
            }
          }
          break;
        }
        case CO_CURL:
          if (f == 0) QG_ST(slotA, e, nspec, st, X);                                  // u
          else {
            const T kx = T(g.kscale) * T(mx);
            QG_ST(slotA, e, nspec, st, csub(cmul_ik(X, kx), cmul_ik(QG_LD(slotA, e, nspec, st), ky)));  // i kx v - i ky u
          }
          break;
        case CO_AB2CN: {  // E = -J + C D + F_obs: slot A collects -J + F_obs, slot B collects D
          const T kx = T(g.kscale) * T(mx);
          if (f == 0) QG_ST(slotA, e, nspec, st, mk<C>(-X.x, -X.y));
          else if (f < d.nst) QG_ST(slotB, e, nspec, st, (f == 1) ? X : cadd(QG_LD(slotB, e, nspec, st), cmul_ik(X, ky)));
          else if (f == d.nst) QG_ST(slotA, e, nspec, st, cadd(QG_LD(slotA, e, nspec, st), cscale(cmul_ik(X, ky), T(d.inv_eta))));
          else QG_ST(slotA, e, nspec, st, csub(QG_LD(slotA, e, nspec, st), cscale(cmul_ik(X, kx), T(d.inv_eta))));
          break;
        }
        case CO_FORWARD2:
          if (f == 0) QG_ST(slotA, e, nspec, st, X);
          else QG_ST(slotB, e, nspec, st, X);
          break;
        case CO_FORWARD_N:  // field f's band straight to its own spectral array
          if (mx < g.Kc)
            QG_ST(reinterpret_cast<C*>(d.fout[f]), gi, n_spec, st,
                  (d.zero_mean && mx == 0 && my == 0) ? mk<C>(T(0), T(0)) : X);
          break;
        default:  // CO_FORWARD
          QG_ST(slotA, e, nspec, st, X);
          break;
      }
    }
    __syncthreads();
  }

  if (d.op == CO_FORWARD_N) return;  // every field's band is stored
  if (d.op == CO_DYN_REDUCE) {
    // deterministic block reduction of the Germano partial sums
    double hm = acc_hm.value(), mm = acc_mm.value();
    for (int o = 16; o > 0; o >>= 1) {
      hm += __shfl_down_sync(0xffffffffu, hm, o);
      mm += __shfl_down_sync(0xffffffffu, mm, o);
    }
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) {
      red[0][wid] = hm;
      red[1][wid] = mm;
    }
    __syncthreads();
    if (wid == 0) {
      const int nw = (nt + 31) >> 5;
      hm = lane < nw ? red[0][lane] : 0.0;
      mm = lane < nw ? red[1][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        hm += __shfl_down_sync(0xffffffffu, hm, o);
        mm += __shfl_down_sync(0xffffffffu, mm, o);
      }
      if (lane == 0) {
        QG_ST(d.partials, 2LL * blockIdx.x, n_part, st, hm);
        QG_ST(d.partials, 2LL * blockIdx.x + 1, n_part, st, mm);
      }
    }
    return;
  }

  // ---- coefficient of the dynamic closures from the partial sums (same order in every CTA)
  T coeff = T(d.coeff);
  if (d.op == CO_DYN_COMBINE || d.op == CO_AB2CN_COMBINE) {
    if (tid < 32) {
      double a = 0.0, b = 0.0;
      for (int i = tid; i < d.npartials; i += 32) {
        a += QG_LD(d.partials, 2LL * i, n_part, st);
        b += QG_LD(d.partials, 2LL * i + 1, n_part, st);
      }
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (tid == 0) {
        const double C = b > 0.0 ? fmax(0.0, a / b) : 0.0;
        red[0][0] = C;
        if (blockIdx.x == 0 && d.coeff_out) *d.coeff_out = C;
      }
    }
    __syncthreads();
    coeff = T(red[0][0]);
  }

  // ---- Phase S: new vorticity spectrum for the owned columns
  const T dt = T(d.dt), a_rk = T(d.a), b_rk = T(d.b), beta = T(d.beta);
  const T* vx = reinterpret_cast<const T*>(d.visc_x);
  const T* vy = reinterpret_cast<const T*>(d.visc_y);
  const T vmu = T(d.visc_mu);
  for (int e = tid; e < nspec; e += nt) {
    const int c = e / Ny, r = e - c * Ny;
    const int mx = c0 + c;
    const int my = my_of_r(g, r);
    const size_t gi = (size_t)mx * g.SP + r;
    C wn = mk<C>(T(0), T(0));
    if (mx < g.Kc) {
      switch (d.op) {
        case CO_DERIVE:
          wn = QG_LD(w0, gi, n_spec, st);
          break;
        case CO_STAGE_STATIC:
        case CO_DYN_COMBINE: {
          const C wz = QG_LD(w0, gi, n_spec, st);
          const C wst = d.use_ws ? QG_LD(ws, gi, n_spec, st) : wz;
          const T ik2 = InvK2<T>::get(ks2, mx * mx + my * my);
          const C psi = mk<C>(-wst.x * ik2, -wst.y * ik2);
          const T kx = T(g.kscale) * T(mx);
          const C bv = cscale(cmul_ik(psi, kx), beta);
          C L;
          if (d.op == CO_STAGE_STATIC) {
            L = csub(QG_LD(slotA, e, nspec, st), bv);
            if (d.nfwd > 1) L = cadd(L, cscale(QG_LD(slotB, e, nspec, st), coeff));
          } else {
            const C J = QG_LD(jh, gi, n_spec, st);
            L = csub(mk<C>(-J.x, -J.y), bv);
            L = cadd(L, cscale(QG_LD(dh, gi, n_spec, st), coeff));
          }
          const C inner = cadd(wst, cscale(L, dt));
          wn = cadd(cscale(wz, a_rk), cscale(inner, b_rk));
          break;
        }
        case CO_AB2CN:
        case CO_AB2CN_COMBINE: {
          // Eq. 4: w* = ((1 + dt/2 lin) w^t + dt (3/2 E - 1/2 E_prev)) / (1 - dt/2 lin)
          C E;
          if (d.op == CO_AB2CN) {
            E = (d.nst > 1) ? cadd(QG_LD(slotA, e, nspec, st), cscale(QG_LD(slotB, e, nspec, st), coeff)) : QG_LD(slotA, e, nspec, st);
          } else {
            const C J = QG_LD(jh, gi, n_spec, st);
            E = cadd(mk<C>(-J.x, -J.y), cscale(QG_LD(dh, gi, n_spec, st), coeff));
            if (d.brink) E = cadd(E, QG_LD(reinterpret_cast<const C*>(d.bh), gi, n_spec, st));
          }
          C* ep = reinterpret_cast<C*>(d.eprev);
          const C Ep = d.ab2_first ? E : QG_LD(ep, gi, n_spec, st);
          QG_ST(ep, gi, n_spec, st, E);
          const int m2 = mx * mx + my * my;
          const T k2 = T(ks2) * T(m2);
          const T ik2 = InvK2<T>::get(ks2, m2);
          const T kx = T(g.kscale) * T(mx);
          const T hdt = T(0.5) * dt;
          const T lre = -(T(d.nu) * k2 + T(d.mu));
          const T lim = beta * kx * ik2;
          const C wz = QG_LD(w0, gi, n_spec, st);
          const C ab = mk<C>(T(1.5) * E.x - T(0.5) * Ep.x, T(1.5) * E.y - T(0.5) * Ep.y);
          const C num = cadd(cmul(mk<C>(T(1) + hdt * lre, hdt * lim), wz), cscale(ab, dt));
          const T dre = T(1) - hdt * lre, dim = -hdt * lim;
          const T den = dre * dre + dim * dim;
          const C wst = mk<C>((num.x * dre + num.y * dim) / den, (num.y * dre - num.x * dim) / den);
          if (d.sponge_next) {
            C* wsp = reinterpret_cast<C*>(d.wss);
            const C wss = d.ab2_first ? wst : QG_LD(wsp, gi, n_spec, st);
            QG_ST(wsp, gi, n_spec, st, wst);
            wn = mk<C>(T(1.5) * wst.x - T(0.5) * wss.x, T(1.5) * wst.y - T(0.5) * wss.y);
          } else {
            wn = wst;
          }
          break;
        }
        case CO_AB2CN_FINAL:
          wn = csub(QG_LD(reinterpret_cast<const C*>(d.wss), gi, n_spec, st), QG_LD(slotA, e, nspec, st));
          break;
        default:  // CO_CURL, CO_FORWARD, CO_FORWARD2
          wn = QG_LD(slotA, e, nspec, st);
          break;
      }
      if (d.viscous) wn = cscale(wn, QG_LD(vx, mx, g.Kcp, st) * QG_LD(vy, r, g.SP, st) * vmu);
      if (d.zero_mean && mx == 0 && my == 0) wn = mk<C>(T(0), T(0));
      if (d.store_ws) QG_ST(reinterpret_cast<C*>(d.ws_out), gi, n_spec, st, wn);
      if (d.store_w0) QG_ST(w0, gi, n_spec, st, wn);
      if (d.op == CO_FORWARD2) {  // the second field, treated like the first
        C wb = QG_LD(slotB, e, nspec, st);
        if (d.viscous) wb = cscale(wb, QG_LD(vx, mx, g.Kcp, st) * QG_LD(vy, r, g.SP, st) * vmu);
        if (d.zero_mean && mx == 0 && my == 0) wb = mk<C>(T(0), T(0));
        QG_ST(reinterpret_cast<C*>(d.w0b), gi, n_spec, st, wb);
      }
    }
    QG_ST(slotA, e, nspec, st, wn);
  }
  __syncthreads();

  // ---- Phase I: derived fields, inverse y-transforms, mixed arrays out
  const T scale = T(1.0 / (double(N) * double(N)));
  const T U = T(d.U);
  for (int q = 0; q < d.nder; ++q) {
    const int code = d.der[q];
    for (int e = tid; e < N * W; e += nt) {
      const int row = e / W, c = e - row * W;
      const int mx = c0 + c;
      C v = mk<C>(T(0), T(0));
      int r = -1;
      if (row <= g.K) r = row;
      else if (row >= N - g.K) r = row - N + Ny;
      if (r >= 0 && mx < g.Kc) v = derive<T>(code, QG_LD(slotA, (long long)c * Ny + r, nspec, st), mx, my_of_r(g, r), g, ks2, d.test_m2max, scale, U);
      QG_ST(tile, e, n_tile, st, v);
    }
    fft_batched<C>(tile, plan, W, tw, +1, st);
    C* dst = reinterpret_cast<C*>(d.dout[q]);
    for (int e = tid; e < N * W; e += nt) {
      const int y = e / W, c = e - y * W;
      QG_ST(dst, (long long)y * g.IP + c0 + c, n_mixed, st, QG_LD(tile, e, n_tile, st));
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_col(const Geom& g, const FftPlan& plan, const ColDesc& d, const void* tw, int W, int threads,
                       size_t smem, cudaStream_t st) {
  auto k = col_kernel<T>;
  cudaError_t e = raise_smem_limit<col_kernel<T>>(smem);
  if (e != cudaSuccess) return e;
  k<<<g.Kcp / W, threads, smem, st>>>(g, plan, d, reinterpret_cast<const cplx_t<T>*>(tw), W);
  return cudaGetLastError();
}

template cudaError_t launch_col<float>(const Geom&, const FftPlan&, const ColDesc&, const void*, int, int, size_t, cudaStream_t);
template cudaError_t launch_col<double>(const Geom&, const FftPlan&, const ColDesc&, const void*, int, int, size_t, cudaStream_t);

}  // namespace qg
