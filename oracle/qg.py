"""Plain FP64 CPU oracle of the QG beta-plane LES step.  TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It is written for a reader checking it against the paper by eye:
numpy's FFT is the only library step; every spectral operator is built from
its definition, one array operation per term, in the order of the equations.

Model (Sec. II-A, Eq. 1):  dw/dt + J(psi, w) = nu lap w - mu w - beta psi_x
+ F_obs + F_sponge + Pi,  (u, v) = (-psi_y, psi_x),  w = lap psi, with a
uniform inflow U added to the zeroth Fourier mode of u (Sec. II-D).

Discretisation (Sec. II-C): Fourier pseudo-spectral on an N x N periodic grid
of [0, L)^2, derivatives in Fourier space, products by collocation with the
2/3 rule.  Unnormalised forward DFT, inverse carries 1/N^2 (numpy's
convention).  Spectra use numpy's rfft2 layout: rows k_y in FFT order, columns
k_x = 0 .. N/2.

Readings taken where the paper is silent, ambiguous or garbled (each is also
followed by the CUDA path):

R1  time scheme: SSP-RK3 (Shu-Osher form) for J, beta and the SGS term; then
    the exact viscous/friction factor exp(-(nu|k|^2 + mu) dt); then the exact
    Brinkman sub-step; then the exact sponge sub-step (Lie-Trotter order of
    Sec. II-E: the obstacle equation first, the sponge second).  The paper's
    own AB2CN scheme (Eq. 4) is not this step.
R2  2/3 rule: square truncation T, |m_x|, |m_y| <= K = floor((N-1)/3), applied
    to every product output (Jacobian, SGS fluxes, Brinkman curl, sponge).
R3  mean mode: psi_hat(0) = w_hat(0) = 0; U enters only through u's mean.
R4  Brinkman (Eq. 2, u_obs = 0) exactly: the total velocity is multiplied by
    exp(-chi dt / eta) pointwise, then w_hat = T (i k_x v_hat - i k_y u_hat).
R5  sponge (Eq. 3) exactly, target w_sponge = 0: w <- exp(-rate chi_s dt) w,
    then T.
R6  test filter: sharp spectral, radial, kept iff |m| <= N / (2 r), r = 2.
R7  closure width Delta = L / N of the grid the closure runs on.
R8  Germano/Lilly coefficient (Eq. 11, 12, 14): H and M built with the same
    de-aliased operators as the step, <.> the whole-domain mean, U included
    at both levels, C = max(0, <HM>/<MM>), C = 0 when <MM> = 0 (the
    coefficient is clipped, not H pointwise).  C is recomputed at every RK
    stage from that stage's field.
R9  a priori filter (Eq. 5, garbled): H_G = exp(-k^2 Delta_FF^2 / 6) with the
    square restored, Delta_FF = L / N_c, sharp radial cut-off |k| <= pi /
    Delta_FF, then a spectral copy of the retained modes onto the N_c grid
    (the coarse Nyquist lines dropped).  All coarse-grid quantities of Eq. 8
    are taken in the coarse 2/3 band.  The filter constant (6 vs 24) is
    parity-unpinned.

Parity pins (tests/test_oracle_*.py): brute-force DFT, Parseval, exact
derivatives of trigonometric polynomials, 3/2-rule de-aliasing equivalence,
Jacobian antisymmetry and discrete conservation, single-mode Rossby wave
against the RK3 stability polynomial, viscous decay, penalisation and sponge
exponentials, nu_e >= 0, Germano coefficient against brute-force least
squares, a priori invariances; the eddy-viscosity divergence of Eq. 9 with a
prescribed g (constant g = diffusion, single-mode closed forms), its
enstrophy dissipation by summation by parts and its truncation; the obstacle
and sponge forcings of Eq. 2-3 for constant masks and single-mode closed
forms.  Parity unpinned: the absolute a priori PCC
values of Tab. I/III (need the authors' data) and the Gaussian constant of R9.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "NONE", "SMAG", "LEITH", "DSMAG", "DLEITH",
    "Closure", "Params", "Ops", "QGOracle",
    "project", "to_physical", "streamfunction_hat", "velocity", "vorticity_gradient",
    "strain_magnitude", "gradient_magnitude", "eddy_scale", "sgs_divergence_hat", "closure_power",
    "closure_coefficient", "jacobian_hat", "explicit_rhs", "germano_coefficient", "RK3_STAGES",
    "obstacle_forcing_hat", "sponge_forcing_hat",
    "rk3_step", "viscous_substep", "brinkman_substep", "sponge_substep", "full_step",
    "energy", "enstrophy", "sgs_apriori", "pcc", "apriori_filter",
    "AB2CN", "RK3_EXACT", "AB2History", "ab2cn_step",
]

NONE, SMAG, LEITH, DSMAG, DLEITH = 0, 1, 2, 3, 4


@dataclass
class Closure:
    kind: int = NONE
    c: float = 0.0
    test_ratio: float = 2.0


RK3_EXACT, AB2CN = 0, 1


@dataclass
class Params:
    dt: float = 2e-3
    nu: float = 1.0 / 200.0
    mu: float = 0.0
    eta: float = 1e-3
    sponge_rate: float = 50.0
    scheme: int = RK3_EXACT


class Ops:
    """Wavenumbers and spectral masks of an N x N grid on [0, L)^2 (Sec. II-C)."""

    def __init__(self, n: int, L: float = 2 * math.pi):
        self.n, self.L = n, L
        self.mx = np.arange(n // 2 + 1, dtype=np.float64)[None, :]
        self.my = np.fft.fftfreq(n, 1.0 / n)[:, None]
        scale = 2 * math.pi / L
        self.kx = scale * self.mx
        self.ky = scale * self.my
        self.k2 = self.kx ** 2 + self.ky ** 2
        self.inv_k2 = np.zeros_like(self.k2)
        nz = self.k2 > 0
        self.inv_k2[nz] = 1.0 / self.k2[nz]
        self.K = (n - 1) // 3
        self.T = ((np.abs(self.mx) <= self.K) & (np.abs(self.my) <= self.K)).astype(np.float64)
        self.delta = L / n

    def test_filter(self, ratio: float) -> np.ndarray:
        m2 = self.mx ** 2 + self.my ** 2
        return (m2 * (2.0 * ratio) ** 2 <= float(self.n) ** 2).astype(np.float64)

    def fwd(self, f: np.ndarray) -> np.ndarray:
        return np.fft.rfft2(f)

    def inv(self, fh: np.ndarray) -> np.ndarray:
        return np.fft.irfft2(fh, s=(self.n, self.n))


def project(ops: Ops, omega: np.ndarray) -> np.ndarray:
    """State from a physical field: T F[w] with the mean mode removed (R2, R3)."""
    wh = ops.T * ops.fwd(np.asarray(omega, dtype=np.float64))
    wh[0, 0] = 0.0
    return wh


def to_physical(ops: Ops, wh: np.ndarray) -> np.ndarray:
    return ops.inv(wh)


def streamfunction_hat(ops: Ops, wh: np.ndarray) -> np.ndarray:
    """psi_hat = -w_hat / |k|^2 with psi_hat(0) = 0 (Eq. 1, w = lap psi)."""
    return -wh * ops.inv_k2


def velocity(ops: Ops, wh: np.ndarray, U: float):
    """Physical (u_total, v): u = -psi_y + U, v = psi_x (Eq. 1, Sec. II-D)."""
    ph = streamfunction_hat(ops, wh)
    u = ops.inv(-1j * ops.ky * ph) + U
    v = ops.inv(1j * ops.kx * ph)
    return u, v


def vorticity_gradient(ops: Ops, wh: np.ndarray):
    return ops.inv(1j * ops.kx * wh), ops.inv(1j * ops.ky * wh)


def jacobian_hat(ops: Ops, wh: np.ndarray, U: float) -> np.ndarray:
    """T F[u w_x + v w_y]: the de-aliased advection term J(psi, w) (Eq. 1, Sec. II-C)."""
    u, v = velocity(ops, wh, U)
    wx, wy = vorticity_gradient(ops, wh)
    return ops.T * ops.fwd(u * wx + v * wy)


def strain_magnitude(ops: Ops, wh: np.ndarray) -> np.ndarray:
    """|S| = sqrt(4 psi_xy^2 + (psi_xx - psi_yy)^2) (Eq. 10)."""
    ph = streamfunction_hat(ops, wh)
    psi_xy = ops.inv(-(ops.kx * ops.ky) * ph)
    psi_d = ops.inv(-(ops.kx ** 2 - ops.ky ** 2) * ph)
    return np.sqrt(4.0 * psi_xy ** 2 + psi_d ** 2)


def gradient_magnitude(ops: Ops, wh: np.ndarray) -> np.ndarray:
    """|grad w| = sqrt(w_x^2 + w_y^2) (Eq. 13)."""
    wx, wy = vorticity_gradient(ops, wh)
    return np.sqrt(wx ** 2 + wy ** 2)


def eddy_scale(ops: Ops, wh: np.ndarray, kind: int) -> np.ndarray:
    """The field g in nu_e = C g: |S| for the Smagorinsky family, |grad w| for Leith."""
    if kind in (SMAG, DSMAG):
        return strain_magnitude(ops, wh)
    if kind in (LEITH, DLEITH):
        return gradient_magnitude(ops, wh)
    raise ValueError(kind)


def sgs_divergence_hat(ops: Ops, wh: np.ndarray, kind: int) -> np.ndarray:
    """T F[div(g grad w)]: the eddy-viscosity term of Eq. 9 without its coefficient."""
    g = eddy_scale(ops, wh, kind)
    wx, wy = vorticity_gradient(ops, wh)
    return ops.T * (1j * ops.kx * ops.fwd(g * wx) + 1j * ops.ky * ops.fwd(g * wy))


def closure_power(kind: int) -> int:
    return 2 if kind in (SMAG, DSMAG) else 3


def germano_coefficient(ops: Ops, wh: np.ndarray, closure: Closure, U: float):
    """Dynamic coefficient C = (c Delta)^p by Lilly's least squares (Eq. 11, 12, 14; R8).

    Returns (C, <HM>, <MM>).  H = J(psi~, w~) - (J(psi, w))~ ,
    M = r^p div(g~ grad w~) - (div(g grad w))~ , ~ the test filter (R6).
    """
    G = ops.test_filter(closure.test_ratio)
    wt = G * wh
    H_hat = jacobian_hat(ops, wt, U) - G * jacobian_hat(ops, wh, U)
    p = closure_power(closure.kind)
    M_hat = closure.test_ratio ** p * sgs_divergence_hat(ops, wt, closure.kind) - G * sgs_divergence_hat(ops, wh, closure.kind)
    H = ops.inv(H_hat)
    M = ops.inv(M_hat)
    hm = float(np.mean(H * M))
    mm = float(np.mean(M * M))
    C = max(0.0, hm / mm) if mm > 0.0 else 0.0
    return C, hm, mm


def closure_coefficient(ops: Ops, wh: np.ndarray, closure: Closure, U: float) -> float:
    if closure.kind in (SMAG, LEITH):
        return (closure.c * ops.delta) ** closure_power(closure.kind)
    if closure.kind in (DSMAG, DLEITH):
        return germano_coefficient(ops, wh, closure, U)[0]
    return 0.0


def explicit_rhs(ops: Ops, wh: np.ndarray, beta: float, U: float, closure: Closure):
    """L(w) = -J(psi, w) - beta psi_x + C div(g grad w) (Eq. 1 and 9).

    Returns (L_hat, C).
    """
    ph = streamfunction_hat(ops, wh)
    rhs = -jacobian_hat(ops, wh, U) - beta * (1j * ops.kx * ph)
    C = 0.0
    if closure.kind != NONE:
        C = closure_coefficient(ops, wh, closure, U)
        rhs = rhs + C * sgs_divergence_hat(ops, wh, closure.kind)
    return rhs, C


RK3_STAGES = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def rk3_step(ops: Ops, wh: np.ndarray, dt: float, beta: float, U: float, closure: Closure):
    """Shu-Osher SSP-RK3: w_{s+1} = a_s w_0 + b_s (w_s + dt L(w_s)) (R1).

    Returns (w_3, [C_1, C_2, C_3]).
    """
    w0 = wh
    ws = wh
    coeffs = []
    for a, b in RK3_STAGES:
        L_hat, C = explicit_rhs(ops, ws, beta, U, closure)
        coeffs.append(C)
        ws = a * w0 + b * (ws + dt * L_hat)
    return ws, coeffs


def viscous_substep(ops: Ops, wh: np.ndarray, dt: float, nu: float, mu: float) -> np.ndarray:
    """Exact solution of dw/dt = nu lap w - mu w over dt (Eq. 1 linear terms; R1)."""
    return np.exp(-(nu * ops.k2 + mu) * dt) * wh


def brinkman_substep(ops: Ops, wh: np.ndarray, chi: np.ndarray, dt: float, eta: float, U: float) -> np.ndarray:
    """Exact Brinkman penalisation of the total velocity (Eq. 2 with u_obs = 0; R4)."""
    u, v = velocity(ops, wh, U)
    f = np.exp(-chi * dt / eta)
    u = f * u
    v = f * v
    return ops.T * (1j * ops.kx * ops.fwd(v) - 1j * ops.ky * ops.fwd(u))


def sponge_substep(ops: Ops, wh: np.ndarray, chi_s: np.ndarray, dt: float, rate: float) -> np.ndarray:
    """Exact relaxation of w toward 0 inside the sponge (Eq. 3; R5)."""
    w = ops.inv(wh)
    return ops.T * ops.fwd(np.exp(-rate * chi_s * dt) * w)


def full_step(ops: Ops, wh: np.ndarray, beta: float, U: float, closure: Closure, params: Params,
              chi: np.ndarray | None, chi_s: np.ndarray | None):
    """One step: RK3 explicit part, viscous factor, Brinkman, sponge, mean removal (R1-R5)."""
    w, coeffs = rk3_step(ops, wh, params.dt, beta, U, closure)
    w = viscous_substep(ops, w, params.dt, params.nu, params.mu)
    if chi is not None:
        w = brinkman_substep(ops, w, chi, params.dt, params.eta, U)
    if chi_s is not None:
        w = sponge_substep(ops, w, chi_s, params.dt, params.sponge_rate)
    w = ops.T * w
    w[0, 0] = 0.0
    return w, coeffs


@dataclass
class AB2History:
    """History of the paper's scheme: the explicit terms at the previous step and
    the previous step's intermediate field w** (Sec. II-E, Eq. 4)."""
    E: np.ndarray
    w_star: np.ndarray


def ab2cn_step(ops: Ops, wh: np.ndarray, hist, beta: float, U: float, closure: Closure, params: Params,
               chi, chi_s):
    """One step of the paper's scheme (Sec. II-E, Eq. 4).

    w*   = w^t + dt/2 (nu lap - mu - beta d/dx)(w* + w^t) + dt (3/2 E^t - 1/2 E^{t-1})
           with the explicit terms E = -J(psi, w) + C div(g grad w) - curl(chi u / eta)
           (Crank-Nicolson on the linear terms, AB2 on the Jacobian, the closure and
           the Brinkman forcing; the closure term joins the explicit part in LES);
    w^{t+1} = w* - dt rate chi_s (3/2 w* - 1/2 w**), w** the previous step's w*,
           then the 2/3 truncation and the mean mode set to zero.
    The first step (no history) takes E^{t-1} = E^t and w** = w* (Euler start).
    Returns (w^{t+1}, new history, C).
    """
    dt = params.dt
    E = -jacobian_hat(ops, wh, U)
    C = 0.0
    if closure.kind != NONE:
        C = closure_coefficient(ops, wh, closure, U)
        E = E + C * sgs_divergence_hat(ops, wh, closure.kind)
    if chi is not None:
        u, v = velocity(ops, wh, U)
        E = E - ops.T * (1j * ops.kx * ops.fwd(chi * v) - 1j * ops.ky * ops.fwd(chi * u)) / params.eta
    E_prev = E if hist is None else hist.E
    lin = -(params.nu * ops.k2 + params.mu) + 1j * beta * ops.kx * ops.inv_k2
    w_star = ((1.0 + 0.5 * dt * lin) * wh + dt * (1.5 * E - 0.5 * E_prev)) / (1.0 - 0.5 * dt * lin)
    w_new = w_star
    if chi_s is not None:
        w_ss = w_star if hist is None else hist.w_star
        Z = ops.inv(1.5 * w_star - 0.5 * w_ss)
        w_new = w_star - ops.T * ops.fwd(dt * params.sponge_rate * chi_s * Z)
    w_new = ops.T * w_new
    w_new[0, 0] = 0.0
    return w_new, AB2History(E, w_star), C


def energy(ops: Ops, wh: np.ndarray) -> float:
    """E = <|u'|^2> / 2 of the perturbation velocity (no inflow), physical mean."""
    u, v = velocity(ops, wh, 0.0)
    return 0.5 * float(np.mean(u * u + v * v))


def enstrophy(ops: Ops, wh: np.ndarray) -> float:
    """Z = <w^2> / 2, physical mean."""
    w = ops.inv(wh)
    return 0.5 * float(np.mean(w * w))


class QGOracle:
    """Stateful oracle with the same operations as the C-ABI handle."""

    def __init__(self, n: int, L: float, beta: float, U: float, mask, sponge, closure: Closure, params: Params):
        self.ops = Ops(n, L)
        self.beta, self.U = float(beta), float(U)
        self.chi = None if mask is None else np.asarray(mask, dtype=np.float64).reshape(n, n)
        self.chi_s = None if sponge is None else np.asarray(sponge, dtype=np.float64).reshape(n, n)
        self.closure, self.params = closure, params
        self.wh = np.zeros((n, n // 2 + 1), dtype=np.complex128)
        self.hist = None
        self.t = 0.0
        self.step_count = 0
        self.last_coeff = 0.0

    def set_state(self, omega):
        self.wh = project(self.ops, omega)
        self.hist = None

    def get_state(self) -> np.ndarray:
        return to_physical(self.ops, self.wh)

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            if self.params.scheme == AB2CN:
                self.wh, self.hist, C = ab2cn_step(self.ops, self.wh, self.hist, self.beta, self.U, self.closure,
                                                   self.params, self.chi, self.chi_s)
                self.last_coeff = C
            else:
                self.wh, coeffs = full_step(self.ops, self.wh, self.beta, self.U, self.closure, self.params, self.chi,
                                            self.chi_s)
                self.last_coeff = coeffs[-1]
            self.step_count += 1
            self.t += self.params.dt

    def diagnostics(self) -> dict:
        w = self.get_state()
        return {
            "t": self.t,
            "step": self.step_count,
            "energy": energy(self.ops, self.wh),
            "enstrophy": enstrophy(self.ops, self.wh),
            "coeff": self.last_coeff,
            "max_abs_omega": float(np.max(np.abs(w))),
            "finite": bool(np.all(np.isfinite(w))),
        }


# ----------------------------------------------------------------------------
# A priori SGS analysis (Sec. III, Eq. 5-8 and 15)
# ----------------------------------------------------------------------------

def apriori_filter(ops_f: Ops, fh: np.ndarray, n_c: int, gaussian: bool = True) -> np.ndarray:
    """Grid filter of Eq. 5 (R9): Gaussian x radial cut-off, then spectral copy to N_c.

    Input: a spectrum on the fine grid (rfft2 layout).  Output: the filtered
    field's spectrum on the N_c grid (rfft2 layout), scaled so that the
    coarse inverse transform returns the filtered physical values.
    """
    n_f = ops_f.n
    L = ops_f.L
    d_ff = L / n_c
    k2 = ops_f.k2
    h = np.exp(-k2 * d_ff ** 2 / 6.0) if gaussian else np.ones_like(k2)
    # |k| <= pi / Delta_FF  <=>  |m| <= N_c / 2 for integer wavenumbers m, tested exactly
    m2 = ops_f.mx ** 2 + ops_f.my ** 2
    h = h * (4.0 * m2 <= float(n_c) ** 2)
    fh = fh * h
    out = np.zeros((n_c, n_c // 2 + 1), dtype=np.complex128)
    half = n_c // 2
    # retained k_x = 0 .. half-1, k_y = -(half-1) .. half-1 (coarse Nyquist lines dropped)
    mys = list(range(0, half)) + list(range(-(half - 1), 0))
    for my in mys:
        out[my % n_c, :half] = fh[my % n_f, :half]
    return out * (n_c / n_f) ** 2


def pcc(X: np.ndarray, Y: np.ndarray) -> float:
    """Pearson correlation with population moments over all points (Eq. 15)."""
    x = X - X.mean()
    y = Y - Y.mean()
    return float(np.mean(x * y) / (math.sqrt(np.mean(x * x)) * math.sqrt(np.mean(y * y))))


def obstacle_forcing_hat(ops: Ops, wh: np.ndarray, chi: np.ndarray, eta: float, U: float) -> np.ndarray:
    """T F[F_obs] with F_obs = -curl(chi u / eta), u the total velocity (Eq. 2, u_obs = 0)."""
    u, v = velocity(ops, wh, U)
    return -ops.T * (1j * ops.kx * ops.fwd(chi * v) - 1j * ops.ky * ops.fwd(chi * u)) / eta


def sponge_forcing_hat(ops: Ops, wh: np.ndarray, chi_s: np.ndarray, rate: float) -> np.ndarray:
    """T F[F_sponge] with F_sponge = -rate chi_s (w - 0) (Eq. 3, eta_sponge = 1 / rate)."""
    return -rate * ops.T * ops.fwd(chi_s * ops.inv(wh))


def sgs_apriori(omega_fr, n_les: int, L: float, mask_fr, sponge_fr, closure: Closure, params: Params,
                U: float, beta: float, gaussian: bool = True):
    """Ideal SGS forcing Pi of Eq. 8 on the N_c grid, the closure's Pi model and their PCC.

    Returns (pi_exact, pi_model, parts, pcc) with parts = (Pi_J, Pi_obs, Pi_sponge),
    all physical N_c x N_c arrays.  beta does not enter Pi: its term is linear
    and commutes with the spectral filter.
    """
    omega_fr = np.asarray(omega_fr, dtype=np.float64)
    n_f = omega_fr.shape[0]
    of = Ops(n_f, L)
    oc = Ops(n_les, L)
    wh = project(of, omega_fr)

    def filt(fh):
        return oc.T * apriori_filter(of, fh, n_les, gaussian)

    def filt_coeff(field):
        return oc.inv(apriori_filter(of, of.fwd(field), n_les, gaussian))

    wbar = filt(wh)
    J_bar = filt(jacobian_hat(of, wh, U))
    J_les = jacobian_hat(oc, wbar, U)
    pi_j = oc.inv(J_les - J_bar)
    pi_obs = np.zeros((n_les, n_les))
    pi_sp = np.zeros((n_les, n_les))
    if mask_fr is not None:
        chi = np.asarray(mask_fr, dtype=np.float64).reshape(n_f, n_f)
        Fo_bar = filt(obstacle_forcing_hat(of, wh, chi, params.eta, U))
        Fo_les = obstacle_forcing_hat(oc, wbar, filt_coeff(chi), params.eta, U)
        pi_obs = oc.inv(Fo_bar - Fo_les)
    if sponge_fr is not None:
        chs = np.asarray(sponge_fr, dtype=np.float64).reshape(n_f, n_f)
        Fs_bar = filt(sponge_forcing_hat(of, wh, chs, params.sponge_rate))
        Fs_les = sponge_forcing_hat(oc, wbar, filt_coeff(chs), params.sponge_rate)
        pi_sp = oc.inv(Fs_bar - Fs_les)
    pi_exact = pi_j + pi_obs + pi_sp
    if closure.kind == NONE:
        pi_model = np.zeros((n_les, n_les))
        r = float("nan")
    else:
        C = closure_coefficient(oc, wbar, closure, U)
        pi_model = oc.inv(C * sgs_divergence_hat(oc, wbar, closure.kind))
        r = pcc(pi_exact, pi_model) if C != 0.0 else float("nan")
    return pi_exact, pi_model, (pi_j, pi_obs, pi_sp), r
