"""Discrete adjoint of the oracle's time step (Sec. II-E step, R1-R5), plain FP64.  TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU legs use this module; the
product path never imports it.

The step maps the physical vorticity w_n (a band-limited field) to w_{n+1};
this module gives the vector-Jacobian product of that map: for the gradient
lam_{n+1} of a loss with respect to w_{n+1} it returns lam_n, the gradient
with respect to w_n, and the gradients with respect to the closure constant
and the sponge rate.  Inner products are plain sums over the grid points.

Every operator of the step is a spectral multiplier m(k) between transforms,
a pointwise product, or a projection.  For the sum-over-points inner product
the transpose of a multiplier is its complex conjugate (so i k -> -i k and
real multipliers are their own transposes), the 2/3 truncation and the
mean-mode removal are orthogonal projections (their own transposes), and a
pointwise product by a field is its own transpose.  The transposes are taken
in the reverse order of the forward operations; nonlinear terms are
linearised at the forward fields, recomputed from w_n.

Closures covered: none, Smagorinsky and Leith with a fixed coefficient
C = (c Delta)^p (Eq. 10, 13), and their dynamic forms, whose coefficient
C(w) = max(0, <HM>/<MM>) (Eq. 12, 14) is differentiated through the quotient
(zero gradient where it is clipped).

Parity: pinned by central finite differences of the forward oracle (which is
pinned by its own tests) in every direction the gradients cover.
"""
from __future__ import annotations

import numpy as np

from .qg import (DLEITH, DSMAG, LEITH, NONE, RK3_STAGES, SMAG, Closure, Ops, Params, brinkman_substep,
                 closure_power, explicit_rhs, germano_coefficient, gradient_magnitude, jacobian_hat, project,
                 sgs_divergence_hat, sponge_substep, strain_magnitude, velocity, viscous_substep, vorticity_gradient)

__all__ = ["jac_vjp", "sgs_vjp", "germano_vjp", "rhs_vjp", "full_step_vjp", "ADJOINT_CLOSURES"]

ADJOINT_CLOSURES = (NONE, SMAG, LEITH, DSMAG, DLEITH)


def _multipliers(ops: Ops):
    """Spectral multipliers of w -> u, v, w_x, w_y (psi = -w / |k|^2, u = -psi_y, v = psi_x)."""
    du = 1j * ops.ky * ops.inv_k2
    dv = -1j * ops.kx * ops.inv_k2
    dx = 1j * ops.kx
    dy = 1j * ops.ky
    return du, dv, dx, dy


def _safe_ratio(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    """a / g where g > 0, else 0 (the limits used where the eddy scale g vanishes)."""
    out = np.zeros_like(a)
    nz = g > 0
    out[nz] = a[nz] / g[nz]
    return out


def jac_vjp(ops: Ops, wh: np.ndarray, mu: np.ndarray, U: float) -> np.ndarray:
    """J'(w)^T mu: transpose of the linearised J(psi, w) = T F[u w_x + v w_y] (Eq. 1), physical in and out."""
    a = ops.inv(ops.T * ops.fwd(mu))
    du, dv, dx, dy = _multipliers(ops)
    u, v = velocity(ops, wh, U)
    wx, wy = vorticity_gradient(ops, wh)
    fa = ops.fwd
    # each factor's transpose takes the other factor
    return ops.inv(ops.T * (np.conj(du) * fa(a * wx) + np.conj(dv) * fa(a * wy) + np.conj(dx) * fa(a * u)
                            + np.conj(dy) * fa(a * v)))


def sgs_vjp(ops: Ops, wh: np.ndarray, nu: np.ndarray, kind: int) -> np.ndarray:
    """D'(w)^T nu: transpose of the linearised D(w) = T div(g grad w) (Eq. 9 without C; g of Eq. 10 or 13)."""
    a = ops.inv(ops.T * ops.fwd(nu))
    du, dv, dx, dy = _multipliers(ops)
    wx, wy = vorticity_gradient(ops, wh)
    fa = ops.fwd
    # D = d_x(g w_x) + d_y(g w_y); p, q = the transposed derivatives of a
    p = ops.inv(np.conj(dx) * fa(a))
    q = ops.inv(np.conj(dy) * fa(a))
    s = p * wx + q * wy  # the factor that multiplies the variation of g
    if kind in (LEITH, DLEITH):
        g = gradient_magnitude(ops, wh)
        gx = g * p + _safe_ratio(s * wx, g)  # g = |grad w|: dg = (w_x dw_x + w_y dw_y) / g
        gy = g * q + _safe_ratio(s * wy, g)
        out = np.conj(dx) * fa(gx) + np.conj(dy) * fa(gy)
    else:
        g = strain_magnitude(ops, wh)
        ph = -wh * ops.inv_k2
        psi_xy = ops.inv(-(ops.kx * ops.ky) * ph)
        psi_d = ops.inv(-(ops.kx ** 2 - ops.ky ** 2) * ph)
        dxy = ops.kx * ops.ky * ops.inv_k2          # w -> psi_xy (real)
        dd = (ops.kx ** 2 - ops.ky ** 2) * ops.inv_k2  # w -> psi_xx - psi_yy (real)
        out = np.conj(dx) * fa(g * p) + np.conj(dy) * fa(g * q)
        # |S| = sqrt(4 psi_xy^2 + psi_d^2): d|S| = (4 psi_xy dpsi_xy + psi_d dpsi_d) / |S|
        out = out + dxy * fa(_safe_ratio(4.0 * s * psi_xy, g)) + dd * fa(_safe_ratio(s * psi_d, g))
    return ops.inv(ops.T * out)


def germano_vjp(ops: Ops, wh: np.ndarray, closure: Closure, U: float, C_bar: float) -> np.ndarray:
    """C_bar times the gradient of the dynamic coefficient C(w) = max(0, <HM>/<MM>) (Eq. 11, 12, 14; R8).

    Where C > 0: dC = (sum M dH + sum (H - 2 C M) dM) / (N^2 <MM>), with
    H = J(G w) - G J(w) and M = r^p D(G w) - G D(w) (G the test filter), so
    grad C = (H'^T M + M'^T (H - 2 C M)) / (N^2 <MM>) and
    H'^T m = G J'(G w)^T m - J'(w)^T G m,  M'^T m = r^p G D'(G w)^T m - D'(w)^T G m.
    Where the coefficient is clipped to 0 (or <MM> = 0) the gradient is taken as 0.
    """
    C, hm, mm = germano_coefficient(ops, wh, closure, U)
    if not (C > 0.0 and mm > 0.0):
        return np.zeros((ops.n, ops.n))
    G = ops.test_filter(closure.test_ratio)
    wt = G * wh
    p = closure_power(closure.kind)
    rp = closure.test_ratio ** p
    H = ops.inv(jacobian_hat(ops, wt, U) - G * jacobian_hat(ops, wh, U))
    M = ops.inv(rp * sgs_divergence_hat(ops, wt, closure.kind) - G * sgs_divergence_hat(ops, wh, closure.kind))

    def Gp(f):
        return ops.inv(G * ops.fwd(f))

    nu = H - 2.0 * C * M
    grad = (Gp(jac_vjp(ops, wt, M, U)) - jac_vjp(ops, wh, Gp(M), U)
            + rp * Gp(sgs_vjp(ops, wt, nu, closure.kind)) - sgs_vjp(ops, wh, Gp(nu), closure.kind))
    return C_bar * grad / (ops.n * ops.n * mm)


def rhs_vjp(ops: Ops, wh: np.ndarray, lam: np.ndarray, beta: float, U: float, closure: Closure, C: float):
    """Transpose of the linearised L(w) = -J(psi, w) - beta psi_x + C div(g grad w) (Eq. 1, 9), applied to lam.

    wh: the spectral state at which L is linearised; lam: a physical field;
    C: the coefficient of the static closures (the dynamic ones compute theirs
    from wh, Eq. 12, 14, and differentiate it too).
    Returns (w_bar, C_bar): w_bar the physical field (2/3 band) L'(w)^T lam,
    C_bar = sum over points of lam * div(g grad w) (the derivative in C).
    """
    a = ops.inv(ops.T * ops.fwd(lam))
    w_bar = -jac_vjp(ops, wh, a, U)
    # -beta psi_x = (i beta k_x / |k|^2) w: transpose -i beta k_x / |k|^2
    w_bar = w_bar + ops.inv(ops.T * np.conj(1j * beta * ops.kx * ops.inv_k2) * ops.fwd(a))
    C_bar = 0.0
    if closure.kind != NONE:
        if closure.kind in (DSMAG, DLEITH):
            C = germano_coefficient(ops, wh, closure, U)[0]
        w_bar = w_bar + C * sgs_vjp(ops, wh, a, closure.kind)
        C_bar = float(np.sum(a * ops.inv(sgs_divergence_hat(ops, wh, closure.kind))))
        if closure.kind in (DSMAG, DLEITH):
            w_bar = w_bar + germano_vjp(ops, wh, closure, U, C_bar)
    return w_bar, C_bar


def full_step_vjp(ops: Ops, wh: np.ndarray, lam_next: np.ndarray, beta: float, U: float, closure: Closure,
                  params: Params, chi: np.ndarray | None, chi_s: np.ndarray | None):
    """Transpose of the linearised full step (RK3, viscous factor, Brinkman, sponge, projection) applied to lam_next.

    wh: spectral state w_n (projected); lam_next: physical gradient with respect
    to w_{n+1} = inv(full_step(w_n)).  Returns (lam_n, grads) with lam_n the
    physical gradient with respect to the physical input field (projected as
    the state is: 2/3 band, zero mean) and grads = {"C": dloss/dC per RK stage
    summed, "c": dloss/dc for the static closures, "sponge_rate": dloss/drate}.
    """
    dt = params.dt
    C = 0.0
    if closure.kind in (SMAG, LEITH):
        C = (closure.c * ops.delta) ** closure_power(closure.kind)
    # forward stages, recomputed from w_n
    stages = [wh]
    ws = wh
    for a_s, b_s in RK3_STAGES:
        L_hat, _ = explicit_rhs(ops, ws, beta, U, closure)
        ws = a_s * wh + b_s * (ws + dt * L_hat)
        stages.append(ws)
    w_visc = viscous_substep(ops, stages[3], dt, params.nu, params.mu)
    w_brink = brinkman_substep(ops, w_visc, chi, dt, params.eta, U) if chi is not None else w_visc

    grads = {"C": 0.0, "c": 0.0, "sponge_rate": 0.0}
    # mean removal and truncation of the output
    lam = ops.inv(project(ops, lam_next))
    if chi_s is not None:
        s = np.exp(-params.sponge_rate * chi_s * dt)
        grads["sponge_rate"] = float(np.sum(lam * (-chi_s * dt * s) * ops.inv(w_brink)))
        lam = ops.inv(ops.T * ops.fwd(s * lam))
    if chi is not None:
        # w' = T (d_x (f v) - d_y (f u)), u = U + du w, v = dv w: only the linear part carries a gradient
        du, dv, dx, dy = _multipliers(ops)
        f = np.exp(-chi * dt / params.eta)
        px = ops.inv(np.conj(dx) * ops.fwd(lam))
        py = ops.inv(np.conj(dy) * ops.fwd(lam))
        lam = ops.inv(ops.T * (np.conj(dv) * ops.fwd(f * px) - np.conj(du) * ops.fwd(f * py)))
    lam = ops.inv(ops.T * np.exp(-(params.nu * ops.k2 + params.mu) * dt) * ops.fwd(lam))

    # Shu-Osher stages in reverse: w_{s+1} = a_s w_0 + b_s (w_s + dt L(w_s))
    w0_bar = np.zeros_like(lam)
    lam_s = lam
    for s_idx in (2, 1, 0):
        a_s, b_s = RK3_STAGES[s_idx]
        w0_bar = w0_bar + a_s * lam_s
        rb, cb = rhs_vjp(ops, stages[s_idx], b_s * dt * lam_s, beta, U, closure, C)
        grads["C"] += cb
        lam_s = b_s * lam_s + rb
    w0_bar = w0_bar + lam_s
    lam_n = ops.inv(project(ops, w0_bar))
    if closure.kind in (SMAG, LEITH):
        p = closure_power(closure.kind)
        grads["c"] = grads["C"] * p * closure.c ** (p - 1) * ops.delta ** p
    return lam_n, grads
