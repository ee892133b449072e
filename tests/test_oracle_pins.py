"""Pins that tie the FP64 oracle to closed forms, brute force and exact invariants.

Each test names the part of the paper it checks.  None of them compares the
oracle with itself through the same formula: expected values come from
analytic solutions, an independent de-aliasing route (3/2-rule zero padding),
the RK3 stability polynomial, ODE sub-cycling, or a least-squares solve.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import init_field, island_mask, sponge_mask


def grid(n, L=2 * math.pi):
    x = np.arange(n) * (L / n)
    return x[None, :], x[:, None]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------------
# Derivatives, inversion (Eq. 1, Sec. II-C)
# --------------------------------------------------------------------------

def test_spectral_derivatives_and_inversion_exact():
    n, L = 32, 2 * math.pi
    ops = O.Ops(n, L)
    X, Y = grid(n, L)
    # psi = sin(3x) cos(2y) + 0.5 cos(x + 4y)
    psi = np.sin(3 * X) * np.cos(2 * Y) + 0.5 * np.cos(X + 4 * Y)
    w = -13 * np.sin(3 * X) * np.cos(2 * Y) - 0.5 * 17 * np.cos(X + 4 * Y)
    wh = O.project(ops, w)
    ph = O.streamfunction_hat(ops, wh)
    assert np.max(np.abs(ops.inv(ph) - psi)) < 1e-13
    u, v = O.velocity(ops, wh, 0.3)
    u_ref = 2 * np.sin(3 * X) * np.sin(2 * Y) + 0.5 * 4 * np.sin(X + 4 * Y) + 0.3
    v_ref = 3 * np.cos(3 * X) * np.cos(2 * Y) - 0.5 * np.sin(X + 4 * Y)
    assert np.max(np.abs(u - u_ref)) < 1e-13
    assert np.max(np.abs(v - v_ref)) < 1e-13
    wx, wy = O.vorticity_gradient(ops, wh)
    wx_ref = -39 * np.cos(3 * X) * np.cos(2 * Y) + 0.5 * 17 * np.sin(X + 4 * Y)
    wy_ref = 26 * np.sin(3 * X) * np.sin(2 * Y) + 0.5 * 17 * 4 * np.sin(X + 4 * Y)
    assert np.max(np.abs(wx - wx_ref)) < 1e-12
    assert np.max(np.abs(wy - wy_ref)) < 1e-12


def test_strain_and_gradient_magnitude_closed_form():
    n = 32
    ops = O.Ops(n)
    X, Y = grid(n)
    # psi = sin(x) sin(2y): psi_xy = 2 cos x cos 2y, psi_xx - psi_yy = 3 sin x sin 2y
    w = -5 * np.sin(X) * np.sin(2 * Y)
    wh = O.project(ops, w)
    S = O.strain_magnitude(ops, wh)
    S_ref = np.sqrt(4 * (2 * np.cos(X) * np.cos(2 * Y)) ** 2 + (3 * np.sin(X) * np.sin(2 * Y)) ** 2)
    assert np.max(np.abs(S - S_ref)) < 1e-12
    G = O.gradient_magnitude(ops, wh)
    G_ref = 5 * np.sqrt(np.cos(X) ** 2 * np.sin(2 * Y) ** 2 + 4 * np.sin(X) ** 2 * np.cos(2 * Y) ** 2)
    assert np.max(np.abs(G - G_ref)) < 1e-12


# --------------------------------------------------------------------------
# Jacobian and 2/3 de-aliasing (Eq. 1, Sec. II-C)
# --------------------------------------------------------------------------

def test_jacobian_closed_form_two_modes():
    n = 16
    ops = O.Ops(n)
    X, Y = grid(n)
    A, B, U = 0.7, -1.3, 0.4
    # psi = A cos x + B sin 2y -> J = u w_x + v w_y = 6AB sin x cos 2y (+ U A sin x)
    w = -A * np.cos(X) - 4 * B * np.sin(2 * Y)
    J = ops.inv(O.jacobian_hat(ops, O.project(ops, w), U))
    J_ref = 6 * A * B * np.sin(X) * np.cos(2 * Y) + U * A * np.sin(X)
    assert np.max(np.abs(J - J_ref)) < 1e-13


def test_single_mode_jacobian_vanishes():
    n = 24
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.cos(3 * X + 4 * Y) + 0.4 * np.sin(5 * X)  # |k| = 5 for both
    J = ops.inv(O.jacobian_hat(ops, O.project(ops, w), 0.0))
    assert np.max(np.abs(J)) < 1e-12


def _jacobian_three_halves(n, wh, U):
    """J(psi, w) by zero padding to a 3N/2 grid, then truncation to the 2/3 band."""
    m = 3 * n // 2
    ky = np.fft.fftfreq(n, 1.0 / n)
    kx = np.arange(n // 2 + 1)
    K = (n - 1) // 3
    full = np.zeros((m, m // 2 + 1), dtype=np.complex128)

    def pad(fh):
        out = np.zeros_like(full)
        for j, my in enumerate(ky.astype(int)):
            if abs(my) <= K:
                out[my % m, : K + 1] = fh[j, : K + 1]
        return out * (m / n) ** 2

    KX = np.arange(m // 2 + 1)[None, :].astype(float)
    KY = np.fft.fftfreq(m, 1.0 / m)[:, None]
    K2 = KX ** 2 + KY ** 2
    inv = np.where(K2 > 0, 1.0 / np.where(K2 > 0, K2, 1), 0.0)
    W = pad(wh)
    P = -W * inv
    u = np.fft.irfft2(-1j * KY * P, s=(m, m)) + U
    v = np.fft.irfft2(1j * KX * P, s=(m, m))
    wx = np.fft.irfft2(1j * KX * W, s=(m, m))
    wy = np.fft.irfft2(1j * KY * W, s=(m, m))
    Jm = np.fft.rfft2(u * wx + v * wy) * (n / m) ** 2
    out = np.zeros_like(wh)
    for j, my in enumerate(ky.astype(int)):
        if abs(my) <= K:
            out[j, : K + 1] = Jm[my % m, : K + 1]
    return out


@pytest.mark.parametrize("n", [16, 24, 48])
def test_two_thirds_equals_three_halves(n):
    ops = O.Ops(n)
    wh = O.project(ops, init_field(3, n))
    a = O.jacobian_hat(ops, wh, 0.6)
    b = _jacobian_three_halves(n, wh, 0.6)
    assert rel(a, b) < 1e-13


@pytest.mark.parametrize("U", [0.0, 0.8])
def test_discrete_conservation_of_truncated_jacobian(U):
    n = 48
    ops = O.Ops(n)
    wh = O.project(ops, init_field(11, n))
    J = O.jacobian_hat(ops, wh, U)
    ph = O.streamfunction_hat(ops, wh)
    w = np.full(wh.shape, 2.0)
    w[:, 0] = 1.0
    scale = np.sqrt(np.sum(w * np.abs(J) ** 2) * np.sum(w * np.abs(wh) ** 2))
    e_rate = np.sum(w * (np.conj(ph) * J).real)
    z_rate = np.sum(w * (np.conj(wh) * J).real)
    assert abs(z_rate) < 1e-13 * scale
    scale_p = np.sqrt(np.sum(w * np.abs(J) ** 2) * np.sum(w * np.abs(ph) ** 2))
    assert abs(e_rate) < 1e-13 * scale_p


# --------------------------------------------------------------------------
# Time stepping: Rossby wave, viscous decay, conservation (Eq. 1, R1)
# --------------------------------------------------------------------------

def rk3_poly(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


@pytest.mark.parametrize("mode", [(2, 3), (1, -4), (5, 0)])
def test_single_mode_rossby_wave_equals_rk3_polynomial(mode):
    n, beta, U, dt, nsteps = 32, 5.0, 0.5, 2e-3, 50
    mx, my = mode
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.cos(mx * X + my * Y + 0.3)
    wh = O.project(ops, w)
    w0 = wh.copy()
    for _ in range(nsteps):
        wh, _ = O.full_step(ops, wh, beta, U, O.Closure(O.NONE), O.Params(dt=dt, nu=0.0, mu=0.0), None, None)
    k2 = mx * mx + my * my
    lam = 1j * mx * (beta / k2 - U)
    expected = w0 * rk3_poly(dt * lam) ** nsteps
    assert rel(wh, expected) < 1e-13
    # and within O(dt^3) of the exact dispersion relation sigma = -beta k_x/|k|^2 (U = 0 case in lam)
    exact = w0 * np.exp(lam * dt * nsteps)
    assert rel(wh, exact) < 1e-6


def test_rossby_wave_observed_order_three():
    n, beta, T = 16, 20.0, 0.4
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.cos(X + 2 * Y)
    lam = 1j * 1 * (beta / 5.0)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        wh = O.project(ops, w)
        w0 = wh.copy()
        for _ in range(int(round(T / dt))):
            wh, _ = O.full_step(ops, wh, beta, 0.0, O.Closure(O.NONE), O.Params(dt=dt, nu=0.0), None, None)
        errs.append(rel(wh, w0 * np.exp(lam * T)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.8 < p < 3.2 for p in orders), orders


def test_viscous_decay_exact():
    n, nu, mu, dt, nsteps = 32, 0.05, 0.2, 1e-2, 40
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.sin(4 * X - 3 * Y)
    wh = O.project(ops, w)
    for _ in range(nsteps):
        wh, _ = O.full_step(ops, wh, 0.0, 0.0, O.Closure(O.NONE), O.Params(dt=dt, nu=nu, mu=mu), None, None)
    expected = w * math.exp(-(nu * 25 + mu) * dt * nsteps)
    assert np.max(np.abs(ops.inv(wh) - expected)) < 1e-14


def test_inviscid_invariants_rates_vanish():
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(5, n))
    L, _ = O.explicit_rhs(ops, wh, 7.0, 0.0, O.Closure(O.NONE))
    ph = O.streamfunction_hat(ops, wh)
    w = np.full(wh.shape, 2.0)
    w[:, 0] = 1.0
    dZ = np.sum(w * (np.conj(wh) * L).real)
    dE = -np.sum(w * (np.conj(ph) * L).real)
    ref = np.sqrt(np.sum(w * np.abs(wh) ** 2) * np.sum(w * np.abs(L) ** 2))
    assert abs(dZ) < 1e-13 * ref
    assert abs(dE) < 1e-13 * ref


def test_energy_enstrophy_drift_is_third_order():
    n, T = 32, 0.5
    ops = O.Ops(n)
    w_init = init_field(2, n)
    drifts = []
    for dt in (0.02, 0.01):
        wh = O.project(ops, w_init)
        Z0 = O.enstrophy(ops, wh)
        for _ in range(int(round(T / dt))):
            wh, _ = O.full_step(ops, wh, 3.0, 0.0, O.Closure(O.NONE), O.Params(dt=dt, nu=0.0), None, None)
        drifts.append(abs(O.enstrophy(ops, wh) - Z0) / Z0)
    p = math.log2(drifts[0] / drifts[1])
    assert 2.5 < p < 4.5, (drifts, p)


# --------------------------------------------------------------------------
# Penalisation and sponge (Eq. 2, 3; R4, R5)
# --------------------------------------------------------------------------

def test_constant_mask_brinkman_is_exact_exponential():
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(4, n))
    c, dt, eta = 0.37, 2e-3, 1e-3
    out = O.brinkman_substep(ops, wh, np.full((n, n), c), dt, eta, U=0.9)
    assert rel(out, wh * math.exp(-c * dt / eta)) < 1e-14


def test_brinkman_matches_subcycled_rk4_velocity():
    n = 24
    ops = O.Ops(n)
    wh = O.project(ops, init_field(8, n))
    chi = island_mask(n, radius=1.0)
    dt, eta, U = 2e-3, 1e-3, 0.5
    u, v = O.velocity(ops, wh, U)
    # integrate du/dt = -chi u / eta with RK4, 1e4 sub-steps, independent of the exponential
    h = dt / 10000
    a = -chi / eta
    for _ in range(10000):
        k1u, k1v = a * u, a * v
        k2u, k2v = a * (u + 0.5 * h * k1u), a * (v + 0.5 * h * k1v)
        k3u, k3v = a * (u + 0.5 * h * k2u), a * (v + 0.5 * h * k2v)
        k4u, k4v = a * (u + h * k3u), a * (v + h * k3v)
        u = u + h / 6 * (k1u + 2 * k2u + 2 * k3u + k4u)
        v = v + h / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
    # curl, truncated, computed here with explicit wavenumbers
    mx = np.arange(n // 2 + 1)[None, :]
    my = np.fft.fftfreq(n, 1.0 / n)[:, None]
    K = (n - 1) // 3
    T = (np.abs(mx) <= K) & (np.abs(my) <= K)
    ref = T * (1j * mx * np.fft.rfft2(v) - 1j * my * np.fft.rfft2(u))
    out = O.brinkman_substep(ops, wh, chi, dt, eta, U)
    assert rel(out, ref) < 1e-10


def test_sponge_unit_mask_exact():
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(9, n))
    out = O.sponge_substep(ops, wh, np.ones((n, n)), 2e-3, 50.0)
    assert rel(out, wh * math.exp(-50.0 * 2e-3)) < 1e-14


# --------------------------------------------------------------------------
# Closures (Eq. 9-14; R6-R8)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [O.SMAG, O.LEITH])
def test_eddy_viscosity_nonnegative(kind):
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(12, n))
    assert np.all(O.eddy_scale(ops, wh, kind) >= 0)


@pytest.mark.parametrize("kind", [O.DSMAG, O.DLEITH])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_germano_is_least_squares_and_nonnegative(kind, seed):
    n = 16
    ops = O.Ops(n)
    wh = O.project(ops, init_field(seed, n, k_peak=3.0))
    cl = O.Closure(kind, test_ratio=2.0)
    C, hm, mm = O.germano_coefficient(ops, wh, cl, 0.5)
    assert C >= 0.0
    # rebuild H and M on the grid and solve the 256 x 1 least-squares system directly
    G = ops.test_filter(2.0)
    wt = G * wh
    p = O.closure_power(kind)
    H = ops.inv(O.jacobian_hat(ops, wt, 0.5) - G * O.jacobian_hat(ops, wh, 0.5)).ravel()
    M = ops.inv(2.0 ** p * O.sgs_divergence_hat(ops, wt, kind) - G * O.sgs_divergence_hat(ops, wh, kind)).ravel()
    c_ls = np.linalg.lstsq(M[:, None], H, rcond=None)[0][0]
    assert abs(hm / mm - c_ls) < 1e-12 * max(1.0, abs(c_ls))
    # dense scan + golden section on the residual
    f = lambda c: np.sum((H - c * M) ** 2)
    grid_c = np.linspace(c_ls - 10 * abs(c_ls) - 1, c_ls + 10 * abs(c_ls) + 1, 2001)
    c0 = grid_c[np.argmin([f(c) for c in grid_c])]
    a, b = c0 - (grid_c[1] - grid_c[0]), c0 + (grid_c[1] - grid_c[0])
    g = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        c1, c2 = b - g * (b - a), a + g * (b - a)
        if f(c1) < f(c2):
            b = c2
        else:
            a = c1
    assert abs(0.5 * (a + b) - c_ls) < 1e-6 * max(1.0, abs(c_ls))
    assert C == (max(0.0, c_ls) if mm > 0 else 0.0) or abs(C - max(0.0, c_ls)) < 1e-12 * max(1.0, abs(c_ls))
    # physical mean equals the Parseval sum over the half spectrum
    Hh = np.fft.rfft2(H.reshape(n, n))
    Mh = np.fft.rfft2(M.reshape(n, n))
    w = np.full(Hh.shape, 2.0)
    w[:, 0] = 1.0
    w[:, -1] = 1.0
    assert abs(np.sum(w * (Hh * np.conj(Mh)).real) / n ** 4 - hm) < 1e-12 * math.sqrt(hm * hm + mm * mm)


@pytest.mark.parametrize("kind", [O.DSMAG, O.DLEITH])
def test_germano_closed_form_for_test_filter_invariant_field(kind):
    """Field band-limited inside the test filter: w~ = w, so H = (1-G)J and
    M = r^p (1-G)D + (r^p - 1) G D; the projections are orthogonal, giving
    <HM> = r^p |(1-G)J . (1-G)D| and <MM> = r^2p |(1-G)D|^2 + (r^p-1)^2 |GD|^2."""
    n = 48
    ops = O.Ops(n)
    G = ops.test_filter(2.0)
    wh = G * O.project(ops, init_field(21, n, k_peak=4.0))
    J = O.jacobian_hat(ops, wh, 0.3)
    D = O.sgs_divergence_hat(ops, wh, kind)
    p = O.closure_power(kind)
    r = 2.0 ** p

    def mean(a, b):
        return float(np.mean(ops.inv(a) * ops.inv(b)))

    hm_ref = r * mean((1 - G) * J, (1 - G) * D)
    mm_ref = r * r * mean((1 - G) * D, (1 - G) * D) + (r - 1) ** 2 * mean(G * D, G * D)
    C, hm, mm = O.germano_coefficient(ops, wh, O.Closure(kind), 0.3)
    assert abs(hm - hm_ref) < 1e-12 * math.sqrt(hm_ref ** 2 + mm_ref ** 2)
    assert abs(mm - mm_ref) < 1e-12 * mm_ref


def test_germano_H_independent_of_inflow_and_single_mode_zero():
    n = 16
    ops = O.Ops(n)
    wh = O.project(ops, init_field(1, n, k_peak=3.0))
    G = ops.test_filter(2.0)
    H0 = O.jacobian_hat(ops, G * wh, 0.0) - G * O.jacobian_hat(ops, wh, 0.0)
    H1 = O.jacobian_hat(ops, G * wh, 0.9) - G * O.jacobian_hat(ops, wh, 0.9)
    assert np.max(np.abs(H0 - H1)) < 1e-12 * np.max(np.abs(H0))
    X, Y = grid(n)
    single = O.project(ops, np.cos(X + 2 * Y))
    C, hm, mm = O.germano_coefficient(ops, single, O.Closure(O.DLEITH), 0.0)
    assert abs(hm) < 1e-14 * mm and C < 1e-12


def test_static_coefficient_values():
    ops = O.Ops(64, L=2 * math.pi)
    wh = O.project(ops, init_field(0, 64))
    d = 2 * math.pi / 64
    assert O.closure_coefficient(ops, wh, O.Closure(O.SMAG, c=0.17), 0) == pytest.approx((0.17 * d) ** 2, rel=1e-15)
    assert O.closure_coefficient(ops, wh, O.Closure(O.LEITH, c=0.25), 0) == pytest.approx((0.25 * d) ** 3, rel=1e-15)


# --------------------------------------------------------------------------
# Diagnostics and a full step
# --------------------------------------------------------------------------

def test_energy_enstrophy_parseval_forms():
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(6, n))
    w = np.full(wh.shape, 2.0)
    w[:, 0] = 1.0
    k2 = ops.k2
    E = np.sum(w * k2 * np.abs(wh * ops.inv_k2) ** 2) / (2 * n ** 4)
    Z = np.sum(w * np.abs(wh) ** 2) / (2 * n ** 4)
    assert O.energy(ops, wh) == pytest.approx(E, rel=1e-13)
    assert O.enstrophy(ops, wh) == pytest.approx(Z, rel=1e-13)


def test_full_step_keeps_band_and_zero_mean():
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(0, n))
    chi = island_mask(n, radius=0.6)
    chs = sponge_mask(n)
    out, coeffs = O.full_step(ops, wh, 5.0, 0.5, O.Closure(O.DSMAG), O.Params(), chi, chs)
    assert out[0, 0] == 0
    assert np.all(out[ops.T == 0] == 0)
    assert all(c >= 0 for c in coeffs)
    assert np.all(np.isfinite(out))


# --------------------------------------------------------------------------
# A priori analysis (Eq. 5-8, 15)
# --------------------------------------------------------------------------

def _bandlimited_mask(n):
    X, Y = grid(n)
    return np.broadcast_to(0.5 + 0.25 * np.cos(X) * np.cos(2 * Y) + 0.1 * np.sin(3 * X), (n, n)).copy()


def test_apriori_identity_filter_gives_zero_pi():
    n = 32
    w = init_field(3, n)
    chi = _bandlimited_mask(n)
    X, Y = grid(n)
    chs = np.broadcast_to(0.3 + 0.2 * np.cos(X), (n, n)).copy()
    pe, pm, parts, r = O.sgs_apriori(w, n, 2 * math.pi, chi, chs, O.Closure(O.SMAG, c=0.17), O.Params(), 0.5, 5.0, gaussian=False)
    scale = np.max(np.abs(O.Ops(n).inv(O.jacobian_hat(O.Ops(n), O.project(O.Ops(n), w), 0.5))))
    assert np.max(np.abs(pe)) < 1e-11 * scale


@pytest.mark.parametrize("pair", [(O.SMAG, O.DSMAG), (O.LEITH, O.DLEITH)])
def test_apriori_pcc_independent_of_coefficient(pair):
    n_f, n_c = 64, 32
    w = init_field(4, n_f, k_peak=6.0)
    chi = island_mask(n_f, radius=0.8)
    chs = sponge_mask(n_f)
    static, dyn = pair
    out_s = O.sgs_apriori(w, n_c, 2 * math.pi, chi, chs, O.Closure(static, c=0.2), O.Params(), 0.5, 5.0)
    out_d = O.sgs_apriori(w, n_c, 2 * math.pi, chi, chs, O.Closure(dyn), O.Params(), 0.5, 5.0)
    if math.isnan(out_d[3]):
        pytest.skip("dynamic coefficient clipped to zero for this field")
    assert abs(out_s[3] - out_d[3]) < 1e-12
    assert np.allclose(out_s[0], out_d[0], rtol=0, atol=0)


def test_pcc_properties():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((16, 16))
    Y = X + 0.5 * rng.standard_normal((16, 16))
    assert O.pcc(X, X) == pytest.approx(1.0, abs=1e-15)
    assert O.pcc(X, 3.0 * Y - 2.0) == pytest.approx(O.pcc(X, Y), abs=1e-14)
    assert O.pcc(X, -Y) == pytest.approx(-O.pcc(X, Y), abs=1e-14)


# --------------------------------------------------------------------------
# The eddy-viscosity term div(g grad w) (Eq. 9) and the forcings of Eq. 8
# (Eq. 2, 3).  g is replaced by a prescribed field through the module's
# eddy_scale hook, so the divergence itself is checked against closed forms.
# --------------------------------------------------------------------------

import oracle.qg as OQ


def _prescribe_g(monkeypatch, g):
    monkeypatch.setattr(OQ, "eddy_scale", lambda ops, wh, kind: g)


def _half_weights(shape):
    w = np.full(shape, 2.0)
    w[:, 0] = 1.0
    w[:, -1] = 1.0
    return w


@pytest.mark.parametrize("kind", [O.SMAG, O.LEITH])
def test_sgs_divergence_constant_g_is_diffusion(monkeypatch, kind):
    """g = gamma constant: div(gamma grad w) = gamma lap w, i.e. -gamma |k|^2 w_hat."""
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(31, n))
    gamma = 0.73
    _prescribe_g(monkeypatch, np.full((n, n), gamma))
    D = O.sgs_divergence_hat(ops, wh, kind)
    ref = -gamma * ops.k2 * wh
    assert np.max(np.abs(D - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("p,q", [((1, 2), (3, -1)), ((2, 0), (3, 0)), ((0, 3), (4, 0)), ((-1, 1), (2, 5))])
def test_sgs_divergence_closed_form_single_modes(monkeypatch, p, q):
    """g = 1 + e cos(p.x), w = cos(q.x):
    div(g grad w) = e (p.q) sin(p.x) sin(q.x) - |q|^2 (1 + e cos(p.x)) cos(q.x).
    Pairs p parallel and perpendicular to q fix the pairing of k_x with w_x and the sign."""
    n = 48
    ops = O.Ops(n)
    X, Y = grid(n)
    e = 0.4
    px, py = p
    qx, qy = q
    ph = px * X + py * Y
    qh = qx * X + qy * Y
    _prescribe_g(monkeypatch, 1.0 + e * np.cos(ph))
    wh = O.project(ops, np.cos(qh) + 0 * X * Y)
    D = ops.inv(O.sgs_divergence_hat(ops, wh, O.LEITH))
    ref = e * (px * qx + py * qy) * np.sin(ph) * np.sin(qh) - (qx * qx + qy * qy) * (1 + e * np.cos(ph)) * np.cos(qh)
    assert np.max(np.abs(D - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind", [O.SMAG, O.LEITH, O.DSMAG, O.DLEITH])
def test_sgs_term_dissipates_enstrophy_parseval(kind):
    """Summation by parts on the grid: sum_x w div(g grad w) = -sum_x g |grad w|^2,
    written in the half spectrum as sum w_k Re(conj(w_hat) D_hat) / N^2."""
    n = 48
    ops = O.Ops(n)
    wh = O.project(ops, init_field(32 + kind, n, k_peak=6.0))
    D = O.sgs_divergence_hat(ops, wh, kind)
    lhs = np.sum(_half_weights(wh.shape) * (np.conj(wh) * D).real) / n ** 2
    g = O.eddy_scale(ops, wh, kind)
    wx, wy = O.vorticity_gradient(ops, wh)
    rhs = -np.sum(g * (wx * wx + wy * wy))
    assert rhs < 0
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


@pytest.mark.parametrize("kind", [O.SMAG, O.LEITH])
def test_sgs_divergence_is_truncated(kind):
    """The flux divergence is a product output: zero outside the 2/3 band (R2)."""
    n = 48
    ops = O.Ops(n)
    wh = O.project(ops, init_field(40, n, k_peak=12.0))
    D = O.sgs_divergence_hat(ops, wh, kind)
    assert np.all(D[ops.T == 0] == 0)
    assert np.max(np.abs(D)) > 0


def test_obstacle_forcing_constant_mask():
    """chi = c: F_obs = -curl(c u / eta) = -(c / eta) w (the uniform inflow has no curl)."""
    n = 32
    ops = O.Ops(n)
    wh = O.project(ops, init_field(41, n))
    c, eta = 0.6, 1e-3
    F = O.obstacle_forcing_hat(ops, wh, np.full((n, n), c), eta, U=0.8)
    assert rel(F, -(c / eta) * wh) < 1e-14


@pytest.mark.parametrize("p,q", [((0, 1), (3, 0)), ((1, 2), (2, -3)), ((2, 1), (0, 4))])
def test_obstacle_forcing_closed_form(p, q):
    """chi = 1 + e cos(p.x), w = cos(q.x) (psi = -cos(q.x)/|q|^2, u = -psi_y + U, v = psi_x):
    -curl(chi u)/eta = -(chi w + chi_x v - chi_y u) / eta, evaluated pointwise."""
    n = 48
    ops = O.Ops(n)
    X, Y = grid(n)
    e, eta, U = 0.3, 1e-3, 0.7
    px, py = p
    qx, qy = q
    q2 = qx * qx + qy * qy
    ph = px * X + py * Y
    qh = qx * X + qy * Y
    chi = 1 + e * np.cos(ph) + 0 * X * Y
    w = np.cos(qh) + 0 * X * Y
    u = -qy * np.sin(qh) / q2 + U
    v = qx * np.sin(qh) / q2
    chi_x = -e * px * np.sin(ph)
    chi_y = -e * py * np.sin(ph)
    ref = -(chi * w + chi_x * v - chi_y * u) / eta
    F = ops.inv(O.obstacle_forcing_hat(ops, O.project(ops, w), chi, eta, U))
    assert np.max(np.abs(F - ref)) < 1e-12 * np.max(np.abs(ref))


def test_sponge_forcing_unit_mask():
    """chi_s = 1: F_sp = -rate (w - 0) = -rate w (Eq. 3, target 0)."""
    n = 48
    ops = O.Ops(n)
    rate = 50.0
    wh = O.project(ops, init_field(42, n))
    assert rel(O.sponge_forcing_hat(ops, wh, np.ones((n, n)), rate), -rate * wh) < 1e-14


def test_sponge_forcing_closed_form():
    """chi_s = 1 + e cos(p.x), w = cos(q.x): F_sp = -rate chi_s w pointwise, inside the band."""
    n = 48
    ops = O.Ops(n)
    rate = 50.0
    X, Y = grid(n)
    chs = 1 + 0.25 * np.cos(2 * X - Y)
    w = np.cos(3 * X + 4 * Y)
    F = ops.inv(O.sponge_forcing_hat(ops, O.project(ops, w), chs, rate))
    ref = -rate * chs * w
    assert np.max(np.abs(F - ref)) < 1e-12 * np.max(np.abs(ref))
