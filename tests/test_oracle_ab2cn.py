"""Pins of the paper's own time scheme (Sec. II-E, Eq. 4) in the oracle.

Each test reduces the scheme to a scalar recurrence per Fourier mode that is
written out here independently of the oracle's array code: Crank-Nicolson on
the linear terms, AB2 on the explicit ones, and the AB2 sponge split.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import init_field


def grid(n):
    x = np.arange(n) * (2 * math.pi / n)
    return x[None, :], x[:, None]


def run(ops, w, nsteps, beta, U, params, chi=None, chi_s=None, closure=None):
    q = O.QGOracle(ops.n, ops.L, beta, U, chi, chi_s, closure or O.Closure(O.NONE), params)
    q.set_state(w)
    q.step(nsteps)
    return q.wh


def scalar_ab2cn(z0, steps, dt, lin, lam_e, sponge=0.0):
    """w* = ((1 + dt/2 lin) w + dt (3/2 lam_e w - 1/2 lam_e w_prev)) / (1 - dt/2 lin);
    w_new = w* - dt sponge (3/2 w* - 1/2 w**), Euler start."""
    w, w_prev, ws_prev = z0, None, None
    for _ in range(steps):
        e = lam_e * w
        e_prev = e if w_prev is None else lam_e * w_prev
        ws = ((1 + 0.5 * dt * lin) * w + dt * (1.5 * e - 0.5 * e_prev)) / (1 - 0.5 * dt * lin)
        wss = ws if ws_prev is None else ws_prev
        new = ws - dt * sponge * (1.5 * ws - 0.5 * wss)
        w_prev, ws_prev, w = w, ws, new
    return w


@pytest.mark.parametrize("mode", [(2, 3), (1, -4), (3, 0)])
def test_single_mode_matches_scalar_recurrence(mode):
    n, beta, U, nu, mu, dt, steps = 32, 5.0, 0.5, 0.01, 0.1, 2e-3, 60
    mx, my = mode
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.cos(mx * X + my * Y + 0.4)
    wh0 = O.project(ops, w)
    out = run(ops, w, steps, beta, U, O.Params(dt=dt, nu=nu, mu=mu, scheme=O.AB2CN))
    k2 = mx * mx + my * my
    lin = -(nu * k2 + mu) + 1j * beta * mx / k2   # CN part: viscosity, friction, beta
    lam_e = -1j * U * mx                          # AB2 part: advection by the inflow
    idx = (my % n, mx)
    expected = scalar_ab2cn(wh0[idx], steps, dt, lin, lam_e)
    assert abs(out[idx] - expected) < 1e-13 * abs(expected)
    mask = np.ones_like(out, dtype=bool)
    mask[idx] = False
    assert np.max(np.abs(out[mask])) < 1e-12 * abs(expected)


def test_second_order_in_time():
    n, beta, U, T = 16, 20.0, 1.0, 0.4
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.cos(X + 2 * Y)
    lam = 1j * (beta / 5.0 - U)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        wh0 = O.project(ops, w)
        out = run(ops, w, int(round(T / dt)), beta, U, O.Params(dt=dt, nu=0.0, scheme=O.AB2CN))
        errs.append(np.linalg.norm(out - wh0 * np.exp(lam * T)) / np.linalg.norm(wh0))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < p < 2.3 for p in orders), orders


def test_crank_nicolson_viscous_decay():
    n, nu, dt, steps = 32, 0.05, 0.01, 25
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.sin(4 * X - 3 * Y)
    out = O.to_physical(ops, run(ops, w, steps, 0.0, 0.0, O.Params(dt=dt, nu=nu, scheme=O.AB2CN)))
    a = 0.5 * dt * nu * 25
    assert np.max(np.abs(out - w * ((1 - a) / (1 + a)) ** steps)) < 1e-14


def test_ab2_sponge_split_unit_mask():
    n, dt, rate, steps = 32, 1e-3, 50.0, 30
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.cos(2 * X + Y)
    wh0 = O.project(ops, w)
    out = run(ops, w, steps, 0.0, 0.0, O.Params(dt=dt, nu=0.0, sponge_rate=rate, scheme=O.AB2CN),
              chi_s=np.ones((n, n)))
    idx = (1, 2)
    expected = scalar_ab2cn(wh0[idx], steps, dt, 0.0, 0.0, sponge=rate)
    assert abs(out[idx] - expected) < 1e-13 * abs(expected)


def test_ab2_brinkman_constant_mask():
    """chi = c: curl(c u) = c w, so the Brinkman term is -c/eta w, advanced by AB2."""
    n, dt, eta, c, steps = 32, 1e-3, 5e-3, 0.3, 40
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.sin(X - 2 * Y)
    wh0 = O.project(ops, w)
    out = run(ops, w, steps, 0.0, 0.7, O.Params(dt=dt, nu=0.0, eta=eta, scheme=O.AB2CN), chi=np.full((n, n), c))
    idx = ((-2) % n, 1)
    expected = scalar_ab2cn(wh0[idx], steps, dt, 0.0, -c / eta - 1j * 0.7 * 1)
    assert abs(out[idx] - expected) < 1e-13 * abs(expected)


def test_ab2cn_full_configuration_runs_and_keeps_band():
    n = 48
    ops = O.Ops(n)
    from synth import island_mask, sponge_mask
    out = run(ops, init_field(3, n), 5, 5.0, 0.5, O.Params(dt=5e-4, eta=2e-3, scheme=O.AB2CN),
              chi=island_mask(n, radius=0.8), chi_s=sponge_mask(n), closure=O.Closure(O.DLEITH))
    assert np.all(np.isfinite(out)) and out[0, 0] == 0
    assert np.all(out[ops.T == 0] == 0)


@pytest.mark.parametrize("r,grows", [(0.5, False), (0.9, False), (1.2, True), (2.0, True)])
def test_explicit_penalisation_needs_eta_above_dt(r, grows):
    """Sec. II-E: treated explicitly, the penalisation is stable only for eta > dt.  With chi = 1 (and U = 0)
    every mode obeys dw/dt = -w/eta; AB2 gives w_{n+1} = (1 - 3r/2) w_n + r/2 w_{n-1}, r = dt/eta, whose roots
    leave the unit circle for r > 1 (at r = 1.2 the larger one is 1.272, at r = 0.9 it is 0.868).  The RK3
    split's exact implicit sub-step damps the same mode by exactly exp(-r) per step at any eta."""
    n, dt, steps = 16, 1e-3, 200
    eta = dt / r
    ops = O.Ops(n)
    X, Y = grid(n)
    w = np.sin(X + Y)
    wh0 = O.project(ops, w)
    idx = (1, 1)  # the k = (1, 1) mode of the half spectrum
    chi = np.ones((n, n))
    with np.errstate(over="ignore", invalid="ignore"):  # the unstable runs overflow
        ab2 = run(ops, w, steps, 0.0, 0.0, O.Params(dt=dt, nu=0.0, mu=0.0, eta=eta, scheme=O.AB2CN), chi=chi)
        growth = abs(ab2[idx]) / abs(wh0[idx])
    if grows:
        assert not np.isfinite(growth) or growth > 1e10
    else:
        assert growth < 1.0
    # the scalar recurrence written out here agrees where it stays finite
    if not grows:
        expected = scalar_ab2cn(wh0[idx], steps, dt, 0.0, -1.0 / eta)
        assert abs(ab2[idx] - expected) <= 1e-12 * abs(wh0[idx])
    exact = run(ops, w, steps, 0.0, 0.0, O.Params(dt=dt, nu=0.0, mu=0.0, eta=eta), chi=chi)
    assert abs(exact[idx]) / abs(wh0[idx]) == pytest.approx(math.exp(-r * steps), rel=1e-10)

