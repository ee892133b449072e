"""Pins of the oracle's discrete adjoint (the step's vector-Jacobian product) by central finite differences
of the forward oracle, in the state, the closure constant and the sponge rate."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S

L = 2 * math.pi


def setup(n, kind, c, mask=True, sponge=True, seed=2, U=0.5, beta=5.0):
    ops = O.Ops(n, L)
    chi = S.island_mask(n, L, radius=0.9) if mask else None
    chs = S.sponge_mask(n, L) if sponge else None
    w0 = S.init_field(seed, n, L, k_peak=n / 6)
    wh = O.project(ops, w0)
    cl = O.Closure(kind, c=c)
    return ops, chi, chs, wh, cl, U, beta


def loss(ops, wh, lam_next, beta, U, cl, params, chi, chs):
    w1, _ = O.full_step(ops, wh, beta, U, cl, params, chi, chs)
    return float(np.sum(lam_next * ops.inv(w1)))


@pytest.mark.parametrize("kind,c", [(O.NONE, 0.0), (O.SMAG, 0.5), (O.LEITH, 0.6)])
@pytest.mark.parametrize("mask,sponge", [(True, True), (False, False), (True, False)])
def test_state_gradient_matches_central_differences(kind, c, mask, sponge):
    n = 32
    ops, chi, chs, wh, cl, U, beta = setup(n, kind, c, mask, sponge)
    params = O.Params(dt=5e-3, eta=2e-2)
    rng = np.random.default_rng(7)
    lam_next = rng.standard_normal((n, n))
    lam_n, _ = O.full_step_vjp(ops, wh, lam_next, beta, U, cl, params, chi, chs)
    for trial in range(3):
        d = ops.inv(O.project(ops, rng.standard_normal((n, n))))
        eps = 1e-5
        fp = loss(ops, wh + eps * O.project(ops, d), lam_next, beta, U, cl, params, chi, chs)
        fm = loss(ops, wh - eps * O.project(ops, d), lam_next, beta, U, cl, params, chi, chs)
        fd = (fp - fm) / (2 * eps)
        ad = float(np.sum(lam_n * d))
        assert ad == pytest.approx(fd, rel=2e-7, abs=1e-9 * abs(fd) + 1e-10)


@pytest.mark.parametrize("kind,c", [(O.SMAG, 0.5), (O.LEITH, 0.6)])
def test_closure_constant_gradient(kind, c):
    n = 32
    ops, chi, chs, wh, cl, U, beta = setup(n, kind, c)
    params = O.Params(dt=5e-3, eta=2e-2)
    lam_next = np.random.default_rng(3).standard_normal((n, n))
    _, g = O.full_step_vjp(ops, wh, lam_next, beta, U, cl, params, chi, chs)
    eps = 1e-6
    fp = loss(ops, wh, lam_next, beta, U, O.Closure(kind, c=c + eps), params, chi, chs)
    fm = loss(ops, wh, lam_next, beta, U, O.Closure(kind, c=c - eps), params, chi, chs)
    assert g["c"] == pytest.approx((fp - fm) / (2 * eps), rel=1e-7)


def test_sponge_rate_gradient():
    n = 32
    ops, chi, chs, wh, cl, U, beta = setup(n, O.LEITH, 0.6)
    params = O.Params(dt=5e-3, eta=2e-2, sponge_rate=50.0)
    lam_next = np.random.default_rng(4).standard_normal((n, n))
    _, g = O.full_step_vjp(ops, wh, lam_next, beta, U, cl, params, chi, chs)
    eps = 1e-4
    fp = loss(ops, wh, lam_next, beta, U, cl, O.Params(dt=5e-3, eta=2e-2, sponge_rate=50.0 + eps), chi, chs)
    fm = loss(ops, wh, lam_next, beta, U, cl, O.Params(dt=5e-3, eta=2e-2, sponge_rate=50.0 - eps), chi, chs)
    assert g["sponge_rate"] == pytest.approx((fp - fm) / (2 * eps), rel=1e-7)


def test_transpose_at_the_zero_state():
    """At w = 0 the linearised step is A d = (step(e d) - step(-e d)) / 2e up to O(e^2) (RK3 composes the
    quadratic Jacobian, so odd powers up to 7 remain): <lam, A d> = <A^T lam, d>."""
    n = 24
    ops, chi, chs, _, cl, U, beta = setup(n, O.NONE, 0.0)
    params = O.Params(dt=5e-3, eta=2e-2)
    wh0 = np.zeros((n, n // 2 + 1), dtype=complex)
    rng = np.random.default_rng(5)
    lam_next = rng.standard_normal((n, n))
    lam_n, _ = O.full_step_vjp(ops, wh0, lam_next, beta, U, cl, params, chi, chs)
    d = ops.inv(O.project(ops, rng.standard_normal((n, n))))
    base = O.full_step(ops, wh0, beta, U, cl, params, chi, chs)[0]  # the constant part (inflow through the mask)
    e = 1e-3
    Ad = ops.inv(O.full_step(ops, e * O.project(ops, d), beta, U, cl, params, chi, chs)[0] - base)
    Am = ops.inv(O.full_step(ops, -e * O.project(ops, d), beta, U, cl, params, chi, chs)[0] - base)
    lin = (Ad - Am) / (2 * e)
    assert float(np.sum(lam_next * lin)) == pytest.approx(float(np.sum(lam_n * d)), rel=1e-9)


def test_output_is_band_limited_with_zero_mean():
    n = 32
    ops, chi, chs, wh, cl, U, beta = setup(n, O.SMAG, 0.5)
    lam_n, _ = O.full_step_vjp(ops, wh, np.random.default_rng(1).standard_normal((n, n)), beta, U, cl,
                               O.Params(dt=5e-3, eta=2e-2), chi, chs)
    h = np.fft.rfft2(lam_n)
    assert abs(h[0, 0]) < 1e-10
    assert np.max(np.abs(h * (1 - ops.T))) < 1e-10


def dynamic_setup(kind, n=32):
    """A state whose dynamic coefficient is positive (so the quotient, not the clip, is differentiated)."""
    for seed in range(1, 40):
        ops, chi, chs, wh, cl, U, beta = setup(n, kind, 0.0, seed=seed)
        wh = O.project(ops, S.init_field(seed, n, L, k_peak=n / 3))
        if O.germano_coefficient(ops, wh, cl, U)[0] > 0.0:
            return ops, chi, chs, wh, cl, U, beta
    raise RuntimeError("no state with a positive coefficient")


@pytest.mark.parametrize("kind", [O.DSMAG, O.DLEITH])
def test_germano_coefficient_gradient_matches_central_differences(kind):
    ops, chi, chs, wh, cl, U, beta = dynamic_setup(kind)
    grad = O.germano_vjp(ops, wh, cl, U, 1.0)
    rng = np.random.default_rng(11)
    for _ in range(3):
        d = ops.inv(O.project(ops, rng.standard_normal((ops.n, ops.n))))
        eps = 1e-5
        cp = O.germano_coefficient(ops, wh + eps * O.project(ops, d), cl, U)[0]
        cm = O.germano_coefficient(ops, wh - eps * O.project(ops, d), cl, U)[0]
        assert float(np.sum(grad * d)) == pytest.approx((cp - cm) / (2 * eps), rel=1e-6)


@pytest.mark.parametrize("kind", [O.DSMAG, O.DLEITH])
def test_dynamic_step_gradient_matches_central_differences(kind):
    ops, chi, chs, wh, cl, U, beta = dynamic_setup(kind)
    params = O.Params(dt=5e-3, eta=2e-2)
    n = ops.n
    rng = np.random.default_rng(12)
    lam_next = rng.standard_normal((n, n))
    lam_n, g = O.full_step_vjp(ops, wh, lam_next, beta, U, cl, params, chi, chs)
    for _ in range(3):
        d = ops.inv(O.project(ops, rng.standard_normal((n, n))))
        eps = 1e-5
        fp = loss(ops, wh + eps * O.project(ops, d), lam_next, beta, U, cl, params, chi, chs)
        fm = loss(ops, wh - eps * O.project(ops, d), lam_next, beta, U, cl, params, chi, chs)
        assert float(np.sum(lam_n * d)) == pytest.approx((fp - fm) / (2 * eps), rel=2e-7)
    assert g["c"] == 0.0


def test_clipped_dynamic_coefficient_has_no_gradient():
    n = 32
    for seed in range(1, 40):
        ops, chi, chs, wh, cl, U, beta = setup(n, O.DLEITH, 0.0, seed=seed)
        C, hm, mm = O.germano_coefficient(ops, wh, cl, U)
        if C == 0.0 and hm < 0.0:
            break
    else:
        pytest.skip("no clipped state found")
    assert np.all(O.germano_vjp(ops, wh, cl, U, 1.0) == 0.0)
    params = O.Params(dt=5e-3, eta=2e-2)
    lam_next = np.random.default_rng(13).standard_normal((n, n))
    lam_n, _ = O.full_step_vjp(ops, wh, lam_next, beta, U, cl, params, chi, chs)
    d = ops.inv(O.project(ops, np.random.default_rng(14).standard_normal((n, n))))
    eps = 1e-6
    fp = loss(ops, wh + eps * O.project(ops, d), lam_next, beta, U, cl, params, chi, chs)
    fm = loss(ops, wh - eps * O.project(ops, d), lam_next, beta, U, cl, params, chi, chs)
    assert float(np.sum(lam_n * d)) == pytest.approx((fp - fm) / (2 * eps), rel=2e-7)
