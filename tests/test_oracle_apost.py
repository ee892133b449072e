"""Pins of the oracle's a posteriori tools (Sec. IV, Eq. 15-16) against closed forms and identities."""
import math

import numpy as np
import pytest

import oracle
import synth

L = 2 * math.pi


def cosine_series(n, nsnap, m, c, dt_snap, shift=0, theta=0.3):
    """cos(k0 m . (x - c t_i) + theta), t_i = (i + shift) dt_snap, on an n x n grid."""
    x = np.arange(n) * (L / n)
    X, Y = np.meshgrid(x, x)  # [y][x]
    out = []
    for i in range(nsnap):
        t = (i + shift) * dt_snap
        out.append(np.cos(m[0] * (X - c[0] * t) + m[1] * (Y - c[1] * t) + theta))
    return np.array(out)


def test_single_mode_distance_pcc_and_phase_closed_form():
    n, nsnap, dt_snap = 24, 9, 0.1
    m, c = (2, 1), (0.9, -0.4)
    s = 2  # the LES runs s snapshots ahead: omega_LES(t) = omega_FF(t + s)
    ff = cosine_series(n, nsnap, m, c, dt_snap)
    les = cosine_series(n, nsnap, m, c, dt_snap, shift=s)
    lag_min, lag_max = -4, 4
    dist, corr = oracle.lag_table(les, ff, lag_min, lag_max)
    omega = m[0] * c[0] + m[1] * c[1]  # phase speed of the mode in radians per time unit
    for t in range(nsnap):
        for j, phi in enumerate(range(lag_min, lag_max + 1)):
            if not 0 <= t - phi < nsnap:
                assert np.isnan(dist[t, j]) and np.isnan(corr[t, j])
                continue
            da = omega * (s - phi) * dt_snap
            assert dist[t, j] == pytest.approx(n * n * (1 - math.cos(da)), abs=1e-10)
            assert corr[t, j] == pytest.approx(math.cos(da), abs=1e-12)
    phi, mean = oracle.phase_shift(dist, lag_min)
    assert phi == s
    assert mean[s - lag_min] == pytest.approx(0.0, abs=1e-10)


def test_pcc_series_is_cosine_of_the_phase_offset():
    n, nsnap = 16, 5
    ff = cosine_series(n, nsnap, (1, 3), (0.5, 0.2), 0.1)
    les = cosine_series(n, nsnap, (1, 3), (0.5, 0.2), 0.1, theta=1.1)
    r = oracle.pcc_series(les, ff)
    assert np.allclose(r, math.cos(0.8), atol=1e-12)


def test_series_against_itself():
    a = synth.wave_series(3, 20, 7, L, noise=0.05)
    dist, corr = oracle.lag_table(a, a, -3, 3)
    assert np.all(dist[:, 3] == 0.0)
    assert np.allclose(corr[:, 3], 1.0, atol=1e-14)
    phi, _ = oracle.phase_shift(dist, -3)
    assert phi == 0


def test_exchanging_the_series_negates_the_lag():
    n, nsnap = 16, 8
    a = synth.wave_series(5, n, nsnap, L, noise=0.1)
    b = synth.wave_series(5, n, nsnap, L, t0=0.3, noise=0.1, noise_seed=99)
    d_ab, c_ab = oracle.lag_table(a, b, -3, 3)
    d_ba, c_ba = oracle.lag_table(b, a, -3, 3)
    for t in range(nsnap):
        for j, phi in enumerate(range(-3, 4)):
            if 0 <= t - phi < nsnap:
                jj = -phi + 3
                assert d_ab[t, j] == pytest.approx(d_ba[t - phi, jj], rel=1e-14)
                assert c_ab[t, j] == pytest.approx(c_ba[t - phi, jj], rel=1e-13)
    assert oracle.phase_shift(d_ab, -3)[0] == -oracle.phase_shift(d_ba, -3)[0]


def test_noisy_translating_pattern_recovers_the_shift():
    n, nsnap, dt_snap, s = 32, 12, 0.2, -3
    ff = synth.wave_series(11, n, nsnap, L, dt_snap=dt_snap, noise=0.2)
    les = synth.wave_series(11, n, nsnap, L, dt_snap=dt_snap, t0=s * dt_snap, noise=0.2, noise_seed=7)
    dist, _ = oracle.lag_table(les, ff, -5, 5)
    assert oracle.phase_shift(dist, -5)[0] == s


def test_phase_tie_rules_and_empty_lags():
    nan = float("nan")
    d = np.array([[1.0, 2.0, 1.0], [1.0, 2.0, 1.0]])
    assert oracle.phase_shift(d, -1)[0] == -1  # equal means at -1 and +1: the negative lag
    d = np.array([[1.0, 1.0, 1.0]])
    assert oracle.phase_shift(d, -1)[0] == 0  # smallest |phi| first
    d = np.array([[nan, 5.0, nan], [nan, 1.0, 0.5]])
    phi, mean = oracle.phase_shift(d, -1)
    assert np.isnan(mean[0]) and mean[1] == 3.0 and mean[2] == 0.5 and phi == 1
    assert oracle.phase_shift(np.full((2, 3), nan), -1)[0] is None


def test_lag_table_nan_pattern_for_unequal_lengths():
    les = synth.wave_series(1, 8, 3, L)
    ff = synth.wave_series(2, 8, 5, L)
    dist, corr = oracle.lag_table(les, ff, -2, 3)
    for t in range(5):
        for j, phi in enumerate(range(-2, 4)):
            assert np.isnan(dist[t, j]) == (not 0 <= t - phi < 3)
            assert np.isnan(corr[t, j]) == (not 0 <= t - phi < 3)


def test_constant_field_has_undefined_pcc():
    a = np.ones((1, 8, 8))
    b = synth.wave_series(2, 8, 1, L)
    dist, corr = oracle.lag_table(a, b, 0, 0)
    assert np.isnan(corr[0, 0])
    assert dist[0, 0] == pytest.approx(float(np.sum((1.0 - b[0]) ** 2)), rel=1e-14)


@pytest.mark.parametrize("gaussian", [True, False])
def test_grid_filter_on_single_modes(gaussian):
    n_f, n_c = 48, 24
    x_f = np.arange(n_f) * (L / n_f)
    x_c = np.arange(n_c) * (L / n_c)
    delta = L / n_c
    for (mx, my) in [(1, 0), (3, -2), (5, 7), (7, 7)]:  # inside the coarse 2/3 band K_c = 7
        Xf, Yf = np.meshgrid(x_f, x_f)
        Xc, Yc = np.meshgrid(x_c, x_c)
        f = np.cos(mx * Xf + my * Yf + 0.4)
        g = np.exp(-(mx * mx + my * my) * delta ** 2 / 6.0) if gaussian else 1.0
        expect = g * np.cos(mx * Xc + my * Yc + 0.4)
        assert np.allclose(oracle.filter_to_les(f, n_c, L, gaussian), expect, atol=1e-13)
    for (mx, my) in [(8, 0), (0, 9), (10, 12)]:  # outside the coarse band, inside the fine band K_f = 15
        Xf, Yf = np.meshgrid(x_f, x_f)
        f = np.cos(mx * Xf + my * Yf)
        assert np.allclose(oracle.filter_to_les(f, n_c, L, gaussian), 0.0, atol=1e-13)


def test_grid_filter_without_gaussian_samples_band_limited_fields():
    n_f, n_c = 64, 32
    w = synth.init_field(4, n_f, L, k_peak=3.0)
    # keep the part inside the coarse 2/3 band, then the filter is plain sampling
    wh = np.fft.rfft2(w)
    m = np.fft.fftfreq(n_f, 1.0 / n_f)
    kc = (n_c - 1) // 3
    keep = (np.abs(m)[:, None] <= kc) & (np.abs(m[: n_f // 2 + 1])[None, :] <= kc)
    w_low = np.fft.irfft2(wh * keep, s=(n_f, n_f))
    w_low -= w_low.mean()
    out = oracle.filter_to_les(w_low, n_c, L, gaussian=False)
    assert np.allclose(out, w_low[:: n_f // n_c, :: n_f // n_c], atol=1e-13)


def test_grid_filter_series_is_per_snapshot():
    s = synth.wave_series(6, 32, 3, L)
    out = oracle.filter_to_les(s, 16, L)
    for i in range(3):
        assert np.array_equal(out[i], oracle.filter_to_les(s[i], 16, L))


def test_pcc_is_affine_invariant_and_distance_is_not():
    a = synth.wave_series(8, 16, 4, L, noise=0.1)
    b = synth.wave_series(9, 16, 4, L, noise=0.1)
    d0, c0 = oracle.lag_table(a, b, -1, 1)
    d1, c1 = oracle.lag_table(3.0 * a + 5.0, b, -1, 1)
    ok = ~np.isnan(c0)
    assert np.allclose(c1[ok], c0[ok], atol=1e-13)
    assert not np.allclose(d1[ok], d0[ok])
