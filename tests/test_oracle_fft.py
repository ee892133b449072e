"""Pins of the oracle's only library step, the 2-D real FFT, and of its conventions.

Sec. II-C: derivatives in Fourier space on an N x N periodic grid.  The
oracle uses numpy's rfft2/irfft2 (unnormalised forward transform, inverse
with 1/N^2); these tests pin that step against a brute-force O(N^4) DFT and
against the invariants every DFT must satisfy.
"""
import math

import numpy as np
import pytest

from oracle import Ops


def brute_dft2(f):
    n = f.shape[0]
    idx = np.arange(n)
    out = np.zeros((n, n // 2 + 1), dtype=np.complex128)
    for ky in range(n):
        for kx in range(n // 2 + 1):
            ph = np.exp(-2j * math.pi * (kx * idx[None, :] + ky * idx[:, None]) / n)
            out[ky, kx] = np.sum(f * ph)
    return out


@pytest.mark.parametrize("n", [8, 12, 16, 24])
def test_rfft2_matches_brute_force(n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal((n, n))
    ops = Ops(n)
    ref = brute_dft2(f)
    got = ops.fwd(f)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [16, 48, 96])
def test_round_trip_parseval_hermitian(n):
    rng = np.random.default_rng(7 + n)
    f = rng.standard_normal((n, n))
    ops = Ops(n)
    fh = ops.fwd(f)
    assert np.max(np.abs(ops.inv(fh) - f)) < 1e-13
    # Parseval over the half spectrum: weight 1 on the k_x = 0 and k_x = N/2 columns, else 2
    w = np.full(fh.shape, 2.0)
    w[:, 0] = 1.0
    w[:, -1] = 1.0
    lhs = np.sum(f * f)
    rhs = np.sum(w * np.abs(fh) ** 2) / n ** 2
    assert abs(lhs - rhs) < 1e-12 * lhs
    # Hermitian symmetry of the k_x = 0 column: F(0, -ky) = conj F(0, ky)
    col = fh[:, 0]
    assert np.max(np.abs(col[1:] - np.conj(col[1:][::-1]))) < 1e-12 * np.max(np.abs(col))


def test_wavenumber_layout():
    ops = Ops(12, L=4.0)
    assert ops.K == 3
    assert ops.kx.shape == (1, 7) and ops.ky.shape == (12, 1)
    np.testing.assert_allclose(ops.kx[0, 1], 2 * math.pi / 4.0)
    assert ops.my[11, 0] == -1 and ops.my[6, 0] == -6
    assert ops.T.sum() == 4 * 7  # kx 0..3, ky -3..3
