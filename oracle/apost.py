"""A posteriori evaluation tools (Sec. IV, Eq. 15-16), plain FP64.  TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU legs use this module; the
product path never imports it.

What the paper computes from a pair of runs on the LES grid:

* omega_FF: the fully resolved vorticity passed through the grid filter of
  Eq. 5 (the same filter as the a priori analysis, reading R9) and kept in the
  coarse 2/3 band, the field an LES state is compared with;
* PCC_a-post,omega(t) = PCC(omega_LES(t), omega_FF(t)) (Eq. 15) per snapshot;
* the phase shift phi of Eq. 16, the time lag that brings the LES series
  closest to the filtered series in the L2 norm.

Reading R14 (Eq. 16 states one phi per run but not how the snapshot pairs
are combined): lags are whole multiples of the snapshot interval; for a lag
phi the squared discrete L2 distance d(t, phi) = sum over grid points of
(omega_LES(t - phi) - omega_FF(t))^2 is averaged over the snapshots t for
which both fields exist; phi is the lag of the smallest mean (ties: the
smallest |phi|, then the negative lag).  Lags with no overlapping pair take
no part.

Parity: pinned by closed forms of translating cosine patterns (distance
N^2 (1 - cos(a - b)) for one mode, PCC = cos(a - b), phase = the imposed
shift), by identities (a series against itself; exchanging the series
negates the lag), and by the grid filter's action on single Fourier modes.
"""
from __future__ import annotations

import math

import numpy as np

from .qg import Ops, apriori_filter, pcc, project

__all__ = ["filter_to_les", "pcc_series", "lag_table", "phase_shift"]


def filter_to_les(omega_fr, n_les: int, L: float, gaussian: bool = True) -> np.ndarray:
    """omega_FF: the grid filter of Eq. 5 (R9) applied to a fully resolved field, on the N_c grid.

    The fine field is first projected onto its own 2/3 band (zero mean, as the
    solver's state); the filtered spectrum is kept in the coarse 2/3 band.
    Accepts one field (n, n) or a series (nsnap, n, n).
    """
    w = np.asarray(omega_fr, dtype=np.float64)
    if w.ndim == 3:
        return np.stack([filter_to_les(f, n_les, L, gaussian) for f in w])
    of = Ops(w.shape[0], L)
    oc = Ops(n_les, L)
    return oc.inv(oc.T * apriori_filter(of, project(of, w), n_les, gaussian))


def pcc_series(les, ff) -> np.ndarray:
    """PCC(omega_LES(t), omega_FF(t)) for every snapshot t of two equally long series (Eq. 15)."""
    les = np.asarray(les, dtype=np.float64)
    ff = np.asarray(ff, dtype=np.float64)
    return np.array([pcc(a, b) for a, b in zip(les, ff)])


def lag_table(les, ff, lag_min: int, lag_max: int):
    """Squared L2 distances and PCCs of omega_LES(t - phi) against omega_FF(t) (Eq. 15-16).

    Returns (dist, corr), each of shape (n_ff, lag_max - lag_min + 1): column
    j holds phi = lag_min + j; entries whose LES snapshot t - phi lies outside
    the LES series are NaN.  dist is the plain sum of squared differences over
    all grid points; corr is the PCC with population moments.
    """
    les = np.asarray(les, dtype=np.float64).reshape(len(les), -1)
    ff = np.asarray(ff, dtype=np.float64).reshape(len(ff), -1)
    nlag = lag_max - lag_min + 1
    dist = np.full((len(ff), nlag), np.nan)
    corr = np.full((len(ff), nlag), np.nan)
    for t in range(len(ff)):
        for j in range(nlag):
            s = t - (lag_min + j)
            if 0 <= s < len(les):
                diff = les[s] - ff[t]
                dist[t, j] = float(np.sum(diff * diff))
                corr[t, j] = _pcc_or_nan(les[s], ff[t])
    return dist, corr


def _pcc_or_nan(a, b) -> float:
    x = a - a.mean()
    y = b - b.mean()
    vx = float(np.sum(x * x))
    vy = float(np.sum(y * y))
    if not (vx > 0.0 and vy > 0.0):
        return float("nan")
    return float(np.sum(x * y)) / (math.sqrt(vx) * math.sqrt(vy))


def phase_shift(dist, lag_min: int):
    """Eq. 16 under reading R14: (phi, mean_dist) from a lag table's distances.

    mean_dist[j] is the mean of dist[:, j] over the defined entries (NaN if
    none); phi minimises it, ties going to the smallest |phi|, then the
    negative lag.  phi is None when no lag has a pair.
    """
    dist = np.asarray(dist, dtype=np.float64)
    nlag = dist.shape[1]
    mean = np.full(nlag, np.nan)
    for j in range(nlag):
        col = dist[:, j]
        col = col[~np.isnan(col)]
        if col.size:
            mean[j] = float(np.mean(col))
    best = None
    for j in range(nlag):
        if np.isnan(mean[j]):
            continue
        phi = lag_min + j
        if best is None:
            best = (mean[j], phi)
            continue
        m, p = best
        if mean[j] < m or (mean[j] == m and (abs(phi) < abs(p) or (abs(phi) == abs(p) and phi < p))):
            best = (mean[j], phi)
    return (None if best is None else best[1]), mean
