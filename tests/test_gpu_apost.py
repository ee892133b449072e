"""GPU a posteriori tools (qg_grid_filter, qg_series_compare; Sec. IV, Eq. 5, 15, 16) vs the FP64 oracle.

Tolerances: FP64 series 1e-12 relative on distances and 1e-12 absolute on
PCCs (different summation orders only); FP32 series 1e-6 (the difference of
two FP32 values is rounded once before it is squared, about 1.2e-7 relative
per term); the grid filter 1e-12 relative L2.  Shapes span several 16 x 16
pair tiles with ragged tails and point counts that are not multiples of the
staged rounds.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth as S

pytestmark = pytest.mark.gpu

qg = pytest.importorskip("paper_2508_06678_gb300")
L = 2 * math.pi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06678_gb300._lib import LIB_PATH
    import os
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    qg.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check_table(got, ref_dist, ref_pcc, lag_min, dist_tol, pcc_tol, dist_atol=0.0):
    assert np.array_equal(np.isnan(got["dist"]), np.isnan(ref_dist))
    assert np.array_equal(np.isnan(got["pcc"]), np.isnan(ref_pcc))
    ok = ~np.isnan(ref_dist)
    assert np.allclose(got["dist"][ok], ref_dist[ok], rtol=dist_tol, atol=dist_atol)
    okp = ~np.isnan(ref_pcc)
    assert np.allclose(got["pcc"][okp], ref_pcc[okp], rtol=0, atol=pcc_tol)
    phi, mean = O.phase_shift(ref_dist, lag_min)
    okm = ~np.isnan(mean)
    assert np.array_equal(np.isnan(got["mean_dist"]), ~okm)
    assert np.allclose(got["mean_dist"][okm], mean[okm], rtol=dist_tol, atol=dist_atol)
    assert got["phase"] == phi


@pytest.mark.parametrize("n_fr,n_les", [(128, 64), (96, 48), (54, 36), (256, 96)])
@pytest.mark.parametrize("gaussian", [True, False])
def test_grid_filter_parity(n_fr, n_les, gaussian):
    w = np.stack([S.init_field(s, n_fr, L, k_peak=n_fr / 6) for s in range(3)])
    got = qg.qg_grid_filter(w, n_les, L, gaussian)
    ref = O.filter_to_les(w, n_les, L, gaussian)
    assert got.shape == (3, n_les, n_les)
    for i in range(3):
        assert rel(got[i], ref[i]) < 1e-12


def test_grid_filter_rejects_bad_sizes():
    w = np.zeros((64, 64))
    with pytest.raises(qg.QGError):
        qg.qg_grid_filter(w, 128, L)
    with pytest.raises(qg.QGError) as e:
        qg.qg_grid_filter(np.zeros((48, 48)), 48 - 2, L)  # 46 = 2 * 23 is not 2^a 3^b
    assert "bad sizes" in str(e.value) or "QG_ERR_ARG" in str(e.value)
    with pytest.raises(qg.QGError) as e:
        qg.qg_grid_filter(np.zeros((48, 48)), 48, L)  # coarse band 23 > fine band 15
    assert "QG_ERR_UNSUPPORTED" in str(e.value) or "exceeds" in str(e.value)


def series_pair(n_les, n_ff, shape, shift, noise=0.15, seed=4):
    nx = int(np.prod(shape))
    side = int(math.ceil(math.sqrt(nx)))
    ff = S.wave_series(seed, side, n_ff, L, dt_snap=0.2, noise=noise).reshape(n_ff, -1)[:, :nx]
    les = S.wave_series(seed, side, n_les, L, dt_snap=0.2, t0=0.2 * shift, noise=noise,
                        noise_seed=seed + 50).reshape(n_les, -1)[:, :nx]
    return les.reshape((n_les,) + shape).copy(), ff.reshape((n_ff,) + shape).copy()


@pytest.mark.parametrize("n_les,n_ff,shape,lags,shift", [
    (17, 20, (45, 45), (-9, 9), 2),     # two t tiles and two lag tiles, both ragged; 2025 points
    (5, 3, (7, 11), (-2, 6), -1),       # unequal lengths, lags beyond the series
    (33, 33, (64, 64), (-20, 20), 5),   # three lag tiles
    (1, 1, (3, 3), (0, 0), 0),          # single pair
])
@pytest.mark.parametrize("dtype,dist_tol,pcc_tol", [(np.float64, 1e-12, 1e-12), (np.float32, 1e-6, 1e-6)])
def test_series_compare_host_parity(n_les, n_ff, shape, lags, shift, dtype, dist_tol, pcc_tol):
    les, ff = series_pair(n_les, n_ff, shape, shift)
    les, ff = les.astype(dtype), ff.astype(dtype)
    got = qg.qg_series_compare(les, ff, *lags)
    ref_d, ref_p = O.lag_table(les.astype(np.float64), ff.astype(np.float64), *lags)
    check_table(got, ref_d, ref_p, lags[0], dist_tol, pcc_tol)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_series_compare_device_matches_host_bitwise(dtype):
    import torch
    les, ff = series_pair(19, 23, (40, 40), 3)
    les, ff = les.astype(dtype), ff.astype(dtype)
    host = qg.qg_series_compare(les, ff, -6, 7)
    st = torch.cuda.Stream()
    dl = torch.from_numpy(les).cuda()
    df = torch.from_numpy(ff).cuda()
    torch.cuda.synchronize()
    dev = qg.qg_series_compare(dl, df, -6, 7, stream=st)
    for k in ("dist", "pcc", "mean_dist"):
        assert np.array_equal(host[k], dev[k], equal_nan=True)
    assert host["phase"] == dev["phase"]


@pytest.mark.parametrize("dtype,dist_tol,pcc_tol", [("float32", 1e-6, 1e-6), ("float64", 1e-12, 1e-12)])
def test_series_compare_unaligned_device_series(dtype, dist_tol, pcc_tol):
    """Series that start off a 16-byte boundary are staged element by element instead of by bulk copies
    (other round lengths, so other point chunks): the same table up to summation order."""
    import torch
    les, ff = series_pair(21, 18, (32, 48), -2)
    les, ff = les.astype(dtype), ff.astype(dtype)
    aligned = qg.qg_series_compare(torch.from_numpy(les).cuda(), torch.from_numpy(ff).cuda(), -7, 5)
    tdt = getattr(torch, dtype)
    bl = torch.zeros(les.size + 1, dtype=tdt, device="cuda")
    bf = torch.zeros(ff.size + 1, dtype=tdt, device="cuda")
    dl = bl[1:].view(les.shape)
    df = bf[1:].view(ff.shape)
    dl.copy_(torch.from_numpy(les))
    df.copy_(torch.from_numpy(ff))
    assert dl.data_ptr() % 16 != 0
    torch.cuda.synchronize()
    off = qg.qg_series_compare(dl, df, -7, 5)
    ref_d, ref_p = O.lag_table(les.astype(np.float64), ff.astype(np.float64), -7, 5)
    check_table(aligned, ref_d, ref_p, -7, dist_tol, pcc_tol)
    check_table(off, ref_d, ref_p, -7, dist_tol, pcc_tol)
    ok = ~np.isnan(ref_d)
    assert np.allclose(off["dist"][ok], aligned["dist"][ok], rtol=dist_tol, atol=0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_phase_of_a_translating_pattern(dtype):
    for shift in (-4, 0, 3):
        les, ff = series_pair(24, 24, (64, 64), shift, noise=0.3, seed=9)
        got = qg.qg_series_compare(les.astype(dtype), ff.astype(dtype), -8, 8)
        assert got["phase"] == shift


def test_series_compare_edge_cases():
    # a constant field: PCC undefined, distance defined
    a = np.ones((1, 16), dtype=np.float64)
    b = np.arange(16, dtype=np.float64)[None]
    got = qg.qg_series_compare(a, b, 0, 0)
    assert np.isnan(got["pcc"][0, 0])
    assert got["dist"][0, 0] == pytest.approx(float(np.sum((1.0 - b) ** 2)), rel=1e-15)
    # one point per field
    got = qg.qg_series_compare(np.array([[2.0], [3.0]]), np.array([[1.0], [5.0]]), -1, 1)
    ref_d, ref_p = O.lag_table(np.array([[2.0], [3.0]]), np.array([[1.0], [5.0]]), -1, 1)
    check_table(got, ref_d, ref_p, -1, 1e-15, 1e-15)
    # no lag pairs two snapshots; reversed range
    with pytest.raises(qg.QGError):
        qg.qg_series_compare(np.zeros((2, 4)), np.zeros((3, 4)), 3, 5)
    with pytest.raises(qg.QGError):
        qg.qg_series_compare(np.zeros((2, 4)), np.zeros((3, 4)), -1, -3)
    with pytest.raises(qg.QGError):
        qg.qg_series_compare(np.zeros((2, 4)), np.zeros((2, 4)), 1, -1)
    with pytest.raises(ValueError):
        qg.qg_series_compare(np.zeros((2, 4)), np.zeros((2, 5)), 0, 0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_phase_tie_rules(dtype):
    """Integer-valued series: every distance and mean is exact, so ties at the minimum are real ties
    and the argmin must follow the rule (smallest |phi|, then the negative lag)."""
    rng = np.random.default_rng(0)
    kinds = set()
    for _ in range(400):
        n = int(rng.integers(3, 7))
        npts = int(rng.integers(1, 4))
        les = rng.integers(0, 4, (n, npts)).astype(dtype)
        ff = rng.integers(0, 4, (n, npts)).astype(dtype)
        ref_d, ref_p = O.lag_table(les.astype(np.float64), ff.astype(np.float64), -2, 2)
        phi, mean = O.phase_shift(ref_d, -2)
        got = qg.qg_series_compare(les, ff, -2, 2)
        assert np.array_equal(got["dist"], ref_d, equal_nan=True)
        assert np.array_equal(got["mean_dist"], mean, equal_nan=True)
        assert got["phase"] == phi
        tied = [j - 2 for j in range(5) if mean[j] == np.nanmin(mean)]
        if len(tied) > 1:
            kinds.add("sign" if 0 not in tied and -phi in tied else "abs")
    assert kinds == {"abs", "sign"}  # both tie rules were exercised


def test_series_compare_full_size_sampled():
    """512^2 fields, 40 snapshots, 41 lags in FP32: sampled pairs against the oracle one by one."""
    n, nsnap = 512, 40
    ff = S.wave_series(21, n, nsnap, L, dt_snap=0.1, noise=0.2).astype(np.float32)
    les = S.wave_series(21, n, nsnap, L, dt_snap=0.1, t0=0.3, noise=0.2, noise_seed=3).astype(np.float32)
    got = qg.qg_series_compare(les, ff, -20, 20)
    rng = np.random.default_rng(0)
    for _ in range(12):
        t = int(rng.integers(0, nsnap))
        phi = int(rng.integers(-20, 21))
        s = t - phi
        if not 0 <= s < nsnap:
            assert np.isnan(got["dist"][t, phi + 20])
            continue
        d, p = O.lag_table(les[s:s + 1].astype(np.float64), ff[t:t + 1].astype(np.float64), 0, 0)
        assert got["dist"][t, phi + 20] == pytest.approx(d[0, 0], rel=1e-6)
        assert got["pcc"][t, phi + 20] == pytest.approx(p[0, 0], abs=1e-6)
    assert got["phase"] == 3


def run_series(solver_or_oracle, nsteps, every, get):
    out = [get()]
    for _ in range(nsteps // every):
        solver_or_oracle.step(every)
        out.append(get())
    return np.stack(out)


def test_aposteriori_pipeline_parity():
    """Fully resolved run -> grid filter -> LES from the filtered start -> PCC series and phase (Sec. IV)."""
    n_fr, n_les, beta, U, dt = 96, 48, 5.0, 0.5, 2e-3
    nu = 1.0 / 200
    w0 = S.init_field(3, n_fr, L, k_peak=10.0)
    mask_f, mask_c = S.island_mask(n_fr, L, radius=0.8), S.island_mask(n_les, L, radius=0.8)
    sp_f, sp_c = S.sponge_mask(n_fr, L), S.sponge_mask(n_les, L)
    # GPU side
    fr = qg.QGSolver(n_fr, L=L, beta=beta, U=U, mask=mask_f, sponge=sp_f, kind=qg.QG_NONE, dt=dt, nu=nu)
    fr.set_state(w0)
    fr_series = run_series(fr, 30, 5, fr.get_state)
    ff = qg.qg_grid_filter(fr_series, n_les, L)
    les = qg.QGSolver(n_les, L=L, beta=beta, U=U, mask=mask_c, sponge=sp_c, kind=qg.QG_DLEITH, dt=dt, nu=nu)
    les.set_state(ff[0])
    les_series = run_series(les, 30, 5, les.get_state)
    got = qg.qg_series_compare(les_series, ff, -3, 3)
    # oracle side, independently
    ofr = O.QGOracle(n_fr, L, beta, U, mask_f, sp_f, O.Closure(O.NONE), O.Params(dt=dt, nu=nu))
    ofr.set_state(w0)
    o_fr = run_series(ofr, 30, 5, ofr.get_state)
    o_ff = O.filter_to_les(o_fr, n_les, L)
    oles = O.QGOracle(n_les, L, beta, U, mask_c, sp_c, O.Closure(O.DLEITH), O.Params(dt=dt, nu=nu))
    oles.set_state(o_ff[0])
    o_les = run_series(oles, 30, 5, oles.get_state)
    assert rel(ff, o_ff) < 1e-10
    assert rel(les_series, o_les) < 1e-10
    ref_d, ref_p = O.lag_table(o_les, o_ff, -3, 3)
    # (les[0], ff[0]) is the same field on both sides: its distance is zero up to rounding
    check_table(got, ref_d, ref_p, -3, 1e-8, 1e-9, dist_atol=1e-12 * float(np.nanmax(ref_d)))
    assert np.allclose(got["pcc"][:, 3], O.pcc_series(o_les, o_ff), atol=1e-9)
