"""GPU (libqg, through the C-ABI) vs the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 of the vorticity): FP64 1e-11 after 100 steps, FP32
2e-4; single transforms and single steps far tighter.  Grid sizes span several
column tiles with ragged tails (N = 18, 48, 54, 96 keep 6, 16, 18, 32 k_x
columns against a tile width of 4 / 2), radix-3 sizes, and the full 2048^2
production workload.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth as S

pytestmark = pytest.mark.gpu

qg = pytest.importorskip("paper_2508_06678_gb300")


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


def make_pair(n, kind, *, geometry="island", beta=5.0, U=0.5, c=0.2, radius=0.8, sponge=True, seed=1,
              k_peak=None, precision=qg.QG_FP64, dt=2e-3, nu=1.0 / 200, mu=0.0):
    wl = S.Workload("t", n, geometry, beta=beta, U=U, closure=kind, c=c, radius=radius, seed=seed, sponge=sponge,
                    dt=dt, nu=nu, mu=mu)
    w0 = S.init_field(seed, n, k_peak=k_peak or max(4.0, n / 8))
    mask = wl.mask() if geometry != "none" else None
    sp = wl.sponge_field()
    ref = O.QGOracle(n, wl.L, beta, U, mask, sp, O.Closure(kind, c=c), O.Params(dt=dt, nu=nu, mu=mu))
    ref.set_state(w0)
    gpu = qg.QGSolver(n, L=wl.L, precision=precision, beta=beta, U=U, mask=mask, sponge=sp, kind=kind, c=c,
                      dt=dt, nu=nu, mu=mu)
    gpu.set_state(w0)
    return ref, gpu, w0


@pytest.mark.parametrize("n", [16, 18, 24, 48, 54, 96, 128, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096])
@pytest.mark.parametrize("prec,tol", [(qg.QG_FP64, 1e-13), (qg.QG_FP32, 2e-6)])
def test_projection_round_trip(n, prec, tol):
    """set_state/get_state = forward then inverse 2-D transform with the 2/3 band (Sec. II-C)."""
    ops = O.Ops(n)
    rng = np.random.default_rng(n)
    w = rng.standard_normal((n, n))
    with qg.QGSolver(n, precision=prec) as s:
        s.set_state(w)
        got = s.get_state()
    ref = O.to_physical(ops, O.project(ops, w))
    assert rel(got, ref) < tol


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("n", [18, 48, 54])
def test_one_step_parity_fp64(kind, n):
    ref, gpu, _ = make_pair(n, kind, radius=0.9)
    ref.step(1)
    gpu.step(1)
    assert rel(gpu.get_state(), ref.get_state()) < 1e-12
    d = gpu.diagnostics()
    if kind in (S.DSMAG, S.DLEITH):
        assert d["coeff"] == pytest.approx(ref.last_coeff, rel=1e-9, abs=1e-300)
    gpu.close()


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("n", [128, 256, 384])
def test_100_step_parity_fp64_island(kind, n):
    """128^2 runs the generic kernels, 256^2 the register-resident 2^p kernels, 384^2 the 3 * 2^p ones."""
    ref, gpu, _ = make_pair(n, kind, radius=0.4, seed=0, k_peak=16.0)
    ref.step(100)
    gpu.step(100)
    err = rel(gpu.get_state(), ref.get_state())
    assert err < 1e-11, err
    d = gpu.diagnostics()
    r = ref.diagnostics()
    assert d["energy"] == pytest.approx(r["energy"], rel=1e-11)
    assert d["enstrophy"] == pytest.approx(r["enstrophy"], rel=1e-11)
    assert d["max_abs_omega"] == pytest.approx(r["max_abs_omega"], rel=1e-10)
    assert d["step"] == 100 and d["finite"]
    gpu.close()


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("n", [96, 256])
def test_100_step_parity_fp32_cape(kind, n):
    ref, gpu, _ = make_pair(n, kind, geometry="cape", beta=10.0, U=1.0, seed=2, k_peak=12.0,
                            precision=qg.QG_FP32)
    ref.step(100)
    gpu.step(100)
    err = rel(gpu.get_state(), ref.get_state())
    assert err < 2e-4, err
    if kind in (S.DSMAG, S.DLEITH):
        # the closure is active at the end of the run, in both implementations
        assert ref.last_coeff > 0
        assert gpu.diagnostics()["coeff"] == pytest.approx(ref.last_coeff, rel=2e-2)
    gpu.close()


def streamfunction(w):
    """psi = lap^-1 w on [0, 2 pi)^2 with zero mean (plain numpy)."""
    n = w.shape[0]
    wh = np.fft.rfft2(w)
    mx = np.arange(n // 2 + 1)[None, :]
    my = np.fft.fftfreq(n, 1.0 / n)[:, None]
    k2 = (mx * mx + my * my).astype(float)
    k2[0, 0] = 1.0
    ph = -wh / k2
    ph[0, 0] = 0.0
    return np.fft.irfft2(ph, s=(n, n))


def field_errors(got, d, ref):
    """Relative error of each reported field against the oracle: w, psi, C, E, Z."""
    r = ref.diagnostics()
    w_ref = ref.get_state()
    out = {"w": rel(got, w_ref), "psi": rel(streamfunction(got), streamfunction(w_ref)),
           "E": abs(d["energy"] - r["energy"]) / r["energy"], "Z": abs(d["enstrophy"] - r["enstrophy"]) / r["enstrophy"]}
    if ref.last_coeff > 0:
        out["C"] = abs(d["coeff"] - ref.last_coeff) / ref.last_coeff
    return out


@pytest.mark.parametrize("kind", [S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
def test_cape512_100_steps_fp64_and_fp32_against_the_oracle(kind):
    """The closure sweep's own configuration (512^2 cape, beta = 10, U = 1, its seed and spectrum), 100 steps:
    the FP64 form within 1e-11 of the oracle and the FP32 form within 2e-4 (relative L2 of w), per field
    (w, psi, E, Z, and C for the dynamic closures, which are active by then)."""
    wl = S.cape512(kind)
    w0 = wl.omega0()
    ref = O.QGOracle(wl.n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(kind, c=wl.c), O.Params())
    ref.set_state(w0)
    ref.step(100)
    dynamic = kind in (S.DSMAG, S.DLEITH)
    if dynamic:
        assert ref.last_coeff > 0
    for prec, tol, ctol in ((qg.QG_FP64, 1e-11, 1e-9), (qg.QG_FP32, 2e-4, 2e-2)):
        with qg.QGSolver.from_workload(wl, precision=prec) as s:
            s.set_state(w0)
            s.step(100)
            got = s.get_state()
            d = s.diagnostics()
        e = field_errors(got, d, ref)
        assert e["w"] < tol, (prec, e)
        assert e["psi"] < tol, (prec, e)
        assert e["E"] < tol and e["Z"] < tol, (prec, e)
        if dynamic:
            assert d["coeff"] > 0 and e["C"] < ctol, (prec, e, d["coeff"], ref.last_coeff)


@pytest.mark.slow
def test_full_size_fp32_100_steps_against_the_oracle_closure_active():
    """2048^2 dynamic Leith, FP32 form, 100 steps against the oracle with the closure active.  The island
    workload's resolved flow leaves the Germano coefficient clipped to zero at this resolution, so the
    same parameters run past the cape (coastal wall and cape, beta = 5, U = 0.5, nu = 1/200, the workload's
    seeded field), where the penalised coast feeds the small scales and C > 0 from the fourth step on.  Relative
    L2 of w and psi within 2e-4, E and Z within 2e-4, C within 2%.  The oracle takes several minutes here."""
    base = S.island2048_dleith()
    wl = S.Workload("cape2048-dleith", base.n, "cape", beta=base.beta, U=base.U, closure=S.DLEITH, seed=base.seed)
    n = wl.n
    w0 = wl.omega0()
    ref = O.QGOracle(n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(wl.closure), O.Params())
    ref.set_state(w0)
    ref.step(100)
    assert ref.last_coeff > 0
    with qg.QGSolver.from_workload(wl, precision=qg.QG_FP32) as s:
        s.set_state(w0)
        s.step(100)
        got = s.get_state()
        d = s.diagnostics()
    e = field_errors(got, d, ref)
    assert d["coeff"] > 0
    assert e["w"] < 2e-4 and e["psi"] < 2e-4, e
    assert e["E"] < 2e-4 and e["Z"] < 2e-4, e
    assert e["C"] < 2e-2, e


@pytest.mark.parametrize("kind", [S.DSMAG, S.DLEITH])
def test_dynamic_coefficient_is_active_and_matches(kind):
    ref, gpu, _ = make_pair(48, kind, seed=1, k_peak=20.0)
    for _ in range(3):
        ref.step(1)
        gpu.step(1)
        d = gpu.diagnostics()
        assert ref.last_coeff > 0
        assert d["coeff"] == pytest.approx(ref.last_coeff, rel=1e-10)
    gpu.close()


def test_rossby_wave_matches_rk3_polynomial():
    n, beta, U, dt, steps = 32, 5.0, 0.5, 2e-3, 50
    x = np.arange(n) * (2 * math.pi / n)
    w = np.cos(2 * x[None, :] + 3 * x[:, None] + 0.3)
    with qg.QGSolver(n, beta=beta, U=U, dt=dt, nu=0.0) as s:
        s.set_state(w)
        s.step(steps)
        got = s.get_state()
    lam = 1j * 2 * (beta / 13.0 - U)
    R = 1 + dt * lam + (dt * lam) ** 2 / 2 + (dt * lam) ** 3 / 6
    ops = O.Ops(n)
    expected = O.to_physical(ops, O.project(ops, w) * R ** steps)
    assert rel(got, expected) < 1e-13


def test_viscous_decay_exact():
    n, nu, mu, dt, steps = 32, 0.05, 0.2, 1e-2, 40
    x = np.arange(n) * (2 * math.pi / n)
    w = np.sin(4 * x[None, :] - 3 * x[:, None])
    with qg.QGSolver(n, dt=dt, nu=nu, mu=mu) as s:
        s.set_state(w)
        s.step(steps)
        got = s.get_state()
    assert np.max(np.abs(got - w * math.exp(-(nu * 25 + mu) * dt * steps))) < 1e-14


def test_nonfinite_state_stops_and_reports():
    n = 32
    w = S.init_field(0, n)
    w[3, 5] = np.nan
    with qg.QGSolver(n, beta=1.0, U=0.3, kind=S.LEITH, c=0.2) as s:
        s.set_state(w)
        s.step(2)
        with pytest.raises(qg.QGError) as ei:
            s.sync()
        assert ei.value.code == qg.QG_ERR_NONFINITE
        with pytest.raises(qg.QGError):
            s.step(1)
        # a finite state resets the flag and stepping resumes
        s.set_state(S.init_field(0, n))
        s.step(1)
        s.sync()


@pytest.mark.parametrize("n", [15, 14, 20, 8, 8192])
def test_bad_grid_sizes_rejected(n):
    with pytest.raises(qg.QGError) as ei:
        qg.QGSolver(n)
    assert ei.value.code == qg.QG_ERR_ARG


def test_device_state_io_with_torch():
    import torch
    n = 48
    w = S.init_field(5, n)
    with qg.QGSolver(n, precision=qg.QG_FP32, stream=torch.cuda.current_stream()) as s:
        s.set_state(torch.tensor(w, dtype=torch.float32, device="cuda"))
        out = torch.empty((n, n), dtype=torch.float32, device="cuda")
        s.get_state(out=out)
        torch.cuda.synchronize()
        ops = O.Ops(n)
        assert rel(out.double().cpu().numpy(), O.to_physical(ops, O.project(ops, w))) < 2e-6


def test_full_size_production_step_fp32():
    """2048^2 dynamic Leith past an island, in the bench's launch configuration:
    one step compared with the oracle over the whole field."""
    wl = S.island2048_dleith()
    n = wl.n
    w0 = wl.omega0()
    ref = O.QGOracle(n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(wl.closure), O.Params())
    ref.set_state(w0)
    ref.step(1)
    with qg.QGSolver.from_workload(wl, precision=qg.QG_FP32) as s:
        s.set_state(w0)
        s.step(1)
        got = s.get_state()
    assert rel(got, ref.get_state()) < 2e-5


@pytest.mark.parametrize("kind", [S.SMAG, S.DLEITH])
@pytest.mark.parametrize("prec,tol", [(qg.QG_FP64, 1e-12), (qg.QG_FP32, 2e-5)])
@pytest.mark.parametrize("n", [512, 384, 768])
def test_fast_and_generic_kernels_agree(kind, prec, tol, n, monkeypatch):
    """The register-resident kernels (2^p and 3 * 2^p engines) and the generic mixed-radix kernels compute the
    same step."""
    wl = S.Workload("t", n, "island", beta=5.0, U=0.5, closure=kind, c=0.2, radius=0.6, seed=7)
    w0 = S.init_field(7, n, k_peak=40.0)
    out = []
    for generic in (False, True):
        if generic:
            monkeypatch.setenv("QG_FORCE_GENERIC", "1")
        else:
            monkeypatch.delenv("QG_FORCE_GENERIC", raising=False)
        with qg.QGSolver.from_workload(wl, precision=prec) as s:
            s.set_state(w0)
            s.step(10)
            out.append(s.get_state())
    assert rel(out[0], out[1]) < tol


# --------------------------------------------------------------------------
# A priori SGS analysis (Sec. III, Eq. 5-8, 15) through qg_sgs_apriori
# --------------------------------------------------------------------------

def _apriori_pair(n_fr, n_les, kind, seed=4, gaussian=True):
    L = 2 * math.pi
    w = S.init_field(seed, n_fr, k_peak=n_fr / 10)
    chi = S.island_mask(n_fr, radius=0.8)
    chs = S.sponge_mask(n_fr)
    cl = O.Closure(kind, c=0.2)
    pr = O.Params()
    ref = O.sgs_apriori(w, n_les, L, chi, chs, cl, pr, 0.5, 5.0, gaussian=gaussian)
    from paper_2508_06678_gb300._lib import qg_closure, qg_params
    got = qg.qg_sgs_apriori(w, n_les, L, chi, chs, qg_closure(kind, 0, 0.2, 2.0),
                            qg_params(pr.dt, pr.nu, pr.mu, pr.eta, pr.sponge_rate), 0.5, 5.0,
                            0 if gaussian else 1)
    return ref, got


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("sizes", [(128, 64), (96, 48), (192, 64)])
def test_apriori_parity(kind, sizes):
    ref, got = _apriori_pair(*sizes, kind)
    pe, pm, parts, r = got
    assert rel(pe, ref[0]) < 1e-10
    for i in range(3):
        if np.linalg.norm(ref[2][i]) > 0:
            assert rel(parts[i], ref[2][i]) < 1e-10
    if kind == S.NONE:
        assert np.all(pm == 0) and math.isnan(r)
    elif math.isnan(ref[3]):
        assert np.linalg.norm(pm) == 0 or math.isnan(r)
    else:
        assert rel(pm, ref[1]) < 1e-9
        assert abs(r - ref[3]) < 1e-9


def test_apriori_no_gaussian_flag():
    ref, got = _apriori_pair(128, 64, S.LEITH, gaussian=False)
    assert rel(got[0], ref[0]) < 1e-10
    assert abs(got[3] - ref[3]) < 1e-9


def test_apriori_full_size_2048_to_512():
    """The configuration's a priori check: a 2048^2 field filtered to 512^2."""
    ref, got = _apriori_pair(2048, 512, S.DLEITH, seed=5)
    assert rel(got[0], ref[0]) < 1e-10
    if not math.isnan(ref[3]):
        assert abs(got[3] - ref[3]) < 1e-8


def test_apriori_rejects_unsupported_sizes():
    from paper_2508_06678_gb300._lib import qg_closure, qg_params
    w = S.init_field(0, 64)
    with pytest.raises(qg.QGError) as ei:
        qg.qg_sgs_apriori(w, 64, 2 * math.pi, None, None, qg_closure(1, 0, 0.2, 2.0),
                          qg_params(2e-3, 5e-3, 0.0, 1e-3, 50.0), 0.5, 5.0)
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED


def test_full_size_production_step_fp64():
    """2048^2 dynamic Leith, FP64 form: two steps against the oracle."""
    wl = S.island2048_dleith()
    w0 = wl.omega0()
    ref = O.QGOracle(wl.n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(wl.closure), O.Params())
    ref.set_state(w0)
    ref.step(2)
    with qg.QGSolver.from_workload(wl, precision=qg.QG_FP64) as s:
        s.set_state(w0)
        s.step(2)
        got = s.get_state()
    assert rel(got, ref.get_state()) < 1e-12


def test_full_size_fp32_error_against_fp64_100_steps():
    """The FP32 form's vorticity error against the (oracle-pinned) FP64 form at
    2048^2 after 100 steps stays within 2e-4; energy and enstrophy within 0.5%."""
    wl = S.island2048_dleith()
    w0 = wl.omega0()
    out = {}
    for prec in (qg.QG_FP64, qg.QG_FP32):
        with qg.QGSolver.from_workload(wl, precision=prec) as s:
            s.set_state(w0)
            s.step(100)
            out[prec] = (s.get_state(), s.diagnostics())
    err = rel(out[qg.QG_FP32][0], out[qg.QG_FP64][0])
    assert err < 2e-4, err
    for key in ("energy", "enstrophy"):
        a, b = out[qg.QG_FP32][1][key], out[qg.QG_FP64][1][key]
        assert abs(a - b) < 5e-3 * abs(b)


def test_island128_smagorinsky_200_steps_fp64_against_the_oracle():
    """The small FP64 configuration in full: 128^2 island, Smagorinsky c_S = 0.17, 200 steps."""
    wl = S.island128_smag()
    ref = O.QGOracle(wl.n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(wl.closure, c=wl.c),
                     O.Params(dt=wl.dt, nu=wl.nu, mu=wl.mu, eta=wl.eta, sponge_rate=wl.sponge_rate))
    ref.set_state(wl.omega0())
    ref.step(wl.steps)
    with qg.QGSolver.from_workload(wl, precision=qg.QG_FP64) as s:
        s.set_state(wl.omega0())
        s.step(wl.steps)
        got = s.get_state()
        d = s.diagnostics()
    assert rel(got, ref.get_state()) < 1e-11
    r = ref.diagnostics()
    assert d["energy"] == pytest.approx(r["energy"], rel=1e-11)
    assert d["enstrophy"] == pytest.approx(r["enstrophy"], rel=1e-11)


@pytest.mark.parametrize("kind", [S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
def test_cape512_2000_steps_fp32_energy_and_enstrophy_within_half_percent(kind):
    """Long runs of the closure sweep (512^2 cape, beta = 10, U = 1, 2000 steps): the FP32 form's energy and
    enstrophy stay within 0.5% of the FP64 form's (which the oracle pins), every 500 steps."""
    wl = S.cape512(kind)
    w0 = wl.omega0()
    solvers = {p: qg.QGSolver.from_workload(wl, precision=p) for p in (qg.QG_FP64, qg.QG_FP32)}
    for s in solvers.values():
        s.set_state(w0)
    for _ in range(4):
        diag = {}
        for p, s in solvers.items():
            s.step(500)
            diag[p] = s.diagnostics()
        for key in ("energy", "enstrophy"):
            a, b = diag[qg.QG_FP32][key], diag[qg.QG_FP64][key]
            assert abs(a - b) < 5e-3 * abs(b), (key, a, b)
        assert diag[qg.QG_FP32]["finite"]
    for s in solvers.values():
        s.close()


@pytest.mark.parametrize("n,prec", [(256, qg.QG_FP32), (96, qg.QG_FP64), (2048, qg.QG_FP32), (768, qg.QG_FP32)])
def test_graph_replay_is_bitwise_eager(n, prec, monkeypatch):
    """qg_step replays one captured step as a CUDA graph on a capturable stream;
    the result is bit-identical to launching the same kernels one by one."""
    import torch
    wl = S.Workload("t", n, "island", beta=5.0, U=0.5, closure=S.DLEITH, radius=0.5, seed=2)
    w0 = S.init_field(2, n, k_peak=n / 8)
    out = []
    for eager in (False, True):
        if eager:
            monkeypatch.setenv("QG_NO_GRAPH", "1")
        else:
            monkeypatch.delenv("QG_NO_GRAPH", raising=False)
        stream = torch.cuda.Stream()
        with qg.QGSolver.from_workload(wl, precision=prec, stream=stream) as s:
            s.set_state(w0)
            s.step(1)
            s.step(7)
            out.append((s.get_state(), s.diagnostics()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["step"] == out[1][1]["step"] == 8


# --------------------------------------------------------------------------
# The paper's own scheme (Sec. II-E, Eq. 4): CN / AB2 with the AB2 sponge split
# --------------------------------------------------------------------------

def make_ab2_pair(n, kind, precision=qg.QG_FP64, seed=1, k_peak=None, geometry="island", beta=5.0, U=0.5,
                  stream=None):
    dt, eta = 5e-4, 2e-3  # the scheme treats the penalisation explicitly: eta > dt (Sec. II-E)
    wl = S.Workload("t", n, geometry, beta=beta, U=U, closure=kind, c=0.2, radius=0.8, seed=seed, dt=dt, eta=eta)
    w0 = S.init_field(seed, n, k_peak=k_peak or max(4.0, n / 8))
    mask = wl.mask()
    sp = wl.sponge_field()
    ref = O.QGOracle(n, wl.L, beta, U, mask, sp, O.Closure(kind, c=0.2),
                     O.Params(dt=dt, eta=eta, scheme=O.AB2CN))
    ref.set_state(w0)
    gpu = qg.QGSolver(n, L=wl.L, precision=precision, beta=beta, U=U, mask=mask, sponge=sp, kind=kind, c=0.2,
                      dt=dt, eta=eta, scheme=qg.QG_SCHEME_AB2CN, stream=stream)
    gpu.set_state(w0)
    return ref, gpu, w0


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("n", [48, 54, 256])
def test_ab2cn_parity_fp64(kind, n):
    ref, gpu, _ = make_ab2_pair(n, kind, k_peak=n / 6)
    for steps in (1, 59):
        ref.step(steps)
        gpu.step(steps)
        err = rel(gpu.get_state(), ref.get_state())
        assert err < 1e-11, (steps, err)
    if kind in (S.DSMAG, S.DLEITH):
        assert gpu.diagnostics()["coeff"] == pytest.approx(ref.last_coeff, rel=1e-9, abs=1e-300)
    gpu.close()


@pytest.mark.parametrize("kind", [S.SMAG, S.DLEITH])
def test_ab2cn_parity_fp32_cape(kind):
    ref, gpu, _ = make_ab2_pair(256, kind, precision=qg.QG_FP32, geometry="cape", beta=10.0, U=1.0, seed=2)
    ref.step(100)
    gpu.step(100)
    assert rel(gpu.get_state(), ref.get_state()) < 2e-4
    gpu.close()


def test_ab2cn_history_restarts_after_set_state():
    ref, gpu, w0 = make_ab2_pair(48, S.LEITH)
    ref.step(5)
    gpu.step(5)
    w_mid = S.init_field(9, 48, k_peak=8.0)
    ref.set_state(w_mid)
    gpu.set_state(w_mid)
    ref.step(7)
    gpu.step(7)
    assert rel(gpu.get_state(), ref.get_state()) < 1e-12
    gpu.close()


def test_ab2cn_graph_replay_is_bitwise_eager(monkeypatch):
    import torch
    out = []
    for eager in (False, True):
        if eager:
            monkeypatch.setenv("QG_NO_GRAPH", "1")
        else:
            monkeypatch.delenv("QG_NO_GRAPH", raising=False)
        _, gpu, _ = make_ab2_pair(256, S.DSMAG, precision=qg.QG_FP32, stream=torch.cuda.Stream())
        gpu.step(1)
        gpu.step(9)
        out.append(gpu.get_state())
        gpu.close()
    assert np.array_equal(out[0], out[1])
