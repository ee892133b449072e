"""Edge cases of the step on the GPU against the FP64 oracle: the largest grids of each register-resident engine,
degenerate fields (zero, a single Fourier mode, content only at the edge of the 2/3 band), and a zero-step call.
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
    import os
    from paper_2508_06678_gb300._lib import LIB_PATH
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    qg.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pair(n, kind, w0, *, geometry="island", U=0.5, beta=5.0, sponge=True, precision=qg.QG_FP64):
    wl = S.Workload("edge", n, geometry, beta=beta, U=U, closure=kind, c=0.2, radius=0.5, seed=0, sponge=sponge)
    mask = wl.mask() if geometry != "none" else None
    sp = wl.sponge_field()
    ref = O.QGOracle(n, L, beta, U, mask, sp, O.Closure(kind, c=0.2), O.Params())
    ref.set_state(w0)
    gpu = qg.QGSolver(n, L=L, precision=precision, beta=beta, U=U, mask=mask, sponge=sp, kind=kind, c=0.2)
    gpu.set_state(w0)
    return ref, gpu


@pytest.mark.parametrize("n", [4096, 3072])
def test_largest_grids_one_step(n):
    """The largest grid of each engine (2^12 with 16 elements per thread, 3 * 2^10 with 12), past an island with the
    sponge, one step against the oracle: dynamic Leith in FP32, Leith in FP64.  The FP64 form of the dynamic
    closures does not fit the row pass's shared memory at these sizes and is refused with QG_ERR_UNSUPPORTED.

    The FP32 tolerance grows with N: past a coast the penalty term's curl (Eq. 2) carries the mask's one-cell edge,
    so its size, and the FP32 rounding of it, scale with 1/dx.  Measured one-step errors past the island: 1.1e-5
    (1024^2), 2.1e-5 (2048^2), 4.1e-5 (4096^2); 4e-7 at 4096^2 with neither coast nor closure."""
    w0 = S.init_field(17, n, L, k_peak=n / 16)
    for kind, prec, tol in ((S.DLEITH, qg.QG_FP32, 2.5e-8 * n), (S.LEITH, qg.QG_FP64, 1e-12)):
        ref, gpu = pair(n, kind, w0, precision=prec)
        ref.step(1)
        gpu.step(1)
        got = gpu.get_state()
        d = gpu.diagnostics()
        gpu.close()
        assert rel(got, ref.get_state()) < tol, (kind, prec, rel(got, ref.get_state()))
        if kind == S.DLEITH and ref.last_coeff > 0:
            assert d["coeff"] == pytest.approx(ref.last_coeff, rel=2e-2)
    with pytest.raises(qg.QGError) as ei:
        qg.QGSolver(n, precision=qg.QG_FP64, kind=S.DLEITH)
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", [S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("prec", [qg.QG_FP64, qg.QG_FP32])
def test_zero_field_without_forcing_stays_zero(kind, prec):
    """No vorticity, no inflow, no coast, no sponge: every term of Eq. 1 vanishes and the state stays exactly zero
    (the dynamic coefficient takes its <MM> = 0 branch, C = 0)."""
    for n in (48, 256):
        with qg.QGSolver(n, precision=prec, beta=5.0, U=0.0, kind=kind, c=0.2) as s:
            s.set_state(np.zeros((n, n)))
            s.step(5)
            w = s.get_state()
            d = s.diagnostics()
        assert np.all(w == 0.0)
        assert d["coeff"] == (0.0 if kind in (S.DSMAG, S.DLEITH) else d["coeff"])
        assert d["energy"] == 0.0 and d["enstrophy"] == 0.0 and d["finite"]


@pytest.mark.parametrize("n", [48, 256])
def test_zero_field_with_inflow_past_the_island(n):
    """A zero initial field with the uniform inflow: the penalised coast generates vorticity (Eq. 2) from the first
    step on; 10 steps against the oracle."""
    ref, gpu = pair(n, S.DLEITH, np.zeros((n, n)))
    ref.step(10)
    gpu.step(10)
    expect = ref.get_state()
    assert np.linalg.norm(expect) > 0
    assert rel(gpu.get_state(), expect) < 1e-11
    gpu.close()


@pytest.mark.parametrize("kind", [S.DSMAG, S.DLEITH])
@pytest.mark.parametrize("n", [48, 256])
def test_single_mode_field_gives_zero_dynamic_coefficient(kind, n):
    """A single Fourier mode has J(psi, w) = 0 at every filter level, so H vanishes to rounding and the Germano
    coefficient (Eq. 12, 14) is zero to rounding on both sides (static Leith/Smagorinsky values here would be
    ~1e-7); without coast, sponge and inflow the mode then only decays and rotates."""
    x = np.arange(n) * (L / n)
    w0 = np.cos(3 * x[None, :] + 2 * x[:, None] + 0.4)
    ref, gpu = pair(n, kind, w0, geometry="none", U=0.0, sponge=False)
    for _ in range(3):
        ref.step(1)
        gpu.step(1)
        assert ref.last_coeff < 1e-13
        assert gpu.diagnostics()["coeff"] < 1e-13
    assert rel(gpu.get_state(), ref.get_state()) < 1e-12
    gpu.close()


@pytest.mark.parametrize("n", [54, 256, 384])
def test_field_at_the_edge_of_the_band(n):
    """Content only in the outermost kept wavenumbers |m_x| = K or |m_y| = K (the 2/3 rule's edge, where aliasing
    would first appear): 5 steps of Smagorinsky past the island against the oracle."""
    K = (n - 1) // 3
    x = np.arange(n) * (L / n)
    X, Y = x[None, :], x[:, None]
    w0 = np.cos(K * X + 1 * Y) + 0.7 * np.sin(2 * X - K * Y) + 0.3 * np.cos(K * X + K * Y)
    ref, gpu = pair(n, S.SMAG, w0)
    ref.step(5)
    gpu.step(5)
    assert rel(gpu.get_state(), ref.get_state()) < 1e-11
    gpu.close()


def test_zero_steps_leave_the_state_unchanged():
    n = 256
    w0 = S.init_field(5, n, L, k_peak=n / 8)
    with qg.QGSolver(n, precision=qg.QG_FP32, beta=5.0, U=0.5, kind=S.DLEITH) as s:
        s.set_state(w0)
        a = s.get_state()
        s.step(0)
        b = s.get_state()
        d = s.diagnostics()
    assert np.array_equal(a, b) and d["step"] == 0
