"""Device tensors and streams: a solver on its own stream, fed and read by torch ops on the current stream.

QGSolver's methods order the handle's stream against torch's current stream
(qg_stream plus stream waits), so results must not depend on which stream the
solver runs on.  Each check queues a long matmul on the current stream right
before handing the library a tensor that torch writes after it, so a missing
wait would read stale memory.  Results are compared bit for bit with the same
work on the default stream.
"""
import math

import numpy as np
import pytest

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


def busy(torch):
    """A few milliseconds of work on the current stream."""
    a = torch.randn((4096, 4096), device="cuda")
    for _ in range(4):
        a = a @ a
        a = a / a.norm()
    return a


def make(n, precision, stream=None):
    return qg.QGSolver(n, precision=precision, beta=5.0, U=0.5, mask=S.island_mask(n, L, radius=0.9),
                       sponge=S.sponge_mask(n, L), kind=qg.QG_SMAG, c=0.3, dt=5e-3, eta=2e-2, stream=stream)


def test_qg_stream_reports_the_create_stream():
    import torch
    st = torch.cuda.Stream()
    s = make(64, qg.QG_FP64, stream=st)
    assert qg.qg_stream(s.h) == st.cuda_stream
    assert qg.qg_stream(make(64, qg.QG_FP64).h) == 0


@pytest.mark.parametrize("precision", [qg.QG_FP64, qg.QG_FP32])
def test_state_round_trip_on_a_side_stream(precision):
    import torch
    n = 128
    tdt = torch.float64 if precision == qg.QG_FP64 else torch.float32
    w0 = torch.from_numpy(S.init_field(2, n, L, k_peak=10.0)).to(tdt)
    results = []
    for stream in (None, torch.cuda.Stream()):
        s = make(n, precision, stream)
        busy(torch)
        w = w0.cuda() * 1.0  # written on the current stream after the busy work
        s.set_state(w)
        s.step(7)
        out = torch.empty((n, n), dtype=tdt, device="cuda")
        s.get_state(out=out)
        results.append((out * 2.0).cpu().numpy())  # read on the current stream
        del w
    assert np.array_equal(results[0], results[1])


@pytest.mark.parametrize("precision", [qg.QG_FP64, qg.QG_FP32])
def test_checkpointed_gradient_on_a_side_stream(precision):
    import torch
    from paper_2508_06678_gb300.adjoint import rollout_grad
    n, K = 64, 12
    tdt = torch.float64 if precision == qg.QG_FP64 else torch.float32
    w0 = torch.from_numpy(S.init_field(4, n, L, k_peak=8.0)).to(tdt).cuda()
    obs = {k: torch.from_numpy(np.random.default_rng(k).standard_normal((n, n))).to(tdt).cuda() for k in (4, 8, 12)}
    out = []
    for stream in (None, torch.cuda.Stream()):
        s = make(n, precision, stream)
        busy(torch)
        lam, g = rollout_grad(s, w0 * 1.0, K, {k: v * 1.0 for k, v in obs.items()}, checkpoint_every=5)
        out.append((lam.cpu().numpy(), g))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_series_compare_on_a_side_stream(dtype):
    import torch
    les = S.wave_series(3, 48, 12, L, noise=0.1).astype(dtype)
    ff = S.wave_series(3, 48, 12, L, t0=0.2, noise=0.1, noise_seed=5).astype(dtype)
    host = qg.qg_series_compare(les, ff, -4, 4)
    busy(torch)
    dl = torch.from_numpy(les).cuda() * 1.0
    df = torch.from_numpy(ff).cuda() * 1.0
    dev = qg.qg_series_compare(dl, df, -4, 4, stream=torch.cuda.Stream())
    for k in ("dist", "pcc", "mean_dist"):
        assert np.array_equal(host[k], dev[k], equal_nan=True)
    assert host["phase"] == dev["phase"]
