"""Failure handling on the GPU without a fault: a bounded device wait that runs out.

The column pass waits on an mbarrier for each tile its TMA loads bring in, and gives up after about one second of
SM clocks: the kernel then sets a status bit and returns, and the host reports QG_ERR_TIMEOUT.  Here the wait is
made to run out safely: QG_INJECT_TMA_STALL (read at creation, off by default) makes one CTA of the first step's
first column pass arm its mbarrier for a tile it never requests, so nothing is in flight when it leaves.  Every
later kernel of the step sees the status flag and returns at once; qg_step refuses further work until qg_set_state
installs a state, after which the handle steps exactly as a fresh one.
"""
import numpy as np
import pytest

import synth as S

pytestmark = pytest.mark.gpu

qg = pytest.importorskip("paper_2508_06678_gb300")


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


@pytest.mark.parametrize("kind", [S.SMAG, S.DLEITH])
def test_bounded_tma_wait_times_out_and_set_state_recovers(kind, monkeypatch):
    n = 256
    wl = S.Workload("t", n, "island", beta=5.0, U=0.5, closure=kind, c=0.17, radius=0.6, seed=3)
    w0 = S.init_field(3, n, k_peak=n / 8)
    monkeypatch.setenv("QG_INJECT_TMA_STALL", "5")
    s = qg.QGSolver.from_workload(wl, precision=qg.QG_FP32)
    monkeypatch.delenv("QG_INJECT_TMA_STALL")
    try:
        s.set_state(w0)
        s.step(1)
        with pytest.raises(qg.QGError) as ei:
            s.sync()
        assert ei.value.code == qg.QG_ERR_TIMEOUT
        with pytest.raises(qg.QGError) as ei:
            s.step(1)
        assert ei.value.code == qg.QG_ERR_TIMEOUT
        # a new state clears the status; the handle then steps exactly as a fresh one
        s.set_state(w0)
        s.step(4)
        s.sync()
        got = s.get_state()
        d = s.diagnostics()
    finally:
        s.close()
    with qg.QGSolver.from_workload(wl, precision=qg.QG_FP32) as clean:
        clean.set_state(w0)
        clean.step(4)
        ref = clean.get_state()
    assert np.array_equal(got, ref)
    assert d["finite"]
