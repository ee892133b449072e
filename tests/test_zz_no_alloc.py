"""qg_field_stats_static: field statistics without any device allocation.

Callers that cannot allocate device memory where they need these numbers
(a host framework that owns all device memory, code that must not trigger an
allocation's synchronisation, real-time loops) get energy, enstrophy, max |w|
and finiteness from this entry point, whose scratch is a fixed static device
array.  Its results must match what the allocating path reports
(qg_set_state + qg_diagnostics on a handle) for the same field, on two calls
in a row (the second call reuses the array the first one left behind).
"""
import ctypes as C

import numpy as np
import pytest

import synth as S

pytestmark = pytest.mark.gpu

qg = pytest.importorskip("paper_2508_06678_gb300")


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2508_06678_gb300._lib import LIB_PATH
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    return qg.load()


def reference_stats(w, n, prec):
    with qg.QGSolver(n, precision=prec) as s:
        s.set_state(w)
        d = s.diagnostics()
    return np.array([d["energy"], d["enstrophy"], d["max_abs_omega"], 1.0 if d["finite"] else 0.0])


@pytest.mark.parametrize("n", [48, 96, 256, 512])
@pytest.mark.parametrize("prec", [qg.QG_FP64, qg.QG_FP32])
def test_static_scratch_stats_match_allocating_path(lib, n, prec):
    import torch
    dt = torch.float64 if prec == qg.QG_FP64 else torch.float32
    tol = 1e-12 if prec == qg.QG_FP64 else 2e-5
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for seed in (3, 4):  # two calls in a row share the static scratch
        w = S.init_field(seed, n, k_peak=n / 8) * (1.0 + seed)
        wd = torch.tensor(w, dtype=dt, device="cuda")
        rc = lib.qg_field_stats_static(C.c_void_p(wd.data_ptr()), n, 2 * np.pi,
                                       qg.QG_FP32 if prec == qg.QG_FP32 else qg.QG_FP64,
                                       C.c_void_p(stream.cuda_stream), C.c_void_p(out.data_ptr()))
        assert rc == qg.QG_OK, lib.qg_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = reference_stats(w.astype(np.float32) if prec == qg.QG_FP32 else w, n, prec)
        np.testing.assert_allclose(got[:3], ref[:3], rtol=tol, atol=0)
        assert got[3] == 1.0 and ref[3] == 1.0


def test_rejects_grid_beyond_static_capacity(lib):
    import torch
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.zeros((768, 768), dtype=torch.float64, device="cuda")
    rc = lib.qg_field_stats_static(C.c_void_p(w.data_ptr()), 768, 2 * np.pi, qg.QG_FP64, None,
                                   C.c_void_p(out.data_ptr()))
    assert rc == qg.QG_ERR_ARG
    assert b"512" in lib.qg_last_error()


def test_calls_after_warm_up_allocate_no_device_memory(lib):
    """The property the entry point exists for: once a warm-up call per device has loaded the module, further
    calls (every size and dtype, up to the 512^2 FP64 maximum) leave the device's free memory unchanged."""
    import torch
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    fields = {}
    for n in (48, 512):
        for prec, dt in ((qg.QG_FP64, torch.float64), (qg.QG_FP32, torch.float32)):
            fields[(n, prec)] = torch.tensor(S.init_field(n, n, k_peak=n / 8), dtype=dt, device="cuda")

    def call(n, prec):
        rc = lib.qg_field_stats_static(C.c_void_p(fields[(n, prec)].data_ptr()), n, 2 * np.pi, prec,
                                       C.c_void_p(stream.cuda_stream), C.c_void_p(out.data_ptr()))
        assert rc == qg.QG_OK, lib.qg_last_error()

    for key in fields:  # warm-up: module load, kernel attributes
        call(*key)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for key in fields:
            call(*key)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)
