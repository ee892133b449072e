"""GPU discrete adjoint (qg_step_vjp) against the oracle's adjoint, which finite differences pin.

FP64: gradients within 1e-10 relative L2 (the recomputation and transforms differ from the oracle's by
rounding only); parameter derivatives within 1e-9.  FP32: 1e-4.  Grid sizes exercise the generic kernels (48,
54, 96) and the register-resident ones (256).  Multi-step gradients go through checkpointed rollouts.
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


def make(n, kind, c, precision=qg.QG_FP64, mask=True, sponge=True, dt=5e-3, eta=2e-2, rate=50.0, beta=5.0, U=0.5):
    chi = S.island_mask(n, L, radius=0.9) if mask else None
    chs = S.sponge_mask(n, L) if sponge else None
    params = O.Params(dt=dt, eta=eta, sponge_rate=rate)
    solver = qg.QGSolver(n, precision=precision, beta=beta, U=U, mask=chi, sponge=chs, kind=kind, c=c, dt=dt,
                         eta=eta, sponge_rate=rate)
    ops = O.Ops(n, L)
    return solver, ops, chi, chs, params, O.Closure(kind, c=c), beta, U


CASES = [(48, O.NONE, 0.0), (48, O.SMAG, 0.5), (54, O.LEITH, 0.6), (96, O.LEITH, 0.4), (256, O.SMAG, 0.3),
         (256, O.LEITH, 0.5)]


@pytest.mark.parametrize("n,kind,c", CASES)
def test_step_vjp_matches_the_oracle_fp64(n, kind, c):
    solver, ops, chi, chs, params, cl, beta, U = make(n, kind, c)
    w = S.init_field(3, n, L, k_peak=n / 6)
    lam_next = np.random.default_rng(n).standard_normal((n, n))
    got, g = solver.step_vjp(w, lam_next)
    ref, gr = O.full_step_vjp(ops, O.project(ops, w), lam_next, beta, U, cl, params, chi, chs)
    assert rel(got, ref) < 1e-10
    for key in ("C", "c", "sponge_rate"):
        if gr[key] != 0.0:
            assert g[key] == pytest.approx(gr[key], rel=1e-9), key


@pytest.mark.parametrize("mask,sponge", [(False, False), (True, False), (False, True)])
def test_step_vjp_without_mask_or_sponge(mask, sponge):
    solver, ops, chi, chs, params, cl, beta, U = make(64, O.LEITH, 0.5, mask=mask, sponge=sponge)
    w = S.init_field(5, 64, L, k_peak=10)
    lam_next = np.random.default_rng(1).standard_normal((64, 64))
    got, g = solver.step_vjp(w, lam_next)
    ref, gr = O.full_step_vjp(ops, O.project(ops, w), lam_next, beta, U, cl, params, chi, chs)
    assert rel(got, ref) < 1e-10
    assert g["sponge_rate"] == pytest.approx(gr["sponge_rate"], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("n,kind,c", [(256, O.LEITH, 0.5), (96, O.SMAG, 0.4)])
def test_step_vjp_fp32(n, kind, c):
    solver, ops, chi, chs, params, cl, beta, U = make(n, kind, c, precision=qg.QG_FP32)
    w = S.init_field(3, n, L, k_peak=n / 6)
    lam_next = np.random.default_rng(2).standard_normal((n, n))
    got, g = solver.step_vjp(w.astype(np.float32), lam_next.astype(np.float32))
    ref, gr = O.full_step_vjp(ops, O.project(ops, w), lam_next, beta, U, cl, params, chi, chs)
    assert rel(got.astype(np.float64), ref) < 1e-4
    assert g["c"] == pytest.approx(gr["c"], rel=1e-3)


def test_device_buffers_match_host_and_leave_the_state_alone():
    import torch
    n = 256
    solver, ops, chi, chs, params, cl, beta, U = make(n, O.LEITH, 0.5)
    w = S.init_field(3, n, L, k_peak=20)
    lam_next = np.random.default_rng(4).standard_normal((n, n))
    solver.set_state(w)
    solver.step(3)
    before = solver.get_state()
    host, gh = solver.step_vjp(w, lam_next)
    dev, gd = solver.step_vjp(torch.from_numpy(w).cuda(), torch.from_numpy(lam_next).cuda())
    assert np.array_equal(host, dev.cpu().numpy())
    assert gh == gd
    assert np.array_equal(solver.get_state(), before)
    solver.step(2)
    ref = qg.QGSolver(n, beta=beta, U=U, mask=chi, sponge=chs, kind=O.LEITH, c=0.5, dt=5e-3, eta=2e-2)
    ref.set_state(w)
    ref.step(5)
    assert np.array_equal(solver.get_state(), ref.get_state())


def positive_coefficient_state(n, kind):
    """A state whose dynamic coefficient is positive (the quotient, not the clip, is differentiated)."""
    ops = O.Ops(n, L)
    for seed in range(1, 60):
        w = S.init_field(seed, n, L, k_peak=n / 3)
        if O.germano_coefficient(ops, O.project(ops, w), O.Closure(kind), 0.5)[0] > 0.0:
            return w
    raise RuntimeError("no state with a positive coefficient")


@pytest.mark.parametrize("n,kind", [(48, O.DSMAG), (54, O.DLEITH), (256, O.DLEITH), (256, O.DSMAG)])
def test_dynamic_step_vjp_matches_the_oracle_fp64(n, kind):
    solver, ops, chi, chs, params, cl, beta, U = make(n, kind, 0.0)
    w = positive_coefficient_state(n, kind)
    lam_next = np.random.default_rng(n + kind).standard_normal((n, n))
    got, g = solver.step_vjp(w, lam_next)
    ref, gr = O.full_step_vjp(ops, O.project(ops, w), lam_next, beta, U, cl, params, chi, chs)
    assert rel(got, ref) < 1e-10
    assert g["C"] == pytest.approx(gr["C"], rel=1e-9)
    assert g["sponge_rate"] == pytest.approx(gr["sponge_rate"], rel=1e-9)
    assert g["c"] == 0.0


def test_dynamic_step_vjp_fp32():
    n, kind = 256, O.DLEITH
    solver, ops, chi, chs, params, cl, beta, U = make(n, kind, 0.0, precision=qg.QG_FP32)
    w = positive_coefficient_state(n, kind)
    lam_next = np.random.default_rng(3).standard_normal((n, n))
    got, _ = solver.step_vjp(w.astype(np.float32), lam_next.astype(np.float32))
    ref, _ = O.full_step_vjp(ops, O.project(ops, w), lam_next, beta, U, cl, params, chi, chs)
    assert rel(got.astype(np.float64), ref) < 1e-4


def test_unsupported_configurations_are_refused():
    s = qg.QGSolver(48, kind=O.SMAG, c=0.2, scheme=qg.QG_SCHEME_AB2CN, eta=1e-2)
    with pytest.raises(qg.QGError) as e:
        s.step_vjp(np.zeros((48, 48)), np.zeros((48, 48)))
    assert e.value.code == qg.QG_ERR_UNSUPPORTED


def oracle_rollout_grad(ops, w0, nsteps, obs, beta, U, cl, params, chi, chs):
    states = [O.project(ops, w0)]
    for _ in range(nsteps):
        states.append(O.full_step(ops, states[-1], beta, U, cl, params, chi, chs)[0])
    lam = np.zeros((ops.n, ops.n))
    grads = {"C": 0.0, "c": 0.0, "sponge_rate": 0.0}
    for k in range(nsteps - 1, -1, -1):
        if k + 1 in obs:
            lam = lam + obs[k + 1]
        lam, g = O.full_step_vjp(ops, states[k], lam, beta, U, cl, params, chi, chs)
        for key in grads:
            grads[key] += g[key]
    return lam, grads


def test_checkpointed_rollout_gradient_matches_the_oracle():
    from paper_2508_06678_gb300.adjoint import rollout_grad
    n, nsteps = 48, 23
    solver, ops, chi, chs, params, cl, beta, U = make(n, O.SMAG, 0.5)
    w0 = S.init_field(6, n, L, k_peak=8)
    rng = np.random.default_rng(9)
    obs = {k: rng.standard_normal((n, n)) for k in (5, 11, 20, 23)}
    got, g = rollout_grad(solver, w0, nsteps, obs, checkpoint_every=7)
    ref, gr = oracle_rollout_grad(ops, w0, nsteps, obs, beta, U, cl, params, chi, chs)
    assert rel(got.cpu().numpy(), ref) < 1e-9
    assert g["c"] == pytest.approx(gr["c"], rel=1e-8)
    assert g["sponge_rate"] == pytest.approx(gr["sponge_rate"], rel=1e-8)


def test_autograd_rollout_mse_loss():
    import torch
    from paper_2508_06678_gb300.adjoint import rollout
    n, nsteps = 48, 12
    solver, ops, chi, chs, params, cl, beta, U = make(n, O.LEITH, 0.5)
    w0 = torch.from_numpy(S.init_field(7, n, L, k_peak=8)).cuda().requires_grad_(True)
    target = torch.from_numpy(S.init_field(8, n, L, k_peak=8)).cuda()
    states = rollout(solver, w0, nsteps, [4, 8, 12], checkpoint_every=5)
    loss = ((states - target) ** 2).mean()
    loss.backward()
    st = [O.project(ops, w0.detach().cpu().numpy())]
    for _ in range(nsteps):
        st.append(O.full_step(ops, st[-1], beta, U, cl, params, chi, chs)[0])
    tgt = target.cpu().numpy()
    obs = {k: 2.0 * (ops.inv(st[k]) - tgt) / (3 * n * n) for k in (4, 8, 12)}
    ref, _ = oracle_rollout_grad(ops, w0.detach().cpu().numpy(), nsteps, obs, beta, U, cl, params, chi, chs)
    assert rel(w0.grad.cpu().numpy(), ref) < 1e-9
    assert set(solver.param_grads) == {"C", "c", "sponge_rate"}


def test_step_vjp_on_a_three_times_power_of_two_grid():
    solver, ops, chi, chs, params, cl, beta, U = make(384, O.LEITH, 0.5)
    w = S.init_field(3, 384, L, k_peak=40)
    lam_next = np.random.default_rng(5).standard_normal((384, 384))
    got, g = solver.step_vjp(w, lam_next)
    ref, gr = O.full_step_vjp(ops, O.project(ops, w), lam_next, beta, U, cl, params, chi, chs)
    assert rel(got, ref) < 1e-10
    assert g["c"] == pytest.approx(gr["c"], rel=1e-9)
