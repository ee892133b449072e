"""Gradients through many steps with the discrete adjoint (qg_step_vjp) and checkpointing.

A loss that depends on the states w_k at some steps k of a K-step run has the
gradient w.r.t. w_0 (and the closure constant and the sponge rate) given by the
step's vector-Jacobian product applied from step K down to 0, adding dloss/dw_k
on the way.  The forward run stores every ``checkpoint_every``-th state; the
backward sweep re-runs each segment from its checkpoint, keeps that segment's
states and applies ``qg_step_vjp`` in reverse.  Memory: K / checkpoint_every +
checkpoint_every states; work: two forward runs and one adjoint run.

Arithmetic runs in libqg; this module only sequences calls.  States and
gradients are torch CUDA tensors in the solver's precision.  The solver's own
state is overwritten (it ends at a checkpoint of the last segment).
"""
from __future__ import annotations

from ._lib import QG_FP32

__all__ = ["rollout_states", "rollout_grad", "rollout"]


def _dtype(solver):
    import torch
    return torch.float32 if solver.cfg.precision == QG_FP32 else torch.float64


def rollout_states(solver, omega0, nsteps: int, checkpoint_every: int = 20):
    """Run nsteps from omega0; returns (checkpoints {k: state}, final state) as device tensors."""
    import torch
    n = solver.cfg.n
    dt = _dtype(solver)
    w = torch.as_tensor(omega0, device="cuda").to(dt).contiguous()
    solver.set_state(w)
    ckpts = {}
    for k in range(nsteps):
        if k % checkpoint_every == 0:
            ckpts[k] = solver.get_state(out=torch.empty((n, n), dtype=dt, device="cuda"))
        solver.step(1)
    final = solver.get_state(out=torch.empty((n, n), dtype=dt, device="cuda"))
    return ckpts, final


def rollout_grad(solver, omega0, nsteps: int, obs: dict, checkpoint_every: int = 20, ckpts: dict | None = None):
    """Gradient of loss = sum over k in obs of <obs[k], w_k> (obs[k] = dloss/dw_k, physical N x N).

    Returns (dloss/dw_0 on the 2/3 band, {"C", "c", "sponge_rate"}) with the
    parameter derivatives summed over all steps.
    """
    import torch
    n = solver.cfg.n
    dt = _dtype(solver)
    obs = {int(k): torch.as_tensor(v, device="cuda").to(dt).contiguous() for k, v in obs.items()}
    if any(k < 0 or k > nsteps for k in obs):
        raise ValueError("observed steps must lie in [0, nsteps]")
    if ckpts is None:
        ckpts, _ = rollout_states(solver, omega0, nsteps, checkpoint_every)
    lam = torch.zeros((n, n), dtype=dt, device="cuda")
    grads = {"C": 0.0, "c": 0.0, "sponge_rate": 0.0}
    starts = sorted(ckpts)
    for i in reversed(range(len(starts))):
        k0 = starts[i]
        k1 = starts[i + 1] if i + 1 < len(starts) else nsteps
        states = [ckpts[k0]]
        solver.set_state(ckpts[k0])
        for _ in range(k0 + 1, k1):
            solver.step(1)
            states.append(solver.get_state(out=torch.empty((n, n), dtype=dt, device="cuda")))
        for k in range(k1 - 1, k0 - 1, -1):
            if k + 1 in obs:
                lam = lam + obs[k + 1]
            lam, g = solver.step_vjp(states[k - k0], lam)
            for key in grads:
                grads[key] += g[key]
    if 0 in obs:
        # the state is the projection of the input field: its gradient is the projected one
        lam = lam + _project(solver, obs[0])
    return lam, grads


def _project(solver, f):
    """The 2/3-band, zero-mean projection of a physical field (set_state then get_state)."""
    import torch
    solver.set_state(f)
    return solver.get_state(out=torch.empty_like(f))


def rollout(solver, omega0, nsteps: int, obs_steps, checkpoint_every: int = 20):
    """States at ``obs_steps`` as a (len, N, N) tensor that backpropagates to omega0.

    After backward, ``solver.param_grads`` holds the derivatives of the loss in
    C, c and the sponge rate.
    """
    import torch

    class _Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w0):
            n = solver.cfg.n
            dt = _dtype(solver)
            steps = sorted(int(k) for k in obs_steps)
            want = set(steps)
            solver.set_state(w0.detach().to(dt).contiguous())
            ckpts, out = {}, {}
            for k in range(nsteps + 1):
                if k in want or k % checkpoint_every == 0:
                    s = solver.get_state(out=torch.empty((n, n), dtype=dt, device="cuda"))
                    if k in want:
                        out[k] = s
                    if k % checkpoint_every == 0 and k < nsteps:
                        ckpts[k] = s
                if k < nsteps:
                    solver.step(1)
            ctx.ckpts = ckpts
            ctx.steps = steps
            return torch.stack([out[k] for k in [int(x) for x in obs_steps]]).to(w0.dtype)

        @staticmethod
        def backward(ctx, grad_out):
            obs = {}
            for i, k in enumerate(int(x) for x in obs_steps):
                obs[k] = obs.get(k, 0) + grad_out[i]
            lam, g = rollout_grad(solver, None, nsteps, obs, checkpoint_every, ckpts=ctx.ckpts)
            solver.param_grads = g
            return lam.to(grad_out.dtype)

    return _Rollout.apply(torch.as_tensor(omega0, device="cuda"))
