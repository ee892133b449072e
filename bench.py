"""Benchmark: grid-point-steps/s of the QG LES step on one GB300 (or N replicas).

Default workload: 2048^2 island, dynamic Leith, beta = 5, U = 0.5, FP32 fields
with FP64 Germano sums / diagnostics / low-k inversion (the production step).
A "step" is one full time step: three RK3 stages with the dynamic
coefficient, the viscous factor, the Brinkman and the sponge sub-steps.

Prints one JSON line.  Multi-GPU (torchrun, one process per GPU) runs
independent replicas: the step has no data-parallel split on one grid.

The roofline object reports the dominant kernel class (the stage row pass)
against the measured HBM copy peak: "achieved" / "frac" count the
full-field round-trip bytes (every 2-D transform moves one N^2 field between
its passes), "band_model" the arrays this design keeps (2/3 band only), and
"step_frac" the whole step on the full-field model.  Other workloads:
--scheme ab2cn (Eq. 4), --workload ensemble96 | adjoint256 | series512.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth as S  # noqa: E402

WORKLOADS = {
    "island2048-dleith": S.island2048_dleith,
    "island128-smag": S.island128_smag,
    "cape512-dleith": lambda: S.cape512(S.DLEITH),
    "cape512-dsmag": lambda: S.cape512(S.DSMAG),
    "cape512-smag": lambda: S.cape512(S.SMAG),
    "cape512-leith": lambda: S.cape512(S.LEITH),
}

METRIC = "grid-pt-steps/s at 2048^2 dyn-Leith, FP32 vs FP64 at stated err; % HBM peak"
UNIT = "grid-pt-steps/s"
SCHEMES = {"rk3": 0, "ab2cn": 1}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank float over the process group (identity without one).

    Uses a CUDA tensor under NCCL and a CPU tensor under gloo.
    """
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(n: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job grid-point-steps/s of `world` replicas, each advancing an n^2 grid `steps` steps."""
    return world * n * n * steps / (ms_max / 1e3)


def algorithmic_bytes(wl, precision_fp32: bool):
    """Minimal HBM bytes per launch of each kernel class of one step.

    Units: a mixed array holds N x (K+1) complex, a spectral array (K+1) x
    (2K+1) complex, a physical field N x N reals; each is read or written once
    where the algorithm needs it.  Returns {class: (launches_per_step,
    bytes_per_launch)}.
    """
    n = wl.n
    K = (n - 1) // 3
    esz = 4 if precision_fp32 else 8
    csz = 2 * esz
    I = n * (K + 1) * csz
    Sp = (K + 1) * (2 * K + 1) * csz
    R = n * n * esz
    kind = wl.closure
    nin = {S.NONE: 4, S.LEITH: 4, S.SMAG: 6, S.DLEITH: 8, S.DSMAG: 12}[kind]
    nout = {S.NONE: 1, S.LEITH: 3, S.SMAG: 3, S.DLEITH: 6, S.DSMAG: 6}[kind]
    dyn = kind in (S.DSMAG, S.DLEITH)
    has_mask = wl.geometry != "none"
    has_sponge = wl.sponge
    after = 2 if has_mask else (1 if has_sponge else nin)
    out = {"row_stage": (3, (nin + nout) * I)}
    # column pass of the stages: stage 0 reads w0 only; later stages w0 and ws;
    # stages 0, 1 write ws and nin mixed arrays; stage 2 writes `after` mixed arrays
    stage_bytes = []
    for s in range(3):
        b = (2 * Sp if dyn else nout * I)  # J, D (dynamic) or the forward inputs (static)
        b += Sp if s == 0 else 2 * Sp
        b += (Sp + nin * I) if s < 2 else after * I
        stage_bytes.append(b)
    out["col_stage"] = (3, sum(stage_bytes) / 3)
    if dyn:
        out["col_reduce"] = (3, 6 * I + 2 * Sp)
    if has_mask:
        out["row_brinkman"] = (1, 4 * I + R)
        out["col_curl"] = (1, 2 * I + (I if has_sponge else Sp + nin * I))
    if has_sponge:
        out["row_sponge"] = (1, 2 * I + R)
        out["col_final"] = (1, I + Sp + nin * I)
    return out


# Full-field round-trip model of one RK3 step: every 2-D transform moves one
# N x N field (U_N = N^2 b bytes) out of its first pass and into its second;
# stage I/O adds the reads of w_s (and w_0) and the write of w_{s+1}, and the
# dynamic closures write and read J and D.  U_N traversals per RK stage by
# closure; the Brinkman sub-step adds 11 and the sponge sub-step 7 (their
# factor-field reads included).
FIELD_TRAVERSALS_PER_STAGE = {S.NONE: 14, S.SMAG: 22, S.LEITH: 18, S.DSMAG: 43, S.DLEITH: 35}


# 2-D transforms per RK3 step by closure (inverse + forward over the three stages, Brinkman 4, sponge 2) and the
# cost of one real 2-D transform, 2.5 N^2 log2(N^2) flops: the arithmetic model of a step.
TRANSFORMS_PER_STEP = {S.NONE: 21, S.SMAG: 33, S.LEITH: 27, S.DSMAG: 60, S.DLEITH: 48}


def transforms_per_step(wl, scheme: int = 0) -> float:
    """Real 2-D transforms of one step, counted as (x passes + y passes) / 2 over the launch sequence: RK3 from
    the table above (island with sponge); AB2CN (Eq. 4) evaluates the products once, so the stage's nin inverse
    and nout forward transforms, the Brinkman pair (its x passes on u, v and chi u, chi v, its y passes forward)
    and the sponge's field in and out."""
    if scheme == 0:
        return TRANSFORMS_PER_STEP[wl.closure]
    nin = {S.NONE: 4, S.LEITH: 4, S.SMAG: 6, S.DLEITH: 8, S.DSMAG: 12}[wl.closure]
    nout = {S.NONE: 1, S.LEITH: 3, S.SMAG: 3, S.DLEITH: 6, S.DSMAG: 6}[wl.closure]
    mask = 1 if wl.geometry != "none" else 0
    sponge = 1 if wl.sponge else 0
    return nin + nout + 3 * mask + 2 * sponge


def step_flop_model(wl, scheme: int = 0) -> float:
    n2 = wl.n * wl.n
    return transforms_per_step(wl, scheme) * 2.5 * n2 * math.log2(n2)


def host_cpu():
    """CPU model name and logical core count of this host (for the CPU baseline)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


def streamfunction(w):
    """psi = lap^-1 w with zero mean on [0, 2 pi)^2 (plain numpy; for the per-field error report)."""
    n = w.shape[0]
    wh = np.fft.rfft2(w)
    mx = np.arange(n // 2 + 1)[None, :]
    my = np.fft.fftfreq(n, 1.0 / n)[:, None]
    k2 = (mx * mx + my * my).astype(float)
    k2[0, 0] = 1.0
    ph = -wh / k2
    ph[0, 0] = 0.0
    return np.fft.irfft2(ph, s=(n, n))


def precision_errors(qg, wl, w0, steps, stream, scheme):
    """Step the FP64 and FP32 forms side by side from w0 and report the FP32 form's error per field
    (relative L2 of w and psi, relative E and Z at the end, and the dynamic coefficient C at every step)."""
    sol = {p: qg.QGSolver.from_workload(wl, precision=p, stream=stream, scheme=scheme)
           for p in (qg.QG_FP64, qg.QG_FP32)}
    cs = {p: [] for p in sol}
    for s in sol.values():
        s.set_state(w0)
    blown = {}
    z0 = {}
    for k in range(steps):
        for p, s in sol.items():
            s.step(1)
            d = s.diagnostics(raise_nonfinite=False)
            z0.setdefault(p, d["enstrophy"])
            if p not in blown and (not d["finite"] or not d["enstrophy"] <= 1e6 * z0[p]):
                blown[p] = k + 1
            cs[p].append(d["coeff"])
        if blown:
            # keep stepping until both forms have diverged or a few steps passed, to report both
            if len(blown) == len(sol) or k + 1 >= min(blown.values()) + 5:
                break
    if blown:
        # the run diverged (non-finite, or enstrophy grown a millionfold): report at which step, for each form
        for s in sol.values():
            s.close()
        return {"steps": steps, "diverged_at_step": {("fp64" if p == qg.QG_FP64 else "fp32"): blown.get(p)
                                                     for p in sol}}
    a = sol[qg.QG_FP64].get_state()
    b = sol[qg.QG_FP32].get_state()
    d64 = sol[qg.QG_FP64].diagnostics()
    d32 = sol[qg.QG_FP32].diagnostics()
    for s in sol.values():
        s.close()
    c64 = np.array(cs[qg.QG_FP64])
    c32 = np.array(cs[qg.QG_FP32])
    act = c64 > 0
    out = {"steps": steps, "w": float(np.linalg.norm(b - a) / np.linalg.norm(a)),
           "psi": float(np.linalg.norm(streamfunction(b) - streamfunction(a)) / np.linalg.norm(streamfunction(a))),
           "E": abs(d32["energy"] - d64["energy"]) / abs(d64["energy"]),
           "Z": abs(d32["enstrophy"] - d64["enstrophy"]) / abs(d64["enstrophy"]),
           "steps_with_C_positive": int(act.sum()), "C_final_fp64": float(c64[-1]), "C_final_fp32": float(c32[-1])}
    if wl.closure in (S.DSMAG, S.DLEITH):
        # per step where the FP64 coefficient is positive: the largest relative difference (large where C itself
        # is near the clip at 0), the relative L2 difference over those steps, and the largest difference as a
        # fraction of the largest coefficient
        rel = np.abs(c32[act] - c64[act]) / c64[act] if act.any() else np.zeros(0)
        out["C_max_rel_diff"] = float(rel.max()) if act.any() else None
        out["C_median_rel_diff"] = float(np.median(rel)) if act.any() else None
        out["C_steps_rel_diff_over_1pct"] = int((rel > 0.01).sum())
        out["C_rel_l2_diff"] = (float(np.linalg.norm(c32[act] - c64[act]) / np.linalg.norm(c64[act]))
                                if act.any() else None)
        out["C_max_diff_over_max_C"] = (float(np.abs(c32[act] - c64[act]).max() / c64[act].max())
                                        if act.any() else None)
        out["C_mean_fp64"] = float(c64[act].mean()) if act.any() else 0.0
    return out


def field_model_bytes(wl, precision_fp32: bool):
    """(row-pass bytes per launch, RK3 step bytes) in the full-field round-trip model.

    A stage's row pass takes the row halves of its transforms: it reads the nin
    inverse-transform intermediates and writes the nout forward ones, one U_N
    each.
    """
    un = wl.n * wl.n * (4 if precision_fp32 else 8)
    nin = {S.NONE: 4, S.LEITH: 4, S.SMAG: 6, S.DLEITH: 8, S.DSMAG: 12}[wl.closure]
    nout = {S.NONE: 1, S.LEITH: 3, S.SMAG: 3, S.DLEITH: 6, S.DSMAG: 6}[wl.closure]
    step = 3 * FIELD_TRAVERSALS_PER_STAGE[wl.closure]
    step += 11 if wl.geometry != "none" else 0
    step += 7 if wl.sponge else 0
    return (nin + nout) * un, step * un


def algorithmic_bytes_ab2cn(wl, precision_fp32: bool):
    """Minimal HBM bytes per launch of each kernel class of one AB2CN step (Eq. 4), steady state.

    Same units as ``algorithmic_bytes``.  One explicit evaluation per step:
    row pass (products), Brinkman row pass (chi u), Germano reduction writing
    J, D (and the Brinkman forcing) spectra, the AB2CN combine (reads E_prev
    and writes E, reads w^n, and with a sponge reads/writes the w* history and
    writes the field the sponge row pass needs), sponge row pass, final pass.
    """
    n = wl.n
    K = (n - 1) // 3
    esz = 4 if precision_fp32 else 8
    I = n * (K + 1) * 2 * esz
    Sp = (K + 1) * (2 * K + 1) * 2 * esz
    R = n * n * esz
    kind = wl.closure
    nin = {S.NONE: 4, S.LEITH: 4, S.SMAG: 6, S.DLEITH: 8, S.DSMAG: 12}[kind]
    nout = {S.NONE: 1, S.LEITH: 3, S.SMAG: 3, S.DLEITH: 6, S.DSMAG: 6}[kind]
    dyn = kind in (S.DSMAG, S.DLEITH)
    mask = wl.geometry != "none"
    sponge = wl.sponge
    out = {"row_stage": (1, (nin + nout) * I)}
    if mask:
        out["row_brinkman"] = (1, 4 * I + R)
    if dyn:
        out["col_reduce"] = (1, (nout + (2 if mask else 0)) * I + (3 if mask else 2) * Sp)
        forcing = (3 if mask else 2) * Sp
    else:
        forcing = (nout + (2 if mask else 0)) * I
    combine = forcing + 2 * Sp + Sp  # E_prev read + write, w^n read
    if sponge:
        out["col_stage"] = (1, combine + 2 * Sp + I)  # w* history read + write, the sponge's field
        out["row_sponge"] = (1, 2 * I + R)
        out["col_final"] = (1, I + Sp + Sp + nin * I)  # forcing, w*, w^{n+1}, next step's fields
    else:
        out["col_final"] = (1, combine + Sp + nin * I)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_id

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


class TorchFFTStep:
    """The same RK3 step (readings R1-R5) written with torch.fft (cuFFT) and torch elementwise ops, FP32 on the
    GPU, eager: a library-FFT implementation of the method, timed beside libqg as context only.

    Sec. II-A Eq. 1 with the closures of Eq. 9-14, the exact Brinkman (Eq. 2) and sponge (Eq. 3) sub-steps and the
    2/3 rule, in numpy's rfft2 layout.  The dynamic coefficient stays on the device (no host round trip).
    """

    def __init__(self, wl, dtype=None, device="cuda"):
        import torch
        self.torch = torch
        dev = device
        self.dtype = dtype or torch.float32
        n, L = wl.n, wl.L
        self.n, self.wl = n, wl
        mx = torch.arange(n // 2 + 1, device=dev, dtype=torch.float64)[None, :]
        my = torch.fft.fftfreq(n, 1.0 / n, device=dev, dtype=torch.float64)[:, None]
        sc = 2 * math.pi / L
        kx, ky = sc * mx, sc * my
        k2 = kx ** 2 + ky ** 2
        inv_k2 = torch.where(k2 > 0, 1.0 / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
        K = (n - 1) // 3
        T = ((mx.abs() <= K) & (my.abs() <= K)).to(torch.float64)
        G = ((mx ** 2 + my ** 2) * (2.0 * wl.test_ratio) ** 2 <= float(n) ** 2).to(torch.float64)
        rd = self.dtype
        self.kx = kx.to(rd)
        self.ky = ky.to(rd)
        self.inv_k2 = inv_k2.to(rd)
        self.T = T.to(rd)
        self.G = G.to(rd)
        self.visc = torch.exp(-(wl.nu * k2 + wl.mu) * wl.dt).to(rd)
        self.fb = torch.exp(torch.from_numpy(-wl.mask() * wl.dt / wl.eta)).to(dev, rd) if wl.geometry != "none" else None
        sp = wl.sponge_field()
        self.fs = torch.exp(torch.from_numpy(-wl.sponge_rate * sp * wl.dt)).to(dev, rd) if sp is not None else None
        self.delta = L / n

    def inv(self, fh):
        return self.torch.fft.irfft2(fh, s=(self.n, self.n))

    def fwd(self, f):
        return self.torch.fft.rfft2(f)

    def project(self, w):
        wh = self.T * self.fwd(w.to(self.dtype))
        wh[0, 0] = 0
        return wh

    def velocity(self, wh):
        ph = -wh * self.inv_k2
        return self.inv(-1j * self.ky * ph) + self.wl.U, self.inv(1j * self.kx * ph)

    def grad(self, wh):
        return self.inv(1j * self.kx * wh), self.inv(1j * self.ky * wh)

    def jac(self, wh):
        u, v = self.velocity(wh)
        wx, wy = self.grad(wh)
        return self.T * self.fwd(u * wx + v * wy)

    def eddy(self, wh, smag):
        if smag:
            ph = -wh * self.inv_k2
            pxy = self.inv(-(self.kx * self.ky) * ph)
            pd = self.inv(-(self.kx ** 2 - self.ky ** 2) * ph)
            return self.torch.sqrt(4 * pxy * pxy + pd * pd)
        wx, wy = self.grad(wh)
        return self.torch.sqrt(wx * wx + wy * wy)

    def sgs(self, wh, smag):
        g = self.eddy(wh, smag)
        wx, wy = self.grad(wh)
        return self.T * (1j * self.kx * self.fwd(g * wx) + 1j * self.ky * self.fwd(g * wy))

    def rhs(self, wh):
        wl = self.wl
        out = -self.jac(wh) - wl.beta * (1j * self.kx * (-wh * self.inv_k2))
        if wl.closure == S.NONE:
            return out
        smag = wl.closure in (S.SMAG, S.DSMAG)
        D = self.sgs(wh, smag)
        if wl.closure in (S.SMAG, S.LEITH):
            C = (wl.c * self.delta) ** (2 if smag else 3)
        else:
            wt = self.G * wh
            H = self.inv(self.jac(wt) - self.G * self.jac(wh))
            M = self.inv(wl.test_ratio ** (2 if smag else 3) * self.sgs(wt, smag) - self.G * D)
            hm, mm = (H * M).mean(), (M * M).mean()
            C = self.torch.where(mm > 0, self.torch.clamp(hm / self.torch.where(mm > 0, mm, self.torch.ones_like(mm)),
                                                          min=0), self.torch.zeros_like(mm))
        return out + C * D

    def step(self, wh):
        dt = self.wl.dt
        w0, ws = wh, wh
        for a, b in ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)):
            ws = a * w0 + b * (ws + dt * self.rhs(ws))
        w = self.visc * ws
        if self.fb is not None:
            u, v = self.velocity(w)
            w = self.T * (1j * self.kx * self.fwd(self.fb * v) - 1j * self.ky * self.fwd(self.fb * u))
        if self.fs is not None:
            w = self.T * self.fwd(self.fs * self.inv(w))
        w = self.T * w
        w[0, 0] = 0
        return w


def torch_fft_context(wl, ours_ms: float, steps: int = 20):
    """Time the torch.fft form of the step and compare its field with libqg's after 20 steps (FP32 both)."""
    import torch
    import paper_2508_06678_gb300 as qg
    ts = TorchFFTStep(wl)
    w0 = wl.omega0()
    wh = ts.project(torch.from_numpy(w0).cuda())
    for _ in range(3):
        wh = ts.step(wh)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        wh = ts.step(wh)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    wh = ts.project(torch.from_numpy(w0).cuda())
    for _ in range(20):
        wh = ts.step(wh)
    a = ts.inv(wh).double().cpu().numpy()
    with qg.QGSolver.from_workload(wl, precision=qg.QG_FP32) as s:
        s.set_state(w0)
        s.step(20)
        b = s.get_state()
    return {"ms_per_step": ms, "value": wl.n * wl.n / (ms / 1e3), "unit": UNIT, "libqg_speedup": ms / ours_ms,
            "rel_l2_diff_vs_libqg_after_20_steps": float(np.linalg.norm(a - b) / np.linalg.norm(b)),
            "what": "the same RK3 step in eager torch (torch.fft rfft2/irfft2 = cuFFT, elementwise torch ops), FP32, "
                    f"{steps} steps after 3 warm-up"}


def time_oracle(wl, max_seconds: float, warmup: int = 1, scheme: int = 0):
    """The FP64 CPU oracle, as it stands, on the workload; bounded wall time."""
    import oracle as O
    ref = O.QGOracle(wl.n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(wl.closure, c=wl.c),
                     O.Params(dt=wl.dt, nu=wl.nu, mu=wl.mu, eta=wl.eta, sponge_rate=wl.sponge_rate, scheme=scheme))
    ref.set_state(wl.omega0())
    for _ in range(warmup):
        ref.step(1)
    steps = 0
    t0 = time.perf_counter()
    while True:
        ref.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= max_seconds or el / steps * (steps + 1) > 1.5 * max_seconds:
            break
    return steps, el


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    budget = float(os.environ.get("QG_REF_SECONDS", "60"))
    if args.workload in TOOLS:
        TOOLS[args.workload]["reference"](args, budget)
        return
    steps, el = time_oracle(wl, budget, warmup=min(args.warmup, 1), scheme=SCHEMES[args.scheme])
    value = wl.n * wl.n * steps / el
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": 1, "steps": steps,
        "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "closure": S.CLOSURE_NAMES[wl.closure], "scheme": args.scheme,
                   "eta": wl.eta},
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": f"{steps} full {wl.n}^2 steps of the FP64 numpy oracle "
                                        f"(bounded to ~{budget:.0f} s)"}, **host_cpu()),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# A posteriori lag table (Eq. 15-16): qg_series_compare on two FP32 snapshot
# series of 512^2 fields, 96 snapshots each, lags -32 .. 32.
# ---------------------------------------------------------------------------
SERIES = {"n": 512, "nsnap": 96, "lag": 32, "seed": 21, "dt_snap": 0.1, "shift": 3}
SERIES_METRIC = "pair-points/s of the Eq. 15-16 lag table, 512^2 FP32 series, 96 snapshots, lags -32..32"
SERIES_UNIT = "pair-points/s"
# FP32 operations per (pair, point) of the plain definition of the two sums:
# a - b and its square added (one FMA), a - a_mean, b - b_mean and their
# product added (one FMA); the FP32-pipe roofline counts these, whatever the
# kernel spends on top (compensation, shared centring)
SERIES_INST = 5


def series_inputs():
    c = SERIES
    L = 2 * math.pi
    ff = S.wave_series(c["seed"], c["n"], c["nsnap"], L, dt_snap=c["dt_snap"], noise=0.2).astype(np.float32)
    les = S.wave_series(c["seed"], c["n"], c["nsnap"], L, dt_snap=c["dt_snap"], t0=c["shift"] * c["dt_snap"],
                        noise=0.2, noise_seed=c["seed"] + 100).astype(np.float32)
    return les, ff


def valid_pairs(n_les: int, n_ff: int, lag_min: int, lag_max: int) -> int:
    """Number of (t, phi) with 0 <= t - phi < n_les, t < n_ff, lag_min <= phi <= lag_max."""
    return sum(1 for t in range(n_ff) for phi in range(lag_min, lag_max + 1) if 0 <= t - phi < n_les)


def time_series_oracle(les, ff, max_seconds: float):
    """The oracle's lag table, one pair at a time over the workload's pairs, bounded wall time."""
    import oracle as O
    lag = SERIES["lag"]
    pairs = [(t, phi) for t in range(len(ff)) for phi in range(-lag, lag + 1) if 0 <= t - phi < len(les)]
    rng = np.random.default_rng(0)
    order = rng.permutation(len(pairs))
    done = 0
    t0 = time.perf_counter()
    for k in order:
        t, phi = pairs[k]
        O.lag_table(les[t - phi:t - phi + 1].astype(np.float64), ff[t:t + 1].astype(np.float64), 0, 0)
        done += 1
        if time.perf_counter() - t0 >= max_seconds:
            break
    return done, time.perf_counter() - t0


def run_series_reference(args, budget):
    rank, _, _ = dist_env()
    if rank != 0:
        return
    les, ff = series_inputs()
    npts = les[0].size
    pairs, el = time_series_oracle(les, ff, budget)
    value = pairs * npts / el
    line = {
        "metric": SERIES_METRIC, "value": value, "unit": SERIES_UNIT, "impl": "reference", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * el, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "series512", **SERIES},
        "cpu_baseline": {"value": value, "unit": SERIES_UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{pairs} (snapshot, lag) pairs of 512^2 fields by the FP64 numpy oracle "
                                   f"(bounded to ~{budget:.0f} s)"},
        "e2e": {"value": value, "unit": SERIES_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_series_bench(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2508_06678_gb300 as qg
    from paper_2508_06678_gb300._lib import LIB_PATH, load
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    load()

    les, ff = series_inputs()
    npts = les[0].size
    lag_min, lag_max = -SERIES["lag"], SERIES["lag"]
    nlag = lag_max - lag_min + 1
    pp = valid_pairs(len(les), len(ff), lag_min, lag_max) * npts  # pair-points per call
    stream = torch.cuda.Stream()
    dl = torch.from_numpy(les).cuda()
    df = torch.from_numpy(ff).cuda()
    torch.cuda.synchronize()

    def call(timing=False):
        return qg.qg_series_compare(dl, df, lag_min, lag_max, stream=stream, timing=timing)

    for _ in range(args.warmup):
        r = call()
    phase = r["phase"]

    def barrier():
        if world > 1:
            dist.barrier()

    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except (AttributeError, RuntimeError):
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        call()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    value = world * pp / (ms / 1e3)

    # kernel durations (CUDA events inside the call, on its stream)
    kms = [call(timing=True)["kernel_ms"] for _ in range(args.steps)]
    avg = {k: sum(d[k] for d in kms) / len(kms) for k in kms[0]}
    props = torch.cuda.get_device_properties(local)
    nsm = props.multi_processor_count
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = nsm * 128 * sm_mhz * 1e6 / 1e12  # FP32-pipe instructions, Tinst/s
    achieved = pp * SERIES_INST / (avg["pairs"] / 1e3) / 1e12
    traffic = None  # ncu DRAM bytes of one pairs launch, recorded beside the launch list
    prof = os.path.join(ROOT, "profiles", "launches_series512_fp32.md")
    if os.path.exists(prof):
        rec = dict(line.split(":", 1) for line in open(prof) if line.startswith("traffic_") and ":" in line)
        if rec.get("traffic_kernel", "").strip() == "series_pairs_kernel":
            traffic = int(rec["traffic_bytes_per_launch"].strip())
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s (FP32 pipe)",
                "frac": achieved / peak, "traffic": traffic, "kernel": "series_pairs_kernel",
                "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz",
                "inst_per_pair_point": SERIES_INST, "avg_launch_us": avg["pairs"] * 1e3,
                "kernel_ms": avg,
                "measured_in": "CUDA events around each kernel group inside the call, second pass"}

    # end to end with host series (copies inside the call)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        qg.qg_series_compare(les, ff, lag_min, lag_max, stream=stream)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps)
    e2e = {"value": world * pp / e2e_s, "unit": SERIES_UNIT, "h2d_bytes_per_step": les.nbytes + ff.nbytes,
           "d2h_bytes_per_step": (2 * len(ff) * nlag + nlag) * 8 + 4,
           "api": "qg_series_compare(host series)"}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            pairs_c, el_c = time_series_oracle(les, ff, args.cpu_seconds)
            cpu = {"value": pairs_c * npts / el_c, "unit": SERIES_UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{pairs_c} (snapshot, lag) pairs of 512^2 fields by the FP64 numpy oracle, {el_c:.1f} s"}
        line = {
            "metric": SERIES_METRIC, "value": value, "unit": SERIES_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "series512", **SERIES, "pair_points_per_call": pp, "phase": phase,
                       "l2": "two 100 MB series, 201 MB > 126 MB L2 (no flush)",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 5 * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Ensemble: 96 independent FP32 members (24 each of 256^2, 384^2, 512^2,
# 768^2; island / cape; the four closures; random beta, U), one CUDA graph
# per ensemble step with the members as parallel branches.
# ---------------------------------------------------------------------------
ENS_METRIC = "grid-pt-steps/s (sum of N_i^2) of a 96-member FP32 LES ensemble, 256^2-768^2, 4 closures"


def ensemble_shard(n_members: int, rank: int, world: int) -> list:
    """Members of one rank when the ensemble is split over ``world`` GPUs: every world-th member from ``rank``
    (the sizes interleave, so every rank gets a similar mix)."""
    return list(range(rank, n_members, world))


def time_ensemble_oracle(wls, max_seconds: float):
    """The oracle stepping the first eight members (two of each size) in turn, bounded wall time."""
    import oracle as O
    refs = []
    for w in wls[:8]:
        ref = O.QGOracle(w.n, w.L, w.beta, w.U, w.mask(), w.sponge_field(), O.Closure(w.closure, c=w.c),
                         O.Params(dt=w.dt, nu=w.nu, mu=w.mu, eta=w.eta, sponge_rate=w.sponge_rate))
        ref.set_state(w.omega0())
        refs.append((ref, w.n * w.n))
    done = 0
    pts = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < max_seconds:
        ref, n2 = refs[done % len(refs)]
        ref.step(1)
        done += 1
        pts += n2
    return done, pts, time.perf_counter() - t0


def run_ensemble_reference(args, budget):
    rank, _, _ = dist_env()
    if rank != 0:
        return
    wls = S.ensemble96()
    done, pts, el = time_ensemble_oracle(wls, budget)
    value = pts / el
    line = {
        "metric": ENS_METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": 1e3 * el, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": "ensemble96", "members": len(wls)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{done} member-steps (256^2-768^2) of the FP64 numpy oracle, {el:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ensemble_bench(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2508_06678_gb300 as qg
    from paper_2508_06678_gb300._lib import LIB_PATH, load
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    load()
    all_wls = S.ensemble96()
    total_pts = sum(w.n * w.n for w in all_wls)
    # one ensemble split by member over the ranks: no data-path collective, the total work is fixed
    wls = [all_wls[i] for i in ensemble_shard(len(all_wls), rank, world)]
    pts = sum(w.n * w.n for w in wls)
    stream = torch.cuda.Stream()
    t_create = time.perf_counter()
    ens = qg.QGEnsemble.from_workloads(wls, precision=qg.QG_FP32, stream=stream)
    ens_form = dict(ens.config(), create_s=time.perf_counter() - t_create)
    w0 = [w.omega0() for w in wls]
    for m, w in zip(ens.members, w0):
        m.set_state(w)
    ens.step(args.warmup)
    ens.sync()

    def barrier():
        if world > 1:
            dist.barrier()

    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except (AttributeError, RuntimeError):
        gpu_id = str(local)
    launches0 = sum(m_launches(m) for m in ens.members)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ens.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ens.sync()
    launches = sum(m_launches(m) for m in ens.members) - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    value = total_pts / (ms / 1e3)

    # the same members stepped one after another (each replaying its own step graph) on one stream
    solo = [qg.QGSolver.from_workload(w, precision=qg.QG_FP32, stream=stream) for w in wls]
    for s_, w in zip(solo, w0):
        s_.set_state(w)
        s_.step(3)
    torch.cuda.synchronize()
    k_seq = max(1, args.steps // 4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k_seq):
        for s_ in solo:
            s_.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / k_seq
    for s_ in solo:
        s_.close()

    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    step_bytes = sum(sum(a * b for a, b in algorithmic_bytes(w, True).values()) for w in wls)
    achieved = step_bytes / (ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "ensemble step (every member's kernels, concurrent graph branches)",
                "peak_source": peak_src, "bytes_per_launch": step_bytes, "avg_launch_us": ms * 1e3,
                "measured_in": "CUDA events around the K replayed ensemble steps"}

    # end to end: host states in, K steps, host states and diagnostics out
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, w in zip(ens.members, w0):
        m.set_state(w.astype(np.float32))
    ens.step(args.steps)
    outs = [m.get_state(dtype=np.float32) for m in ens.members]
    diag = [m.diagnostics() for m in ens.members]
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    nbytes = sum(w.n * w.n * 4 for w in wls)
    e2e = {"value": total_pts * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes / args.steps,
           "d2h_bytes_per_step": (nbytes + 56 * len(wls)) / args.steps,
           "api": "per member qg_set_state(host) + qg_ensemble_step(K) + per member qg_get_state(host), "
                  "qg_diagnostics"}
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            done, cpts, el = time_ensemble_oracle(wls, args.cpu_seconds)
            cpu = {"value": cpts / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{done} member-steps (256^2-768^2) of the FP64 numpy oracle, {el:.1f} s"}
        line = {
            "metric": ENS_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ensemble96", "members": len(all_wls), "members_on_rank0": len(wls),
                       "sizes": "24 x (256, 384, 512, 768)^2",
                       "sum_n2": total_pts, "closures": "smag, leith, dyn-smag, dyn-leith", "scheme": "rk3",
                       "parallelism": f"members split over {world} GPUs" if world > 1 else "single",
                       "l2": "working set ~1 GB > 126 MB L2 (no flush)",
                       "sequential_ms_per_step": seq_ms, "concurrency_speedup": seq_ms / ms,
                       "launch_form": ens_form,
                       "all_finite": all(d["finite"] for d in diag)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ens.close()
    if world > 1:
        dist.destroy_process_group()


def m_launches(m) -> int:
    """Kernel launches of one solver handle so far (every kernel class)."""
    import ctypes as C
    from paper_2508_06678_gb300._lib import load
    from paper_2508_06678_gb300._lib import KERNEL_CLASSES
    nk = len(KERNEL_CLASSES)
    counts = (C.c_int32 * nk)()
    load().qg_kernel_times(m.h, counts, None, nk)
    return int(sum(counts))


# ---------------------------------------------------------------------------
# Adjoint: gradient of an MSE loss of a 256^2 Smagorinsky LES (FP64) against a
# 1024^2 closure-free run filtered to 256^2 at steps 100, 120, ..., 400, with
# respect to the initial field, c_S and the sponge rate; checkpoints every 20.
# ---------------------------------------------------------------------------
ADJ = {"n": 256, "n_fr": 1024, "steps": 400, "obs_first": 100, "obs_every": 20, "checkpoint": 20, "c": 0.17,
       "seed": 5, "beta": 5.0, "U": 0.5, "radius": 0.4}
ADJ_CLOSURES = {"dsmag": (S.DSMAG, "dynamic Smagorinsky"), "smag": (S.SMAG, "Smagorinsky")}


def adj_metric(precision: str = "fp64", closure: str = "dsmag") -> str:
    return (f"grid-pt-steps/s of the loss gradient (forward + checkpointed adjoint), 256^2 "
            f"{ADJ_CLOSURES[closure][1]} {precision.upper()} LES, 400 steps, MSE against a filtered 1024^2 run")


def adjoint_workload(closure: str = "dsmag"):
    """The adjoint configuration: a 256^2 island LES (dynamic Smagorinsky by default, the configuration's closure;
    static Smagorinsky c_S = 0.17 with closure="smag"), gradients over 400 steps."""
    c = ADJ
    kind = ADJ_CLOSURES[closure][0]
    les = S.Workload(f"adjoint256-{closure}", c["n"], "island", beta=c["beta"], U=c["U"], closure=kind,
                     c=c["c"] if kind == S.SMAG else 0.0, radius=c["radius"], seed=c["seed"])
    fr = S.Workload("fr1024", c["n_fr"], "island", beta=c["beta"], U=c["U"], closure=S.NONE, radius=c["radius"],
                    seed=c["seed"])
    obs = list(range(c["obs_first"], c["steps"] + 1, c["obs_every"]))
    return les, fr, obs


def adjoint_targets(qg, fr, obs, stream):
    """The 1024^2 run (FP64, no closure: the form the oracle pins) at the observed steps, filtered to 256^2
    (Eq. 5), and its filtered start."""
    s = qg.QGSolver.from_workload(fr, precision=qg.QG_FP64, stream=stream)
    w0 = fr.omega0()
    s.set_state(w0)
    snaps = []
    k = 0
    for t in obs:
        s.step(t - k)
        k = t
        snaps.append(s.get_state())
    s.close()
    n = ADJ["n"]
    return qg.qg_grid_filter(w0, n, fr.L), qg.qg_grid_filter(np.stack(snaps), n, fr.L)


def time_adjoint_oracle(les, max_seconds: float):
    import oracle as O
    ops = O.Ops(les.n, les.L)
    wh = O.project(ops, les.omega0())
    lam = np.random.default_rng(0).standard_normal((les.n, les.n))
    params = O.Params(dt=les.dt, nu=les.nu, mu=les.mu, eta=les.eta, sponge_rate=les.sponge_rate)
    chi, chs = les.mask(), les.sponge_field()
    cl = O.Closure(les.closure, c=les.c)
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < max_seconds:
        # per step of a checkpointed gradient: the forward run, its recomputation, one adjoint step
        w1, _ = O.full_step(ops, wh, les.beta, les.U, cl, params, chi, chs)
        O.full_step(ops, wh, les.beta, les.U, cl, params, chi, chs)
        lam, _ = O.full_step_vjp(ops, wh, lam, les.beta, les.U, cl, params, chi, chs)
        wh = w1
        done += 1
    return done, time.perf_counter() - t0


def run_adjoint_reference(args, budget):
    rank, _, _ = dist_env()
    if rank != 0:
        return
    les, _, _ = adjoint_workload(args.closure)
    done, el = time_adjoint_oracle(les, budget)
    value = les.n * les.n * done / el
    line = {
        "metric": adj_metric(args.precision, args.closure), "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": 1,
        "steps": done,
        "warmup": 0, "ms_per_step": 1e3 * el / done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": "adjoint256", "closure": args.closure, **ADJ},
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": f"{done} steps of the FP64 numpy oracle's checkpointed gradient (2 forward "
                                        f"steps + 1 full_step_vjp each) of the 256^2 LES, {el:.1f} s"}, **host_cpu()),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_adjoint_bench(args):
    import torch
    import torch.distributed as dist
    import ctypes as C

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2508_06678_gb300 as qg
    from paper_2508_06678_gb300._lib import KERNEL_CLASSES, LIB_PATH, load
    from paper_2508_06678_gb300.adjoint import rollout_grad
    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    lib = load()
    les, fr, obs = adjoint_workload(args.closure)
    stream = torch.cuda.Stream()
    w0_les, targets = adjoint_targets(qg, fr, obs, stream)
    n, K, ce = les.n, ADJ["steps"], ADJ["checkpoint"]
    fp32 = args.precision == "fp32"
    tdt = torch.float32 if fp32 else torch.float64
    ndt = np.float32 if fp32 else np.float64
    solver = qg.QGSolver.from_workload(les, precision=qg.QG_FP32 if fp32 else qg.QG_FP64, stream=stream)
    tgt = {k: torch.from_numpy(t.astype(ndt)).cuda() for k, t in zip(obs, targets)}
    w0 = torch.from_numpy(w0_les.astype(ndt)).cuda()
    scale = 2.0 / (len(obs) * n * n)

    need = sorted(set(range(0, K, ce)) | set(obs))

    def forward(w_start):
        """One forward run keeping the checkpoints and the observed states."""
        solver.set_state(w_start)
        ckpts, states = {}, {}
        k = 0
        for t in need:
            solver.step(t - k)
            k = t
            st_ = solver.get_state(out=torch.empty((n, n), dtype=tdt, device="cuda"))
            if t % ce == 0 and t < K:
                ckpts[t] = st_
            if t in tgt:
                states[t] = st_
        return ckpts, states

    def gradient():
        ckpts, states = forward(w0)
        # dloss/dw_k of loss = mean over the observed steps and points of (w_k - target_k)^2
        g_obs = {t: scale * (states[t] - tgt[t]) for t in obs}
        loss = float(sum(((states[t] - tgt[t]) ** 2).sum().item() for t in obs)) * scale / 2.0
        lam, g = rollout_grad(solver, None, K, g_obs, ce, ckpts=ckpts)
        return loss, lam, g

    for _ in range(max(1, args.warmup // 3)):
        loss, lam, g = gradient()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except (AttributeError, RuntimeError):
        gpu_id = str(local)
    reps = max(1, args.steps)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        loss, lam, g = gradient()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / reps)
    value = world * n * n * K / (ms / 1e3)

    # the plain forward run and one adjoint step, for the cost ratio
    solver.set_state(w0)
    solver.step(5)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / K
    st = solver.get_state(out=torch.empty((n, n), dtype=tdt, device="cuda"))
    lam1 = torch.randn((n, n), dtype=tdt, device="cuda")
    for _ in range(3):
        solver.step_vjp(st, lam1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(50):
        solver.step_vjp(st, lam1)
    e1.record(stream)
    torch.cuda.synchronize()
    vjp_ms = e0.elapsed_time(e1) / 50

    # per-class device times of adjoint steps (eager, a CUDA event pair around every launch)
    nk = len(KERNEL_CLASSES)
    lib.qg_profile(solver.h, 1)
    for _ in range(5):
        solver.step_vjp(st, lam1)
    counts = (C.c_int32 * nk)()
    kms = (C.c_double * nk)()
    lib.qg_kernel_times(solver.h, counts, kms, nk)
    lib.qg_profile(solver.h, 0)
    cls = {KERNEL_CLASSES[i]: (int(counts[i]), float(kms[i])) for i in range(nk) if counts[i]}
    Kb = (n - 1) // 3
    esz = 4 if fp32 else 8
    I = n * (Kb + 1) * 2 * esz
    R = n * n * esz
    n_row, t_row = cls.get("adj_row", (0, 0.0))
    achieved = (R + I) * n_row / (t_row / 1e3) / 1e9 if t_row else 0.0
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "adj_row (row pass of one field into or out of physical space)",
                "peak_source": peak_src, "bytes_per_launch": R + I,
                "avg_launch_us": 1e3 * t_row / n_row if n_row else None,
                "class_ms_per_vjp": {k: v[1] / 5 for k, v in cls.items()},
                "class_launches_per_vjp": {k: v[0] / 5 for k, v in cls.items()},
                "note": f"256^2 {args.precision.upper()} fields ({R / 2**20:.2f} MB) stay in the 126 MB L2: "
                        "these launches are latency-bound",
                "measured_in": "CUDA events around each launch of 5 eager adjoint steps"}

    # end to end: host initial field and targets in, gradient out
    barrier()
    t0 = time.perf_counter()
    w_host = w0_les.astype(ndt)
    tg_host = {k: t.astype(ndt) for k, t in zip(obs, targets)}
    tgt = {k: torch.from_numpy(t).cuda() for k, t in tg_host.items()}
    ck, states = forward(torch.from_numpy(w_host).cuda())
    g_obs = {t: scale * (states[t] - tgt[t]) for t in obs}
    lam_h, _ = rollout_grad(solver, None, K, g_obs, ce, ckpts=ck)
    lam_h = lam_h.cpu().numpy()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            done, el = time_adjoint_oracle(les, args.cpu_seconds)
            cpu = {"value": n * n * done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{done} steps of the FP64 numpy oracle's checkpointed gradient (2 forward steps + 1 "
                             f"full_step_vjp each) of the 256^2 LES, {el:.1f} s"}
            cpu.update(host_cpu())
        line = {
            "metric": adj_metric(args.precision, args.closure), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": reps,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
            "data": "synthetic",
            "config": {"workload": "adjoint256", "closure": args.closure, **ADJ, "observed_steps": len(obs),
                       "loss": loss, "dloss_dC": g.get("C"),
                       "grad_norm": float(lam.norm().item()), "dloss_dc": g["c"], "dloss_drate": g["sponge_rate"],
                       "ms_per_gradient": ms, "forward_ms_per_step": fwd_ms, "vjp_ms_per_step": vjp_ms,
                       "adjoint_over_forward": vjp_ms / fwd_ms,
                       "gradient_over_forward_run": ms / (fwd_ms * K),
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "256^2 working set fits the L2 (latency-bound sizes)"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": world * n * n * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": (len(obs) + 1) * R / K,
                    "d2h_bytes_per_step": (len(obs) + 1) * R / K,
                    "api": "initial field and targets from host, rollout + qg_step_vjp sweep, gradient to host"},
            "gpu_launches": int(sum(v[0] for v in cls.values()) / 5 * K), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


TOOLS = {"series512": {"ours": run_series_bench, "reference": run_series_reference},
         "adjoint256": {"ours": run_adjoint_bench, "reference": run_adjoint_reference},
         "ensemble96": {"ours": run_ensemble_bench, "reference": run_ensemble_reference}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=1000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="island2048-dleith", choices=sorted(WORKLOADS) + sorted(TOOLS))
    ap.add_argument("--scheme", default="rk3", choices=sorted(SCHEMES),
                    help="time scheme: rk3 (SSP-RK3 with exact sub-steps) or ab2cn (the paper's Eq. 4)")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"],
                    help="working precision (default: fp64 for the adjoint workload, fp32 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 throughput / error leg")
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--err-steps", type=int, default=300,
                    help="steps of the FP32-vs-FP64 error comparison (the configuration's 300)")
    ap.add_argument("--closure", default="dsmag", choices=sorted(ADJ_CLOSURES),
                    help="adjoint256 only: the LES closure (the configuration's dynamic Smagorinsky by default)")
    ap.add_argument("--spinup", type=int, default=1000,
                    help="untimed steps before the warm-up: the configuration times steps 1000-5000")
    ap.add_argument("--no-torch-context", action="store_true",
                    help="skip timing the torch.fft (cuFFT) form of the step beside libqg")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp64" if args.workload == "adjoint256" else "fp32"
    if args.warmup < 3 and args.impl != "reference":
        raise SystemExit("--warmup must be >= 3")
    if args.workload in TOOLS:
        if args.impl == "reference":
            run_reference(args, None)
        else:
            TOOLS[args.workload]["ours"](args)
        return
    wl = WORKLOADS[args.workload]()
    if args.scheme == "ab2cn":
        # AB2 treats the Brinkman term explicitly, which is stable only for
        # eta > dt (Sec. II-E); the paper's runs use eta = 1.025 dt
        wl.eta = 1.025 * wl.dt
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2508_06678_gb300 as qg
    from paper_2508_06678_gb300._lib import KERNEL_CLASSES, LIB_PATH, load

    if not os.path.exists(LIB_PATH):
        from paper_2508_06678_gb300.build import build
        build()
    lib = load()
    import ctypes as C

    fp32 = args.precision == "fp32"
    stream = torch.cuda.Stream()
    scheme = SCHEMES[args.scheme]
    solver = qg.QGSolver.from_workload(wl, precision=qg.QG_FP32 if fp32 else qg.QG_FP64, stream=stream,
                                       scheme=scheme)
    w0 = wl.omega0()
    solver.set_state(w0)
    solver.step(args.spinup + args.warmup)
    solver.sync()
    spun = solver.diagnostics(raise_nonfinite=False)

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- timed region: K steps on device-resident state
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gpu_id = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except (AttributeError, RuntimeError):
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    qg_h = solver.h
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solver.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    solver.sync()
    ms = max_over_ranks(ms)
    value = replica_value(wl.n, args.steps, world, ms)

    # ---- per-kernel durations: a second pass of the same K steps with a CUDA
    # event pair recorded around every launch on the solver's stream (the
    # brackets add a few per cent to the step, so the value above is taken
    # without them)
    lib.qg_profile(qg_h, 1)
    torch.cuda.synchronize()
    solver.step(args.steps)
    nk = len(KERNEL_CLASSES)
    counts = (C.c_int32 * nk)()
    kms = (C.c_double * nk)()
    lib.qg_kernel_times(qg_h, counts, kms, nk)
    lib.qg_profile(qg_h, 0)
    solver.sync()
    launches = int(sum(counts))  # our kernels per K-step pass (the timed pass launches the same)

    # ---- roofline of the dominant kernel class
    peaks, peak_src = measured_peaks()
    model = algorithmic_bytes(wl, fp32) if scheme == 0 else algorithmic_bytes_ab2cn(wl, fp32)
    per_class = {KERNEL_CLASSES[i]: (int(counts[i]), float(kms[i])) for i in range(nk)}
    dom = max((k for k in per_class if per_class[k][0] > 0 and k in model), key=lambda k: per_class[k][1])
    n_l, t_l = per_class[dom]
    avg_s = t_l / n_l / 1e3
    bytes_launch = model[dom][1]
    achieved = bytes_launch / avg_s / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    step_bytes = sum(a * b for a, b in model.values())
    traffic = None
    prof_path = os.path.join(ROOT, "profiles", f"row_pass_{wl.name}_{args.precision}.md")
    if os.path.exists(prof_path):
        rec = {}
        for line in open(prof_path):
            if ":" in line and line.split(":")[0].startswith("traffic_"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        if rec.get("traffic_kernel_class") == dom and rec.get("traffic_bytes_per_launch"):
            traffic = int(rec["traffic_bytes_per_launch"])
    step_s = ms / 1e3 / args.steps
    band = {"bytes_per_launch": bytes_launch, "achieved": achieved, "frac": achieved / peak,
            "step_bytes": step_bytes, "step_frac": step_bytes / step_s / 1e9 / peak,
            "model": "band storage: the arrays this design keeps (N x (K+1) mixed, (K+1) x (2K+1) spectral, "
                     "N x N physical), each read or written once"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "peak_source": peak_src,
                "bytes_per_launch": bytes_launch, "avg_launch_us": avg_s * 1e6,
                "measured_in": "CUDA events around each launch, second pass of the same K steps"}
    if dom == "row_stage":
        # the full-field round-trip model: the reported achieved / frac; the band model beside it
        row_b, step_fb = field_model_bytes(wl, fp32)
        roofline.update({"achieved": row_b / avg_s / 1e9, "frac": row_b / avg_s / 1e9 / peak,
                         "bytes_per_launch": row_b,
                         "model": "full-field round trips: each 2-D transform moves one N^2 field between "
                                  "its passes; the row pass reads nin and writes nout such fields"})
        if scheme == 0:
            roofline.update({"step_model_bytes": step_fb, "step_frac": step_fb / step_s / 1e9 / peak})
    roofline["band_model"] = band

    # ---- end to end through the public API with host buffers
    torch.cuda.synchronize()
    host_in = torch.from_numpy(w0.astype(np.float32 if fp32 else np.float64)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dtype_code = qg.QG_FP32 if fp32 else qg.QG_FP64
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lib.qg_set_state(qg_h, C.c_void_p(host_in.data_ptr()), 0, dtype_code)
    lib.qg_step(qg_h, args.steps)
    lib.qg_get_state(qg_h, C.c_void_p(host_out.data_ptr()), 0, dtype_code)
    diag = solver.diagnostics(raise_nonfinite=False)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s)
    esz = 4 if fp32 else 8
    e2e = {"value": world * wl.n * wl.n * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": wl.n * wl.n * esz / args.steps,
           "d2h_bytes_per_step": (wl.n * wl.n * esz + 56) / args.steps,
           "api": "qg_set_state(host) + qg_step(K) + qg_get_state(host) + qg_diagnostics"}

    # ---- the FP64 form on the same workload: throughput against its arithmetic roofline, and the FP32 form's
    # error per field against it (the FP64 form is pinned to the oracle at 1e-12), on the workload's own field
    # and on a rough seeded field (spectral peak N/8) that keeps the dynamic coefficient active from the start
    fp64 = None
    if fp32 and not args.no_fp64:
        s64 = qg.QGSolver.from_workload(wl, precision=qg.QG_FP64, stream=stream, scheme=scheme)
        s64.set_state(w0)
        s64.step(5)
        s64.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k64 = args.fp64_steps
        e0.record(stream)
        s64.step(k64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        s64.close()
        f64 = C.c_double()
        f32 = C.c_double()
        rc64 = lib.qg_probe_fma_rate(qg.QG_FP64, C.byref(f64), None)
        rc32 = lib.qg_probe_fma_rate(qg.QG_FP32, C.byref(f32), None)
        flops = step_flop_model(wl, scheme)
        alu = None
        if rc64 == 0 and f64.value > 0:
            ach = flops / (ms64 / 1e3) / 1e12
            alu = {"bound": "alu", "achieved": ach, "peak": f64.value / 1e12, "unit": "TFLOP/s",
                   "frac": ach / (f64.value / 1e12), "peak_source": "measured FP64 FMA rate (qg_probe_fma_rate)",
                   "flops_per_step": flops,
                   "model": f"{transforms_per_step(wl, scheme):g} real 2-D transforms per step x 2.5 N^2 log2(N^2)",
                   "hbm_model_frac": (field_model_bytes(wl, False)[1] if scheme == 0 else
                                      sum(a * b for a, b in algorithmic_bytes_ab2cn(wl, False).values()))
                   / (ms64 / 1e3) / 1e9 / float(measured_peaks()[0].get("hbm_gbs", 6800.0)),
                   "hbm_model": "full-field round trips" if scheme == 0 else "band storage"}
        err_own = precision_errors(qg, wl, w0, args.err_steps, stream, scheme)
        # the same parameters past the cape: the coast feeds the small scales and the closure is active
        cape = S.Workload(wl.name.replace("island", "cape"), wl.n, "cape", beta=wl.beta, U=wl.U, closure=wl.closure,
                          c=wl.c, dt=wl.dt, nu=wl.nu, mu=wl.mu, eta=wl.eta, sponge_rate=wl.sponge_rate, seed=wl.seed)
        err_cape = precision_errors(qg, cape, cape.omega0(), args.err_steps, stream, scheme)
        fp32_errors = {"workload": err_own, "same_parameters_past_the_cape": err_cape}
        if "diverged_at_step" in err_cape and scheme == 1:
            # AB2CN past the cape at this dt diverges in both forms (and in the oracle): the explicit AB2 part is
            # unstable there.  The FP32 error with the closure active then comes from a quarter of the time step.
            cq = S.Workload(cape.name + "-dt4", wl.n, "cape", beta=wl.beta, U=wl.U, closure=wl.closure, c=wl.c,
                            dt=wl.dt / 4, nu=wl.nu, mu=wl.mu, eta=wl.eta / 4, sponge_rate=wl.sponge_rate,
                            seed=wl.seed)
            fp32_errors["past_the_cape_quarter_dt"] = precision_errors(qg, cq, cq.omega0(), args.err_steps, stream,
                                                                       scheme)
        fp64 = {"value": wl.n * wl.n / (ms64 / 1e3), "ms_per_step": ms64, "steps_timed": k64,
                "fp32_speedup": ms64 / (ms / args.steps),
                "fp32_rel_l2_err_vs_fp64": err_own.get("w"), "err_steps": args.err_steps,
                "energy_rel_diff": err_own.get("E"), "enstrophy_rel_diff": err_own.get("Z"),
                "fp32_errors": fp32_errors,
                "roofline": alu,
                "fma_tflops": {"fp64": f64.value / 1e12 if rc64 == 0 else None,
                               "fp32": f32.value / 1e12 if rc32 == 0 else None}}

    torch_ctx = None
    if rank == 0 and scheme == 0 and fp32 and not args.no_torch_context:
        torch_ctx = torch_fft_context(wl, ms / args.steps)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            steps_c, el_c = time_oracle(wl, args.cpu_seconds, warmup=0, scheme=scheme)
            cpu = {"value": wl.n * wl.n * steps_c / el_c, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{steps_c} full {wl.n}^2 step(s) of the FP64 numpy oracle (single-threaded), "
                             f"{el_c:.1f} s"}
            cpu.update(host_cpu())
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "closure": S.CLOSURE_NAMES[wl.closure], "scheme": args.scheme,
                       "geometry": wl.geometry, "beta": wl.beta, "U": wl.U, "dt": wl.dt, "eta": wl.eta,
                       "precision": args.precision + (" (FP64 Germano sums, diagnostics, low-k inversion)"
                                                      if fp32 else ""),
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "working set > 126 MB L2 (inputs larger than L2, no flush)",
                       "timed_steps_from": args.spinup + args.warmup,
                       "coeff_after_spinup": spun["coeff"],
                       "final_energy": diag["energy"], "final_coeff": diag["coeff"], "finite": diag["finite"]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "fp64": fp64,
            "torch_fft_context": torch_ctx,
            "kernel_ms": {k: v[1] for k, v in per_class.items() if v[0]},
            "kernel_launches": {k: v[0] for k, v in per_class.items() if v[0]},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
