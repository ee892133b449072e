"""Python names of the libqg C-ABI (include/qg.h).  Argument marshalling only.

Host arrays are numpy float64/float32; device arrays are torch CUDA tensors
(passed by data pointer, borrowed for the call).  Streams are torch streams
or raw cudaStream_t integers.  The functional calls leave the ordering of a
handle's stream against other streams to the caller; QGSolver's methods and
qg_series_compare order it against torch's current stream themselves.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from ._lib import (QG_ERR_NONFINITE, QG_FP32, QG_FP64, QG_OK, QGError, check, load, qg_closure, qg_diag, qg_grid,
                   qg_member, qg_params)

__all__ = ["qg_create", "qg_set_state", "qg_get_state", "qg_stream", "qg_step", "qg_sync", "qg_diagnostics",
           "qg_destroy",
           "qg_sgs_apriori", "qg_grid_filter", "qg_series_compare", "qg_step_vjp", "qg_last_error", "qg_version",
           "QGSolver",
           "QGEnsemble"]


def _dptr(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def qg_last_error() -> str:
    return load().qg_last_error().decode()


def qg_version() -> str:
    return load().qg_version().decode()


def qg_create(grid: qg_grid, beta: float, U: float, mask, sponge, closure: qg_closure, params: qg_params,
              stream=None) -> int:
    """Create a solver; returns the opaque handle (int)."""
    lib = load()
    m = _dptr(mask)
    s = _dptr(sponge)
    n = grid.n
    for name, arr in (("mask", m), ("sponge", s)):
        if arr is not None and arr[0].size != n * n:
            raise ValueError(f"{name} must hold n*n values")
    out = C.c_void_p()
    rc = lib.qg_create(C.byref(grid), float(beta), float(U), m[1] if m else None, s[1] if s else None,
                       C.byref(closure), C.byref(params), _stream_ptr(stream), C.byref(out))
    check(rc, "qg_create")
    return out.value


def _buffer(omega, n):
    """(pointer, on_device, dtype, keepalive) of a host numpy array or a torch CUDA tensor."""
    if hasattr(omega, "is_cuda") and omega.is_cuda:
        import torch
        if omega.numel() != n * n or not omega.is_contiguous():
            raise ValueError("device field must be a contiguous tensor of n*n values")
        if omega.dtype == torch.float64:
            dt = QG_FP64
        elif omega.dtype == torch.float32:
            dt = QG_FP32
        else:
            raise TypeError("device field must be float32 or float64")
        return omega.data_ptr(), 1, dt, omega
    a = np.asarray(omega)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    a = np.ascontiguousarray(a)
    if a.size != n * n:
        raise ValueError("field must hold n*n values")
    return a.ctypes.data, 0, (QG_FP32 if a.dtype == np.float32 else QG_FP64), a


def qg_set_state(h: int, omega, n: int) -> None:
    ptr, dev, dt, keep = _buffer(omega, n)
    check(load().qg_set_state(h, ptr, dev, dt), "qg_set_state")
    del keep


def qg_get_state(h: int, n: int, out=None, dtype=np.float64):
    """Physical vorticity: into ``out`` (numpy or torch CUDA tensor) or a new numpy array."""
    if out is None:
        out = np.empty((n, n), dtype=dtype)
    ptr, dev, dt, keep = _buffer(out, n)
    check(load().qg_get_state(h, ptr, dev, dt), "qg_get_state")
    return out


def qg_stream(h: int) -> int:
    """The cudaStream_t (as an int, 0 = legacy default stream) the handle enqueues its work on."""
    out = C.c_void_p(0)
    check(load().qg_stream(h, C.byref(out)), "qg_stream")
    return int(out.value or 0)


class _Ordered:
    """Orders a handle's stream against torch's current stream around a call with device tensors.

    On entry the handle's stream waits for the current stream (whatever torch
    queued that writes the inputs); on exit the current stream waits for the
    handle's stream (so torch's later reads of the outputs, and the caching
    allocator's reuse of their memory, come after the library's writes).
    """

    def __init__(self, h: int, active: bool):
        self.h, self.active = h, active

    def __enter__(self):
        if self.active:
            import torch
            self.cur = torch.cuda.current_stream()
            ptr = qg_stream(self.h)
            self.hs = self.cur if ptr == self.cur.cuda_stream else (
                torch.cuda.default_stream() if ptr == 0 else torch.cuda.ExternalStream(ptr))
            if self.hs is not self.cur:
                self.hs.wait_stream(self.cur)
        return self

    def __exit__(self, *exc):
        if self.active and self.hs is not self.cur:
            self.cur.wait_stream(self.hs)


def _on_device(*xs) -> bool:
    return any(hasattr(x, "is_cuda") and x.is_cuda for x in xs if x is not None)


def qg_step(h: int, nsteps: int = 1) -> None:
    check(load().qg_step(h, int(nsteps)), "qg_step")


def qg_sync(h: int) -> None:
    check(load().qg_sync(h), "qg_sync")


def qg_diagnostics(h: int, raise_nonfinite: bool = True) -> dict:
    d = qg_diag()
    rc = load().qg_diagnostics(h, C.byref(d))
    if rc != QG_OK and not (rc == QG_ERR_NONFINITE and not raise_nonfinite):
        check(rc, "qg_diagnostics")
    return {"t": d.t, "step": d.step, "energy": d.energy, "enstrophy": d.enstrophy, "coeff": d.coeff,
            "max_abs_omega": d.max_abs_omega, "finite": bool(d.finite)}


def qg_step_vjp(h: int, n: int, omega_n, lam_next, lam_n=None):
    """Vector-Jacobian product of one step; returns (lam_n, grads) with grads = {"C", "c", "sponge_rate"}.

    omega_n and lam_next are both numpy arrays (host) or both torch CUDA
    tensors of the same dtype; lam_n (optional) is the output buffer.
    """
    pa, dev_a, dt_a, ka = _buffer(omega_n, n)
    pb, dev_b, dt_b, kb = _buffer(lam_next, n)
    if dev_a != dev_b or dt_a != dt_b:
        raise ValueError("omega_n and lam_next must share location and dtype")
    if lam_n is None:
        if dev_a:
            import torch
            lam_n = torch.empty_like(lam_next)
        else:
            lam_n = np.empty((n, n), dtype=np.float32 if dt_a == QG_FP32 else np.float64)
    pc, dev_c, dt_c, kc = _buffer(lam_n, n)
    if dev_c != dev_a or dt_c != dt_a:
        raise ValueError("lam_n must share location and dtype with the inputs")
    g = np.zeros(3)
    check(load().qg_step_vjp(h, pa, pb, pc, dev_a, dt_a, g.ctypes.data_as(C.POINTER(C.c_double))), "qg_step_vjp")
    del ka, kb, kc
    return lam_n, {"C": float(g[0]), "c": float(g[1]), "sponge_rate": float(g[2])}


def qg_destroy(h: int) -> None:
    if h:
        load().qg_destroy(h)


def qg_sgs_apriori(omega_fr, n_les: int, L: float, mask_fr, sponge_fr, closure: qg_closure, params: qg_params,
                   U: float, beta: float, flags: int = 0):
    """A priori SGS analysis; returns (pi_exact, pi_model, parts[3], pcc) as numpy arrays."""
    w = _dptr(omega_fr)
    n_fr = int(round(math.sqrt(w[0].size)))
    m = _dptr(mask_fr)
    s = _dptr(sponge_fr)
    pe = np.zeros((n_les, n_les))
    pm = np.zeros((n_les, n_les))
    parts = np.zeros((3, n_les, n_les))
    r = C.c_double(0.0)
    P = C.POINTER(C.c_double)
    rc = load().qg_sgs_apriori(w[1], n_fr, int(n_les), float(L), m[1] if m else None, s[1] if s else None,
                               C.byref(closure), C.byref(params), float(U), float(beta), int(flags),
                               pe.ctypes.data_as(P), pm.ctypes.data_as(P), parts.ctypes.data_as(P), C.byref(r))
    check(rc, "qg_sgs_apriori")
    return pe, pm, parts, r.value


def qg_grid_filter(omega_fr, n_les: int, L: float, gaussian: bool = True):
    """Grid filter of Eq. 5 on one fine field (n, n) or a series (nsnap, n, n); FP64 numpy out."""
    w = np.ascontiguousarray(omega_fr, dtype=np.float64)
    single = w.ndim == 2
    if single:
        w = w[None]
    if w.ndim != 3 or w.shape[1] != w.shape[2]:
        raise ValueError("omega_fr must be (n, n) or (nsnap, n, n)")
    out = np.empty((w.shape[0], n_les, n_les))
    P = C.POINTER(C.c_double)
    rc = load().qg_grid_filter(w.ctypes.data_as(P), w.shape[0], w.shape[1], int(n_les), float(L),
                               0 if gaussian else 1, out.ctypes.data_as(P))
    check(rc, "qg_grid_filter")
    return out[0] if single else out


def _series(a):
    """(pointer, nsnap, npts, dtype, on_device, keepalive) of a snapshot series."""
    if hasattr(a, "is_cuda") and a.is_cuda:
        import torch
        if not a.is_contiguous():
            raise ValueError("device series must be contiguous")
        if a.dtype not in (torch.float32, torch.float64):
            raise TypeError("device series must be float32 or float64")
        nsnap = a.shape[0]
        return a.data_ptr(), nsnap, a.numel() // max(nsnap, 1), (QG_FP32 if a.dtype == torch.float32 else QG_FP64), 1, a
    x = np.asarray(a)
    if x.dtype != np.float32:
        x = x.astype(np.float64)
    x = np.ascontiguousarray(x)
    nsnap = x.shape[0]
    return x.ctypes.data, nsnap, x.size // max(nsnap, 1), (QG_FP32 if x.dtype == np.float32 else QG_FP64), 0, x


def qg_series_compare(les, ff, lag_min: int, lag_max: int, stream=None, timing: bool = False):
    """Lag table of two snapshot series (Eq. 15-16): dist, pcc (n_ff, nlag), mean_dist (nlag,), phase.

    ``les`` and ``ff`` are (nsnap, ...) arrays of one dtype: both numpy (host)
    or both torch CUDA tensors (device).  ``timing`` adds ``kernel_ms``, the
    device time of the moments, pairs, finish and phase kernels.
    """
    pa, na, npa, da, dev_a, ka = _series(les)
    pb, nb, npb, db, dev_b, kb = _series(ff)
    if npa != npb or da != db or dev_a != dev_b:
        raise ValueError("series must have the same field size, dtype and location")
    nlag = int(lag_max) - int(lag_min) + 1
    dist = np.empty((nb, max(nlag, 0)))
    pcc = np.empty((nb, max(nlag, 0)))
    mean = np.empty(max(nlag, 0))
    phase = C.c_int32(0)
    kms = np.zeros(4)
    P = C.POINTER(C.c_double)
    if dev_a:
        # the call's stream waits for torch's current stream (the series' producer); the call
        # synchronises its stream before it returns
        import torch
        cur = torch.cuda.current_stream()
        sp = _stream_ptr(stream) or 0
        if sp != cur.cuda_stream:
            (torch.cuda.default_stream() if sp == 0 else torch.cuda.ExternalStream(sp)).wait_stream(cur)
    rc = load().qg_series_compare(pa, na, pb, nb, npa, da, dev_a, int(lag_min), int(lag_max), _stream_ptr(stream),
                                  dist.ctypes.data_as(P), pcc.ctypes.data_as(P), mean.ctypes.data_as(P),
                                  C.byref(phase), kms.ctypes.data_as(P) if timing else None)
    check(rc, "qg_series_compare")
    del ka, kb
    out = {"dist": dist, "pcc": pcc, "mean_dist": mean, "phase": phase.value}
    if timing:
        out["kernel_ms"] = {"moments": kms[0], "pairs": kms[1], "finish": kms[2], "phase": kms[3]}
    return out


@dataclass
class _Cfg:
    n: int
    L: float
    precision: int


class QGSolver:
    """Owning wrapper of one libqg handle."""

    def __init__(self, n: int, *, L: float = 2 * math.pi, precision: int = QG_FP64, beta: float = 0.0,
                 U: float = 0.0, mask=None, sponge=None, kind: int = 0, c: float = 0.0, test_ratio: float = 2.0,
                 dt: float = 2e-3, nu: float = 1.0 / 200.0, mu: float = 0.0, eta: float = 1e-3,
                 sponge_rate: float = 50.0, scheme: int = 0, stream=None):
        self.cfg = _Cfg(n, L, precision)
        self.h = 0
        self.h = qg_create(qg_grid(n, precision, L), beta, U, mask, sponge, qg_closure(kind, 0, c, test_ratio),
                           qg_params(dt, nu, mu, eta, sponge_rate, scheme, 0), stream)

    @classmethod
    def from_workload(cls, wl, precision: int = QG_FP64, stream=None, scheme: int = 0) -> "QGSolver":
        return cls(wl.n, L=wl.L, precision=precision, beta=wl.beta, U=wl.U, mask=wl.mask(),
                   sponge=wl.sponge_field(), kind=wl.closure, c=wl.c, test_ratio=wl.test_ratio, dt=wl.dt,
                   nu=wl.nu, mu=wl.mu, eta=wl.eta, sponge_rate=wl.sponge_rate, scheme=scheme, stream=stream)

    # Device tensors are ordered against torch's current stream (see _Ordered),
    # so callers may mix these calls with torch ops on any stream.
    def set_state(self, omega) -> None:
        with _Ordered(self.h, _on_device(omega)):
            qg_set_state(self.h, omega, self.cfg.n)

    def get_state(self, out=None, dtype=np.float64):
        with _Ordered(self.h, _on_device(out)):
            return qg_get_state(self.h, self.cfg.n, out, dtype)

    def step(self, nsteps: int = 1) -> None:
        qg_step(self.h, nsteps)

    def sync(self) -> None:
        qg_sync(self.h)

    def step_vjp(self, omega_n, lam_next, lam_n=None):
        with _Ordered(self.h, _on_device(omega_n, lam_next, lam_n)):
            return qg_step_vjp(self.h, self.cfg.n, omega_n, lam_next, lam_n)

    def diagnostics(self, raise_nonfinite: bool = True) -> dict:
        return qg_diagnostics(self.h, raise_nonfinite)

    @classmethod
    def _borrow(cls, h: int, n: int, L: float, precision: int) -> "QGSolver":
        """A view of a handle owned elsewhere (an ensemble member): close() leaves it alone."""
        obj = cls.__new__(cls)
        obj.cfg = _Cfg(n, L, precision)
        obj.h = h
        obj._owned = False
        return obj

    def close(self) -> None:
        if self.h and getattr(self, "_owned", True):
            qg_destroy(self.h)
        self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _member_args(n, *, L=2 * math.pi, precision=QG_FP64, beta=0.0, U=0.0, mask=None, sponge=None, kind=0, c=0.0,
                 test_ratio=2.0, dt=2e-3, nu=1.0 / 200.0, mu=0.0, eta=1e-3, sponge_rate=50.0, scheme=0):
    return dict(n=n, L=L, precision=precision, beta=beta, U=U, mask=mask, sponge=sponge, kind=kind, c=c,
                test_ratio=test_ratio, dt=dt, nu=nu, mu=mu, eta=eta, sponge_rate=sponge_rate, scheme=scheme)


class QGEnsemble:
    """Owning wrapper of a libqg ensemble.  ``members[i]`` is a borrowed QGSolver view of member i.

    Each entry of ``specs`` holds QGSolver's keyword arguments plus ``n``.
    """

    def __init__(self, specs, stream=None):
        self.e = 0
        args = [_member_args(**sp) for sp in specs]
        arr = (qg_member * len(args))()
        keep = []
        for i, a in enumerate(args):
            n = a["n"]
            m = arr[i]
            m.grid = qg_grid(n, a["precision"], a["L"])
            m.closure = qg_closure(a["kind"], 0, a["c"], a["test_ratio"])
            m.params = qg_params(a["dt"], a["nu"], a["mu"], a["eta"], a["sponge_rate"], a["scheme"], 0)
            m.beta = a["beta"]
            m.U = a["U"]
            for name in ("mask", "sponge"):
                d = _dptr(a[name])
                if d is not None:
                    if d[0].size != n * n:
                        raise ValueError(f"member {i}: {name} must hold n*n values")
                    keep.append(d[0])
                    setattr(m, name, d[1])
        out = C.c_void_p()
        check(load().qg_ensemble_create(arr, len(args), _stream_ptr(stream), C.byref(out)), "qg_ensemble_create")
        self.e = out.value
        self.members = []
        for i, a in enumerate(args):
            h = C.c_void_p()
            check(load().qg_ensemble_handle(self.e, i, C.byref(h)), "qg_ensemble_handle")
            self.members.append(QGSolver._borrow(h.value, a["n"], a["L"], a["precision"]))

    @classmethod
    def from_workloads(cls, wls, precision: int = QG_FP32, scheme: int = 0, stream=None) -> "QGEnsemble":
        return cls([dict(n=w.n, L=w.L, precision=precision, beta=w.beta, U=w.U, mask=w.mask(),
                         sponge=w.sponge_field(), kind=w.closure, c=w.c, test_ratio=w.test_ratio, dt=w.dt, nu=w.nu,
                         mu=w.mu, eta=w.eta, sponge_rate=w.sponge_rate, scheme=scheme) for w in wls], stream)

    def __len__(self):
        return len(self.members)

    def step(self, nsteps: int = 1) -> None:
        check(load().qg_ensemble_step(self.e, int(nsteps)), "qg_ensemble_step")

    def config(self) -> dict:
        """The launch form the tuner chose (qg_ensemble_config)."""
        form = (C.c_int32 * 4)()
        ms = C.c_double()
        check(load().qg_ensemble_config(self.e, form, C.byref(ms)), "qg_ensemble_config")
        return {"lanes": int(form[0]), "pdl": int(form[1]), "lean": int(form[2]),
                "source": {0: "default", 1: "timed", 2: "cached"}.get(int(form[3]), str(form[3])),
                "ms_per_step": ms.value}

    def sync(self) -> None:
        bad = C.c_int32(-1)
        rc = load().qg_ensemble_sync(self.e, C.byref(bad))
        if rc != QG_OK:
            err = QGError(rc, "qg_ensemble_sync", load().qg_last_error().decode())
            err.member = bad.value
            raise err

    def close(self) -> None:
        for m in getattr(self, "members", []):
            m.h = 0
        if self.e:
            load().qg_ensemble_destroy(self.e)
            self.e = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
