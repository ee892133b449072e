"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only manufactures inputs: a counter-based random stream, the
initial vorticity field, the smoothed land mask and the sponge mask.  It holds
none of the time-stepping arithmetic (no Jacobian, no closure, no penalisation
step); both sides receive these arrays as plain FP64 host data.

Conventions: an N x N grid on [0, L)^2 with spacing d = L/N, x_i = i d,
arrays are row-major ``[y][x]`` (x fastest), dtype float64.

Input recipe (stands in for the paper's fully-resolved island and cape runs,
Sec. IV-A and IV-B, whose data is not available):

* initial vorticity: SplitMix64 -> Box-Muller white noise on the grid, shaped
  in Fourier space by sqrt(k^4 exp(-(k/8)^2)) (k in integer wavenumber units),
  mean removed, band-limited to |m_x|,|m_y| <= floor((N-1)/3), rescaled to
  rms 1;
* land mask chi = (1 - tanh(s / (2 d))) / 2 with s the signed distance to the
  coast (positive in the ocean); island = disc, cape = coastal strip
  y < 0.3 L plus a 0.5 L x 0.15 L rectangle centred in x;
* sponge mask chi_s = max(0, 1 - dist_to_x_edge / (0.1 L)), independent of y
  (the linear ramp of the sponge definition in Eq. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of SplitMix64 started from ``seed`` (uint64).

    Output i (0-based) is mix(seed + (i+1) * 0x9E3779B97F4A7C15) with the
    published SplitMix64 finaliser (shifts 30/27/31).
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform on SplitMix64 pairs."""
    npair = (count + 1) // 2
    u = uniform01(seed, 2 * npair)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


def band_limit(n: int) -> int:
    """Largest retained integer wavenumber of the 2/3 rule, floor((N-1)/3)."""
    return (n - 1) // 3


def init_field(seed: int, n: int, L: float = 2 * math.pi, k_peak: float = 8.0) -> np.ndarray:
    """Seeded random vorticity with spectrum k^4 exp(-(k/k_peak)^2), rms 1."""
    noise = normal(seed, n * n).reshape(n, n)
    spec = np.fft.rfft2(noise)
    mx = np.arange(n // 2 + 1)[None, :]
    my = np.fft.fftfreq(n, 1.0 / n)[:, None]
    k = np.sqrt(mx * mx + my * my)
    spec = spec * np.sqrt(k ** 4 * np.exp(-((k / k_peak) ** 2)))
    spec[0, 0] = 0.0
    kmax = band_limit(n)
    spec[(np.abs(my) > kmax) | (mx > kmax)] = 0.0
    w = np.fft.irfft2(spec, s=(n, n))
    rms = math.sqrt(float(np.mean(w * w)))
    return w / rms


def _coords(n: int, L: float):
    d = L / n
    x = np.arange(n) * d
    return x[None, :], x[:, None], d


def _periodic(a: np.ndarray, L: float) -> np.ndarray:
    """Minimum-image signed offset in a periodic box of length L."""
    return a - L * np.round(a / L)


def _smooth(s: np.ndarray, d: float) -> np.ndarray:
    return 0.5 * (1.0 - np.tanh(s / (2.0 * d)))


def island_mask(n: int, L: float = 2 * math.pi, center=(math.pi / 2, math.pi), radius: float = 0.4) -> np.ndarray:
    """Smoothed disc-shaped land mask (1 on land, 0 in the ocean)."""
    x, y, d = _coords(n, L)
    dx = _periodic(x - center[0], L)
    dy = _periodic(y - center[1], L)
    s = np.sqrt(dx * dx + dy * dy) - radius
    return _smooth(s, d)


def _box_sdf(px, py, hx, hy):
    qx = np.abs(px) - hx
    qy = np.abs(py) - hy
    outside = np.sqrt(np.maximum(qx, 0.0) ** 2 + np.maximum(qy, 0.0) ** 2)
    inside = np.minimum(np.maximum(qx, qy), 0.0)
    return outside + inside


def cape_mask(n: int, L: float = 2 * math.pi, wall: float = 0.3, cape_w: float = 0.5, cape_h: float = 0.15) -> np.ndarray:
    """Smoothed coastline-plus-cape land mask (1 on land).

    Land = {y < wall*L} U {|x - L/2| <= cape_w*L/2, y < (wall+cape_h)*L}; the
    signed distance of the union is the minimum of the two box distances.
    """
    x, y, d = _coords(n, L)
    hy_wall = 0.5 * wall * L
    s_wall = _box_sdf(np.zeros_like(x), _periodic(y - hy_wall, L), np.inf, hy_wall)
    s_wall = np.broadcast_to(s_wall, (n, n))
    top = (wall + cape_h) * L
    s_cape = _box_sdf(_periodic(x - 0.5 * L, L), _periodic(y - 0.5 * top, L), 0.5 * cape_w * L, 0.5 * top)
    return _smooth(np.minimum(s_wall, s_cape), d)


def sponge_mask(n: int, L: float = 2 * math.pi, width: float = 0.1) -> np.ndarray:
    """Linear sponge ramp at the two x-boundaries, 1 at the edge, 0 beyond width*L."""
    x, _, _ = _coords(n, L)
    dist = np.minimum(x, L - x)
    chi = np.maximum(0.0, 1.0 - dist / (width * L))
    return np.broadcast_to(chi, (n, n)).copy()


# Closure kinds, same numbering as the C-ABI.
NONE, SMAG, LEITH, DSMAG, DLEITH = 0, 1, 2, 3, 4
CLOSURE_NAMES = {NONE: "none", SMAG: "smagorinsky", LEITH: "leith", DSMAG: "dyn-smagorinsky", DLEITH: "dyn-leith"}


@dataclass
class Workload:
    """A named synthetic run: grid, physics, closure, geometry and seed."""
    name: str
    n: int
    geometry: str  # "island", "cape", "none"
    beta: float
    U: float
    closure: int
    c: float = 0.0
    test_ratio: float = 2.0
    dt: float = 2e-3
    nu: float = 1.0 / 200.0
    mu: float = 0.0
    eta: float = 1e-3
    sponge_rate: float = 50.0
    radius: float = 0.4
    seed: int = 0
    L: float = 2 * math.pi
    steps: int = 100
    sponge: bool = True
    extra: dict = field(default_factory=dict)

    def mask(self) -> np.ndarray:
        if self.geometry == "island":
            return island_mask(self.n, self.L, radius=self.radius)
        if self.geometry == "cape":
            return cape_mask(self.n, self.L)
        return np.zeros((self.n, self.n))

    def sponge_field(self):
        return sponge_mask(self.n, self.L) if self.sponge else None

    def omega0(self) -> np.ndarray:
        return init_field(self.seed, self.n, self.L)


def island128_smag() -> Workload:
    """Plain FP64 LES past an island at 128^2 with Smagorinsky c_S = 0.17."""
    return Workload("island128-smag", 128, "island", beta=5.0, U=0.5, closure=SMAG, c=0.17, radius=0.4, seed=0, steps=200)


def cape512(closure: int, seed: int = 1) -> Workload:
    """Closure sweep past a cape at 512^2 (beta = 10, U = 1)."""
    c = {SMAG: 0.17, LEITH: 0.25}.get(closure, 0.0)
    return Workload(f"cape512-{CLOSURE_NAMES[closure]}", 512, "cape", beta=10.0, U=1.0, closure=closure, c=c, seed=seed, steps=2000)


def island2048_dleith() -> Workload:
    """Production step past an island at 2048^2 with the dynamic Leith closure."""
    return Workload("island2048-dleith", 2048, "island", beta=5.0, U=0.5, closure=DLEITH, radius=0.2, seed=0, steps=5000)


def ensemble96(seed: int = 7) -> list:
    """96 independent LES members: 24 each of 256^2, 384^2, 512^2 and 768^2; island and cape geometries; the four
    closures; beta ~ U[2, 12) and U ~ U[0.3, 1.0) from SplitMix64(seed); member i starts from init_field(100 + i)."""
    sizes = [256, 384, 512, 768]
    kinds = [SMAG, LEITH, DSMAG, DLEITH]
    u = uniform01(seed, 2 * 96)
    out = []
    for i in range(96):
        n = sizes[i % 4]
        kind = kinds[(i // 4) % 4]
        geometry = "island" if (i // 16) % 2 == 0 else "cape"
        c = {SMAG: 0.17, LEITH: 0.25}.get(kind, 0.0)
        out.append(Workload(f"ens{i:02d}-{geometry}{n}-{CLOSURE_NAMES[kind]}", n, geometry, beta=2.0 + 10.0 * u[2 * i],
                            U=0.3 + 0.7 * u[2 * i + 1], closure=kind, c=c, seed=100 + i, steps=1000))
    return out


def wave_series(seed: int, n: int, nsnap: int, L: float = 2 * math.pi, speed=(0.5, 0.25), t0: float = 0.0,
                dt_snap: float = 1.0, nmodes: int = 6, noise: float = 0.0, noise_seed: int | None = None) -> np.ndarray:
    """A seeded snapshot series of a pattern translating at a uniform speed.

    Snapshot i is f(x - c_x t_i, y - c_y t_i) + noise, t_i = t0 + i dt_snap,
    where f = sum of ``nmodes`` cosines with integer wavevectors |m| <= 6,
    amplitudes in [0.5, 1.5) and phases in [0, 2 pi), all drawn from
    SplitMix64(seed).  ``noise`` adds white noise of that standard deviation
    (stream ``noise_seed``, default seed + 1).  Evaluated pointwise (no
    transforms).  Returns float64 of shape (nsnap, n, n).
    """
    u = uniform01(seed, 4 * nmodes)
    mx = np.floor(u[0::4] * 13).astype(int) - 6
    my = np.floor(u[1::4] * 13).astype(int) - 6
    mx[(mx == 0) & (my == 0)] = 1
    amp = 0.5 + u[2::4]
    phase = 2 * math.pi * u[3::4]
    x, y, _ = _coords(n, L)
    k0 = 2 * math.pi / L
    out = np.zeros((nsnap, n, n))
    for i in range(nsnap):
        t = t0 + i * dt_snap
        xs, ys = x - speed[0] * t, y - speed[1] * t
        for j in range(nmodes):
            out[i] += amp[j] * np.cos(k0 * (mx[j] * xs + my[j] * ys) + phase[j])
    if noise > 0:
        out += noise * normal(seed + 1 if noise_seed is None else noise_seed, out.size).reshape(out.shape)
    return out
