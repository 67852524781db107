"""Seeded synthetic electron loads in Debye units.

Units: plasma frequency, Debye length, thermal speed, vacuum permittivity and
mean electron density are all 1; electrons carry q = -1, m = 1.  A macro
particle then stands for w = V / N_p electrons (V the box volume), so the
mean electron charge density is -1 and the immobile ion background is +1.

Every generator takes a seed and returns host FP64 arrays.  Positions lie in
[0, L) on each spatial axis; velocities have `nv` components.  The loading
recipes follow the paper's worked example (Sec. 3.1: two beams at +-3 v_te,
an oblique mode seeded by the displacement of Eq. 1) and the workload shapes
the benchmark names (1D cold Langmuir, 2D two-stream, 3D magnetised, 3D
precision study, a batch of uneven 1D/2D instances).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Rows drawn per chunk when filling large arrays, so that temporaries stay small.
_CHUNK = 1 << 22


@dataclasses.dataclass
class Workload:
    name: str
    ndim: int
    n: tuple            # grid nodes per axis (3 entries, unused axes = 1)
    dx: tuple           # node spacing per axis (3 entries)
    dt: float
    steps: int
    x: np.ndarray       # (np, ndim) float64, in [0, L)
    v: np.ndarray       # (np, nv) float64
    q: float = -1.0
    m: float = 1.0
    weight: float = 1.0
    B0: tuple = (0.0, 0.0, 0.0)
    E0: tuple = (0.0, 0.0, 0.0)
    sort_every: int = 20
    mode: Optional[tuple] = None   # seeded Fourier mode (integers per axis)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def np_(self) -> int:
        return int(self.x.shape[0])

    @property
    def nv(self) -> int:
        return int(self.v.shape[1])

    @property
    def L(self) -> tuple:
        return tuple(self.n[a] * self.dx[a] for a in range(3))

    @property
    def cells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def config(self) -> dict:
        """Grid, species and push parameters as plain Python values."""
        return dict(ndim=self.ndim, n=tuple(self.n), dx=tuple(self.dx), dt=self.dt,
                    q=self.q, m=self.m, weight=self.weight, B0=tuple(self.B0),
                    E0=tuple(self.E0), nv=self.nv, sort_every=self.sort_every)


def _pad3(t, fill):
    t = tuple(t)
    return t + (fill,) * (3 - len(t))


def _box(ndim, n, dx):
    n3 = _pad3(n, 1)
    dx3 = _pad3(dx, 1.0)
    L = tuple(n3[a] * dx3[a] for a in range(ndim))
    return n3, dx3, L


def _uniform_positions(rng, npart, L):
    x = np.empty((npart, len(L)), dtype=np.float64)
    for s in range(0, npart, _CHUNK):
        e = min(npart, s + _CHUNK)
        x[s:e] = rng.random((e - s, len(L))) * np.asarray(L)
    return x


def _maxwellian(rng, npart, nv, vth):
    v = np.empty((npart, nv), dtype=np.float64)
    for s in range(0, npart, _CHUNK):
        e = min(npart, s + _CHUNK)
        v[s:e] = rng.standard_normal((e - s, nv)) * vth
    return v


def _wrap(x, L):
    """Bring positions back into [0, L) per axis (x == L maps to 0)."""
    for a, La in enumerate(L):
        col = x[:, a]
        np.subtract(col, La * np.floor(col / La), out=col)
        col[col >= La] = 0.0
        col[col < 0.0] = 0.0


def _displace(x, L, mode, delta0):
    """Seed a Fourier mode by the displacement of Eq. 1 (Sec. 3.1):
    xi = delta0 k / |k|^2 sin(k . x), k = 2 pi (m_a / L_a)."""
    k = np.array([2.0 * math.pi * mode[a] / L[a] for a in range(len(L))])
    k2 = float(np.dot(k, k))
    for s in range(0, x.shape[0], _CHUNK):
        e = min(x.shape[0], s + _CHUNK)
        phase = x[s:e] @ k
        x[s:e] += (delta0 / k2) * np.sin(phase)[:, None] * k[None, :]
    _wrap(x, L)


def langmuir_1d(n=64, k=0.5, npart=10_000, delta=0.01, dt=0.1, steps=200, seed=1):
    """Cold 1D Langmuir oscillation: a quiet lattice of electrons displaced by
    (delta / k) sin(k x), zero velocity.  L = 2 pi / k so the mode is m = 1."""
    L = 2.0 * math.pi / k
    n3, dx3, Lt = _box(1, (n,), (L / n,))
    x = ((np.arange(npart, dtype=np.float64) + 0.5) * (L / npart))[:, None].copy()
    # seed is unused by the lattice; kept so every generator has the same signature
    _ = np.random.default_rng(seed)
    _displace(x, Lt, (1,), delta)
    v = np.zeros((npart, 1), dtype=np.float64)
    return Workload("langmuir_1d", 1, n3, dx3, dt, steps, x, v, weight=L / npart,
                    mode=(1,), meta=dict(k=k, delta=delta))


def _lattice_positions(n, dx, sub):
    """A quiet start: sub[0] x sub[1] particles per cell on a regular sub-lattice
    ((i + 1/2) / sub_a of the cell on each axis); rows ordered with axis 0 fastest."""
    gx = (np.arange(n[0] * sub[0], dtype=np.float64) + 0.5) * (dx[0] / sub[0])
    gy = (np.arange(n[1] * sub[1], dtype=np.float64) + 0.5) * (dx[1] / sub[1])
    X, Y = np.meshgrid(gx, gy, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def _two_stream(name, n, dx, ppc_total, v0, vth, mode, delta0, dt, steps, nv, seed,
                sort_every=20, quiet=False):
    rng = np.random.default_rng(seed)
    n3, dx3, L = _box(2, n, dx)
    npart = int(n[0] * n[1] * ppc_total)
    half = npart // 2
    if quiet:
        side = int(round(math.sqrt(ppc_total // 2)))
        if 2 * side * side != ppc_total:
            raise ValueError("a quiet start needs ppc_total / 2 to be a perfect square")
        xb = _lattice_positions(n, dx, (side, side))
        x = np.concatenate([xb, xb])
    else:
        x = _uniform_positions(rng, npart, L)
    v = _maxwellian(rng, npart, nv, vth)
    v[:half, 0] += v0
    v[half:, 0] -= v0
    _displace(x, L, mode, delta0)
    V = L[0] * L[1]
    return Workload(name, 2, n3, dx3, dt, steps, x, v, weight=V / npart, mode=tuple(mode),
                    sort_every=sort_every,
                    meta=dict(v0=v0, vth=vth, delta0=delta0, ppc=ppc_total, quiet=quiet))


def two_stream_2d(n=(512, 512), ppc=64, v0=3.0, vth=1.0, mode=(16, 8), delta0=0.005,
                  dt=0.1, steps=500, nv=2, seed=2, sort_every=20):
    """2D electrostatic two-stream plasma: two equal beams at +-v0 along x with a
    Maxwellian spread vth on both axes, uniform random positions, and the oblique
    mode `mode` seeded by Eq. 1.  On a 512^2 box the default mode (16, 8) has the
    same wave vector as the paper's (2, 1) on its 64^2 box."""
    return _two_stream("two_stream_2d", n, (1.0, 1.0), ppc, v0, vth, mode, delta0, dt,
                       steps, nv, seed, sort_every)


def paper_two_stream(seed=7, nv=3, steps=800, quiet=True):
    """The paper's worked example (Sec. 3.1): 64 x 64 cells of one Debye length,
    64 macro-electrons per cell per beam (524,288 in total), beams at +-3 v_te,
    dt = 0.05, run to t = 40, mode (2, 1) seeded with delta0 = 0.005; 2D3V.
    The paper does not say how positions are loaded; the default here is a quiet
    start (each beam on an 8 x 8 sub-lattice per cell) so that the seeded mode,
    not particle noise, dominates the linear phase."""
    return _two_stream("paper_two_stream", (64, 64), (1.0, 1.0), 128, 3.0, 1.0, (2, 1),
                       0.005, 0.05, steps, nv, seed, quiet=quiet)


def cold_two_stream_1d(k=0.2, n=64, per_beam=8192, delta=1e-4, dt=0.05, steps=600):
    """Two cold counter-streaming beams in 1D, quiet lattice start, drift u chosen
    so that k u = sqrt(3/8) (the fastest-growing cold mode, gamma = 1/(2 sqrt 2));
    mode 1 seeded by the displacement of Eq. 1 with amplitude delta."""
    L = 2.0 * math.pi / k
    u = math.sqrt(3.0 / 8.0) / k
    n3, dx3, Lt = _box(1, (n,), (L / n,))
    xb = ((np.arange(per_beam, dtype=np.float64) + 0.5) * (L / per_beam))[:, None]
    x = np.concatenate([xb, xb])
    v = np.zeros((2 * per_beam, 1), dtype=np.float64)
    v[:per_beam, 0] = u
    v[per_beam:, 0] = -u
    _displace(x, Lt, (1,), delta)
    return Workload("cold_two_stream_1d", 1, n3, dx3, dt, steps, x, v, weight=L / (2 * per_beam),
                    mode=(1,), meta=dict(k=k, u=u, delta=delta))


def _bit_reversed(count):
    """The bit-reversal permutation of range(count), count a power of two."""
    bits = count.bit_length() - 1
    if 1 << bits != count:
        raise ValueError("count must be a power of two")
    idx = np.arange(count, dtype=np.int64)
    rev = np.zeros(count, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def two_stream_eigenmode_1d(k, u_d, gamma, n=64, per_beam=65536, amp=1e-3, dt=0.05,
                            steps=400):
    """Two warm 1D beams (Maxwellian v_te = 1 drifting at +-u_d) in a box of one
    wavelength L = 2 pi / k, loaded on the purely growing eigenmode omega = i gamma
    of mode 1 (gamma is supplied by the caller).

    Quiet start: each beam's positions sit on a regular lattice and its thermal
    velocities are the Maxwellian quantiles Phi^-1((i + 1/2) / N), assigned in
    bit-reversed order so that position and velocity are uncorrelated.  Each
    particle (position x0, velocity v) then takes the linear Lagrangian
    displacement of the mode, xi = Re[A e^{i k x0} / (k v - omega)^2] with
    A = amp gamma^2 (a particle at rest would move by amp / k), and the velocity
    change d xi / dt = Re[i (k v - omega) A e^{i k x0} / (k v - omega)^2].  Only the
    growing root is excited, so the seeded mode grows as e^{gamma t} from t = 0."""
    from scipy.special import ndtri

    L = 2.0 * math.pi / k
    n3, dx3, Lt = _box(1, (n,), (L / n,))
    x0 = (np.arange(per_beam, dtype=np.float64) + 0.5) * (L / per_beam)
    vq = ndtri((_bit_reversed(per_beam) + 0.5) / per_beam)
    x = np.concatenate([x0, x0])
    v = np.concatenate([u_d + vq, -u_d + vq])
    omega = 1j * gamma
    den = k * v - omega
    xi = (amp * gamma * gamma) * np.exp(1j * k * x) / (den * den)
    x = x + xi.real
    v = v + (1j * den * xi).real
    x = x[:, None].copy()
    _wrap(x, Lt)
    return Workload("two_stream_eigenmode_1d", 1, n3, dx3, dt, steps, x, v[:, None].copy(),
                    weight=L / (2 * per_beam), mode=(1,),
                    meta=dict(k=k, u_d=u_d, gamma=gamma, amp=amp))


def maxwellian_box(ndim, n, ppc, vth=1.0, nv=3, dt=0.1, B0=(0.0, 0.0, 0.0), steps=100,
                   seed=3, dx=None, name="maxwellian_box", sort_every=20):
    """Uniform random positions, isotropic Maxwellian velocities."""
    rng = np.random.default_rng(seed)
    dx = dx or (1.0,) * ndim
    n3, dx3, L = _box(ndim, n, dx)
    npart = int(np.prod(n)) * ppc
    x = _uniform_positions(rng, npart, L)
    v = _maxwellian(rng, npart, nv, vth)
    V = float(np.prod(L))
    return Workload(name, ndim, n3, dx3, dt, steps, x, v, weight=V / npart, B0=_pad3(B0, 0.0),
                    sort_every=sort_every, meta=dict(vth=vth, ppc=ppc))


def sparse_box(ndim, n, npart, vth=1.0, nv=None, dt=0.1, seed=8):
    """A dilute Maxwellian plasma (far fewer particles than cells), uniform random
    positions: sorted tiles of particles then span large parts of the grid."""
    rng = np.random.default_rng(seed)
    nv = nv or ndim
    n3, dx3, L = _box(ndim, n, (1.0,) * ndim)
    x = _uniform_positions(rng, npart, L)
    v = _maxwellian(rng, npart, nv, vth)
    V = float(np.prod(L))
    return Workload("sparse_box", ndim, n3, dx3, dt, 10, x, v, weight=V / npart,
                    meta=dict(vth=vth))


def magnetized_3d(n=(128, 128, 128), ppc=64, vth=1.0, wc=2.0, dt=0.05, steps=100, seed=3):
    """3D magnetised Maxwellian plasma with a uniform B0 along z such that the
    electron cyclotron frequency |q| B0 / m equals wc (in units of the plasma
    frequency)."""
    return maxwellian_box(3, n, ppc, vth=vth, nv=3, dt=dt, B0=(0.0, 0.0, wc), steps=steps,
                          seed=seed, name="magnetized_3d")


def precision_3d(n=(256, 256, 256), ppc=16, vth=1.0, noise=0.01, dt=0.1, steps=1000, seed=4):
    """3D Maxwellian plasma whose density carries white per-cell noise of
    relative amplitude `noise`: cells are drawn with probability proportional to
    1 + noise * u_c (u_c uniform in [-1, 1]), positions uniform inside the cell."""
    rng = np.random.default_rng(seed)
    n3, dx3, L = _box(3, n, (1.0, 1.0, 1.0))
    cells = int(np.prod(n))
    npart = cells * ppc
    dens = 1.0 + noise * (2.0 * rng.random(cells) - 1.0)
    cdf = np.cumsum(dens)
    cdf /= cdf[-1]
    x = np.empty((npart, 3), dtype=np.float64)
    for s in range(0, npart, _CHUNK):
        e = min(npart, s + _CHUNK)
        c = np.searchsorted(cdf, rng.random(e - s), side="right")
        c = np.minimum(c, cells - 1)
        ix = c % n[0]
        iy = (c // n[0]) % n[1]
        iz = c // (n[0] * n[1])
        x[s:e, 0] = (ix + rng.random(e - s)) * dx3[0]
        x[s:e, 1] = (iy + rng.random(e - s)) * dx3[1]
        x[s:e, 2] = (iz + rng.random(e - s)) * dx3[2]
    _wrap(x, L)
    v = _maxwellian(rng, npart, 3, vth)
    V = float(np.prod(L))
    return Workload("precision_3d", 3, n3, dx3, dt, steps, x, v, weight=V / npart,
                    meta=dict(vth=vth, ppc=ppc, noise=noise))


def batch_instances(count=1024, seed=5, n_range=(32, 1024), np_range=(1_000, 200_000),
                    vth=1.0, delta=0.01, dt=0.1, steps=200, nv=2, max_mode=4):
    """A batch of independent periodic 1D/2D instances of uneven size: each draws
    its dimension (1 or 2, even odds), nodes per axis log-uniform in n_range,
    particle count log-uniform in np_range, Maxwellian velocities and one random
    Fourier mode seeded by Eq. 1 with relative amplitude `delta`."""
    rng = np.random.default_rng(seed)
    out = []
    lo_n, hi_n = math.log(n_range[0]), math.log(n_range[1])
    lo_p, hi_p = math.log(np_range[0]), math.log(np_range[1])
    for i in range(count):
        ndim = int(rng.integers(1, 3))
        n = tuple(int(round(math.exp(rng.uniform(lo_n, hi_n)))) for _ in range(ndim))
        npart = int(round(math.exp(rng.uniform(lo_p, hi_p))))
        n3, dx3, L = _box(ndim, n, (1.0,) * ndim)
        x = _uniform_positions(rng, npart, L)
        v = _maxwellian(rng, npart, nv, vth)
        mode = tuple(int(rng.integers(1, max_mode + 1)) for _ in range(ndim))
        _displace(x, L, mode, delta)
        V = float(np.prod(L))
        out.append(Workload(f"batch[{i}]", ndim, n3, dx3, dt, steps, x, v, weight=V / npart,
                            mode=mode, meta=dict(vth=vth)))
    return out


def fp32_exact(w: Workload) -> Workload:
    """Round a load so that an FP32 cell + offset store and an FP64 store hold the same
    state: each offset x / dx - floor(x / dx) and each velocity is rounded to the
    nearest FP32 value (offsets that would round up to 1 are clamped below 1).  Exact
    only when every dx is a power of two, which is asserted."""
    for a in range(w.ndim):
        m, _ = math.frexp(w.dx[a])
        assert m == 0.5, "fp32_exact needs power-of-two dx"
    x = w.x.copy()
    for a in range(w.ndim):
        u = x[:, a] / w.dx[a]
        c = np.floor(u)
        f = (u - c).astype(np.float32)
        f = np.minimum(f, np.float32(np.nextafter(np.float32(1), np.float32(0))))
        x[:, a] = (c + f.astype(np.float64)) * w.dx[a]
    v = w.v.astype(np.float32).astype(np.float64)
    return dataclasses.replace(w, x=x, v=v)


def by_name(name: str, **kw) -> Workload:
    table = {
        "langmuir_1d": langmuir_1d,
        "two_stream_2d": two_stream_2d,
        "paper_two_stream": paper_two_stream,
        "cold_two_stream_1d": cold_two_stream_1d,
        "magnetized_3d": magnetized_3d,
        "precision_3d": precision_3d,
    }
    return table[name](**kw)
