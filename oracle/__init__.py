"""FP64 CPU oracle of the electrostatic PIC cycle (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package.  It wraps the plain C reference in `pic_oracle.c` with ctypes and
composes the cycle in the order of the paper's worked example (Sec. 3.1,
Listing 1): load -> field update -> initial half push, then per step: velocity
push (gather + Boris) -> position update with periodic wrap -> field update.
It shares no code with the CUDA path.

Parity status per function (details in the repository's design notes):
  locate, deposit, gather, neg_laplacian, poisson_pcg, efield, boris,
  higuera_cary, move, sort_key, counting_sort, kinetic, kinetic_rel,
  field_energy, momentum, rng24, mcc, yee_b, yee_e, em_gather, boris_eb,
  esirkepov, CpmlField (cpml_b, cpml_e): pinned by the tests under
  tests/test_oracle_*.py.
"""

from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence

import numpy as np

from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int)


def _declare(L):
    i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.orc_set_threads.argtypes = [i]
    L.orc_set_threads.restype = None
    L.orc_get_threads.argtypes = []
    L.orc_get_threads.restype = i
    L.orc_locate.argtypes = [i, _I32, _D, i64, _D, _I64, _D]
    L.orc_deposit.argtypes = [i, _I32, _D, i64, _D, d, _D]
    L.orc_gather.argtypes = [i, _I32, _D, i64, _D, _D, _D]
    L.orc_neg_laplacian.argtypes = [i, _I32, _D, _D, _D]
    L.orc_poisson_pcg.argtypes = [i, _I32, _D, _D, _D, d, i, _I32, _D]
    L.orc_poisson_pcg.restype = i
    L.orc_efield.argtypes = [i, _I32, _D, _D, _D]
    L.orc_boris.argtypes = [i, i, i64, _D, _D, _D, _D, d, d]
    L.orc_move.argtypes = [i, _I32, _D, i, i64, _D, _D, d]
    L.orc_sort_key.argtypes = [i, _I32, _I32, i64, _I64, _I64]
    L.orc_counting_sort.argtypes = [i64, _I64, i64, _I64]
    L.orc_counting_sort.restype = i
    L.orc_kinetic.argtypes = [i, i64, _D, d]
    L.orc_kinetic.restype = d
    L.orc_field_energy.argtypes = [i, _I32, _D, _D]
    L.orc_field_energy.restype = d
    L.orc_momentum.argtypes = [i, i64, _D, d, _D]
    u32, u64 = ctypes.c_uint32, ctypes.c_uint64
    L.orc_rng24.argtypes = [u64, u64, u64, i]
    L.orc_rng24.restype = u32
    L.orc_rng24_fill.argtypes = [u64, u64, u64, i64, i, ctypes.POINTER(ctypes.c_uint32)]
    L.orc_rng24_fill.restype = None
    L.orc_mcc_threshold.argtypes = [d, d, d, d, d]
    L.orc_mcc_threshold.restype = u32
    L.orc_mcc.argtypes = [i64, _D, ctypes.POINTER(ctypes.c_uint32), u64, u64, d, d, d, d, d, d,
                          d, d, _I64]
    L.orc_mcc.restype = None
    L.orc_yee_b.argtypes = [_I32, _D, _D, _D, d]
    L.orc_yee_b.restype = None
    L.orc_yee_e.argtypes = [_I32, _D, _D, _D, d, d, _D]
    L.orc_yee_e.restype = None
    L.orc_yee_div_e.argtypes = [_I32, _D, _D, _D]
    L.orc_yee_div_e.restype = None
    L.orc_yee_div_b.argtypes = [_I32, _D, _D, _D]
    L.orc_yee_div_b.restype = None
    L.orc_em_gather.argtypes = [_I32, _D, i64, _D, _D, _D, _D]
    L.orc_em_gather.restype = None
    L.orc_boris_eb.argtypes = [i64, _D, _D, d, d]
    L.orc_boris_eb.restype = None
    L.orc_esirkepov.argtypes = [_I32, _D, i64, _D, _D, _D, d, d, _D]
    L.orc_esirkepov.restype = None
    PP = ctypes.POINTER(_D)
    L.orc_cpml_b.argtypes = [_I32, _D, _D, _D, d, PP, PP]
    L.orc_cpml_b.restype = None
    L.orc_cpml_e.argtypes = [_I32, _D, _D, _D, d, d, _D, PP, PP]
    L.orc_cpml_e.restype = None
    L.orc_yee3_b.argtypes = [_I32, _D, _D, _D, d]
    L.orc_yee3_b.restype = None
    L.orc_yee3_e.argtypes = [_I32, _D, _D, _D, d, d, _D]
    L.orc_yee3_e.restype = None
    L.orc_yee3_div_e.argtypes = [_I32, _D, _D, _D]
    L.orc_yee3_div_e.restype = None
    L.orc_yee3_div_b.argtypes = [_I32, _D, _D, _D]
    L.orc_yee3_div_b.restype = None
    L.orc_em3_gather.argtypes = [_I32, _D, i64, _D, _D, _D, _D]
    L.orc_em3_gather.restype = None
    L.orc_esirkepov3.argtypes = [_I32, _D, i64, _D, _D, d, d, _D]
    L.orc_esirkepov3.restype = None
    L.orc_em_gather_np.argtypes = [_I32, _D, i64, _D, _D, _D, _D]
    L.orc_em_gather_np.restype = None
    L.orc_esirkepov_np.argtypes = [_I32, _D, i64, _D, _D, _D, d, d, _D]
    L.orc_esirkepov_np.restype = None
    L.orc_deposit_np.argtypes = [_I32, _D, i64, _D, d, _D]
    L.orc_deposit_np.restype = None
    L.orc_hc.argtypes = [i, i, i64, _D, _D, _D, _D, d, d, d]
    L.orc_hc.restype = None
    L.orc_kinetic_rel.argtypes = [i, i64, _D, d, d]
    L.orc_kinetic_rel.restype = d


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _i64p(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_I64)


def _n3(n: Sequence[int]):
    t = list(n) + [1] * (3 - len(n))
    return (ctypes.c_int * 3)(*t[:3])


def _dx3(dx: Sequence[float]):
    t = list(dx) + [1.0] * (3 - len(dx))
    return (ctypes.c_double * 3)(*t[:3])


def _cells(ndim, n):
    return int(np.prod(list(n)[:ndim]))


# ---- thin functional wrappers -------------------------------------------------------------

def set_threads(n):
    """Threads of the particle loops (deposit, gather, pushers, move): each takes a
    contiguous range of particles; the deposit sums per-thread copies of rho in
    thread order.  1 (the default) is the sequential code."""
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())


def locate(ndim, n, dx, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    npart = x.shape[0]
    cell = np.empty(npart, np.int64)
    off = np.empty((npart, ndim), np.float64)
    lib().orc_locate(ndim, _n3(n), _dx3(dx), npart, _dp(x), _i64p(cell), _dp(off))
    return cell, off


def deposit(ndim, n, dx, x, qw):
    """Electron charge density on the nodes (Sec. 2.2 B_Scatter)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    rho = np.empty(_cells(ndim, n), np.float64)
    lib().orc_deposit(ndim, _n3(n), _dx3(dx), x.shape[0], _dp(x), float(qw), _dp(rho))
    return rho


def gather(ndim, n, dx, x, E):
    """Grid field at the particles (Sec. 2.2 C_Gather)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    Ep = np.empty((x.shape[0], ndim), np.float64)
    lib().orc_gather(ndim, _n3(n), _dx3(dx), x.shape[0], _dp(x), _dp(E), _dp(Ep))
    return Ep


def neg_laplacian(ndim, n, dx, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    lib().orc_neg_laplacian(ndim, _n3(n), _dx3(dx), _dp(u), _dp(out))
    return out


def poisson(ndim, n, dx, rho, rtol=1e-12, maxit=200000):
    """-lap(phi) = rho - mean(rho), zero-mean phi (Sec. 2.2 D_Poisson)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.empty_like(rho)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib().orc_poisson_pcg(ndim, _n3(n), _dx3(dx), _dp(rho), _dp(phi), rtol, maxit,
                               ctypes.byref(it), ctypes.byref(rel))
    if st != 0:
        raise RuntimeError(f"oracle PCG did not converge: {it.value} iterations, "
                           f"relative residual {rel.value:.3e}")
    return phi, it.value, rel.value


def efield(ndim, n, dx, phi):
    """E = -grad(phi), centred differences (module D06, Sec. 3.1)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    E = np.empty(ndim * phi.size, np.float64)
    lib().orc_efield(ndim, _n3(n), _dx3(dx), _dp(phi), _dp(E))
    return E


def boris(ndim, v, Ep, E0, B0, qm, h):
    """In-place Boris velocity advance by step h (Sec. 2.2 A_Pusher)."""
    assert v.dtype == np.float64 and v.flags.c_contiguous
    npart, nv = v.shape
    Epp = _dp(np.ascontiguousarray(Ep, dtype=np.float64)) if Ep is not None else None
    e0 = (ctypes.c_double * 3)(*(list(E0) + [0.0] * 3)[:3])
    b0 = (ctypes.c_double * 3)(*(list(B0) + [0.0] * 3)[:3])
    keep = Ep  # noqa: F841  (keep the array alive during the call)
    lib().orc_boris(ndim, nv, npart, _dp(v), Epp, e0, b0, float(qm), float(h))
    return v


def move(ndim, n, dx, x, v, dt):
    """In-place x += v dt with periodic wrap (application code, Sec. 3.1)."""
    assert x.dtype == np.float64 and x.flags.c_contiguous
    v = np.ascontiguousarray(v, dtype=np.float64)
    lib().orc_move(ndim, _n3(n), _dx3(dx), v.shape[1], x.shape[0], _dp(x), _dp(v), float(dt))
    return x


def sort_key(ndim, n, brick, cell):
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    key = np.empty_like(cell)
    b = (ctypes.c_int * 3)(*(list(brick) + [1, 1, 1])[:3])
    lib().orc_sort_key(ndim, _n3(n), b, cell.size, _i64p(cell), _i64p(key))
    return key


def num_keys(ndim, n, brick):
    nk = 1
    for a in range(ndim):
        nb = -(-n[a] // brick[a])
        nk *= nb * brick[a]
    return nk


def counting_sort(key, nkeys):
    key = np.ascontiguousarray(key, dtype=np.int64)
    perm = np.empty_like(key)
    if lib().orc_counting_sort(key.size, _i64p(key), int(nkeys), _i64p(perm)) != 0:
        raise ValueError("sort key out of range")
    return perm


def higuera_cary(ndim, u, Ep, E0, B0, qm, h, c=None):
    """In-place Higuera-Cary advance of the momentum per mass u = gamma v by step h
    (Sec. 2.2 A_Pusher); c=None is the non-relativistic limit."""
    assert u.dtype == np.float64 and u.flags.c_contiguous
    npart, nv = u.shape
    Epp = _dp(np.ascontiguousarray(Ep, dtype=np.float64)) if Ep is not None else None
    e0 = (ctypes.c_double * 3)(*(list(E0) + [0.0] * 3)[:3])
    b0 = (ctypes.c_double * 3)(*(list(B0) + [0.0] * 3)[:3])
    keep = Ep  # noqa: F841  (keep the array alive during the call)
    lib().orc_hc(ndim, nv, npart, _dp(u), Epp, e0, b0, float(qm), float(h), _inv_c2(c))
    return u


def _inv_c2(c):
    return 0.0 if c is None or c == math.inf else 1.0 / (float(c) * float(c))


def lorentz_gamma(u, c=None):
    """gamma = sqrt(1 + |u|^2 / c^2) per particle."""
    u = np.asarray(u, dtype=np.float64)
    return np.sqrt(1.0 + np.sum(u * u, axis=1) * _inv_c2(c))


def kinetic_rel(u, mw, c=None):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_kinetic_rel(u.shape[1], u.shape[0], _dp(u), float(mw), _inv_c2(c))


def rng24(seed, step, pid, k):
    """The counter-based 24-bit draw k of particle `pid` at `step` (SplitMix64 output
    function); what both the oracle and the CUDA path draw."""
    return int(lib().orc_rng24(int(seed), int(step), int(pid), int(k)))


def rng24_fill(seed, step, id0, n, k):
    out = np.empty(n, np.uint32)
    lib().orc_rng24_fill(int(seed), int(step), int(id0), int(n), int(k),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def mcc_threshold(ng, sig_el, sig_exc, vmax, dt):
    return int(lib().orc_mcc_threshold(float(ng), float(sig_el), float(sig_exc), float(vmax),
                                       float(dt)))


MCC_FIELDS = ("density", "sigma_el", "sigma_exc", "eps_exc", "mass_ratio", "vmax", "seed")


def mcc(v, ids, step, p, m, dt):
    """In-place null-collision step (Sec. 2.2 G_collision) of velocities v (np x 3)
    with particle ids; p: dict with MCC_FIELDS.  Returns the counts (elastic,
    excitation, bound exceeded)."""
    assert v.dtype == np.float64 and v.flags.c_contiguous and v.shape[1] == 3
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    counts = np.zeros(3, np.int64)
    lib().orc_mcc(v.shape[0], _dp(v), ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                  int(step), int(p["seed"]), float(p["density"]), float(p["sigma_el"]),
                  float(p["sigma_exc"]), float(p["eps_exc"]), float(p["mass_ratio"]),
                  float(p["vmax"]), float(m), float(dt), _i64p(counts))
    return counts


def kinetic(v, mw):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().orc_kinetic(v.shape[1], v.shape[0], _dp(v), float(mw))


def field_energy(ndim, n, dx, E):
    E = np.ascontiguousarray(E, dtype=np.float64)
    return lib().orc_field_energy(ndim, _n3(n), _dx3(dx), _dp(E))


def momentum(v, mw):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(3, np.float64)
    lib().orc_momentum(v.shape[1], v.shape[0], _dp(v), float(mw), _dp(out))
    return out[: v.shape[1]]


# ---- the cycle ----------------------------------------------------------------------------

class Simulation:
    """The electrostatic PIC cycle of Listing 1 (Sec. 3.1) in FP64.

    `rho_background=None` neutralises the loaded electrons exactly:
    rho_ion = -q w N_p / V.
    """

    def __init__(self, ndim, n, dx, dt, q=-1.0, m=1.0, weight=1.0, B0=(0, 0, 0),
                 E0=(0, 0, 0), rho_background: Optional[float] = None, rtol=1e-12,
                 maxit=200000, pusher="boris", c=None, collisions=None):
        self.ndim = ndim
        self.n = tuple(list(n)[:3]) + (1,) * (3 - len(n))
        self.dx = tuple(list(dx)[:3]) + (1.0,) * (3 - len(dx))
        self.dt, self.q, self.m, self.w = float(dt), float(q), float(m), float(weight)
        self.B0 = tuple(B0) + (0.0,) * (3 - len(B0))
        self.E0 = tuple(E0) + (0.0,) * (3 - len(E0))
        self.rho_background = rho_background
        self.rtol, self.maxit = rtol, maxit
        # "boris", or "hc" (Higuera-Cary): v then holds u = gamma v, positions move
        # with u / gamma, and the kinetic energy is the relativistic one
        assert pusher in ("boris", "hc")
        self.pusher, self.c = pusher, c
        # null-collision Monte Carlo after each move (dict with MCC_FIELDS, or None);
        # particle ids are the load order
        self.collisions = collisions
        self.mcc_counts = np.zeros(3, np.int64)
        self.cells = _cells(ndim, self.n)
        self.dV = float(np.prod(self.dx[:ndim]))
        self.V = self.dV * self.cells
        self.t = 0.0
        self.step_count = 0
        self.cg_iters = 0
        self.ke = 0.0

    # field update: B01 -> D02 -> D05/D06
    def update_field(self):
        npart = self.x.shape[0]
        self.rho_e = deposit(self.ndim, self.n, self.dx, self.x, self.q * self.w)
        bg = (-self.q * self.w * npart / self.V if self.rho_background is None
              else float(self.rho_background))
        self.rho = self.rho_e + bg
        self.phi, self.cg_iters, self.cg_res = poisson(self.ndim, self.n, self.dx, self.rho,
                                                       self.rtol, self.maxit)
        self.E = efield(self.ndim, self.n, self.dx, self.phi)

    def load(self, x, v, half_push=True):
        self.x = np.array(x, dtype=np.float64, order="C")
        self.v = np.array(v, dtype=np.float64, order="C")
        self.ids = np.arange(self.x.shape[0], dtype=np.uint32)
        self.update_field()
        if half_push:
            Ep = gather(self.ndim, self.n, self.dx, self.x, self.E)
            v0 = self.v.copy()
            self._advance(Ep, -0.5 * self.dt)
            self.ke = self._kinetic(v0)
        return self

    def _advance(self, Ep, h):
        if self.pusher == "hc":
            higuera_cary(self.ndim, self.v, Ep, self.E0, self.B0, self.q / self.m, h, self.c)
        else:
            boris(self.ndim, self.v, Ep, self.E0, self.B0, self.q / self.m, h)

    def _kinetic(self, v):
        if self.pusher == "hc":
            return kinetic_rel(v, self.m * self.w, self.c)
        return kinetic(v, self.m * self.w)

    def push(self):
        """Gather (C01) + the pusher (A01 Boris, or Higuera-Cary) by one full step;
        returns the time-centred kinetic energy (mean of the two half-step energies)."""
        Ep = gather(self.ndim, self.n, self.dx, self.x, self.E)
        ke_old = self._kinetic(self.v)
        self._advance(Ep, self.dt)
        self.ke = 0.5 * (ke_old + self._kinetic(self.v))
        return self.ke

    def velocity(self):
        """dx/dt of each particle: v, or u / gamma with the Higuera-Cary pusher."""
        if self.pusher == "hc":
            return np.ascontiguousarray(self.v / lorentz_gamma(self.v, self.c)[:, None])
        return self.v

    def move(self):
        move(self.ndim, self.n, self.dx, self.x, self.velocity(), self.dt)

    def collide(self):
        """Null-collision step of this time step (the step count it draws with is
        the step being completed, 1 for the first)."""
        self.mcc_counts = mcc(self.v, self.ids, self.step_count + 1, self.collisions, self.m,
                              self.dt)
        return self.mcc_counts

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self.push()
            self.move()
            if self.collisions is not None:
                self.collide()
            self.update_field()
            self.t += self.dt
            self.step_count += 1
        return self

    def field_energy(self):
        return field_energy(self.ndim, self.n, self.dx, self.E)

    def momentum(self):
        return momentum(self.v, self.m * self.w)

    def cells_offsets(self):
        return locate(self.ndim, self.n, self.dx, self.x)

    def sort(self, brick):
        cell, _ = self.cells_offsets()
        key = sort_key(self.ndim, self.n, brick, cell)
        perm = counting_sort(key, num_keys(self.ndim, self.n, brick))
        self.x = np.ascontiguousarray(self.x[perm])
        self.v = np.ascontiguousarray(self.v[perm])
        self.ids = np.ascontiguousarray(self.ids[perm])
        return perm


# ---- electromagnetic step (E_Maxwell, Sec. 2.2): periodic 2D3V Yee grid ----------------------

def _n2(n):
    return (ctypes.c_int * 2)(int(n[0]), int(n[1]))


def _dx2(dx):
    return (ctypes.c_double * 2)(float(dx[0]), float(dx[1]))


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def yee_b(n, dx, E, B, h):
    """In-place B -= h curl E on the Yee grid ([3][cells] arrays)."""
    assert B.dtype == np.float64 and B.flags.c_contiguous
    E = _f(E)
    lib().orc_yee_b(_n2(n), _dx2(dx), _dp(E), _dp(B), float(h))
    return B


def yee_e(n, dx, B, J, c, dt, E):
    """In-place E += dt (c^2 curl B - J)."""
    assert E.dtype == np.float64 and E.flags.c_contiguous
    B, J = _f(B), _f(J)
    lib().orc_yee_e(_n2(n), _dx2(dx), _dp(B), _dp(J), float(c) ** 2, float(dt), _dp(E))
    return E


def yee_div_e(n, dx, E):
    out = np.empty(int(n[0]) * int(n[1]))
    E = _f(E)
    lib().orc_yee_div_e(_n2(n), _dx2(dx), _dp(E), _dp(out))
    return out


def yee_div_b(n, dx, B):
    out = np.empty(int(n[0]) * int(n[1]))
    B = _f(B)
    lib().orc_yee_div_b(_n2(n), _dx2(dx), _dp(B), _dp(out))
    return out


def em_gather(n, dx, x, E, B):
    """E and B at the particles (np x 6), CIC on each component's staggered lattice."""
    x, E, B = _f(x), _f(E), _f(B)
    out = np.empty((x.shape[0], 6))
    lib().orc_em_gather(_n2(n), _dx2(dx), x.shape[0], _dp(x), _dp(E), _dp(B), _dp(out))
    return out


def boris_eb(v, EB, qm, h):
    assert v.dtype == np.float64 and v.flags.c_contiguous and v.shape[1] == 3
    EB = _f(EB)
    lib().orc_boris_eb(v.shape[0], _dp(v), _dp(EB), float(qm), float(h))
    return v


def esirkepov(n, dx, x0, x1, vz, qw, dt, J):
    """Add the charge-conserving current of the moves x0 -> x1 into J ([3][cells])."""
    assert J.dtype == np.float64 and J.flags.c_contiguous
    x0, x1, vz = _f(x0), _f(x1), _f(vz)
    lib().orc_esirkepov(_n2(n), _dx2(dx), x0.shape[0], _dp(x0), _dp(x1), _dp(vz), float(qw),
                        float(dt), _dp(J))
    return J


class EmSimulation:
    """The electromagnetic PIC cycle on a periodic 2D3V Yee grid (E_Maxwell with the
    particle modules of Sec. 2.2), FP64.  Fields E^n and B^n at integer times; each
    step: gather E^n, B^n (+ uniform B0) -> Boris -> move -> Esirkepov current
    J^(n+1/2) -> B -= (dt/2) curl E -> E += dt (c^2 curl B - J) -> B -= (dt/2) curl E.
    Loading solves the Poisson equation of the loaded charge for the initial E
    (E = -grad phi by forward differences onto the staggered points, so that
    div E = rho exactly), B = 0, then the backward half push."""

    def __init__(self, n, dx, dt, c, q=-1.0, m=1.0, weight=1.0, B0=(0, 0, 0), rtol=1e-12):
        self.n = (int(n[0]), int(n[1]))
        self.dx = (float(dx[0]), float(dx[1]))
        self.dt, self.c, self.q, self.m, self.w = float(dt), float(c), float(q), float(m), float(weight)
        self.B0 = np.array(list(B0) + [0.0] * (3 - len(B0)))[:3]
        self.rtol = rtol
        self.cells = self.n[0] * self.n[1]
        self.dV = self.dx[0] * self.dx[1]
        self.V = self.dV * self.cells
        self.step_count = 0

    def _rho(self):
        rho_e = deposit(2, self.n, self.dx, self.x, self.q * self.w)
        return rho_e + (-self.q * self.w * self.x.shape[0] / self.V)

    def load(self, x, v, half_push=True):
        self.x = np.array(x, dtype=np.float64, order="C")
        self.v = np.array(v, dtype=np.float64, order="C")
        assert self.v.shape[1] == 3
        rho = self._rho()
        phi, _, _ = poisson(2, self.n, self.dx, rho, self.rtol, 200000)
        ph = phi.reshape(self.n[1], self.n[0])
        self.E = np.zeros((3, self.cells))
        self.E[0] = (-(np.roll(ph, -1, axis=1) - ph) / self.dx[0]).ravel()
        self.E[1] = (-(np.roll(ph, -1, axis=0) - ph) / self.dx[1]).ravel()
        self.B = np.zeros((3, self.cells))
        self.J = np.zeros((3, self.cells))
        self.rho = rho
        if half_push:
            boris_eb(self.v, self._fields_at(self.x), self.q / self.m, -0.5 * self.dt)
        return self

    def _fields_at(self, x):
        EB = em_gather(self.n, self.dx, x, self.E, self.B)
        EB[:, 3:] += self.B0
        return EB

    def step(self, nsteps=1):
        for _ in range(nsteps):
            boris_eb(self.v, self._fields_at(self.x), self.q / self.m, self.dt)
            x0 = self.x.copy()
            move(2, self.n + (1,), self.dx + (1.0,), self.x, self.v, self.dt)
            self.J = np.zeros((3, self.cells))
            esirkepov(self.n, self.dx, x0, self.x, self.v[:, 2], self.q * self.w, self.dt, self.J)
            yee_b(self.n, self.dx, self.E, self.B, 0.5 * self.dt)
            yee_e(self.n, self.dx, self.B, self.J, self.c, self.dt, self.E)
            yee_b(self.n, self.dx, self.E, self.B, 0.5 * self.dt)
            self.rho = self._rho()
            self.step_count += 1
        return self

    def gauss_residual(self):
        return yee_div_e(self.n, self.dx, self.E) - self.rho


# ---- electromagnetic step in 3D (E_Maxwell, Sec. 2.2): periodic Yee lattice --------------------
# Ex (1/2,0,0), Ey (0,1/2,0), Ez (0,0,1/2); Bx (0,1/2,1/2), By (1/2,0,1/2), Bz (1/2,1/2,0);
# arrays [3][cells] with x fastest.

def _cells3(n):
    return int(n[0]) * int(n[1]) * int(n[2])


def yee3_b(n, dx, E, B, h):
    """In-place B -= h curl E on the 3D Yee lattice."""
    assert B.dtype == np.float64 and B.flags.c_contiguous
    lib().orc_yee3_b(_n3(n), _dx3(dx), _dp(_f(E)), _dp(B), float(h))
    return B


def yee3_e(n, dx, B, J, c, dt, E):
    """In-place E += dt (c^2 curl B - J) on the 3D Yee lattice."""
    assert E.dtype == np.float64 and E.flags.c_contiguous
    lib().orc_yee3_e(_n3(n), _dx3(dx), _dp(_f(B)), _dp(_f(J)), float(c) ** 2, float(dt), _dp(E))
    return E


def yee3_div_e(n, dx, E):
    out = np.empty(_cells3(n))
    lib().orc_yee3_div_e(_n3(n), _dx3(dx), _dp(_f(E)), _dp(out))
    return out


def yee3_div_b(n, dx, B):
    out = np.empty(_cells3(n))
    lib().orc_yee3_div_b(_n3(n), _dx3(dx), _dp(_f(B)), _dp(out))
    return out


def em3_gather(n, dx, x, E, B):
    """E and B at the particles (np x 6), trilinear CIC on each staggered lattice."""
    x = _f(x)
    out = np.empty((x.shape[0], 6))
    lib().orc_em3_gather(_n3(n), _dx3(dx), x.shape[0], _dp(x), _dp(_f(E)), _dp(_f(B)), _dp(out))
    return out


def esirkepov3(n, dx, x0, x1, qw, dt, J):
    """Add the charge-conserving 3D current of the moves x0 -> x1 into J ([3][cells])."""
    assert J.dtype == np.float64 and J.flags.c_contiguous
    x0, x1 = _f(x0), _f(x1)
    lib().orc_esirkepov3(_n3(n), _dx3(dx), x0.shape[0], _dp(x0), _dp(x1), float(qw), float(dt),
                         _dp(J))
    return J


class EmSimulation3:
    """The electromagnetic PIC cycle on a periodic 3D Yee lattice, FP64: the 3D form of
    EmSimulation.  Each step: gather E^n, B^n (+ uniform B0) -> Boris -> move ->
    Esirkepov current J^(n+1/2) -> B -= (dt/2) curl E -> E += dt (c^2 curl B - J) ->
    B -= (dt/2) curl E.  Loading solves the Poisson equation of the loaded charge for
    the initial E (forward differences of phi onto the staggered points, so that
    div E = rho exactly), B = 0, then the backward half push."""

    def __init__(self, n, dx, dt, c, q=-1.0, m=1.0, weight=1.0, B0=(0, 0, 0), rtol=1e-12):
        self.n = tuple(int(k) for k in n[:3])
        self.dx = tuple(float(h) for h in dx[:3])
        self.dt, self.c, self.q, self.m, self.w = float(dt), float(c), float(q), float(m), float(weight)
        self.B0 = np.array(list(B0) + [0.0] * (3 - len(B0)))[:3]
        self.rtol = rtol
        self.cells = _cells3(self.n)
        self.dV = self.dx[0] * self.dx[1] * self.dx[2]
        self.V = self.dV * self.cells
        self.step_count = 0

    def _rho(self):
        rho_e = deposit(3, self.n, self.dx, self.x, self.q * self.w)
        return rho_e + (-self.q * self.w * self.x.shape[0] / self.V)

    def load(self, x, v, half_push=True):
        self.x = np.array(x, dtype=np.float64, order="C")
        self.v = np.array(v, dtype=np.float64, order="C")
        assert self.x.shape[1] == 3 and self.v.shape[1] == 3
        rho = self._rho()
        phi, _, _ = poisson(3, self.n, self.dx, rho, self.rtol, 200000)
        ph = phi.reshape(self.n[2], self.n[1], self.n[0])
        self.E = np.zeros((3, self.cells))
        for a, axis in ((0, 2), (1, 1), (2, 0)):  # numpy axis of x, y, z
            self.E[a] = (-(np.roll(ph, -1, axis=axis) - ph) / self.dx[a]).ravel()
        self.B = np.zeros((3, self.cells))
        self.J = np.zeros((3, self.cells))
        self.rho = rho
        if half_push:
            boris_eb(self.v, self._fields_at(self.x), self.q / self.m, -0.5 * self.dt)
        return self

    def _fields_at(self, x):
        EB = em3_gather(self.n, self.dx, x, self.E, self.B)
        EB[:, 3:] += self.B0
        return EB

    def step(self, nsteps=1):
        for _ in range(nsteps):
            boris_eb(self.v, self._fields_at(self.x), self.q / self.m, self.dt)
            x0 = self.x.copy()
            move(3, self.n, self.dx, self.x, self.v, self.dt)
            self.J = np.zeros((3, self.cells))
            esirkepov3(self.n, self.dx, x0, self.x, self.q * self.w, self.dt, self.J)
            yee3_b(self.n, self.dx, self.E, self.B, 0.5 * self.dt)
            yee3_e(self.n, self.dx, self.B, self.J, self.c, self.dt, self.E)
            yee3_b(self.n, self.dx, self.E, self.B, 0.5 * self.dt)
            self.rho = self._rho()
            self.step_count += 1
        return self

    def gauss_residual(self):
        return yee3_div_e(self.n, self.dx, self.E) - self.rho


# ---- convolutional PML (E_Maxwell, Sec. 2.2; Roden and Gedney 2000) ---------------------------

def cpml_axis(n, npml, d, h, c, m=3, kappa_max=1.0, alpha_max=0.0):
    """(b, c, 1/kappa) along one axis of n nodes, at integer positions i and half
    positions i + 1/2, for an update of step h: depth = distance into a layer of npml
    cells / npml, sigma = sigma_max depth^m with sigma_max = 0.8 (m + 1) c / d (the
    matched value for eta = 1 / c, eps0 = 1), kappa = 1 + (kappa_max - 1) depth^m,
    alpha = alpha_max (1 - depth) inside the layer."""
    sigma_max = 0.8 * (m + 1) * c / d
    out = {}
    for name, shift in (("int", 0.0), ("half", 0.5)):
        b, cc, ik = np.ones(n), np.zeros(n), np.ones(n)
        if npml > 0:
            for i in range(n):
                x = i + shift
                depth = max(npml - x, x - (n - 1 - npml), 0.0) / npml
                if depth <= 0.0:
                    continue
                sigma = sigma_max * depth ** m
                kappa = 1.0 + (kappa_max - 1.0) * depth ** m
                alpha = alpha_max * (1.0 - depth)
                b[i] = math.exp(-(sigma / kappa + alpha) * h)
                cc[i] = sigma * (b[i] - 1.0) / (sigma * kappa + kappa * kappa * alpha)
                ik[i] = 1.0 / kappa
        out[name] = (b, cc, ik)
    return out


class CpmlField:
    """The Yee field update of the electromagnetic step on a non-periodic 2D grid with
    a convolutional PML of npml cells on every side, backed by a conducting wall;
    fields only (a prescribed current J drives it).  Each step: B half step, E step,
    B half step, as in EmSimulation."""

    def __init__(self, n, dx, dt, c, npml, m=3, kappa_max=1.0, alpha_max=0.0):
        self.n = (int(n[0]), int(n[1]))
        self.dx = (float(dx[0]), float(dx[1]))
        self.dt, self.c = float(dt), float(c)
        cells = self.n[0] * self.n[1]
        self.E = np.zeros((3, cells))
        self.B = np.zeros((3, cells))
        self.psi_b = [np.zeros(cells) for _ in range(4)]
        self.psi_e = [np.zeros(cells) for _ in range(4)]
        ax = [cpml_axis(self.n[a], npml, self.dx[a], 0.5 * self.dt, self.c, m, kappa_max, alpha_max)
              for a in range(2)]
        ae = [cpml_axis(self.n[a], npml, self.dx[a], self.dt, self.c, m, kappa_max, alpha_max)
              for a in range(2)]
        self.prof_b = [np.ascontiguousarray(v) for v in ax[0]["half"] + ax[1]["half"]]
        self.prof_e = [np.ascontiguousarray(v) for v in ae[0]["int"] + ae[1]["int"]]

    @staticmethod
    def _pp(arrs):
        return (_D * len(arrs))(*[a.ctypes.data_as(_D) for a in arrs])

    def step(self, J=None, nsteps=1):
        J = np.zeros_like(self.E) if J is None else _f(J)
        for _ in range(nsteps):
            for half in (0, 1):
                lib().orc_cpml_b(_n2(self.n), _dx2(self.dx), _dp(self.E), _dp(self.B),
                                 0.5 * self.dt, self._pp(self.prof_b), self._pp(self.psi_b))
                if half == 0:
                    lib().orc_cpml_e(_n2(self.n), _dx2(self.dx), _dp(self.B), _dp(J),
                                     self.c ** 2, self.dt, _dp(self.E), self._pp(self.prof_e),
                                     self._pp(self.psi_e))
        return self

    def energy(self):
        return 0.5 * float(np.sum(self.E ** 2) + self.c ** 2 * np.sum(self.B ** 2)) * \
            self.dx[0] * self.dx[1]


# ---- particles in the CPML mode (non-periodic 2D3V grid, absorbing particle walls) -----------

class CpmlPlasma(CpmlField):
    """Particles on the non-periodic grid of CpmlField: the electromagnetic cycle of
    EmSimulation with the CPML field update, gathers and currents that leave out the
    nodes outside the grid, and absorbing particle walls.  Particles live in the box
    [0, (n0 - 1) dx) x [0, (n1 - 1) dy); one that leaves it during a move deposits the
    current of its whole move (what falls outside the grid is dropped) and is then
    removed.  Fields start at zero (E = B = 0): the load solves no Poisson equation, so
    div E - rho starts at -rho and, by charge conservation, keeps its value at every
    node where neither the layer nor the wall modifies the update."""

    def __init__(self, n, dx, dt, c, npml, q=-1.0, m=1.0, weight=1.0, B0=(0, 0, 0), **kw):
        super().__init__(n, dx, dt, c, npml, **kw)
        self.q, self.m, self.w = float(q), float(m), float(weight)
        self.B0 = np.array(list(B0) + [0.0] * (3 - len(B0)))[:3]
        self.box = np.array([(self.n[0] - 1) * self.dx[0], (self.n[1] - 1) * self.dx[1]])
        self.absorbed = 0
        self.step_count = 0

    def _inside(self, x):
        return np.all((x >= 0.0) & (x < self.box), axis=1)

    def rho_e(self):
        rho = np.empty(self.n[0] * self.n[1])
        lib().orc_deposit_np(_n2(self.n), _dx2(self.dx), self.x.shape[0], _dp(self.x),
                             self.q * self.w, _dp(rho))
        return rho

    def _fields_at(self, x):
        out = np.empty((x.shape[0], 6))
        lib().orc_em_gather_np(_n2(self.n), _dx2(self.dx), x.shape[0], _dp(_f(x)), _dp(self.E),
                               _dp(self.B), _dp(out))
        out[:, 3:] += self.B0
        return out

    def load(self, x, v, half_push=True):
        self.x = np.array(x, dtype=np.float64, order="C")
        self.v = np.array(v, dtype=np.float64, order="C")
        assert self.x.shape[1] == 2 and self.v.shape[1] == 3
        assert np.all(self._inside(self.x)), "particles must start inside the walls"
        self.ids = np.arange(self.x.shape[0])  # load order of the particles still in the box
        if half_push:
            boris_eb(self.v, self._fields_at(self.x), self.q / self.m, -0.5 * self.dt)
        self.rho = self.rho_e()
        return self

    def step(self, nsteps=1):
        for _ in range(nsteps):
            boris_eb(self.v, self._fields_at(self.x), self.q / self.m, self.dt)
            x0 = self.x.copy()
            self.x += self.v[:, :2] * self.dt
            J = np.zeros((3, self.n[0] * self.n[1]))
            lib().orc_esirkepov_np(_n2(self.n), _dx2(self.dx), x0.shape[0], _dp(x0),
                                   _dp(self.x), _dp(np.ascontiguousarray(self.v[:, 2])),
                                   self.q * self.w, self.dt, _dp(J))
            CpmlField.step(self, J)
            keep = self._inside(self.x)
            self.absorbed += int(np.count_nonzero(~keep))
            self.x = np.ascontiguousarray(self.x[keep])
            self.v = np.ascontiguousarray(self.v[keep])
            self.ids = self.ids[keep]
            self.rho = self.rho_e()
            self.step_count += 1
        return self

    def div_e(self):
        """Discrete div E at the nodes, E outside the grid counting as zero."""
        ex = self.E[0].reshape(self.n[1], self.n[0])
        ey = self.E[1].reshape(self.n[1], self.n[0])
        dx = ex - np.pad(ex, ((0, 0), (1, 0)))[:, :-1]
        dy = ey - np.pad(ey, ((1, 0), (0, 0)))[:-1, :]
        return (dx / self.dx[0] + dy / self.dx[1]).ravel()

    def gauss_residual(self):
        return self.div_e() - self.rho
